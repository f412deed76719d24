"""CPU oracle of the PSO iteration -- TEST INFRASTRUCTURE ONLY.

Imported by the tests, by ``__graft_entry__.smoke()`` and by the benchmark's
CPU-baseline leg, never by the library. See ``oracle.py`` for the Python view.
"""
