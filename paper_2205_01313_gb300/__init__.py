"""GB300-native particle swarm optimizer (cuPSO's hot path, sm_103a).

The library is `_build/libcupso.so` behind the C ABI of `include/cupso.h`;
`cupso` is its Python binding. Build with `paper_2205_01313_gb300.build.build()`.
"""
