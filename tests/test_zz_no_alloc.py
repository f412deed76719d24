"""The allocation-free iteration, cupso_tree_step_noalloc, through the C ABI.

Its users are callers that cannot allocate device memory themselves because
another allocator owns their GPU memory; here the test plays that caller and
holds the swarm in torch tensors. Two calls in a row must reproduce what the
regular entry points give for the same swarm (cupso_step in tree mode), within
the tests' single-step bar of 2 ulp (the arithmetic is the same, so in fact
bit for bit).
"""
import numpy as np
import pytest

from tests.gpu_common import W, C12, BOUNDS, load_cupso, same_bits, ulp_distance

pytestmark = pytest.mark.gpu


def _planes(torch, a, ld, fill=0.0):
    """Host [N][D] -> device [D][ld] float32 (columns N..ld-1 = fill)."""
    N, D = a.shape
    out = torch.full((D, ld), fill, dtype=torch.float32, device="cuda")
    out[:, :N] = torch.from_numpy(np.ascontiguousarray(a.T)).to("cuda")
    return out


# (fitness, N, D, extra stride beyond N rounded up to 128). With the sphere and a
# padded stride the padding columns hold x = 0, whose fitness is the global
# optimum 0, with pbest_fit = +inf: they improve every call, and the test shows
# that they still never win the global best.
@pytest.mark.parametrize("fid,N,D,pad", [(1, 3000, 7, 0), (3, 1024, 32, 0), (0, 1000, 5, 1152)])
def test_noalloc_two_calls_match_cupso_step(fid, N, D, pad):
    P = load_cupso()
    import torch

    seed, ld = 13, (N + 127) // 128 * 128 + pad
    b = BOUNDS[fid]
    with P.Swarm(D, N, b, W, C12, C12, fid, seed, mode="tree") as s:
        states = [s.state()]
        bests = [s.gbest()]
        for _ in range(2):
            s.step(1)
            states.append(s.state())
            bests.append(s.gbest())

    st0 = states[0]
    pos = _planes(torch, st0["pos"], ld)
    v = _planes(torch, st0["v"], ld)
    pb = _planes(torch, st0["pbest_pos"], ld)
    pf = torch.full((ld,), float("inf"), dtype=torch.float32, device="cuda")
    pf[:N] = torch.from_numpy(st0["pbest_fit"]).to("cuda")
    gpos = torch.from_numpy(bests[0][3].copy()).to("cuda")
    gfit = torch.empty(1, dtype=torch.float32, device="cuda")
    gidx = torch.empty(1, dtype=torch.int64, device="cuda")
    status = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    for t in (1, 2):
        P.cupso_tree_step_noalloc(D, N, b, W, C12, C12, fid, seed, 0, t, pos.data_ptr(), v.data_ptr(),
                                  pb.data_ptr(), pf.data_ptr(), ld, gpos.data_ptr(), gfit.data_ptr(),
                                  gidx.data_ptr(), status.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        ref = states[t]
        _, ref_fit, ref_idx, ref_gpos = bests[t]
        got = {"pos": pos[:, :N].T.cpu().numpy(), "v": v[:, :N].T.cpu().numpy(),
               "pbest_pos": pb[:, :N].T.cpu().numpy(), "pbest_fit": pf[:N].cpu().numpy()}
        for k in ("pos", "v", "pbest_pos", "pbest_fit"):
            assert ulp_distance(got[k], ref[k]).max() <= 2, (t, k)
            assert same_bits(got[k], ref[k]), (t, k)
        assert int(gidx.item()) == ref_idx
        assert ulp_distance(gfit.cpu().numpy(), np.array([ref_fit], np.float32)).max() <= 2
        assert ulp_distance(gpos.cpu().numpy(), ref_gpos).max() <= 2
        assert int(status.item()) == 0


def test_noalloc_rejects_sizes_beyond_its_limit():
    P = load_cupso()
    import torch

    buf = torch.zeros(1024, dtype=torch.float32, device="cuda")
    p = buf.data_ptr()
    # The arguments are checked on the host before anything is queued, so none
    # of these calls launches a kernel on the one-element buffer.
    M = P.CUPSO_NOALLOC_MAX_N
    for D, N, ld in [(4, M + 1, M + 128),             # N beyond the limit
                     (P.CUPSO_NOALLOC_MAX_D + 1, 128, 128),
                     (4, 200, 200),                    # stride not a multiple of 128
                     (4, M, M + 128),                  # N at the limit, stride one tile row beyond
                     (4, 100, 2 * M)]:                 # small N, stride far beyond the scratch
        with pytest.raises(P.CupsoError) as e:
            P.cupso_tree_step_noalloc(D, N, BOUNDS[0], W, C12, C12, 0, 1, 0, 1, p, p, p, p, ld, p)
        assert e.value.code == P.CUPSO_ERR_INVALID_ARG
        msg = P.last_error()
        assert ("supports N <=" in msg) or ("multiple of" in msg) or ("supports ld <=" in msg), msg


def test_noalloc_calls_leave_free_device_memory_unchanged():
    """The property the entry point exists for: after a first call (which may
    load the library's kernels into the context), further calls take no device
    memory. torch's allocator is idle between the two readings."""
    P = load_cupso()
    import torch

    N, D, fid, seed = 2048, 16, 1, 5
    ld = N
    b = BOUNDS[fid]
    with P.Swarm(D, N, b, W, C12, C12, fid, seed, mode="tree") as s:
        st0 = s.state()
        g0 = s.gbest()
    pos = _planes(torch, st0["pos"], ld)
    v = _planes(torch, st0["v"], ld)
    pb = _planes(torch, st0["pbest_pos"], ld)
    pf = torch.from_numpy(st0["pbest_fit"].copy()).to("cuda")
    gpos = torch.from_numpy(g0[3].copy()).to("cuda")
    gfit = torch.empty(1, dtype=torch.float32, device="cuda")
    gidx = torch.empty(1, dtype=torch.int64, device="cuda")
    status = torch.empty(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    def call(t):
        P.cupso_tree_step_noalloc(D, N, b, W, C12, C12, fid, seed, 0, t, pos.data_ptr(), v.data_ptr(),
                                  pb.data_ptr(), pf.data_ptr(), ld, gpos.data_ptr(), gfit.data_ptr(),
                                  gidx.data_ptr(), status.data_ptr(), stream.cuda_stream)

    call(1)
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    reserved_before = torch.cuda.memory_reserved()
    for t in (2, 3, 4):
        call(t)
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_reserved() == reserved_before
    assert free_after == free_before, (free_before, free_after)
    assert int(status.item()) == 0
