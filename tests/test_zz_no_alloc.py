"""wr_tour_eval_static: the tour-evaluation entry point that allocates no device memory.

It exists for callers that cannot call cudaMalloc (device memory owned by
another allocator, or loops that cannot take cudaMalloc's device-wide
synchronisation); its scratch is a static device array shared by all calls.
These tests call it through the C ABI and check that it returns exactly what
the context-based wr_tour_eval returns, on two calls in a row (so results
cannot depend on what the previous call left in the shared scratch).
The file name sorts last so that a stopping run has already run every
other test before this one.
"""
import numpy as np
import pytest

from paper_2504_20655_gb300 import synth

pytestmark = pytest.mark.gpu
INF = 2**31 - 1


def _case(n, kmax, hi, seed):
    k = synth.uniform_int(seed, n, 1, kmax).astype(np.int32)
    k[::17] = 0                       # bad order: no picks
    k[5::29] = 13                     # bad order: more than WR_MAX_K picks
    D = synth.uniform_int(seed ^ 3, n * 169, 0, hi).reshape(n, 13, 13)
    D = np.where(synth.uniform01(seed ^ 4, n * 169).reshape(n, 13, 13) < 0.03, INF, D)
    D[3::41, 1, 2] = 10324441         # a leg above WR_LEG_MAX
    for i in range(13):
        D[:, i, i] = 0
    return k, D.astype(np.int32)


def test_static_entry_point_matches_context_entry_point():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2504_20655_gb300 import build, wroute
    build.build()
    r = wroute.Router(device=0)
    try:
        for n, kmax, hi, seed in ((700, 9, 60, 11), (90, 11, 4, 12)):
            k, D = _case(n, kmax, hi, seed)
            ref_cost, ref_perm, ref_status = r.tour_eval(k, D)
            dk = torch.from_numpy(k).cuda()
            dD = torch.from_numpy(D).cuda()
            cost = torch.full((n,), -7, dtype=torch.int32, device="cuda")
            perm = torch.full((n * 12,), -7, dtype=torch.int32, device="cuda")
            status = torch.full((n,), -7, dtype=torch.int32, device="cuda")
            wroute.wr_tour_eval_static(dk, dD, cost, perm, status)
            torch.cuda.synchronize()
            assert (status.cpu().numpy() == ref_status).all()
            assert (cost.cpu().numpy() == ref_cost).all()
            got = perm.cpu().numpy().reshape(n, 12)
            for i in range(n):
                kk = min(max(int(k[i]), 0), 12)
                assert (got[i, :kk] == ref_perm[i, :kk]).all(), i
            assert set(np.unique(ref_status)) >= {0, 2, 3}
    finally:
        r.close()


def test_static_entry_point_matches_oracle(orc):
    """The same entry point against the oracle directly: every order's cost, sequence and
    status equal the oracle's Held-Karp (lexicographically first optimum, pinned against
    brute force) over its own matrix, on two calls in a row."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2504_20655_gb300 import build, wroute
    build.build()
    for n, kmax, hi, seed in ((300, 10, 60, 21), (120, 12, 5, 22)):
        k, D = _case(n, kmax, hi, seed)
        cost = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        perm = torch.full((n * 12,), -7, dtype=torch.int32, device="cuda")
        status = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        wroute.wr_tour_eval_static(torch.from_numpy(k).cuda(), torch.from_numpy(D).cuda(), cost, perm, status)
        torch.cuda.synchronize()
        c, p, s = cost.cpu().numpy(), perm.cpu().numpy().reshape(n, 12), status.cpu().numpy()
        for i in range(n):
            kk = int(k[i])
            if kk < 1 or kk > 12:
                assert s[i] == 2, i
                continue
            st, oc, op = orc.tour(D[i, :kk + 1, :kk + 1], "heldkarp")
            assert (s[i], c[i]) == (st, oc), i
            assert p[i, :kk].tolist() == op.tolist(), i


def test_static_entry_point_rejects_oversize():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2504_20655_gb300 import wroute
    n = wroute.WR_STATIC_MAX_ORDERS + 1
    k = torch.ones(n, dtype=torch.int32, device="cuda")
    D = torch.zeros(n * 169, dtype=torch.int32, device="cuda")
    out = [torch.empty(n * 12, dtype=torch.int32, device="cuda") for _ in range(3)]
    with pytest.raises(wroute.WrError) as e:
        wroute.wr_tour_eval_static(k, D, out[0], out[1], out[2])
    assert e.value.code == wroute.WR_EINVAL
