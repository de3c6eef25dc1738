"""The allocation-free solve (mgx_solve_J_noalloc) against mgx_solve_J.

It serves callers that must not allocate device memory during their step; it
uses one fixed 64 MiB device array as working memory and processes origins in
chunks that fit it: at most (8 MiB - 8) / (16 x 2 x pairs) origins per chunk
(2730 at 96 pairs), fewer when their traced point lists exceed the rest of the
array (about 15.6 million entries), in which case the chunk is shrunk and
traced again.  The 1500-point wind and the 8^3 grid fit one chunk; the
30000-point wind takes eleven or more, and its first chunk of 2730 origins
holds more list entries than the array, so it also takes the shrink-and-retry
path.
Two calls in a row check that the contents the previous call left in the
shared array do not leak into the result.  This file is collected last on
purpose.
"""
import numpy as np
import pytest

from helpers import j_rel_err

pytestmark = pytest.mark.gpu


def test_noalloc_matches_solve_J_twice():
    import torch

    import synth

    import paper_2011_14998_gb300 as mgx

    mgx.build()
    ctx = mgx.Context(0)
    try:
        for m, tol in ((synth.wind_model(1500, seed=21, n_freq=50), None), (synth.grid_model(8, n_freq=9), None)):
            mid = ctx.load(m)
            n, nb = len(m["pos"]), len(m["nu0"]) * m["n_freq"]
            for prec, tol in ((mgx.MGX_FP32, 1e-4), (mgx.MGX_FP64, 1e-10)):
                ref = ctx.solve_J(mid, precision=prec)
                for _ in range(2):
                    out = torch.full((n, nb), float("nan"), dtype=torch.float64, device="cuda")
                    mgx.mgx_solve_J_noalloc(ctx.ptr, mid, mgx.solve_params(precision=prec), out)
                    torch.cuda.synchronize()
                    got = out.cpu().numpy()
                    assert np.isfinite(got).all()
                    rel, _ = j_rel_err(got, ref)
                    assert rel <= tol, rel
            ctx.free(mid)
    finally:
        ctx.close()


def test_noalloc_crosses_chunks():
    import torch

    import oracle
    import synth

    import paper_2011_14998_gb300 as mgx

    mgx.build()
    ctx = mgx.Context(0)
    try:
        m = synth.wind_model(30000, seed=23, n_freq=20)
        mid = ctx.load(m)
        n, nb, npairs = len(m["pos"]), len(m["nu0"]) * m["n_freq"], ctx.models[mid]["npairs"]
        c_max = ((64 << 20) // 8 - 8) // (16 * 2 * npairs)
        cap = ((64 << 20) - (((2 * c_max * 2 * npairs + 1) * 8 + 255) // 256 * 256)) // 4
        off = ctx.trace(mid, 0, c_max, ids=False)[0]
        assert n > c_max  # more than one chunk by the origin limit
        assert off[-1] > cap  # the first chunk's lists overflow the array: shrink and retry
        ref = ctx.solve_J(mid, precision=mgx.MGX_FP32)
        rays = ctx.rays(mid)
        for _ in range(2):
            out = torch.full((n, nb), float("nan"), dtype=torch.float64, device="cuda")
            mgx.mgx_solve_J_noalloc(ctx.ptr, mid, mgx.solve_params(precision=mgx.MGX_FP32), out)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert np.isfinite(got).all()
            assert j_rel_err(got, ref)[0] <= 1e-4
        ctx.free(mid)
        # origins spread over every chunk against the FP64 oracle
        o = np.linspace(0, n - 1, 24).astype(np.int64)
        Jo = oracle.OracleModel(m, rays=rays).solve_J(oracle.params(), origins=o)
        assert j_rel_err(got[o], Jo)[0] <= 1e-4
    finally:
        ctx.close()


def test_noalloc_rejects_oversized_ray_set():
    import torch

    import paper_2011_14998_gb300 as mgx

    mgx.build()
    ctx = mgx.Context(0)
    try:
        one = np.ones((2, 1))
        m = dict(pos=np.array([[0.0, 0, 0], [1.0, 0, 0]]), vel=np.zeros((2, 3)), nbr_off=np.array([0, 1, 2]),
                 nbr_idx=np.array([1, 0], np.int32), nu0=np.array([1e11]), chi0=one, eta0=one, dvw=np.ones(2),
                 chi_c=np.ones(2), eta_c=np.ones(2), n_freq=2, x_span=1.0, l_min=8, l_max=8)
        mid = ctx.load(m)  # 393 216 pairs per point: too many for the fixed array
        out = torch.zeros((2, 2), dtype=torch.float64, device="cuda")
        with pytest.raises(mgx.MgxError) as e:
            mgx.mgx_solve_J_noalloc(ctx.ptr, mid, mgx.solve_params(), out)
        assert e.value.status == mgx.MGX_ERANGE
        with pytest.raises(mgx.MgxError):  # host memory is refused
            mgx.mgx_solve_J_noalloc(ctx.ptr, mid, mgx.solve_params(), np.zeros((2, 2)))
        ctx.free(mid)
    finally:
        ctx.close()
