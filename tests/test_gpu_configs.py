"""Parity on two of the workloads at their stated sizes, in the batched
launch that times them (FP32, ray sets rebuilt inside the graph):

* the clump octree of about 3e5 leaf centres (levels 3-8, three Gaussian
  clumps of contrast 1e3, two lines x 64 bins, adaptive rays l 0-3, 2 km/s
  Fourier velocity field);
* models 0, 16, 32 and 48 of the 64-model draw (sizes log-uniform in
  [1e4, 2e5]; grid, wind and octree in turn; four lines x 100 bins; adaptive
  rays l 0-3), solved together in one persistent launch.

J is compared with the FP64 oracle at sampled origins (1e-4), and the
adaptive ray sets of sampled origins bit for bit with the oracle's own ray
set of each origin (Section 2.1.3), computed from the mesh independently of
the GPU's."""
import numpy as np
import pytest

from helpers import j_rel_err

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-4


@pytest.fixture(scope="module")
def ctx():
    import paper_2011_14998_gb300 as mgx

    mgx.build()
    c = mgx.Context(0)
    yield c
    c.close()


def _check(ctx, orc, models, mids, outs, n_origins, seed):
    worst = []
    for j, (m, k) in enumerate(zip(models, mids)):
        n = len(m["pos"])
        rays = ctx.rays(k)
        o = np.sort(np.random.default_rng(seed + j).choice(n, size=min(n_origins, n), replace=False))
        ref_rays = orc.rayset_at(m["pos"], o, m["l_min"], m["l_max"], m["sample"])
        assert np.array_equal(rays[o], ref_rays), m["name"]
        Jo = orc.OracleModel(m, rays=rays).solve_J(orc.params(), origins=o)
        r = j_rel_err(outs[j].cpu().numpy()[o], Jo)[0]
        worst.append((m["name"], n, r))
    print(worst)
    for name, n, r in worst:
        assert r < FP32_TOL, (name, n, r)


def test_octree_full_size(ctx, orc):
    import synth

    import paper_2011_14998_gb300 as mgx

    m = synth.octree_model(300_000, seed=3)
    assert 250_000 < len(m["pos"]) < 350_000
    mid = ctx.load(m)
    flags = mgx.MGX_BATCH_GRAPH | mgx.MGX_BATCH_RAYS
    outs = ctx.solve_J_batch([mid], precision=mgx.MGX_FP32, flags=flags)
    ctx.solve_J_batch([mid], precision=mgx.MGX_FP32, outs=outs, flags=flags)
    _check(ctx, orc, [m], [mid], outs, 24, 31)
    ctx.free(mid)


def test_batch_members_full_size(ctx, orc):
    import synth

    import paper_2011_14998_gb300 as mgx

    models = synth.batch_models(n_models=64, seed=5, only=(0, 16, 32, 48))
    assert len(models) == 4 and all(10_000 * 0.8 <= len(m["pos"]) <= 200_000 * 1.2 for m in models)
    mids = [ctx.load(m) for m in models]
    flags = mgx.MGX_BATCH_GRAPH | mgx.MGX_BATCH_RAYS
    outs = ctx.solve_J_batch(mids, precision=mgx.MGX_FP32, flags=flags)
    ctx.solve_J_batch(mids, precision=mgx.MGX_FP32, outs=outs, flags=flags)
    _check(ctx, orc, models, mids, outs, 12, 51)
    for k in mids:
        ctx.free(k)
