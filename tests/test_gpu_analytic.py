"""The element-size field of analytic models (Section 2.2.1, Eq. 5) on the GPU
against the oracle, bit for bit (Gf, ell and the kept points), on a Gaussian,
an exponential and a flat (one-point axis) background mesh; invalid inputs;
and the meshing pipeline on the spiral-wind tracer (the paper's analytic
example: 1200 AU box, ell_min 15 AU, ell_max 50 AU, here on a coarser
background) producing a mesh the solver accepts."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2011_14998_gb300 as mgx

    mgx.build()
    c = mgx.Context(0)
    yield c
    c.close()


def _fields():
    g = np.linspace(-0.5, 0.5, 33)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    gauss = np.exp(-(X**2 + Y**2 + Z**2) / (2 * 0.2**2)), g[1] - g[0]
    x = np.arange(20) * 0.3
    expo = np.repeat(np.exp(0.7 * x)[:, None, None], 7, axis=1) * (1 + 0.1 * np.arange(7))[None, :, None], 0.3
    return {"gauss": gauss, "expo": expo}


@pytest.mark.parametrize("name", ["gauss", "expo"])
def test_size_field_bit_exact(ctx, orc, name):
    import paper_2011_14998_gb300 as mgx

    f, h = _fields()[name]
    for ell_min, ell_max, seed in ((h, 4 * h, 1), (1.5 * h, 10 * h, 2**63 + 5)):
        Gf, ell, keep, nk = mgx.mgx_analytic_mesh(ctx.ptr, f, h, ell_min, ell_max, seed)
        Go, eo, ko = orc.analytic_mesh(f, h, ell_min, ell_max, seed)
        assert np.array_equal(Gf, Go)
        assert np.array_equal(ell, eo)
        assert np.array_equal(keep, ko)
        assert nk == int(ko.sum())


def test_invalid_inputs(ctx):
    import paper_2011_14998_gb300 as mgx

    f = np.ones((4, 4, 4))
    with pytest.raises(mgx.MgxError):
        mgx.mgx_analytic_mesh(ctx.ptr, f * 0.0, 0.1, 0.1, 0.4)  # tracer must be > 0
    with pytest.raises(mgx.MgxError):
        mgx.mgx_analytic_mesh(ctx.ptr, f, 0.2, 0.1, 0.4)  # h > ell_min
    with pytest.raises(mgx.MgxError):
        mgx.mgx_analytic_mesh(ctx.ptr, f, 0.1, 0.5, 0.4)  # ell_min > ell_max


def test_spiral_wind_mesh_solves(ctx):
    import synth

    import paper_2011_14998_gb300 as mgx
    from paper_2011_14998_gb300 import meshing

    h = 24.0  # 51^3 background over the 1200 AU box (the paper: 100^3, 12 AU)
    mesh = meshing.analytic_mesh(ctx, synth.spiral_density, [-600] * 3, [600] * 3, h, 30.0, 100.0, seed=7)
    n = len(mesh["pos"])
    assert 0 < n == mesh["n_kept"] < np.prod(mesh["shape"])
    # the kept count follows the target density ell^-3, and the kept points sit
    # where the desired elements are smaller
    p = (h / mesh["ell"].ravel()) ** 3
    assert abs(n - p.sum()) < 5 * np.sqrt((p * (1 - p)).sum())
    keep = mesh["keep"].ravel() != 0
    assert mesh["ell"].ravel()[keep].mean() < mesh["ell"].ravel().mean()
    rho = synth.spiral_density(mesh["pos"])
    T = 2000.0 * (np.maximum(np.sqrt((mesh["pos"] ** 2).sum(1)), 10.0) / 10.0) ** -0.7
    chi0 = (0.01 * rho)[:, None]
    model = dict(pos=mesh["pos"], vel=np.zeros((n, 3)), nbr_off=mesh["nbr_off"], nbr_idx=mesh["nbr_idx"],
                 nu0=np.array([synth.NU_CO10]), chi0=chi0, eta0=chi0 * (T / 2000.0)[:, None],
                 dvw=synth.doppler_width(T), chi_c=1e-4 * chi0[:, 0], eta_c=1e-4 * chi0[:, 0] * T / 2000.0,
                 n_freq=11, x_span=4.0, l_min=1, l_max=1, sample=synth.sample_indices(n))
    mid = ctx.load(model)
    J = ctx.solve_J(mid, precision=mgx.MGX_FP32)
    ctx.free(mid)
    assert J.shape == (n, 11) and np.all(np.isfinite(J)) and J.min() >= 0
