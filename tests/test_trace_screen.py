"""The certification logic of the tracer's single-precision screen (k_trace.cu,
step_screen), restated here in NumPy float32 with the kernel's operands, order
and bounds: neighbour records holding the float offset of each neighbour from
its point, the walk's lateral offset carried in float with its error bound, and
a step decided only when the leading candidate is surely forward and its
q-interval lies below every other candidate's.  Walking every half-ray with the
oracle's exact next-point rule (Section 2.1, Fig. 2), each step the screen
certifies must be the oracle's step, and a half-ray the screen ends must end
there; undecided steps continue from the exact step, as the kernel's
double-precision path does.  The meshes include random clouds, a cloud far from
the coordinate origin, and a lattice with directions along its axes and
diagonals (exact ties, which must all be left undecided).  Fused multiply-adds
are emulated as the exact product in double plus one rounding to float, within
the unit roundoff the bounds take.  CPU only."""
import numpy as np
import pytest

from helpers import oracle_model_of as _model

f32 = np.float32
U = f32(2.0 ** -24)
INF = f32(np.inf)


def fma(a, b, c):
    return (np.float64(a) * np.float64(b) + np.float64(c)).astype(f32) if np.ndim(a) or np.ndim(b) or np.ndim(c) \
        else f32(np.float64(a) * np.float64(b) + np.float64(c))


def mesh_tables(pos, off, nbr):
    """Float positions, per-edge offset records, each point's largest record
    |.|_1, and the floor g0 of the bounds, as the mesh ingest forms them."""
    x32 = pos.astype(f32)
    src = np.repeat(np.arange(len(pos)), np.diff(off))
    rec = (x32[nbr] - x32[src]).astype(f32)
    S = ((np.abs(rec[:, 0]) + np.abs(rec[:, 1])).astype(f32) + np.abs(rec[:, 2])).astype(f32)
    smax = np.zeros(len(pos), f32)
    np.maximum.at(smax, src, S)
    s64 = (np.abs(pos[:, 0]) + np.abs(pos[:, 1])) + np.abs(pos[:, 2])
    s32 = s64.astype(f32)
    s32 = np.where(s32.astype(np.float64) < s64, np.nextafter(s32, INF), s32)  # rounded up
    g0 = f32(32.0 * 2.0 ** -48 * float(s32.max()) * (1.0 + 1e-6)) + f32(1e-37)
    return x32, rec, smax, g0


def screen_step(c, e_c, eec, f, x32, rec, smax, g0, off, nbr, margins=True):
    """One step of the screen from point c: (decision, new lateral offset, its bound).
    decision: a point id, -1 (the half-ray ends) or -2 (undecided)."""
    f0, f1, f2 = f
    ecx, ecy, ecz = e_c
    hcw = f32(f32(abs(x32[c, 0]) + abs(x32[c, 1])) + abs(x32[c, 2]))
    bz, be0 = fma(f32(4) * U, hcw, g0), fma(f32(8) * U, hcw, eec)
    sm = smax[c]
    k16 = f32(1) + f32(16) * U
    edZs = f32(fma(f32(8) * U, sm, bz) * k16)
    E1max = f32(f32(f32(f32(abs(ecx) + abs(ecy)) + abs(ecz)) + f32(f32(2.74) * sm)) * k16)
    des = f32(fma(f32(15) * U, sm, fma(f32(2) * U, E1max, be0)) * k16)
    k1 = fma(f32(2.02), des, g0)
    k0 = fma(fma(f32(3.03), des, g0), des, f32(g0 * g0))
    if not margins:  # a planted mistake: no error bounds at all
        edZs = k1 = k0 = f32(0)
    r = rec[off[c]:off[c + 1]]
    if len(r) == 0:
        return -1, None, None
    dx, dy, dz = r[:, 0], r[:, 1], r[:, 2]
    dZ = fma(dz, f2, fma(dy, f1, (dx * f0).astype(f32)))
    ex = (ecx + fma(-dZ, f0, dx)).astype(f32)
    ey = (ecy + fma(-dZ, f1, dy)).astype(f32)
    ez = (ecz + fma(-dZ, f2, dz)).astype(f32)
    q = fma(ez, ez, fma(ey, ey, (ex * ex).astype(f32)))
    E1 = ((np.abs(ex) + np.abs(ey)).astype(f32) + np.abs(ez)).astype(f32)
    eq = fma(k1, E1, fma(f32(6) * U, q, k0))
    lo = np.where(dZ < -edZs, INF, (q - eq).astype(f32))
    if not np.isfinite(lo).any():
        return -1, None, None
    b = int(np.argmin(lo))  # the first of equal lower bounds leads, as the kernel's strict test
    lo2 = np.min(np.delete(lo, b)) if len(lo) > 1 else INF
    hi1 = f32(q[b] + eq[b])
    if not (dZ[b] > edZs) or not (hi1 < lo2):
        return -2, None, None
    S = f32(f32(abs(dx[b]) + abs(dy[b])) + abs(dz[b]))
    bound = fma(f32(15) * U, S, fma(f32(2) * U, E1[b], be0))
    return int(nbr[off[c] + b]), (ex[b], ey[b], ez[b]), f32(bound * (f32(1) + f32(8) * U))


def lateral(pos, n, xo, Z, d, g0):
    """The lateral offset of point n (exact Z given) in double, rounded to float, and its bound."""
    e = tuple(f32((pos[n, i] - xo[i]) - Z * d[i]) for i in range(3))
    return e, fma(f32(f32(1.01) * U), max(abs(v) for v in e), g0)


def check_walks(orc_model, pos, off, nbr, origins, dirs, margins=True):
    """Walk every (origin, direction) half-ray; returns (certified, undecided, wrong) step counts."""
    x32, rec, smax, g0 = mesh_tables(pos, off, nbr)
    certified = undecided = wrong = 0
    for o in origins:
        for d in dirs:
            idx, Z = orc_model.trace_half(int(o), d)
            f = tuple(f32(v) for v in d)
            c, e_c, eec = int(o), (f32(0), f32(0), f32(0)), f32(0)
            for k in range(len(idx) + 1):
                exact = int(idx[k]) if k < len(idx) else -1
                got, e_n, eec_n = screen_step(c, e_c, eec, f, x32, rec, smax, g0, off, nbr, margins)
                if got == -2:
                    undecided += 1
                    if exact < 0:
                        break
                    e_n, eec_n = lateral(pos, exact, pos[o], Z[k], d, g0)
                else:
                    certified += 1
                    if got != exact:
                        wrong += 1
                        break
                    if exact < 0:
                        break
                c, e_c, eec = exact, e_n, eec_n
    return certified, undecided, wrong


def _healpix_dirs(orc, l):
    return [orc.pix2vec(l, p) for p in range(12 * 4 ** l)]


# far from the coordinate origin the float positions carry rounding of a few
# thousandths of the spacing, so fewer steps can be certified there
@pytest.mark.parametrize("shift,ratio", [(0.0, 10.0), (1.0e4, 1.0)])
def test_screen_certifies_only_exact_steps_on_clouds(orc, shift, ratio):
    from paper_2011_14998_gb300.learned import delaunay_neighbours

    rng = np.random.default_rng(11)
    pos = rng.normal(size=(500, 3)) * np.array([1.0, 0.7, 1.3]) + shift
    off, nbr = delaunay_neighbours(pos)
    om = _model(orc, pos, off, nbr)
    origins = rng.choice(len(pos), 12, replace=False)
    cert, und, wrong = check_walks(om, pos, off, nbr, origins, _healpix_dirs(orc, 2))
    assert wrong == 0
    assert cert > ratio * und  # the screen decides most steps of a generic cloud


def test_screen_certifies_only_exact_steps_on_the_wind(orc):
    # element sizes growing a hundredfold from the star outwards
    import synth

    m = synth.wind_model(1500, seed=9, n_freq=3)
    pos, off, nbr = m["pos"], np.asarray(m["nbr_off"]), np.asarray(m["nbr_idx"], np.int32)
    om = _model(orc, pos, off, nbr)
    r = np.linalg.norm(pos, axis=1)
    origins = [int(np.argmin(r)), int(np.argmax(r))] + list(np.random.default_rng(2).choice(len(pos), 6, replace=False))
    cert, und, wrong = check_walks(om, pos, off, nbr, origins, _healpix_dirs(orc, 2))
    assert wrong == 0
    assert cert > 10 * und


def test_screen_leaves_lattice_ties_undecided(orc):
    import synth

    g = synth.grid_model(6, n_freq=3)
    pos, off, nbr = g["pos"], np.asarray(g["nbr_off"]), np.asarray(g["nbr_idx"], np.int32)
    om = _model(orc, pos, off, nbr)
    axes = [np.array(v, float) / np.linalg.norm(v) for v in
            ([1, 0, 0], [0, -1, 0], [0, 0, 1], [1, 1, 0], [1, -1, 1], [0, 1, 1], [2, 1, 0])]
    dirs = axes + [-a for a in axes] + _healpix_dirs(orc, 1)
    origins = range(0, len(pos), 7)
    cert, und, wrong = check_walks(om, pos, off, nbr, origins, dirs)
    assert wrong == 0
    assert und > 0 and cert > 0


def test_screen_without_margins_fails_the_check(orc):
    # the planted mistake: with the error bounds set to zero the screen certifies
    # steps that the exact rule takes differently on the lattice's near-ties
    import synth

    g = synth.grid_model(6, n_freq=3)
    pos, off, nbr = g["pos"], np.asarray(g["nbr_off"]), np.asarray(g["nbr_idx"], np.int32)
    om = _model(orc, pos, off, nbr)
    axes = [np.array(v, float) / np.linalg.norm(v) for v in
            ([1, 0, 0], [0, -1, 0], [0, 0, 1], [1, 1, 0], [1, -1, 1], [0, 1, 1], [2, 1, 0])]
    dirs = axes + [-a for a in axes] + _healpix_dirs(orc, 1)
    _, _, wrong = check_walks(om, pos, off, nbr, range(0, len(pos), 7), dirs, margins=False)
    assert wrong > 0
