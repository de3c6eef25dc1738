"""The bound E that certifies the single-precision solve's Eq. 2 decisions
(k_solve_impl.cuh, stage_interval): at every velocity sample of an interval,
both ends included, the kernel's single-precision opacity must lie within E of
the definition's double-precision one (Section 2.1.1 sample layout, the
profile argument as the oracle forms it, exp(-a^2)).  The single-precision
side is restated in NumPy float32 with the kernel's operands and order: the
points' float data and the error bound of delta, interpolation from the
farther point with t = j (1/nv) by fused multiply-adds, the prescaled profile
constants, rcp.approx for 1/dv and ex2.approx.ftz for the profile, the two
approximations taken at their measured error limits on GB300 (2^-23 and 2^-22
relative, drawn at random and at both extremes).  Removing the profile term
of the bound fails the check.  The decision itself is restated as well: with
the interval's spacing taken in single precision and its margin kappa, every
count the kernel certifies (the no-split threshold, or the ceilings of the
lower and upper bounds agreeing) is the definition's ceil(max(chi) ds /
dtau_max) on the definition's samples, including counts placed within 2^-23
to 2^-8 of an integer; without the bounds some are not.  One line, CPU only."""
import numpy as np
import pytest

f32 = np.float32
U = f32(2.0 ** -24)
K_ERCP = f32(2.0 ** -22)
K_EEX2 = f32(2.0 ** -20)
K_DELTA = f32(6.5) * U
ARG_SCALE = 1.2011224087864498  # sqrt(log2(e)): exp(-a^2) = 2^(-(a sqrt(log2 e))^2)
KC = 299792.458


def fma(a, b, c):
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def delta32(v, vo, e):
    f = e.astype(f32)
    v32, vo32 = v.astype(f32), vo.astype(f32)
    ux, uy, uz = (v32 - vo32).astype(f32)
    d = fma(uz, f[2], fma(uy, f[1], f32(ux * f[0])))
    de = f32(K_DELTA * f32(f32(f32(f32(abs(v32[0]) + abs(vo32[0])) * abs(f[0])) +
                               f32(f32(abs(v32[1]) + abs(vo32[1])) * abs(f[1]))) +
                           f32(f32(abs(v32[2]) + abs(vo32[2])) * abs(f[2]))))
    return d, de


def bound_E(da, dea, db, deb, wa, wb, cca, ccb, c0a, c0b, Am, Bm, drop_profile=False):
    """E of stage_interval for one line."""
    k6 = f32(f32(6) * U + K_ERCP)
    ada, adb = abs(da), abs(db)
    dmax = max(ada, adb)
    edi = f32(f32(dea + deb) + f32(k6 * f32(ada + adb)))
    rdvmin = f32(f32(1) / min(wa, wb))
    rho = f32(f32(K_ERCP + f32(f32(k6 * f32(wa + wb)) * rdvmin)) + f32(4) * U)
    dA = f32(f32(f32(f32(f32(3) * U * f32(Am + f32(Bm * dmax))) + f32(Bm * edi)) * rdvmin) * f32(f32(1) + rho))
    Eg = f32(f32(f32(f32(f32(0.7142) * dA) + f32(f32(f32(0.7358) * rho) * f32(1.001))) + f32(0.3679) * U) + K_EEX2)
    Eg = f32(Eg + f32(f32(2) * dA * dA))
    if drop_profile:
        Eg = f32(0)
    c0m = max(c0a, c0b)
    E = f32(f32(f32(c0m * Eg) + f32(k6 * f32(c0a + c0b))) + f32(U * c0m))
    csum = f32(max(cca, ccb) + c0m)
    E = f32(E + f32(f32(f32(k6 * f32(cca + ccb)) + f32(U * max(cca, ccb))) + f32(f32(2) * U * csum)))
    return f32(E * f32(1.0625))


def chi32(j, nv, pa, pb, A, B, e_rcp, e_ex2):
    """The kernel's opacity at sample j of nv (from the farther point a)."""
    d, w, cc, c0 = (pb if j == nv else tuple(
        fma(f32(y - x), f32(f32(j) * f32(f32(1) / f32(nv))), x) for x, y in zip(pa, pb)))
    if j == 0:
        d, w, cc, c0 = pa
    rdv = f32(f32(np.float64(1.0) / np.float64(w)) * (1.0 + e_rcp))
    a = f32(fma(B, d, A) * rdv)
    g = f32(2.0 ** -float(f32(a * a)) * (1.0 + e_ex2))
    if g < 2.0 ** -126:
        g = f32(0)  # flushed to zero
    return fma(c0, g, cc)


def chi64(orc, j, nv, qa, qb, forward, x, dvo):
    """The definition's opacity at the same sample: interpolated in double from
    the earlier point along +r (b on the forward half, a on the backward half)."""
    if j in (0, nv):
        d, w, cc, c0 = qa if j == 0 else qb
    else:
        x0, x1, i = (qb, qa, nv - j) if forward else (qa, qb, j)
        t = i / nv
        d, w, cc, c0 = (u0 + (u1 - u0) * t for u0, u1 in zip(x0, x1))
    a = orc.profile_arg(1.0, 1.0, x, dvo, d, w)
    return cc + c0 * np.exp(-(a * a))


def _check(orc, seed, n, extremes, drop_profile=False):
    rng = np.random.default_rng(seed)
    worst = 0.0
    for it in range(n):
        e = rng.normal(size=3)
        e /= np.linalg.norm(e)
        vo = rng.normal(0, 8, 3)
        dvo = rng.uniform(0.4, 1.5)
        x = rng.uniform(-4, 4)
        ub = x * dvo
        A = f32(ub * ARG_SCALE)
        B = f32((1.0 + ub / KC) * ARG_SCALE)
        va = vo + rng.normal(0, 3, 3)
        vb = va + rng.normal(0, 1.5, 3)
        wa, wb = rng.uniform(0.3, 2.0, 2)
        c0a, c0b = 10.0 ** rng.uniform(-2, 3, 2)
        cca, ccb = 1e-4 * c0a, 1e-4 * c0b
        da64 = (((va - vo)[0] * e[0] + (va - vo)[1] * e[1]) + (va - vo)[2] * e[2])
        db64 = (((vb - vo)[0] * e[0] + (vb - vo)[1] * e[1]) + (vb - vo)[2] * e[2])
        (da, dea), (db, deb) = delta32(va, vo, e), delta32(vb, vo, e)
        pa = (da, f32(wa), f32(cca), f32(c0a))
        pb = (db, f32(wb), f32(ccb), f32(c0b))
        qa, qb = (da64, wa, cca, c0a), (db64, wb, ccb, c0b)
        E = bound_E(da, dea, db, deb, pa[1], pb[1], pa[2], pb[2], pa[3], pb[3], abs(A), abs(B), drop_profile)
        nv = int(rng.integers(1, 6))
        forward = bool(rng.integers(0, 2))
        for j in range(nv + 1):
            if extremes:
                errs = [(s1 * 2.0 ** -23, s2 * 2.0 ** -22) for s1 in (-1, 1) for s2 in (-1, 1)]
            else:
                errs = [(rng.uniform(-1, 1) * 2.0 ** -23, rng.uniform(-1, 1) * 2.0 ** -22)]
            c64 = chi64(orc, j, nv, qa, qb, forward, x, dvo)
            for er, ee in errs:
                diff = abs(float(chi32(j, nv, pa, pb, A, B, er, ee)) - c64)
                worst = max(worst, diff / float(E))
    return worst


@pytest.mark.parametrize("extremes", [False, True])
def test_bound_covers_the_single_precision_opacity(orc, extremes):
    worst = _check(orc, 5 + int(extremes), 1500, extremes)
    assert worst <= 1.0, worst


def test_bound_without_the_profile_term_fails(orc):
    # the planted mistake: only the interpolation and sum terms, no profile error
    assert _check(orc, 7, 1500, True, drop_profile=True) > 1.0


def _interval(rng):
    e = rng.normal(size=3)
    e /= np.linalg.norm(e)
    vo = rng.normal(0, 8, 3)
    dvo = rng.uniform(0.4, 1.5)
    x = rng.uniform(-4, 4)
    ub = x * dvo
    A, B = f32(ub * ARG_SCALE), f32((1.0 + ub / KC) * ARG_SCALE)
    va = vo + rng.normal(0, 3, 3)
    vb = va + rng.normal(0, 1.5, 3)
    wa, wb = rng.uniform(0.3, 2.0, 2)
    c0a, c0b = 10.0 ** rng.uniform(-2, 3, 2)
    cca, ccb = 1e-4 * c0a, 1e-4 * c0b
    u = lambda v: ((v - vo)[0] * e[0] + (v - vo)[1] * e[1]) + (v - vo)[2] * e[2]
    (da, dea), (db, deb) = delta32(va, vo, e), delta32(vb, vo, e)
    pa, pb = (da, f32(wa), f32(cca), f32(c0a)), (db, f32(wb), f32(ccb), f32(c0b))
    qa, qb = (u(va), wa, cca, c0a), (u(vb), wb, ccb, c0b)
    E = bound_E(da, dea, db, deb, pa[1], pb[1], pa[2], pb[2], pa[3], pb[3], abs(A), abs(B))
    zb = rng.uniform(0.05, 60.0)
    za = zb + rng.uniform(0.002, 4.0)
    return pa, pb, qa, qb, A, B, x, dvo, E, za, zb


def _s_def(za, zb, nv, forward):
    """The definition's signed distances of the interval's samples along +r,
    listed from the farther point a (the kernel's order)."""
    if forward:  # s = +Z, interpolated from the nearer point b
        s0, s1 = zb, za
        s = [s0 if i == 0 else s1 if i == nv else s0 + (s1 - s0) * (i / nv) for i in range(nv + 1)]
        return s[::-1]
    s0, s1 = -za, -zb  # backward half: s = -Z, interpolated from the farther point a
    return [s0 if i == 0 else s1 if i == nv else s0 + (s1 - s0) * (i / nv) for i in range(nv + 1)]


def kernel_n(cm, E, za, zb, nv, dtau_max, cb, bounds=True):
    """Eq. 2's count as the single-precision solve decides it (0: left to double precision)."""
    ds = f32(za - zb)
    hs = f32(ds * f32(f32(1) / f32(nv)))
    zmax = f32(max(za, zb))
    kap = f32(f32(f32(15) * U + f32(f32(f32(9.0e-16) * zmax) / hs)) + f32(1e-15))
    if not bounds:
        kap, E = f32(0), f32(0)
    dtm = f32(dtau_max)
    qs = f32(hs * f32(1.0 / dtau_max))
    thr = f32(f32(f32(dtm / hs) * f32(f32(1) - kap)) - f32(E * f32(f32(1) + f32(4) * U)))
    if bounds and f32(cb * f32(f32(1) + f32(8) * U)) <= thr:
        return 1  # no bin can split anywhere on the interval
    if not cm > thr:
        return 1
    nhi = np.ceil(f32(f32(cm + E) * f32(qs * f32(f32(1) + kap))))
    if nhi <= 1:
        return 1
    nlo = np.ceil(f32(f32(cm - E) * f32(qs * f32(f32(1) - kap))))
    return int(nhi) if nlo == nhi else 0


def _decisions(orc, seed, n, bounds=True):
    rng = np.random.default_rng(seed)
    certified = undecided = wrong = 0
    for _ in range(n):
        pa, pb, qa, qb, A, B, x, dvo, E, za, zb = _interval(rng)
        nv = int(rng.integers(1, 5))
        forward = bool(rng.integers(0, 2))
        s = _s_def(za, zb, nv, forward)
        c64 = [chi64(orc, j, nv, qa, qb, forward, x, dvo) for j in range(nv + 1)]
        er, ee = rng.uniform(-1, 1) * 2.0 ** -23, rng.uniform(-1, 1) * 2.0 ** -22
        c32 = [chi32(j, nv, pa, pb, A, B, er, ee) for j in range(nv + 1)]
        cb = f32(max(pa[2], pb[2]) + max(pa[3], pb[3]))
        # dtau_max puts the first sub-interval's count within 2^-23 .. 2^-8 of an integer
        ds1 = abs(s[1] - s[0])
        k = int(rng.integers(1, 40))
        dtau_max = max(c64[0], c64[1]) * ds1 / (k * (1.0 + rng.integers(-3, 4) * 2.0 ** -float(rng.integers(8, 24))))
        for j in range(1, nv + 1):
            ds = abs(s[j] - s[j - 1])
            n_def = max(1, int(np.ceil(max(c64[j - 1], c64[j]) * ds / dtau_max)))
            got = kernel_n(max(c32[j - 1], c32[j]), E, za, zb, nv, dtau_max, cb, bounds)
            if got == 0:
                undecided += 1
            else:
                certified += 1
                wrong += got != n_def
    return certified, undecided, wrong


def test_certified_eq2_counts_are_the_definitions(orc):
    cert, und, wrong = _decisions(orc, 11, 3000)
    assert wrong == 0
    assert cert > 1000 and und > 0  # counts next to an integer are left to double precision


def test_eq2_counts_without_bounds_go_wrong(orc):
    # the planted mistake: no opacity bound and no spacing margin
    _, _, wrong = _decisions(orc, 11, 3000, bounds=False)
    assert wrong > 0
