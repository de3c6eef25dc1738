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
of the bound fails the check.  One line, CPU only."""
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
