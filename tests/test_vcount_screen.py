"""The certification of the single-precision solve's velocity-sample count
(k_solve_impl.cuh, stage_interval), restated in NumPy float32 with the kernel's
operands and bounds: the projected velocity differences in float with their
error bounds, then ceil of the jump over the limit taken at both ends of its
interval.  Where the two ends agree the count must be the definition's
(Section 2.1.1: ceil(|delta_b - delta_a| / (dv_max min(dv_a, dv_b))) parts when
the jump exceeds the limit, delta in double precision in the definition's
order), and everywhere else the kernel redoes it in double precision.  Jumps
are drawn both at random and close to an integer multiple of the limit (2^-23
to 2^-10 relative); with the error bounds removed the restatement takes wrong
counts there.  CPU only."""
import numpy as np

f32 = np.float32
U = f32(2.0 ** -24)
K_DELTA = f32(6.5) * U


def delta64(v, vo, e):
    """(v - vo).d in double, (x + y) + z, every operation rounded."""
    u = v - vo
    return (u[0] * e[0] + u[1] * e[1]) + u[2] * e[2]


def delta32(v, vo, e):
    """The kernel's single-precision delta and its error bound."""
    f = e.astype(f32)
    v32, vo32 = v.astype(f32), vo.astype(f32)
    ux, uy, uz = (v32 - vo32).astype(f32)
    fma = lambda a, b, c: f32(np.float64(a) * np.float64(b) + np.float64(c))
    d = fma(uz, f[2], fma(uy, f[1], f32(ux * f[0])))
    de = f32(K_DELTA * f32(f32(f32(f32(abs(v32[0]) + abs(vo32[0])) * abs(f[0])) +
                               f32(f32(abs(v32[1]) + abs(vo32[1])) * abs(f[1]))) +
                           f32(f32(abs(v32[2]) + abs(vo32[2])) * abs(f[2]))))
    return d, de


def count64(da, db, wa, wb, dv_max):
    jump, lim = abs(db - da), dv_max * min(wa, wb)
    return int(np.ceil(jump / lim)) if jump > lim else 1


def count32(da, dea, db, deb, wa, wb, dv_max, margins=True):
    """(certified, count) as the kernel's single-precision decision takes it."""
    jump = f32(abs(f32(db - da)))
    ej = f32(f32(dea + deb) + f32(f32(2) * U * jump)) if margins else f32(0)
    rl = f32(f32(1) / f32(f32(dv_max) * min(f32(wa), f32(wb))))
    up, dn = (f32(1) + f32(16) * U, f32(1) - f32(16) * U) if margins else (f32(1), f32(1))
    nhi = np.ceil(f32(f32(f32(jump + ej) * rl) * up))
    if not nhi > 1:
        return True, 1
    nlo = np.ceil(f32(f32(f32(jump - ej) * rl) * dn))
    return bool(nlo == nhi), int(nhi)


def _cases(rng, n, near):
    dv_max = 1.0 / 3.0
    for _ in range(n):
        e = rng.normal(size=3)
        e /= np.linalg.norm(e)
        vo = rng.normal(0, 10, 3)
        va = vo + rng.normal(0, 10, 3)
        wa, wb = rng.uniform(0.3, 2.0, 2)
        lim = dv_max * min(wa, wb)
        if near:  # a jump near an integer multiple of the limit: 2^-23 to 2^-10 relative
            t = rng.integers(1, 12) * (1.0 + rng.integers(-4, 5) * 2.0 ** -float(rng.integers(10, 24)))
        else:
            t = rng.uniform(0.0, 12.0)
        side = rng.normal(size=3)
        side -= side.dot(e) * e
        vb = va + t * lim * e + rng.uniform(0, 5) * side
        yield e, vo, va, vb, wa, wb, dv_max


def _run(near, margins, n=4000, seed=0):
    rng = np.random.default_rng(seed)
    certified = wrong = 0
    for e, vo, va, vb, wa, wb, dv_max in _cases(rng, n, near):
        da, db = delta64(va, vo, e), delta64(vb, vo, e)
        (d32a, dea), (d32b, deb) = delta32(va, vo, e), delta32(vb, vo, e)
        ok, nv = count32(d32a, dea, d32b, deb, wa, wb, dv_max, margins)
        if ok:
            certified += 1
            wrong += nv != count64(da, db, wa, wb, dv_max)
    return certified, wrong


def test_certified_counts_are_the_definitions():
    cert, wrong = _run(near=False, margins=True)
    assert wrong == 0 and cert > 3900  # almost every random jump is decided in single precision
    cert, wrong = _run(near=True, margins=True, seed=1)
    assert wrong == 0 and cert > 0


def test_origin_interval():
    # the origin's own delta is exactly 0 with no error; the other end carries its bound
    rng = np.random.default_rng(4)
    for e, vo, va, vb, wa, wb, dv_max in _cases(rng, 2000, near=True):
        db = delta64(vb, vo, e)
        d32b, deb = delta32(vb, vo, e)
        ok, nv = count32(f32(0), f32(0), d32b, deb, wa, wb, dv_max)
        if ok:
            assert nv == count64(0.0, db, wa, wb, dv_max)


def test_counts_without_bounds_go_wrong_near_multiples():
    # the planted mistake: without the error bounds some near-multiple jumps take
    # the wrong count, which the bounded decision leaves to double precision
    _, wrong = _run(near=True, margins=False, seed=1)
    assert wrong > 0
