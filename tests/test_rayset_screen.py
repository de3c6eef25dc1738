"""The certification logic of the adaptive ray set's single-precision HEALPix
screen (k_rays.cu, vec2pix_nest_f), restated here in NumPy float32 with the
same operation order and bounds (NumPy's own atan2f standing in for CUDA's:
both lie well inside the 2^-20 rad the bound takes).  Wherever the screen
certifies a pixel it must be the pixel of the oracle's double-precision
vec2pix (Gorski et al. 2005 nested scheme); the directions include random
ones and ones next to every kind of pixel boundary, where most must be left
to double precision.  CPU only."""
import numpy as np

f32 = np.float32
U = f32(2.0 ** -24)
KA = f32(2.0 ** -20)


def _trunc_certain(v, e):
    """(ok, k): trunc of every value within e of v is k (trunc maps (-1, 1) to 0)."""
    ok = v > f32(-1.0) + e
    small = v < f32(1.0) - e
    f = np.floor(v)
    far = ((v - f) >= e) & ((f + f32(1.0) - v) >= e)
    k = np.where(small, 0, f).astype(np.int64)
    return ok & (small | far), k


def _spread2(v):
    out = np.zeros_like(v)
    for b in range(16):
        out |= ((v >> b) & 1) << (2 * b)
    return out


def screen(l, a, b, c):
    """Pixel and certified flag of each direction, in the screen's float32 arithmetic."""
    a, b, c = a.astype(f32), b.astype(f32), c.astype(f32)
    ns = 1 << l
    fns = f32(ns)
    with np.errstate(divide="ignore", invalid="ignore"):
        ln = np.sqrt((a * a + b * b) + c * c)
        z = c / ln
        za = np.abs(z)
        ez = f32(7.0) * U * za + f32(1e-30)
        t = np.arctan2(b, a) * f32(0.636619772367581343)
        et = f32(0.64) * KA + f32(12.0) * U
        ok = np.abs(t) >= et
        t = np.where(t < 0, t + f32(4.0), t)
        t = np.where(t >= 4, t - f32(4.0), t).astype(f32)
        tt = f32(0.666666666666666667)
        equ = za <= tt - ez - f32(2) * U
        pol = za > tt + ez + f32(2) * U
        ok &= equ | pol
        # equatorial
        c1 = fns * (f32(0.5) + t)
        c2 = fns * (f32(0.75) * z)
        eA = fns * (et + f32(0.75) * ez + f32(11) * U)
        oka, asc = _trunc_certain((c1 - c2).astype(f32), eA)
        okd, dsc = _trunc_certain((c1 + c2).astype(f32), eA)
        fa, fd = asc >> l, dsc >> l
        face_e = np.where(fa == fd, fa | 4, np.where(fa < fd, fa, fd + 8))
        x_e = dsc & (ns - 1)
        y_e = ns - 1 - (asc & (ns - 1))
        # polar
        okq, q = _trunc_certain(t, et)
        q = np.where(t > f32(3) + et, 3, q)
        okq = okq | (t > f32(3) + et)
        tp = (t - q.astype(f32)).astype(f32)
        om = (f32(1) - za).astype(f32)
        w = fns * np.sqrt(f32(3) * om)
        ew = w * ((ez + f32(2) * U) / (f32(2) * om) + f32(2) * U)
        okw = ew < 0.25
        e2 = et * w + ew + f32(2) * U * w
        oki, ia = _trunc_certain((tp * w).astype(f32), e2)
        okj, ib = _trunc_certain(((f32(1) - tp) * w).astype(f32), e2)
        ia, ib = np.minimum(ia, ns - 1), np.minimum(ib, ns - 1)
        north = z >= 0
        face_p = np.where(north, q, q + 8)
        x_p = np.where(north, ns - 1 - ib, ia)
        y_p = np.where(north, ns - 1 - ia, ib)
        ok &= np.where(equ, oka & okd, okq & okw & oki & okj)
    face = np.where(equ, face_e, face_p)
    x = np.where(equ, x_e, x_p)
    y = np.where(equ, y_e, y_p)
    pix = (face << (2 * l)) + _spread2(x) + 2 * _spread2(y)
    return np.where(ok, pix, -1), ok


def _boundary_directions(rng, l, n):
    ns = 1 << l
    out = []
    for i in range(n):
        kind = i % 4
        d = rng.uniform(-3e-5, 3e-5) * 10 ** rng.uniform(-6, 0)
        if kind < 2:  # equatorial diagonals: ns (0.5 + t) -+ 0.75 ns z = k + d
            z = rng.uniform(-0.66, 0.66)
            k = rng.integers(0, 5 * ns)
            t = (k + d + (0.75 if kind == 0 else -0.75) * ns * z) / ns - 0.5
        elif kind == 2:  # the zone boundary
            z = (2 / 3 + 3e-2 * d) * rng.choice([-1, 1])
            t = rng.uniform(0, 4)
        else:  # polar in-face boundaries: tp w = k + d
            za = rng.uniform(0.67, 0.9999)
            w = ns * np.sqrt(3 * (1 - za))
            k = rng.integers(0, int(w) + 1)
            tp = min(max((k + d) / w, 0.0), 0.9999999)
            if rng.random() < 0.5:
                tp = 1 - tp
            t = rng.integers(0, 4) + tp
            z = za * rng.choice([-1, 1])
        phi = (t % 4.0) * np.pi / 2
        st = np.sqrt(max(0.0, 1 - z * z))
        out.append(np.array([st * np.cos(phi), st * np.sin(phi), z]) * 10 ** rng.uniform(-2, 2))
    return np.array(out)


def test_certified_pixels_are_the_definitions():
    import oracle

    rng = np.random.default_rng(11)
    for l in (0, 2, 3, 5):
        rnd = rng.normal(size=(20000, 3)) * 10 ** rng.uniform(-2, 2, (20000, 1))
        adv = _boundary_directions(rng, l, 6000)
        axes = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1], [1, 1, 0], [-1, -1, 1e-9]])
        for d, kind in ((rnd, "random"), (adv, "boundary"), (axes.astype(float), "axes")):
            # the kernel rounds the double differences to float
            pix, ok = screen(l, d[:, 0].astype(f32), d[:, 1].astype(f32), d[:, 2].astype(f32))
            ref = oracle.vec2pix(l, d)
            assert np.array_equal(pix[ok], ref[ok]), (l, kind, int((pix[ok] != ref[ok]).sum()))
            if kind == "random":
                assert ok.mean() > 0.995, (l, ok.mean())  # almost all certified
            elif kind == "boundary":
                assert ok.mean() < 0.5, (l, ok.mean())  # most left to double precision
