"""The far-wing test of the single-precision solve's sample records
(k_solve_impl.cuh, gen_sample, one line): a record is marked far-wing when the
profile argument of the tile's first and last bin, widened by the spread of B
between them, stays beyond 12.1 in magnitude; the lanes then take the continuum
alone, which is the result only if every bin's own argument a, formed as the
kernel forms it (fl(fl(B delta + A) rdv), A and B rising with the bin), has
fl(a a) >= 128, where ex2.approx.ftz(-a a) is exactly +0.  Restated in NumPy
float32 over random and boundary cases; rcp.approx for rdv taken at its
measured error limit.  With the threshold moved below sqrt(128) it marks
records whose profile is not zero.  CPU only."""
import numpy as np

f32 = np.float32
ARG_SCALE = 1.2011224087864498
KC = 299792.458


def fma(a, b, c):
    return (np.float64(a) * np.float64(b) + np.float64(c)).astype(f32)


def tile_constants(n_freq, x_span, dvo):
    x = -x_span + 2.0 * x_span * np.arange(n_freq) / (n_freq - 1)
    ub = x * dvo
    return (ub * ARG_SCALE).astype(f32), ((1.0 + ub / KC) * ARG_SCALE).astype(f32)


def marked(A, B, dl, rdv, thr=12.1):
    tf, tl = fma(B[0], dl, A[0]), fma(B[-1], dl, A[-1])
    W = f32(f32(f32(1.01) * f32(B[-1] - B[0])) * abs(dl))
    lo = f32(f32(min(tf, tl) - W) * rdv)
    hi = f32(f32(max(tf, tl) + W) * rdv)
    return lo >= f32(thr) or hi <= f32(-thr)


def all_far(A, B, dl, rdv):
    a = (fma(B, dl, A) * rdv).astype(f32)
    return bool(np.all((a * a).astype(f32) >= f32(128.0)))


def _cases(rng, n):
    for _ in range(n):
        n_freq = int(rng.integers(2, 65))
        x_span = rng.uniform(0.5, 8.0)
        dvo = rng.uniform(0.2, 3.0)
        A, B = tile_constants(n_freq, x_span, dvo)
        w = rng.uniform(0.1, 3.0)
        rdv = f32(f32(1.0 / w) * (1.0 + rng.uniform(-1, 1) * 2.0 ** -23))
        if rng.uniform() < 0.5:  # a sample whose first or last bin sits at |a| = 12.1 or so
            end = int(rng.integers(0, 2))
            sign = rng.choice([-1.0, 1.0])
            target = sign * 12.1 * (1.0 + rng.uniform(-1e-3, 1e-3))
            dl = f32((target / float(rdv) - float(A[-end])) / float(B[-end]))
        else:
            dl = f32(rng.uniform(-60.0, 60.0))
        yield A, B, dl, rdv


def test_marked_records_have_every_bin_in_the_far_wing():
    rng = np.random.default_rng(3)
    n_marked = 0
    for A, B, dl, rdv in _cases(rng, 20000):
        if marked(A, B, dl, rdv):
            n_marked += 1
            assert all_far(A, B, dl, rdv)
    assert n_marked > 1000


def test_marking_below_the_flush_point_goes_wrong():
    # the planted mistake: a threshold of 11, below sqrt(128) = 11.31, marks
    # records whose bins still have a nonzero profile
    rng = np.random.default_rng(4)
    bad = 0
    for A, B, dl, rdv in _cases(rng, 20000):
        dl = f32(dl * f32(11.0 / 12.1))  # move the boundary cases to |a| = 11
        if marked(A, B, dl, rdv, thr=11.0) and not all_far(A, B, dl, rdv):
            bad += 1
    assert bad > 0
