// k_trace.cu -- long-characteristic tracer (Section 2.1, Fig. 2).
//
// One thread per half-ray.  From the current point c the next point is the
// neighbour of c that lies strictly further along the ray (Z_n > Z_c with
// Z = (x_n - x_o).d) and closest to it (smallest q = |(x_n - x_o) - Z d|^2),
// ties to the smaller index; the half-ray ends when c has no such neighbour.
// The decisions are those of the double-precision definition, with every
// product and sum explicitly rounded in a fixed order, so the traced point
// lists and distances are bit-reproducible.
//
// GB300 executes double precision at a small fraction of its single-precision
// rate, so each step first screens the neighbours in single precision: each
// CSR edge carries its neighbour's position rounded to float, the offset
// x_n - x_o, Z and q are formed in float, and each gets a rigorous bound on its
// distance from the double-precision value (derived from the unit roundoff
// u = 2^-24 and the positions' own rounding; see step_screen).
// A neighbour is surely (not) forward when Z32 - Z_c clears eZ plus the
// rounding of Z_c; the step is decided in single precision when one surely
// forward neighbour's interval [q32 - eq, q32 + eq] lies strictly below the
// intervals of every other candidate.  Otherwise (near-ties, exact ties of
// lattice meshes, ambiguous forward tests) the step is redone exactly in
// double precision.  The winner's Z is always computed exactly in double.
//
// The fast path carries the winner's single-precision Z and its error bound
// into the next step's forward test, so it executes no double-precision
// operation at all; the exact Z is formed only on undecided steps (and for
// the inspection output of mgx_trace).
//
// The walk serves three layouts of the traced lists (the solver re-forms each
// point's exact Z from its position, so only point ids are stored):
//   * packed: a count pass stores the half-ray lengths, which are prefix-summed
//     into arena offsets, and an emit pass writes the ids at those offsets;
//   * padded (batched solves): one pass writes the first `pad` ids of each
//     half-ray into a fixed-width row h * pad, stores the full length and its
//     excess over the row, and for a half-ray longer than the row the walk's
//     state after its pad-th point; a tail pass resumes those walks from
//     their states and writes the remaining ids into a packed overflow arena
//     at the prefix sums of the excesses.  Every step is walked once by the
//     padded pass and the tail steps once more, so the lists cost about one
//     walk instead of two.
#include "mgx_internal.cuh"

namespace mgx {

namespace {

constexpr float kU = 5.9604644775390625e-8f;  // 2^-24

struct Step {
    int32_t next;  // -1: the half-ray ends
    double Z;
};

__device__ __forceinline__ double exact_Z(const DevMesh &m, int32_t c, double xo, double yo, double zo, double d0,
                                          double d1, double d2) {
    const double dx = __dsub_rn(__ldg(m.x + c), xo);
    const double dy = __dsub_rn(__ldg(m.y + c), yo);
    const double dz = __dsub_rn(__ldg(m.z + c), zo);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, d0), __dmul_rn(dy, d1)), __dmul_rn(dz, d2));
}

struct FStep {
    int32_t next;  // -1: the half-ray ends; -2: undecided
    float z32;     // single-precision Z of next; when undecided, H (see step_contenders)
    float ez;      // bound on |z32 - Z(next)|, Z the double-precision value
};

// Single-precision screen of one step over the neighbour records of c (the
// float position of each neighbour stored next to its id, read sequentially).
// zc32 approximates the double Z of the current point within ezc; Xo is
// |x_o|_1 in float.  With hi-only positions the bounds carry the rounding of
// both positions: eZ = 3u (X_n + X_o) + 12u S + g0, eq = 32u (X_n + X_o) S +
// 128u S^2 + 32 g0 S (about 2.5 to 3 times the worst case).  Returns
// next = -2 when it cannot decide.
__device__ __forceinline__ FStep step_screen(const DevMesh &m, int32_t c, float4 oh, float Xo, float f0, float f1,
                                             float f2, float zc32, float ezc) {
    const float zcm = ezc + 4.0f * kU * fabsf(zc32);
    int32_t best = -1, lo1_id = -1;
    float hib = INFINITY, lo1 = INFINITY, lo2 = INFINITY, zb = 0.0f, ezb = 0.0f;
    const int32_t e1 = m.off[c + 1];
    for (int32_t e = m.off[c]; e < e1; ++e) {
        const float4 rec = __ldg(m.nrec + e);
        const int32_t nb = __float_as_int(rec.w);
        const float dx = rec.x - oh.x, dy = rec.y - oh.y, dz = rec.z - oh.z;
        const float S = fabsf(dx) + fabsf(dy) + fabsf(dz);
        const float XS = fabsf(rec.x) + fabsf(rec.y) + fabsf(rec.z) + Xo;
        const float z32 = fmaf(dz, f2, fmaf(dy, f1, dx * f0));
        const float ez = fmaf(3.0f * kU, XS, fmaf(12.0f * kU, S, m.g0));
        const float diff = z32 - zc32;
        const float E = ez + zcm + 4.0f * kU * fabsf(diff);
        if (diff < -E) continue;  // surely not forward
        const float ex = fmaf(-z32, f0, dx), ey = fmaf(-z32, f1, dy), ez2 = fmaf(-z32, f2, dz);
        const float q = fmaf(ez2, ez2, fmaf(ey, ey, ex * ex));
        const float eq = fmaf(fmaf(32.0f * kU, XS, 128.0f * kU * S), S, fmaf(32.0f * m.g0, S, 1e-37f));
        const float lo = q - eq, hi = q + eq;
        if (lo < lo1) {
            lo2 = lo1;
            lo1 = lo;
            lo1_id = nb;
        } else if (lo < lo2) {
            lo2 = lo;
        }
        if (diff > E && hi < hib) {  // surely forward
            hib = hi;
            best = nb;
            zb = z32;
            ezb = ez;
        }
    }
    if (lo1_id < 0) return FStep{-1, 0.0f, 0.0f};  // no neighbour can be forward
    if (best >= 0 && best == lo1_id && hib < lo2) return FStep{best, zb, ezb};
    return FStep{-2, hib, 0.0f};
}

// An undecided step, exactly: only neighbours that are not surely backward and
// whose interval reaches down to H (the smallest upper bound of a surely
// forward neighbour, or infinity) can be the winner; every other neighbour has
// a strictly larger double-precision q than that surely forward one.  The
// contenders are re-screened (same single-precision values) and decided by
// the defining rule in double precision.
__device__ Step step_contenders(const DevMesh &m, int32_t c, float4 oh, float Xo, float f0, float f1, float f2,
                                float zc32, float ezc, float H, double zc, double xo, double yo, double zo,
                                double d0, double d1, double d2) {
    const float zcm = ezc + 4.0f * kU * fabsf(zc32);
    int32_t best = -1;
    double qbest = 0.0, zbest = 0.0;
    const int32_t e1 = m.off[c + 1];
    for (int32_t e = m.off[c]; e < e1; ++e) {
        const float4 rec = __ldg(m.nrec + e);
        const int32_t nb = __float_as_int(rec.w);
        const float dx = rec.x - oh.x, dy = rec.y - oh.y, dz = rec.z - oh.z;
        const float S = fabsf(dx) + fabsf(dy) + fabsf(dz);
        const float XS = fabsf(rec.x) + fabsf(rec.y) + fabsf(rec.z) + Xo;
        const float z32 = fmaf(dz, f2, fmaf(dy, f1, dx * f0));
        const float ez = fmaf(3.0f * kU, XS, fmaf(12.0f * kU, S, m.g0));
        const float diff = z32 - zc32;
        const float E = ez + zcm + 4.0f * kU * fabsf(diff);
        if (diff < -E) continue;
        const float ex = fmaf(-z32, f0, dx), ey = fmaf(-z32, f1, dy), ez2 = fmaf(-z32, f2, dz);
        const float q = fmaf(ez2, ez2, fmaf(ey, ey, ex * ex));
        const float eq = fmaf(fmaf(32.0f * kU, XS, 128.0f * kU * S), S, fmaf(32.0f * m.g0, S, 1e-37f));
        if (q - eq > H) continue;
        const double ddx = __dsub_rn(__ldg(m.x + nb), xo);
        const double ddy = __dsub_rn(__ldg(m.y + nb), yo);
        const double ddz = __dsub_rn(__ldg(m.z + nb), zo);
        const double zn = __dadd_rn(__dadd_rn(__dmul_rn(ddx, d0), __dmul_rn(ddy, d1)), __dmul_rn(ddz, d2));
        if (!(zn > zc)) continue;
        const double qx = __dsub_rn(ddx, __dmul_rn(zn, d0));
        const double qy = __dsub_rn(ddy, __dmul_rn(zn, d1));
        const double qz = __dsub_rn(ddz, __dmul_rn(zn, d2));
        const double qd = __dadd_rn(__dadd_rn(__dmul_rn(qx, qx), __dmul_rn(qy, qy)), __dmul_rn(qz, qz));
        if (best < 0 || qd < qbest || (qd == qbest && nb < best)) {
            best = nb;
            qbest = qd;
            zbest = zn;
        }
    }
    return Step{best, zbest};
}

// MODE 0: count the points of each half-ray; MODE 1: write their ids;
// MODE 2: write ids, exact double Z and (optionally) projected velocities;
// MODE 3: padded pass (ids k < pad to row h, length to lens[h], excess over
// the row to excess[h], the walk state after entry pad - 1 to resume[h] when
// the half-ray is longer); MODE 4: tail pass (ids k >= pad of the half-rays
// longer than the row, at offs[h] - base + k - pad, resumed from resume[h]).
// Each thread walks half-rays h = tid, tid + T, ... (T = all threads), which
// evens out the very different lengths of the rays a warp's lanes trace.
template <int MODE>
__global__ void __launch_bounds__(128)
k_trace(DevMesh m, DevRays R, int32_t o_begin, int64_t n_half, int64_t *__restrict__ lens,
        const int64_t *__restrict__ offs, int64_t base, int64_t cap, int32_t *__restrict__ idx_out,
        double *__restrict__ Z_out, double *__restrict__ delta_out, int *status,
        unsigned long long *__restrict__ counters, int32_t pad, int64_t *__restrict__ excess,
        int4 *__restrict__ resume) {
    const int64_t T = int64_t(gridDim.x) * blockDim.x;
    unsigned long long n_steps = 0, n_exact = 0;
    for (int64_t h = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; h < n_half; h += T) {
        int64_t expect_len = 0;
        if (MODE == 4) {  // only the half-rays longer than their row
            expect_len = lens[h];
            if (expect_len <= pad) continue;
        }
        const int64_t pr = h >> 1;
        const int32_t o = o_begin + int32_t(pr / R.npairs);
        const uint32_t ray = R.rays[int64_t(o) * R.npairs + (pr % R.npairs)];
        const double *r = R.dir + 3 * (level_offset(int(ray >> 28)) + (ray & 0x0FFFFFFFu));
        double d0 = r[0], d1 = r[1], d2 = r[2];
        if ((h & 1) == 0) {  // backward half: exact negation of the pair direction
            d0 = -d0;
            d1 = -d1;
            d2 = -d2;
        }
        const float f0 = __double2float_rn(d0), f1 = __double2float_rn(d1), f2 = __double2float_rn(d2);
        const float4 oh = m.phi[o];
        const float Xo = fabsf(oh.x) + fabsf(oh.y) + fabsf(oh.z);
        int64_t w = 0;
        int32_t expect = 0;
        if (MODE == 1 || MODE == 2) {
            w = offs[h] - base;
            expect = int32_t(offs[h + 1] - offs[h]);
            if (w < 0 || offs[h + 1] - base > cap) {
                dev_fail(status, kDevArenaOverflow);
                continue;
            }
        } else if (MODE == 3) {
            w = h * int64_t(pad);
        } else if (MODE == 4) {
            w = offs[h] - base - pad;  // entry k >= pad goes to w + k
            expect = int32_t(expect_len);
            if (offs[h] - base < 0 || offs[h + 1] - base > cap || offs[h + 1] - offs[h] != expect_len - pad) {
                dev_fail(status, kDevArenaOverflow);
                continue;
            }
        }
        int32_t c = o, k = 0;
        float zc32 = 0.0f, ezc = 0.0f;  // Z of the origin is exactly 0
        if (MODE == 4) {  // resume after the row's last entry
            const int4 r = resume[h];
            c = r.x;
            zc32 = __int_as_float(r.y);
            ezc = __int_as_float(r.z);
            k = pad;
            if (c < 0 || c >= m.n) {
                dev_fail(status, kDevTraceMismatch);
                continue;
            }
        }
        for (;;) {
            FStep s = step_screen(m, c, oh, Xo, f0, f1, f2, zc32, ezc);
            ++n_steps;
            double zexact = 0.0;
            bool have_exact = false;
            if (s.next == -2) {  // undecided in single precision: its contenders in double
                const double xo = m.x[o], yo = m.y[o], zo = m.z[o];
                const double zc = (c == o) ? 0.0 : exact_Z(m, c, xo, yo, zo, d0, d1, d2);
                const Step x = step_contenders(m, c, oh, Xo, f0, f1, f2, zc32, ezc, s.z32, zc, xo, yo, zo, d0, d1,
                                               d2);
                s.next = x.next;
                zexact = x.Z;
                ++n_exact;
                have_exact = true;
                s.z32 = __double2float_rn(x.Z);
                s.ez = 2.0f * kU * fabsf(s.z32);
            }
            if (s.next < 0) break;
            if (MODE == 3) {
                if (k < pad) idx_out[w + k] = s.next;
            } else if (MODE == 4) {
                if (k >= expect) {
                    dev_fail(status, kDevTraceMismatch);
                    return;
                }
                if (k >= pad) idx_out[w + k] = s.next;
            } else if (MODE > 0) {
                if (k >= expect) {
                    dev_fail(status, kDevTraceMismatch);
                    return;
                }
                idx_out[w + k] = s.next;
                if (MODE == 2) {
                    const double xo = m.x[o], yo = m.y[o], zo = m.z[o];
                    Z_out[w + k] = have_exact ? zexact : exact_Z(m, s.next, xo, yo, zo, d0, d1, d2);
                    if (delta_out) {
                        const double ux = __dsub_rn(m.vx[s.next], m.vx[o]);
                        const double uy = __dsub_rn(m.vy[s.next], m.vy[o]);
                        const double uz = __dsub_rn(m.vz[s.next], m.vz[o]);
                        delta_out[w + k] =
                            __dadd_rn(__dadd_rn(__dmul_rn(ux, d0), __dmul_rn(uy, d1)), __dmul_rn(uz, d2));
                    }
                }
            }
            ++k;
            c = s.next;
            zc32 = s.z32;
            ezc = s.ez;
            if (MODE == 3 && k == pad) resume[h] = make_int4(c, __float_as_int(zc32), __float_as_int(ezc), 0);
            if (k > m.n) {  // Z increases strictly, so this cannot happen
                dev_fail(status, kDevTraceGuard);
                break;
            }
        }
        if (MODE == 0) {
            lens[h] = k;
        } else if (MODE == 3) {
            lens[h] = k;
            excess[h] = k > pad ? k - pad : 0;
        } else if (k != expect) {
            dev_fail(status, kDevTraceMismatch);
        }
    }
    if (counters) {
        atomicAdd(counters + 2, n_steps);
        atomicAdd(counters + 3, n_exact);
    }
}

unsigned trace_grid(int64_t n_half) {
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n_half + 127) / 128;
    const int64_t cap = int64_t(sms) * 8;  // 8 CTAs of 128 threads per SM
    return unsigned(want < cap ? want : cap);
}

}  // namespace

void launch_trace_count(const DevMesh &m, const DevRays &R, int32_t o_begin, int32_t o_end,
                        int64_t *lens, int *status, unsigned long long *counters, cudaStream_t st) {
    const int64_t n_half = int64_t(o_end - o_begin) * R.npairs * 2;
    if (n_half == 0) return;
    k_trace<0><<<trace_grid(n_half), 128, 0, st>>>(m, R, o_begin, n_half, lens, nullptr, 0, 0, nullptr, nullptr,
                                                  nullptr, status, counters, 0, nullptr, nullptr);
}

void launch_trace_emit(const DevMesh &m, const DevRays &R, int32_t o_begin, int32_t o_end,
                       const int64_t *offs, int64_t base, int64_t cap, int32_t *idx, double *Z, double *delta,
                       int *status, cudaStream_t st) {
    const int64_t n_half = int64_t(o_end - o_begin) * R.npairs * 2;
    if (n_half == 0) return;
    if (Z) {
        k_trace<2><<<trace_grid(n_half), 128, 0, st>>>(m, R, o_begin, n_half, nullptr, offs, base, cap, idx, Z,
                                                      delta, status, nullptr, 0, nullptr, nullptr);
    } else {
        k_trace<1><<<trace_grid(n_half), 128, 0, st>>>(m, R, o_begin, n_half, nullptr, offs, base, cap, idx,
                                                      nullptr, nullptr, status, nullptr, 0, nullptr, nullptr);
    }
}

void launch_trace_pad(const DevMesh &m, const DevRays &R, int32_t o_begin, int32_t o_end, int32_t pad,
                      int64_t *lens, int64_t *excess, int4 *resume, int32_t *rows, int *status,
                      unsigned long long *counters, cudaStream_t st) {
    const int64_t n_half = int64_t(o_end - o_begin) * R.npairs * 2;
    if (n_half == 0) return;
    k_trace<3><<<trace_grid(n_half), 128, 0, st>>>(m, R, o_begin, n_half, lens, nullptr, 0, 0, rows, nullptr,
                                                  nullptr, status, counters, pad, excess, resume);
}

void launch_trace_tail(const DevMesh &m, const DevRays &R, int32_t o_begin, int32_t o_end, int32_t pad,
                       const int64_t *lens, const int4 *resume, const int64_t *offs, int64_t base, int64_t cap,
                       int32_t *tail, int *status, cudaStream_t st) {
    const int64_t n_half = int64_t(o_end - o_begin) * R.npairs * 2;
    if (n_half == 0) return;
    k_trace<4><<<trace_grid(n_half), 128, 0, st>>>(m, R, o_begin, n_half, const_cast<int64_t *>(lens), offs, base,
                                                  cap, tail, nullptr, nullptr, status, nullptr, pad, nullptr,
                                                  const_cast<int4 *>(resume));
}

}  // namespace mgx
