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
// rate, so each step first screens the neighbours in single precision:
// positions are held as float hi + lo pairs (x = hi + lo to 2^-48 |x|), the
// offset x_n - x_o, Z and q are formed in float, and each gets a rigorous
// bound on its distance from the double-precision value (derived from the
// unit roundoff u = 2^-24; three to four times the worst case):
//     |Z32 - Z| <= eZ = 16 u S + g0,           S = |dx| + |dy| + |dz|,
//     |q32 - q| <= eq = 256 u S^2 + 32 g0 S,   g0 = 32 u^2 max_n |x_n|_1.
// A neighbour is surely (not) forward when Z32 - Z_c clears eZ plus the
// rounding of Z_c; the step is decided in single precision when one surely
// forward neighbour's interval [q32 - eq, q32 + eq] lies strictly below the
// intervals of every other candidate.  Otherwise (near-ties, exact ties of
// lattice meshes, ambiguous forward tests) the step is redone exactly in
// double precision.  The winner's Z is always computed exactly in double.
//
// Two passes share the walk: the count pass stores the half-ray lengths, which
// are prefix-summed into arena offsets; the emit pass writes point ids and
// distances at those offsets.
#include "mgx_internal.cuh"

namespace mgx {

namespace {

constexpr float kU = 5.9604644775390625e-8f;  // 2^-24

struct Step {
    int32_t next;  // -1: the half-ray ends
    double Z;
};

// The defining rule, exactly in double precision.
__device__ Step step_exact(const DevMesh &m, int32_t c, double xo, double yo, double zo, double d0, double d1,
                           double d2, double zc) {
    int32_t best = -1;
    double qbest = 0.0, zbest = 0.0;
    const int32_t e1 = m.off[c + 1];
    for (int32_t e = m.off[c]; e < e1; ++e) {
        const int32_t nb = __ldg(m.nbr + e);
        const double dx = __dsub_rn(__ldg(m.x + nb), xo);
        const double dy = __dsub_rn(__ldg(m.y + nb), yo);
        const double dz = __dsub_rn(__ldg(m.z + nb), zo);
        const double zn = __dadd_rn(__dadd_rn(__dmul_rn(dx, d0), __dmul_rn(dy, d1)), __dmul_rn(dz, d2));
        if (!(zn > zc)) continue;
        const double ex = __dsub_rn(dx, __dmul_rn(zn, d0));
        const double ey = __dsub_rn(dy, __dmul_rn(zn, d1));
        const double ez = __dsub_rn(dz, __dmul_rn(zn, d2));
        const double q = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
        if (best < 0 || q < qbest || (q == qbest && nb < best)) {
            best = nb;
            qbest = q;
            zbest = zn;
        }
    }
    return Step{best, zbest};
}

// Single-precision screen; falls back to step_exact when it cannot decide.
__device__ __forceinline__ Step step_filtered(const DevMesh &m, int32_t c, float4 oh, float4 ol, double xo,
                                              double yo, double zo, double d0, double d1, double d2, float f0,
                                              float f1, float f2, double zc) {
    const float zc32 = __double2float_rn(zc);
    const float zcm = 4.0f * kU * fabsf(zc32);
    int32_t best = -1, lo1_id = -1;
    float hib = INFINITY, lo1 = INFINITY, lo2 = INFINITY;
    const int32_t e1 = m.off[c + 1];
    for (int32_t e = m.off[c]; e < e1; ++e) {
        const int32_t nb = __ldg(m.nbr + e);
        const float4 h = __ldg(m.phi + nb), l = __ldg(m.plo + nb);
        const float dx = (h.x - oh.x) + (l.x - ol.x);
        const float dy = (h.y - oh.y) + (l.y - ol.y);
        const float dz = (h.z - oh.z) + (l.z - ol.z);
        const float S = fabsf(dx) + fabsf(dy) + fabsf(dz);
        const float z32 = fmaf(dz, f2, fmaf(dy, f1, dx * f0));
        const float diff = z32 - zc32;
        const float E = fmaf(16.0f * kU, S, m.g0) + zcm + 4.0f * kU * fabsf(diff);
        if (diff < -E) continue;  // surely not forward
        const float ex = fmaf(-z32, f0, dx), ey = fmaf(-z32, f1, dy), ez = fmaf(-z32, f2, dz);
        const float q = fmaf(ez, ez, fmaf(ey, ey, ex * ex));
        const float eq = fmaf(256.0f * kU * S, S, 32.0f * m.g0 * S) + 1e-37f;  // floor covers subnormals
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
        }
    }
    if (lo1_id < 0) return Step{-1, 0.0};  // no neighbour can be forward
    if (best >= 0 && best == lo1_id && hib < lo2) {
        const double dx = __dsub_rn(__ldg(m.x + best), xo);
        const double dy = __dsub_rn(__ldg(m.y + best), yo);
        const double dz = __dsub_rn(__ldg(m.z + best), zo);
        return Step{best, __dadd_rn(__dadd_rn(__dmul_rn(dx, d0), __dmul_rn(dy, d1)), __dmul_rn(dz, d2))};
    }
    return step_exact(m, c, xo, yo, zo, d0, d1, d2, zc);
}

template <bool EMIT>
__global__ void __launch_bounds__(128)
k_trace(DevMesh m, DevRays R, int32_t o_begin, int64_t n_half, int64_t *__restrict__ lens,
        const int64_t *__restrict__ offs, int64_t base, int32_t *__restrict__ idx_out,
        double *__restrict__ Z_out, double *__restrict__ delta_out, int *status) {
    const int64_t h = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (h >= n_half) return;
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
    const double xo = m.x[o], yo = m.y[o], zo = m.z[o];
    const float4 oh = m.phi[o], ol = m.plo[o];
    int64_t w = 0;
    int32_t expect = 0;
    if (EMIT) {
        w = offs[h] - base;
        expect = int32_t(offs[h + 1] - offs[h]);
    }
    int32_t c = o, k = 0;
    double zc = 0.0;
    for (;;) {
        const Step s = step_filtered(m, c, oh, ol, xo, yo, zo, d0, d1, d2, f0, f1, f2, zc);
        if (s.next < 0) break;
        if (EMIT) {
            if (k >= expect) {
                dev_fail(status, kDevTraceMismatch);
                return;
            }
            idx_out[w + k] = s.next;
            Z_out[w + k] = s.Z;
            if (delta_out) {
                const double ux = __dsub_rn(m.vx[s.next], m.vx[o]);
                const double uy = __dsub_rn(m.vy[s.next], m.vy[o]);
                const double uz = __dsub_rn(m.vz[s.next], m.vz[o]);
                delta_out[w + k] =
                    __dadd_rn(__dadd_rn(__dmul_rn(ux, d0), __dmul_rn(uy, d1)), __dmul_rn(uz, d2));
            }
        }
        ++k;
        c = s.next;
        zc = s.Z;
        if (k > m.n) {  // Z increases strictly, so this cannot happen
            dev_fail(status, kDevTraceGuard);
            break;
        }
    }
    if (EMIT) {
        if (k != expect) dev_fail(status, kDevTraceMismatch);
    } else {
        lens[h] = k;
    }
}

}  // namespace

void launch_trace_count(const DevMesh &m, const DevRays &R, int32_t o_begin, int32_t o_end,
                        int64_t *lens, int *status, cudaStream_t st) {
    const int64_t n_half = int64_t(o_end - o_begin) * R.npairs * 2;
    if (n_half == 0) return;
    const int tb = 128;
    k_trace<false><<<unsigned((n_half + tb - 1) / tb), tb, 0, st>>>(m, R, o_begin, n_half, lens, nullptr,
                                                                    0, nullptr, nullptr, nullptr, status);
}

void launch_trace_emit(const DevMesh &m, const DevRays &R, int32_t o_begin, int32_t o_end,
                       const int64_t *offs, int64_t base, int32_t *idx, double *Z, double *delta,
                       int *status, cudaStream_t st) {
    const int64_t n_half = int64_t(o_end - o_begin) * R.npairs * 2;
    if (n_half == 0) return;
    const int tb = 128;
    k_trace<true><<<unsigned((n_half + tb - 1) / tb), tb, 0, st>>>(m, R, o_begin, n_half, nullptr, offs,
                                                                   base, idx, Z, delta, status);
}

}  // namespace mgx
