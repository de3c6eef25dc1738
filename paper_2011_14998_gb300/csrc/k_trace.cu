// k_trace.cu -- long-characteristic tracer (Section 2.1, Fig. 2).
//
// One thread per half-ray.  From the current point c the next point is the
// neighbour of c that lies strictly further along the ray (Z_n > Z_c with
// Z = (x_n - x_o).d) and closest to it (smallest |(x_n - x_o) - Z d|^2), ties to
// the smaller index; the half-ray ends when c has no such neighbour.  Every
// product and sum is an explicitly rounded double operation in a fixed order,
// so the traced point lists and distances are bit-reproducible.
//
// Two passes share the walk: the count pass stores the half-ray lengths, which
// are prefix-summed into arena offsets; the emit pass writes point ids and
// distances at those offsets.
#include "mgx_internal.cuh"

namespace mgx {

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
    const double xo = m.x[o], yo = m.y[o], zo = m.z[o];
    int64_t w = 0;
    int32_t expect = 0;
    if (EMIT) {
        w = offs[h] - base;
        expect = int32_t(offs[h + 1] - offs[h]);
    }
    int32_t c = o, k = 0;
    double zc = 0.0;
    for (;;) {
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
        if (best < 0) break;
        if (EMIT) {
            if (k >= expect) {
                dev_fail(status, kDevTraceMismatch);
                return;
            }
            idx_out[w + k] = best;
            Z_out[w + k] = zbest;
            if (delta_out) {
                const double ux = __dsub_rn(m.vx[best], m.vx[o]);
                const double uy = __dsub_rn(m.vy[best], m.vy[o]);
                const double uz = __dsub_rn(m.vz[best], m.vz[o]);
                delta_out[w + k] =
                    __dadd_rn(__dadd_rn(__dmul_rn(ux, d0), __dmul_rn(uy, d1)), __dmul_rn(uz, d2));
            }
        }
        ++k;
        c = best;
        zc = zbest;
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
