// k_rays.cu -- hierarchical, mesh-adaptive HEALPix ray sets (Section 2.1.3,
// Eq. 4, Fig. 1).
//
// Fixed level: every point gets all antipodal pairs of that level.
// Adaptive (one CTA per point): the directions from the point to the global
// sample of points are counted per pixel of the finest level (vec2pix in
// double precision, explicitly rounded operations); coarser counts come from
// nested downgrading (children 4p..4p+3 of pixel p).  Starting from all pairs
// of l_min, each level ranks the candidate pairs by the count of both members
// (ties to the smaller pixel index), keeps the bottom half as rays of that
// level and refines the top half into their four child pairs; at l_max every
// candidate is a ray.  The pairs are written sorted ascending.
#include "mgx_internal.cuh"

namespace mgx {

namespace {

constexpr double kTwoOverPi = 0.636619772367581343075535053490057448;

__device__ __forceinline__ int64_t spread2(int64_t v) {
    int64_t out = 0;
#pragma unroll
    for (int b = 0; b < 16; ++b) out |= ((v >> b) & 1) << (2 * b);
    return out;
}

// nested pixel of level l containing direction (dx, dy, dz); HEALPix zones of
// Gorski et al. (2005): equatorial |z| <= 2/3, polar caps otherwise
__device__ int32_t vec2pix_nest(int l, double dx, double dy, double dz) {
    const int64_t ns = int64_t(1) << l;
    const double len = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
    const double z = __ddiv_rn(dz, len);
    const double za = fabs(z);
    double t = __dmul_rn(atan2(dy, dx), kTwoOverPi);
    if (t < 0.0) t = __dadd_rn(t, 4.0);
    if (t >= 4.0) t = __dsub_rn(t, 4.0);
    int64_t face, x, y;
    if (za <= 2.0 / 3.0) {
        const double c1 = __dmul_rn(double(ns), __dadd_rn(0.5, t));
        const double c2 = __dmul_rn(double(ns), __dmul_rn(0.75, z));
        const int64_t asc = int64_t(__dsub_rn(c1, c2));
        const int64_t dsc = int64_t(__dadd_rn(c1, c2));
        const int64_t fa = asc >> l, fd = dsc >> l;
        face = (fa == fd) ? (fa | 4) : (fa < fd ? fa : fd + 8);
        x = dsc & (ns - 1);
        y = ns - 1 - (asc & (ns - 1));
    } else {
        int64_t q = int64_t(t);
        if (q > 3) q = 3;
        const double tp = __dsub_rn(t, double(q));
        const double w = __dmul_rn(double(ns), __dsqrt_rn(__dmul_rn(3.0, __dsub_rn(1.0, za))));
        int64_t a = int64_t(__dmul_rn(tp, w));
        int64_t b = int64_t(__dmul_rn(__dsub_rn(1.0, tp), w));
        if (a > ns - 1) a = ns - 1;
        if (b > ns - 1) b = ns - 1;
        if (z >= 0.0) {
            face = q;
            x = ns - 1 - b;
            y = ns - 1 - a;
        } else {
            face = q + 8;
            x = a;
            y = b;
        }
    }
    return int32_t((face << (2 * l)) + spread2(x) + 2 * spread2(y));
}

// The same pixel in single precision, certified: returns false when a
// rounding could move any of the decisions (the zone test, the face and the
// in-face indices, all truncations of non-negative arguments) away from those
// of vec2pix_nest above, which the caller then takes.  The translation unit is
// compiled without contraction, so each operation rounds once (u = 2^-24):
//   z = c / |v| within 7u |z| of the double z (inputs, sum of squares, sqrt, division);
//   phi = atan2f(b, a) within kAtanErr of the double angle (3 ulp documented;
//     the inputs' rounding adds at most u);
//   t = phi 2/pi (+4) within et = 0.64 kAtanErr + 12u (and not within et of 0,
//     where the wrap into [0, 4) jumps);
//   equatorial arguments ns (0.5 + t) -+ ns 0.75 z within ns (et + 0.75 ez + 11u);
//   polar w = ns sqrt(3 (1 - |z|)) within w ((ez + 2u) / (2 (1 - |z|)) + 2u), and
//   a, b = trunc(tp w), trunc((1 - tp) w) within et w + ew + 2u w.
// The double path's own rounding (about 1e-15) is inside these margins.
constexpr float kAtanErr = 9.5367431640625e-7f;  // 2^-20 rad

__device__ __forceinline__ bool trunc_certain(float v, float e, int64_t &k) {
    // trunc of the double value equals trunc(v) when v is farther than e from
    // every integer other than 0 (trunc maps (-1, 1) to 0)
    if (!(v > -1.0f + e)) return false;
    if (v < 1.0f - e) {
        k = 0;
        return true;
    }
    const float f = floorf(v);
    if (v - f < e || f + 1.0f - v < e) return false;
    k = int64_t(f);
    return true;
}

__device__ bool vec2pix_nest_f(int l, float a, float b, float c, int32_t &pix) {
    constexpr float kU = 5.9604644775390625e-8f;  // 2^-24
    const int64_t ns = int64_t(1) << l;
    const float fns = float(ns);
    const float len = sqrtf(a * a + b * b + c * c);
    const float z = c / len;
    const float za = fabsf(z);
    const float ez = 7.0f * kU * za + 1e-30f;
    float t = atan2f(b, a) * 0.636619772367581343f;
    const float et = 0.64f * kAtanErr + 12.0f * kU;
    // the wrap into [0, 4) is discontinuous at t = 0: both precisions must be on the same side
    if (fabsf(t) < et) return false;
    if (t < 0.0f) t = t + 4.0f;
    if (t >= 4.0f) t = t - 4.0f;
    constexpr float kTwoThirds = 0.666666666666666667f;
    int64_t face, x, y;
    if (za <= kTwoThirds - ez - 2.0f * kU) {
        const float c1 = fns * (0.5f + t), c2 = fns * (0.75f * z);
        const float eA = fns * (et + 0.75f * ez + 11.0f * kU);
        int64_t asc, dsc;
        if (!trunc_certain(c1 - c2, eA, asc) || !trunc_certain(c1 + c2, eA, dsc)) return false;
        const int64_t fa = asc >> l, fd = dsc >> l;
        face = (fa == fd) ? (fa | 4) : (fa < fd ? fa : fd + 8);
        x = dsc & (ns - 1);
        y = ns - 1 - (asc & (ns - 1));
    } else if (za > kTwoThirds + ez + 2.0f * kU) {
        int64_t q;
        if (t > 3.0f + et) q = 3;
        else if (!trunc_certain(t, et, q)) return false;
        const float tp = t - float(q);
        const float om = 1.0f - za;
        const float w = fns * sqrtf(3.0f * om);
        const float ew = w * ((ez + 2.0f * kU) / (2.0f * om) + 2.0f * kU);
        if (!(ew < 0.25f)) return false;  // next to the pole
        int64_t ia, ib;
        if (!trunc_certain(tp * w, et * w + ew + 2.0f * kU * w, ia)) return false;
        if (!trunc_certain((1.0f - tp) * w, et * w + ew + 2.0f * kU * w, ib)) return false;
        if (ia > ns - 1) ia = ns - 1;
        if (ib > ns - 1) ib = ns - 1;
        if (z >= 0.0f) {
            face = q;
            x = ns - 1 - ib;
            y = ns - 1 - ia;
        } else {
            face = q + 8;
            x = ia;
            y = ib;
        }
    } else {
        return false;  // at the zone boundary
    }
    pix = int32_t((face << (2 * l)) + spread2(x) + 2 * spread2(y));
    return true;
}

// atan2f as the single-precision ray-set screen evaluates it (for the tests of kAtanErr).
__global__ void k_eval_atan2(const float *__restrict__ x, int64_t n, float *__restrict__ y) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        y[i] = atan2f(x[n + i], x[i]);
}

__global__ void k_rays_fixed(int32_t n, int32_t level, int32_t npairs, const uint32_t *__restrict__ pairs,
                             uint32_t *__restrict__ rays) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= int64_t(n) * npairs) return;
    rays[i] = (uint32_t(level) << 28) | pairs[i % npairs];
}

__global__ void __launch_bounds__(256)
k_rays_adaptive(DevMesh m, int32_t lmin, int32_t lmax, int32_t npairs, int64_t n_sample,
                const int32_t *__restrict__ sample, const int32_t *__restrict__ anti,
                const uint32_t *__restrict__ pairs_lmin, int32_t n_pairs_lmin,
                uint32_t *__restrict__ rays, int *status) {
    extern __shared__ uint32_t sm[];
    const int32_t o = blockIdx.x;
    const int tid = threadIdx.x, nt = blockDim.x;
    // shared layout: histograms of levels lmin..lmax, then candidate buffers
    uint32_t *hist[MGX_MAX_ADAPT_LEVEL + 1];
    int64_t off = 0;
    for (int l = lmax; l >= lmin; --l) {
        hist[l] = sm + off;
        off += int64_t(12) << (2 * l);
    }
    const int32_t cmax = int32_t((int64_t(12) << (2 * lmax)) / 2);
    uint32_t *cand = sm + off;
    uint32_t *next = cand + cmax;
    uint32_t *score = next + cmax;
    uint32_t *out = score + cmax;
    __shared__ int32_t nout;

    const int32_t nfine = int32_t(int64_t(12) << (2 * lmax));
    for (int32_t i = tid; i < nfine; i += nt) hist[lmax][i] = 0;
    if (tid == 0) nout = 0;
    __syncthreads();
    const double xo = m.x[o], yo = m.y[o], zo = m.z[o];
    for (int64_t s = tid; s < n_sample; s += nt) {
        const int32_t j = sample[s];
        if (j == o || j < 0 || j >= m.n) continue;
        const double dx = __dsub_rn(m.x[j], xo), dy = __dsub_rn(m.y[j], yo), dz = __dsub_rn(m.z[j], zo);
        if (dx == 0.0 && dy == 0.0 && dz == 0.0) continue;
        // single precision when the screen certifies the pixel, else the double path
        int32_t pix;
        if (!vec2pix_nest_f(lmax, __double2float_rn(dx), __double2float_rn(dy), __double2float_rn(dz), pix))
            pix = vec2pix_nest(lmax, dx, dy, dz);
        atomicAdd(&hist[lmax][pix], 1u);
    }
    __syncthreads();
    for (int l = lmax - 1; l >= lmin; --l) {
        const int32_t np = int32_t(int64_t(12) << (2 * l));
        for (int32_t q = tid; q < np; q += nt)
            hist[l][q] = hist[l + 1][4 * q] + hist[l + 1][4 * q + 1] + hist[l + 1][4 * q + 2] +
                         hist[l + 1][4 * q + 3];
        __syncthreads();
    }
    int32_t ncand = n_pairs_lmin;
    for (int32_t c = tid; c < ncand; c += nt) cand[c] = pairs_lmin[c];
    __syncthreads();
    for (int l = lmin; l < lmax; ++l) {
        const int32_t *al = anti + level_offset(l);
        const int32_t *an = anti + level_offset(l + 1);
        for (int32_t c = tid; c < ncand; c += nt) score[c] = hist[l][cand[c]] + hist[l][al[cand[c]]];
        __syncthreads();
        const int32_t half = ncand / 2;
        for (int32_t c = tid; c < ncand; c += nt) {
            const uint32_t sc = score[c], pc = cand[c];
            int32_t rank = 0;
            for (int32_t c2 = 0; c2 < ncand; ++c2)
                rank += (score[c2] > sc) || (score[c2] == sc && cand[c2] < pc);
            if (rank >= half) {
                const int32_t slot = atomicAdd(&nout, 1);
                if (slot < cmax) out[slot] = (uint32_t(l) << 28) | pc;
            } else {
                for (int ch = 0; ch < 4; ++ch) {
                    const uint32_t cp = 4 * pc + ch, ap = uint32_t(an[cp]);
                    next[4 * rank + ch] = cp < ap ? cp : ap;
                }
            }
        }
        __syncthreads();
        ncand = 4 * half;
        for (int32_t c = tid; c < ncand; c += nt) cand[c] = next[c];
        __syncthreads();
    }
    for (int32_t c = tid; c < ncand; c += nt) {
        const int32_t slot = atomicAdd(&nout, 1);
        if (slot < cmax) out[slot] = (uint32_t(lmax) << 28) | cand[c];
    }
    __syncthreads();
    if (nout != npairs) {
        if (tid == 0) dev_fail(status, kDevBadInput);
        return;
    }
    for (int32_t i = tid; i < npairs; i += nt) {
        const uint32_t v = out[i];
        int32_t rank = 0;
        for (int32_t j = 0; j < npairs; ++j) rank += out[j] < v;
        rays[int64_t(o) * npairs + rank] = v;
    }
}

}  // namespace

void launch_eval_atan2(const float *x, int64_t n, float *y, cudaStream_t st) {
    if (n <= 0) return;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_eval_atan2<<<unsigned(blocks), 256, 0, st>>>(x, n, y);
}

float atan2_bound() { return kAtanErr; }

void launch_rays_fixed(int32_t n, int32_t level, int32_t npairs, const uint32_t *pairs, uint32_t *rays,
                       cudaStream_t st) {
    const int64_t tot = int64_t(n) * npairs;
    const int tb = 256;
    k_rays_fixed<<<unsigned((tot + tb - 1) / tb), tb, 0, st>>>(n, level, npairs, pairs, rays);
}

void launch_rays_adaptive(const DevMesh &m, int32_t lmin, int32_t lmax, int32_t npairs, int64_t n_sample,
                          const int32_t *sample, const int32_t *anti, const uint32_t *pairs_lmin,
                          int32_t n_pairs_lmin, uint32_t *rays, int *status, cudaStream_t st) {
    int64_t words = 0;
    for (int l = lmin; l <= lmax; ++l) words += int64_t(12) << (2 * l);
    const int64_t cmax = (int64_t(12) << (2 * lmax)) / 2;
    words += 4 * cmax;
    const size_t smem = size_t(words) * sizeof(uint32_t);
    cudaFuncSetAttribute(k_rays_adaptive, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    k_rays_adaptive<<<unsigned(m.n), 256, smem, st>>>(m, lmin, lmax, npairs, n_sample, sample, anti,
                                                      pairs_lmin, n_pairs_lmin, rays, status);
}

}  // namespace mgx
