// k_analytic.cu -- element-size field of an analytic model (Section 2.2.1, Eq. 5).
//
// On a regular Cartesian background mesh of spacing h with the tracer f > 0 at
// its points (index (i ny + j) nz + k):
//   Gf = max_n n.grad f / f = ||grad f|| / f,
// the gradient by central differences (first differences on the faces, 0 along
// an axis with a single point); the desired element size maps [max Gf, min Gf]
// linearly onto [ell_min, ell_max] (all ell_max when Gf is constant).  In place
// of Gmsh, the mesh is the background mesh (point density h^-3) thinned to the
// density ell^-3: point q is kept when u_q < (h / ell_q)^3, u_q the SplitMix64
// uniform of (seed, q).  Every operation is explicitly rounded, so Gf, ell and the kept set
// are reproducible bit for bit.
#include "mgx_internal.cuh"

namespace mgx {

namespace {

__device__ __forceinline__ double axis_diff(const double *__restrict__ f, int64_t q, int64_t stride, int32_t pos,
                                            int32_t n, double h) {
    if (n < 2) return 0.0;
    if (pos == 0) return __ddiv_rn(__dsub_rn(f[q + stride], f[q]), h);
    if (pos == n - 1) return __ddiv_rn(__dsub_rn(f[q], f[q - stride]), h);
    return __ddiv_rn(__dsub_rn(f[q + stride], f[q - stride]), __dmul_rn(2.0, h));
}

__global__ void k_size_field(int32_t nx, int32_t ny, int32_t nz, const double *__restrict__ f, double h,
                             double *__restrict__ Gf, unsigned long long *__restrict__ mm) {
    const int64_t n = int64_t(nx) * ny * nz;
    unsigned long long lo = ~0ull, hi = 0ull;
    for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < n; q += int64_t(gridDim.x) * blockDim.x) {
        const int32_t k = int32_t(q % nz);
        const int32_t j = int32_t((q / nz) % ny);
        const int32_t i = int32_t(q / (int64_t(ny) * nz));
        const double gx = axis_diff(f, q, int64_t(ny) * nz, i, nx, h);
        const double gy = axis_diff(f, q, nz, j, ny, h);
        const double gz = axis_diff(f, q, 1, k, nz, h);
        const double s = __dadd_rn(__dadd_rn(__dmul_rn(gx, gx), __dmul_rn(gy, gy)), __dmul_rn(gz, gz));
        const double g = __ddiv_rn(__dsqrt_rn(s), f[q]);
        Gf[q] = g;
        const unsigned long long b = (unsigned long long)__double_as_longlong(g);  // g >= 0
        lo = b < lo ? b : lo;
        hi = b > hi ? b : hi;
    }
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) {
        const unsigned long long l2 = __shfl_down_sync(0xffffffffu, lo, sh);
        const unsigned long long h2 = __shfl_down_sync(0xffffffffu, hi, sh);
        lo = l2 < lo ? l2 : lo;
        hi = h2 > hi ? h2 : hi;
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(mm, lo);
        atomicMax(mm + 1, hi);
    }
}

__global__ void k_size_map(int64_t n, const double *__restrict__ Gf, const unsigned long long *__restrict__ mm,
                           double h, double ell_min, double ell_max, uint64_t seed, double *__restrict__ ell,
                           uint8_t *__restrict__ keep, unsigned long long *__restrict__ kept) {
    const double gmin = __longlong_as_double((long long)mm[0]), gmax = __longlong_as_double((long long)mm[1]);
    unsigned long long cnt = 0;
    for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < n; q += int64_t(gridDim.x) * blockDim.x) {
        const double e = gmax > gmin ? __dsub_rn(ell_max, __ddiv_rn(__dmul_rn(__dsub_rn(Gf[q], gmin),
                                                                              __dsub_rn(ell_max, ell_min)),
                                                                    __dsub_rn(gmax, gmin)))
                                     : ell_max;
        const double r = __ddiv_rn(h, e);
        const uint8_t kq = splitmix_uniform(seed, q) < __dmul_rn(__dmul_rn(r, r), r) ? 1 : 0;
        if (ell) ell[q] = e;
        keep[q] = kq;
        cnt += kq;
    }
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, sh);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(kept, cnt);
}

unsigned grid_for(int64_t n) {
    int64_t g = (n + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    return unsigned(g < 1 ? 1 : g);
}

}  // namespace

void launch_size_field(int32_t nx, int32_t ny, int32_t nz, const double *f, double h, double *Gf,
                       unsigned long long *mm, cudaStream_t st) {
    const int64_t n = int64_t(nx) * ny * nz;
    k_size_field<<<grid_for(n), 256, 0, st>>>(nx, ny, nz, f, h, Gf, mm);
}

void launch_size_map(int64_t n, const double *Gf, const unsigned long long *mm, double h, double ell_min,
                     double ell_max, uint64_t seed, double *ell, uint8_t *keep, unsigned long long *kept,
                     cudaStream_t st) {
    k_size_map<<<grid_for(n), 256, 0, st>>>(n, Gf, mm, h, ell_min, ell_max, seed, ell, keep, kept);
}

}  // namespace mgx
