// k_thin.cu -- thinning with keep-probabilities weighted by a score (the
// learned reduction's prediction), in the spirit of the random thinning that
// replaces re-meshing (Section 2.2.2): point i is kept when
//   u_i < min(1, c w_i),   w_i = 10^(alpha y_i),
// y_i the predicted log10 J error if i is dropped, u_i the SplitMix64 uniform
// of (seed, i), and c the scale at which the expected kept count
// sum_i min(1, c w_i) equals the target (found by bisection on log2 c).  Unlike
// keeping the top-ranked points, every region keeps some points.
#include "mgx_internal.cuh"

namespace mgx {

namespace {

__global__ void k_thin_weights(const float *__restrict__ y, int64_t n, float alpha, float *__restrict__ w) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    float e = alpha * y[i] * 3.3219280948873622f;  // log2(10)
    e = fminf(fmaxf(e, -100.0f), 100.0f);
    w[i] = exp2f(e);
}

__global__ void k_thin_expected(const float *__restrict__ w, int64_t n, double c, double *__restrict__ sum) {
    double acc = 0.0;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const double p = c * double(w[i]);
        acc += p < 1.0 ? p : 1.0;
    }
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, sh);
    if ((threadIdx.x & 31) == 0) atomicAdd(sum, acc);
}

__global__ void k_thin_mark(const float *__restrict__ w, int64_t n, double c, uint64_t seed,
                            uint8_t *__restrict__ keep, unsigned long long *__restrict__ kept) {
    unsigned long long cnt = 0;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const double p = __dmul_rn(c, double(w[i]));
        const uint8_t k = splitmix_uniform(seed, i) < (p < 1.0 ? p : 1.0) ? 1 : 0;
        keep[i] = k;
        cnt += k;
    }
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, sh);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(kept, cnt);
}

unsigned thin_grid(int64_t n) {
    int64_t g = (n + 255) / 256;
    if (g > 152 * 8) g = 152 * 8;
    return unsigned(g < 1 ? 1 : g);
}

}  // namespace

void launch_thin_weights(const float *y, int64_t n, float alpha, float *w, cudaStream_t st) {
    if (n > 0) k_thin_weights<<<unsigned((n + 255) / 256), 256, 0, st>>>(y, n, alpha, w);
}

void launch_thin_expected(const float *w, int64_t n, double c, double *sum, cudaStream_t st) {
    cudaMemsetAsync(sum, 0, sizeof(double), st);
    if (n > 0) k_thin_expected<<<thin_grid(n), 256, 0, st>>>(w, n, c, sum);
}

void launch_thin_mark(const float *w, int64_t n, double c, uint64_t seed, uint8_t *keep, unsigned long long *kept,
                      cudaStream_t st) {
    cudaMemsetAsync(kept, 0, sizeof(unsigned long long), st);
    if (n > 0) k_thin_mark<<<thin_grid(n), 256, 0, st>>>(w, n, c, seed, keep, kept);
}

}  // namespace mgx
