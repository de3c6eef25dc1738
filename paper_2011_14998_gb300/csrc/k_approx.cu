// k_approx.cu -- evaluation of the approximate single-precision functions the
// formal solution uses (k_solve_impl.cuh), so that tests can check the error
// bounds its single-precision integer decisions are certified with.
#include "k_solve_impl.cuh"

namespace mgx {

namespace {

__global__ void k_eval_approx(int kind, const float *__restrict__ x, int64_t n, float *__restrict__ y) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        float r;
        const float v = x[i];
        if (kind == 0) asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
        else r = Ar<float>::rcp(v);
        y[i] = r;
    }
}

}  // namespace

void launch_eval_approx(int kind, const float *x, int64_t n, float *y, cudaStream_t st) {
    if (n <= 0) return;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_eval_approx<<<unsigned(blocks), 256, 0, st>>>(kind, x, n, y);
}

// bounds the certification takes, for the tests
float approx_bound(int kind) { return kind == 0 ? kEEx2 : kERcp; }

}  // namespace mgx
