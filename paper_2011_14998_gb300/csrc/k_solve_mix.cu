// k_solve_mix.cu -- the second-order formal solution (k_solve_impl.cuh) with
// the optical-depth increments and the elimination pivots (Fh, D) in double
// precision and the rest in single precision (MGX_FP32_DT64), compiled apart
// from the other forms.
#include "k_solve_impl.cuh"

namespace mgx {

void launch_solve_dt64(const DevMesh &m, const DevLines &Ln, const DevRays &R, const SolveArgs &a, int bins_per_lane,
                       cudaStream_t st) {
    if (bins_per_lane == 2) launch_RB<float, 2, 2, double>(m, Ln, R, a, st);
    else launch_RB<float, 1, 2, double>(m, Ln, R, a, st);
}

void launch_solve_queue_dt64(int bins_per_lane, int max_lines, const BatchSlot *slots, const uint2 *work,
                             int64_t n_work, unsigned long long *next, cudaStream_t st) {
    if (n_work == 0) return;
    if (bins_per_lane == 2) launch_queue_RB<float, 2, 2, double>(max_lines, slots, work, n_work, next, st);
    else launch_queue_RB<float, 1, 2, double>(max_lines, slots, work, n_work, next, st);
}

}  // namespace mgx
