// k_solve.cu -- the second-order instantiation of the formal solution
// (k_solve_impl.cuh) and the dispatch on the scheme's order; the Hermitian
// instantiation is compiled separately (k_solve_herm.cu).
#include "k_solve_impl.cuh"

namespace mgx {

// Bins per lane of the single-precision kernel: 2 when there are more bins than
// lanes (the frequency-independent work is then shared by two bins), else 1.
int solve_bins_per_lane(int precision, int32_t n_bins) {
    if (precision != MGX_FP32 && precision != MGX_FP32_DT64) return 1;
    return n_bins > 32 ? 2 : 1;
}

template void launch_solve_ord<2>(const DevMesh &, const DevLines &, const DevRays &, const SolveArgs &, int,
                                  cudaStream_t);
template void launch_solve_queue_ord<2>(int, int, int, const BatchSlot *, const uint2 *, int64_t,
                                        unsigned long long *, cudaStream_t);
extern template void launch_solve_ord<4>(const DevMesh &, const DevLines &, const DevRays &, const SolveArgs &, int,
                                         cudaStream_t);
extern template void launch_solve_queue_ord<4>(int, int, int, const BatchSlot *, const uint2 *, int64_t,
                                               unsigned long long *, cudaStream_t);

void launch_solve(const DevMesh &m, const DevLines &Ln, const DevRays &R, const SolveArgs &a, int precision,
                  int order, cudaStream_t st) {
    if (order == 4) launch_solve_ord<4>(m, Ln, R, a, precision, st);
    else launch_solve_ord<2>(m, Ln, R, a, precision, st);
}

void launch_solve_queue(int precision, int order, int bins_per_lane, int max_lines, const BatchSlot *slots,
                        const uint2 *work, int64_t n_work, unsigned long long *next, cudaStream_t st) {
    if (order == 4) launch_solve_queue_ord<4>(precision, bins_per_lane, max_lines, slots, work, n_work, next, st);
    else launch_solve_queue_ord<2>(precision, bins_per_lane, max_lines, slots, work, n_work, next, st);
}

}  // namespace mgx
