// k_solve_herm.cu -- the Hermitian (fourth-order, Auer 1976; Section 2.1)
// instantiation of the formal solution in k_solve_impl.cuh, compiled in its own
// translation unit so that the two schemes build in parallel.
#include "k_solve_impl.cuh"

namespace mgx {

template void launch_solve_ord<4>(const DevMesh &, const DevLines &, const DevRays &, const SolveArgs &, int,
                                  cudaStream_t);
template void launch_solve_queue_ord<4>(int, int, int, const BatchSlot *, const uint2 *, int64_t,
                                        unsigned long long *, cudaStream_t);

}  // namespace mgx
