// k_batch.cu -- work list of a batched, length-binned solve.
//
// Many models (or one model with very uneven rays) share one persistent solve
// launch.  The cost of an origin is the number of traced points over all its
// ray pairs (its work is proportional to it); origins are binned by log2 of
// that cost and the (model, origin, tile) items are laid out bin by bin,
// longest bin first, so that the persistent warps start the longest items
// first and the end of the launch is not held up by one long straggler.
// The order within a bin follows atomics and does not affect any result:
// every item writes only its own J entries.
#include "mgx_internal.cuh"

namespace mgx {

namespace {

constexpr int kBins = 32;

// model of global origin g: last k with origin_base[k] <= g
__device__ __forceinline__ int32_t model_of(const int64_t *__restrict__ origin_base, int32_t n_models, int64_t g) {
    int32_t lo = 0, hi = n_models - 1;
    while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (origin_base[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int cost_bin(int64_t cost) {
    // bins in decreasing order of cost: bin 0 holds costs >= 2^31
    const unsigned long long c = (unsigned long long)(cost < 1 ? 1 : cost);
    const int lg = 63 - __clzll(c);
    const int b = kBins - 1 - (lg < kBins - 1 ? lg : kBins - 1);
    return b;
}

__global__ void k_cost_hist(const BatchGeom *__restrict__ geo, const int64_t *__restrict__ origin_base,
                            int32_t n_models, int64_t n_origins, const int64_t *__restrict__ offs,
                            unsigned long long *__restrict__ hist) {
    const int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (g >= n_origins) return;
    const int32_t k = model_of(origin_base, n_models, g);
    const int64_t o = g - origin_base[k];
    const int64_t h0 = geo[k].half_base + o * geo[k].npairs2;
    const int64_t cost = offs[h0 + geo[k].npairs2] - offs[h0];
    atomicAdd(&hist[cost_bin(cost)], (unsigned long long)geo[k].n_tiles);
}

__global__ void k_cost_scan(unsigned long long *__restrict__ hist, unsigned long long *__restrict__ cursor) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned long long run = 0;
    for (int b = 0; b < kBins; ++b) {
        cursor[b] = run;
        run += hist[b];
    }
}

__global__ void k_cost_scatter(const BatchGeom *__restrict__ geo, const int64_t *__restrict__ origin_base,
                               int32_t n_models, int64_t n_origins, const int64_t *__restrict__ offs,
                               unsigned long long *__restrict__ cursor, uint2 *__restrict__ work) {
    const int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (g >= n_origins) return;
    const int32_t k = model_of(origin_base, n_models, g);
    const int64_t o = g - origin_base[k];
    const int64_t h0 = geo[k].half_base + o * geo[k].npairs2;
    const int64_t cost = offs[h0 + geo[k].npairs2] - offs[h0];
    const int32_t nt = geo[k].n_tiles;
    const unsigned long long pos = atomicAdd(&cursor[cost_bin(cost)], (unsigned long long)nt);
    for (int32_t t = 0; t < nt; ++t) work[pos + t] = make_uint2((uint32_t(k) << 16) | uint32_t(t), uint32_t(o));
}

}  // namespace

void launch_batch_worklist(const BatchGeom *geo, const int64_t *origin_base, int32_t n_models, int64_t n_origins,
                           const int64_t *offs, unsigned long long *scratch64, uint2 *work, cudaStream_t st) {
    unsigned long long *hist = scratch64, *cursor = scratch64 + kBins;
    cudaMemsetAsync(hist, 0, kBins * sizeof(unsigned long long), st);
    const int tb = 256;
    const unsigned grid = unsigned((n_origins + tb - 1) / tb);
    k_cost_hist<<<grid, tb, 0, st>>>(geo, origin_base, n_models, n_origins, offs, hist);
    k_cost_scan<<<1, 32, 0, st>>>(hist, cursor);
    k_cost_scatter<<<grid, tb, 0, st>>>(geo, origin_base, n_models, n_origins, offs, cursor, work);
}

}  // namespace mgx
