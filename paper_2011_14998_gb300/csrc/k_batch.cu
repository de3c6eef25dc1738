// k_batch.cu -- work list of a batched, length-binned solve.
//
// Many models (or one model with very uneven rays) share one persistent solve
// launch.  The cost of an origin is the number of traced points over all its
// ray pairs (its work is proportional to it), summed from the half-ray
// lengths; origins are binned by log2 of
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

__device__ __forceinline__ int64_t origin_cost(const BatchGeom &g, int64_t o, const int64_t *__restrict__ lens) {
    const int64_t h0 = g.half_base + o * g.npairs2;
    int64_t cost = 0;
    for (int32_t j = 0; j < g.npairs2; ++j) cost += lens[h0 + j];
    return cost;
}

__global__ void k_cost_hist(const BatchGeom *__restrict__ geo, const int64_t *__restrict__ origin_base,
                            int32_t n_models, int64_t n_origins, const int64_t *__restrict__ lens,
                            unsigned long long *__restrict__ hist) {
    const int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (g >= n_origins) return;
    const int32_t k = model_of(origin_base, n_models, g);
    const int64_t cost = origin_cost(geo[k], g - origin_base[k], lens);
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
                               int32_t n_models, int64_t n_origins, const int64_t *__restrict__ lens,
                               unsigned long long *__restrict__ cursor, uint2 *__restrict__ work) {
    const int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (g >= n_origins) return;
    const int32_t k = model_of(origin_base, n_models, g);
    const int64_t o = g - origin_base[k];
    const int64_t cost = origin_cost(geo[k], o, lens);
    const int32_t nt = geo[k].n_tiles;
    const unsigned long long pos = atomicAdd(&cursor[cost_bin(cost)], (unsigned long long)nt);
    for (int32_t t = 0; t < nt; ++t) work[pos + t] = make_uint2((uint32_t(k) << 16) | uint32_t(t), uint32_t(o));
}

// Points beyond a row of width 2^j, sum over half-rays of max(0, len - 2^j),
// for j < kPadCandidates, and the total points (slot kPadCandidates).
__global__ void k_excess_totals(const int64_t *__restrict__ lens, int64_t n, unsigned long long *__restrict__ out) {
    unsigned long long acc[kPadCandidates + 1] = {};
    for (int64_t h = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; h < n; h += int64_t(gridDim.x) * blockDim.x) {
        const int64_t len = lens[h];
#pragma unroll
        for (int j = 0; j < kPadCandidates; ++j) {
            const int64_t e = len - (int64_t(1) << j);
            acc[j] += e > 0 ? (unsigned long long)e : 0ull;
        }
        acc[kPadCandidates] += (unsigned long long)len;
    }
#pragma unroll
    for (int j = 0; j <= kPadCandidates; ++j) {
        unsigned long long v = acc[j];
#pragma unroll
        for (int sh = 16; sh > 0; sh >>= 1) v += __shfl_down_sync(0xffffffffu, v, sh);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(out + j, v);
    }
}

}  // namespace

void launch_excess_totals(const int64_t *lens, int64_t n, unsigned long long *out, cudaStream_t st) {
    cudaMemsetAsync(out, 0, (kPadCandidates + 1) * sizeof(unsigned long long), st);
    if (n == 0) return;
    int64_t grid = (n + 255) / 256;
    if (grid > 152 * 8) grid = 152 * 8;
    k_excess_totals<<<unsigned(grid), 256, 0, st>>>(lens, n, out);
}

void launch_batch_worklist(const BatchGeom *geo, const int64_t *origin_base, int32_t n_models, int64_t n_origins,
                           const int64_t *lens, unsigned long long *scratch64, uint2 *work, cudaStream_t st) {
    unsigned long long *hist = scratch64, *cursor = scratch64 + kBins;
    cudaMemsetAsync(hist, 0, kBins * sizeof(unsigned long long), st);
    const int tb = 256;
    const unsigned grid = unsigned((n_origins + tb - 1) / tb);
    k_cost_hist<<<grid, tb, 0, st>>>(geo, origin_base, n_models, n_origins, lens, hist);
    k_cost_scan<<<1, 32, 0, st>>>(hist, cursor);
    k_cost_scatter<<<grid, tb, 0, st>>>(geo, origin_base, n_models, n_origins, lens, cursor, work);
}

}  // namespace mgx
