// k_batch.cu -- work list of a batched, length-binned solve.
//
// Many models (or one model with very uneven rays) share one persistent solve
// launch.  The cost of an origin is the number of traced points over all its
// ray pairs (its work is proportional to it), summed from the half-ray
// lengths; origins are binned by log2 of
// that cost and the (model, origin, tile) items are laid out bin by bin,
// longest bin first, so that the persistent warps start the longest items
// first and the end of the launch is not held up by one long straggler.
// The binning is a stable radix sort of the origins by bin, so within a bin
// the items keep ascending (model, origin) order and neighbouring origins,
// whose traced points overlap, stay together for the cache.  No order affects
// a result: every item writes only its own J entries.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

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

// Key (cost bin) and value (global origin) of every origin for the stable sort.
__global__ void k_cost_keys(const BatchGeom *__restrict__ geo, const int64_t *__restrict__ origin_base,
                            int32_t n_models, int64_t n_origins, const int64_t *__restrict__ lens,
                            uint8_t *__restrict__ key, int32_t *__restrict__ val) {
    const int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (g >= n_origins) return;
    const int32_t k = model_of(origin_base, n_models, g);
    key[g] = uint8_t(cost_bin(origin_cost(geo[k], g - origin_base[k], lens)));
    val[g] = int32_t(g);
}

// Work items of the s-th origin in sorted order.
__global__ void k_sorted_tiles(const BatchGeom *__restrict__ geo, const int64_t *__restrict__ origin_base,
                               int32_t n_models, int64_t n_origins, const int32_t *__restrict__ val,
                               int64_t *__restrict__ tiles) {
    const int64_t s = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (s >= n_origins) return;
    tiles[s] = geo[model_of(origin_base, n_models, val[s])].n_tiles;
}

__global__ void k_emit_items(const BatchGeom *__restrict__ geo, const int64_t *__restrict__ origin_base,
                             int32_t n_models, int64_t n_origins, const int32_t *__restrict__ val,
                             const int64_t *__restrict__ toff, uint2 *__restrict__ work) {
    const int64_t s = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (s >= n_origins) return;
    const int64_t g = val[s];
    const int32_t k = model_of(origin_base, n_models, g);
    const int64_t o = g - origin_base[k];
    const int32_t nt = geo[k].n_tiles;
    const int64_t pos = s == 0 ? 0 : toff[s - 1];
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

// Plain order (for comparison with the cost bins): item (model k, origin o,
// tile t) at work_base[k] + o n_tiles[k] + t.
__global__ void k_work_natural(const BatchGeom *__restrict__ geo, const int64_t *__restrict__ origin_base,
                               int32_t n_models, int64_t n_origins, uint2 *__restrict__ work) {
    const int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (g >= n_origins) return;
    const int32_t k = model_of(origin_base, n_models, g);
    const int64_t o = g - origin_base[k];
    const int32_t nt = geo[k].n_tiles;
    const int64_t pos = geo[k].work_base + o * nt;
    for (int32_t t = 0; t < nt; ++t) work[pos + t] = make_uint2((uint32_t(k) << 16) | uint32_t(t), uint32_t(o));
}

}  // namespace

void launch_excess_totals(const int64_t *lens, int64_t n, unsigned long long *out, cudaStream_t st) {
    cudaMemsetAsync(out, 0, (kPadCandidates + 1) * sizeof(unsigned long long), st);
    if (n == 0) return;
    int64_t grid = (n + 255) / 256;
    if (grid > 152 * 8) grid = 152 * 8;
    k_excess_totals<<<unsigned(grid), 256, 0, st>>>(lens, n, out);
}

size_t batch_worklist_temp_bytes(int64_t n_origins) {
    size_t a = 0, b = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, a, (const uint8_t *)nullptr, (uint8_t *)nullptr,
                                    (const int32_t *)nullptr, (int32_t *)nullptr, int(n_origins), 0, 5);
    cub::DeviceScan::InclusiveSum(nullptr, b, (const int64_t *)nullptr, (int64_t *)nullptr, int(n_origins));
    return a > b ? a : b;
}

void launch_batch_worklist(const BatchGeom *geo, const int64_t *origin_base, int32_t n_models, int64_t n_origins,
                           const int64_t *lens, const WorkListBufs &b, uint2 *work, bool natural, cudaStream_t st) {
    const int tb = 256;
    const unsigned grid = unsigned((n_origins + tb - 1) / tb);
    if (n_origins == 0) return;
    if (natural) {
        k_work_natural<<<grid, tb, 0, st>>>(geo, origin_base, n_models, n_origins, work);
        return;
    }
    k_cost_keys<<<grid, tb, 0, st>>>(geo, origin_base, n_models, n_origins, lens, b.key_in, b.val_in);
    size_t bytes = b.tmp_bytes;
    cub::DeviceRadixSort::SortPairs(b.tmp, bytes, b.key_in, b.key_out, b.val_in, b.val_out, int(n_origins), 0, 5,
                                    st);
    k_sorted_tiles<<<grid, tb, 0, st>>>(geo, origin_base, n_models, n_origins, b.val_out, b.tiles);
    bytes = b.tmp_bytes;
    cub::DeviceScan::InclusiveSum(b.tmp, bytes, b.tiles, b.toff, int(n_origins), st);
    k_emit_items<<<grid, tb, 0, st>>>(geo, origin_base, n_models, n_origins, b.val_out, b.toff, work);
}

}  // namespace mgx
