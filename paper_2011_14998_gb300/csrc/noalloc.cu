// noalloc.cu -- scratch for the allocation-free variant of the solve.
//
// mgx_solve_J allocates its working memory (half-ray lengths, their offsets
// and the traced point lists) from the stream-ordered pool on every call.
// Some callers cannot allow that: code that runs while a framework owns all
// device memory and forbids third-party allocations during its step, or code
// inside a region where no allocation may be enqueued.  For them,
// mgx_solve_J_noalloc takes its working memory from the fixed array below
// instead and processes the origins in chunks that fit it.
//
// The array is a file-scope __device__ variable: every GPU that loads this
// library holds its 64 MiB until the process exits.  Host code cannot use the
// variable's name as a device address; the first call on each device looks
// the address up with cudaGetSymbolAddress (with that device current) and
// caches it, so that first call should come before any stream capture.  Every
// call shares the array and leaves the previous call's
// contents in it; calls that overlap on the GPU (different streams, or several
// contexts on one device) race on it.
#include <algorithm>
#include <cstdio>
#include <mutex>

#include "mgx_internal.cuh"

namespace mgx {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// offs[0] = 0, offs[i+1] = lens[0] + ... + lens[i]; one CTA, no temporary memory
__global__ void __launch_bounds__(1024) k_scan_lengths(const int64_t *__restrict__ lens, int64_t n,
                                                       int64_t *__restrict__ offs) {
    __shared__ int64_t part[1024];
    const int t = threadIdx.x, T = blockDim.x;
    const int64_t per = (n + T - 1) / T;
    const int64_t b = min(n, int64_t(t) * per), e = min(n, b + per);
    int64_t s = 0;
    for (int64_t i = b; i < e; ++i) s += lens[i];
    part[t] = s;
    __syncthreads();
    for (int d = 1; d < T; d <<= 1) {
        const int64_t v = t >= d ? part[t - d] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int64_t run = t > 0 ? part[t - 1] : 0;
    if (t == 0) offs[0] = 0;
    for (int64_t i = b; i < e; ++i) {
        run += lens[i];
        offs[i + 1] = run;
    }
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

// Device address of the scratch array on the current device (looked up once).
static cudaError_t scratch_address(int device, unsigned char **out) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[device] = p;
    }
    *out = static_cast<unsigned char *>(g_scratch_addr[device]);
    return cudaSuccess;
}

int noalloc_solve(int device, const DevMesh &m, const DevLines &Ln, const DevRays &R, double dtau_max,
                  double dv_max, double I_bdy, int precision, int order, double *J, int *status, cudaStream_t st,
                  char *err, size_t errlen) {
    unsigned char *base = nullptr;
    cudaError_t ce = scratch_address(device, &base);
    if (ce != cudaSuccess) {
        snprintf(err, errlen, "cudaGetSymbolAddress of the scratch array failed: %s", cudaGetErrorString(ce));
        return MGX_ECUDA;
    }
    const int64_t np2 = int64_t(R.npairs) * 2;
    // lengths and offsets of a chunk take at most an eighth of the array
    const int64_t c_max = int64_t(kNoAllocScratchBytes / 8 - 8) / (16 * np2);
    if (c_max < 1) {
        snprintf(err, errlen, "ray set of %d pairs too large for the %zu MiB scratch", R.npairs,
                 kNoAllocScratchBytes >> 20);
        return MGX_ERANGE;
    }
    const int64_t NB = int64_t(Ln.L) * Ln.F;
    int64_t o0 = 0;
    while (o0 < m.n) {
        int64_t c = std::min<int64_t>(c_max, m.n - o0);
        int64_t *lens = nullptr, *offs = nullptr;
        int32_t *idx = nullptr;
        int64_t cap_used = 0;
        for (;;) {
            const int64_t nh = c * np2;
            lens = reinterpret_cast<int64_t *>(base);
            offs = lens + nh;
            const size_t arena0 = align256(size_t(2 * nh + 1) * sizeof(int64_t));
            const int64_t cap = int64_t((kNoAllocScratchBytes - arena0) / sizeof(int32_t));
            idx = reinterpret_cast<int32_t *>(base + arena0);
            cap_used = cap;
            launch_trace_count(m, R, int32_t(o0), int32_t(o0 + c), lens, status, nullptr, st);
            k_scan_lengths<<<1, 1024, 0, st>>>(lens, nh, offs);
            int64_t total = 0;
            if ((ce = cudaGetLastError()) != cudaSuccess ||
                (ce = cudaMemcpyAsync(&total, offs + nh, sizeof total, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
                (ce = cudaStreamSynchronize(st)) != cudaSuccess) {
                snprintf(err, errlen, "CUDA error in the allocation-free solve: %s", cudaGetErrorString(ce));
                return MGX_ECUDA;
            }
            if (total <= cap) break;
            if (c == 1) {
                snprintf(err, errlen,
                         "the traced point lists of origin %lld hold %lld entries; the %zu MiB scratch holds %lld",
                         (long long)o0, (long long)total, kNoAllocScratchBytes >> 20, (long long)cap);
                return MGX_ERANGE;
            }
            c = std::max<int64_t>(1, int64_t(double(c) * double(cap) / double(total) * 0.9));
        }
        launch_trace_emit(m, R, int32_t(o0), int32_t(o0 + c), offs, 0, cap_used, idx, nullptr, nullptr, status, st);
        SolveArgs a;
        a.dtau_max = dtau_max;
        a.dv_max = dv_max;
        a.I_bdy = I_bdy;
        a.o_begin = int32_t(o0);
        a.o_end = int32_t(o0 + c);
        {
            const int64_t per = 32 * solve_bins_per_lane(precision, int32_t(NB));
            a.n_tiles = int32_t((NB + per - 1) / per);
        }
        a.offs = offs;
        a.base = 0;
        a.idx = idx;
        a.J = J;
        a.status = status;
        a.counters = nullptr;
        fill_pair_weights(a);
        launch_solve(m, Ln, R, a, precision, order, st);
        if ((ce = cudaGetLastError()) != cudaSuccess) {
            snprintf(err, errlen, "CUDA error in the allocation-free solve: %s", cudaGetErrorString(ce));
            return MGX_ECUDA;
        }
        o0 += c;
    }
    return MGX_OK;
}

}  // namespace mgx
