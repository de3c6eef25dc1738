// k_mlp.cu -- the learned mesh-reduction network: per-point features, BF16
// tensor-core forward and backward passes with FP32 accumulation, Adam.
//
// Network 8 -> 64 -> 64 -> 1 with ReLU (parameters as one FP32 vector theta:
// W1 [8][64], b1 [64], W2 [64][64], b2 [64], W3 [64], b3 [1]).  Inputs and
// the two hidden weight matrices are held in bfloat16 (W1 padded to 16 input
// rows), as are the activations h1 and the back-propagated gradients of both
// hidden layers, the operands of the tensor-core products; accumulators,
// biases, h2, the output layer and all gradient sums are FP32.
//
// One CTA of 4 warps handles 64 points; each warp computes 16-row blocks with
// 16x16x16 bf16 WMMA fragments.  The backward pass recomputes the forward
// pass of its 64 points in shared memory and adds its parameter gradients to
// a global FP32 accumulator.
#include <cub/device/device_radix_sort.cuh>
#include <cuda_bf16.h>
#include <mma.h>

#include "mgx_internal.cuh"

namespace mgx {

namespace {

using namespace nvcuda;
using bf16 = __nv_bfloat16;

constexpr int kPts = 64;  // points per CTA
constexpr int kHid = 64;
constexpr int kInPad = 16;

struct Smem {
    bf16 W1[kInPad * kHid];
    bf16 W2[kHid * kHid];
    bf16 X[kPts * kInPad];
    bf16 H1[kPts * kHid];
    float H2[kPts * kHid];
    float Acc[kPts * kHid];
    bf16 D2[kPts * kHid];
    bf16 D1[kPts * kHid];
    float dy[kPts];
    float red[4][kHid];
};

__global__ void k_mlp_convert(const float *__restrict__ theta, bf16 *__restrict__ W1b, bf16 *__restrict__ W2b) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kInPad * kHid) {
        const int r = i / kHid;
        W1b[i] = __float2bfloat16_rn(r < 8 ? theta[kMlpW1 + i] : 0.0f);
    }
    if (i < kHid * kHid) W2b[i] = __float2bfloat16_rn(theta[kMlpW2 + i]);
}

template <bool TRAIN>
__global__ void __launch_bounds__(128)
k_mlp(const float *__restrict__ X, const float *__restrict__ t, const int32_t *__restrict__ perm, int64_t rows,
      const bf16 *__restrict__ W1b, const bf16 *__restrict__ W2b, const float *__restrict__ theta,
      float *__restrict__ y_out, float *__restrict__ grad, float *__restrict__ loss, float inv_batch) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem &s = *reinterpret_cast<Smem *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t r0 = int64_t(blockIdx.x) * kPts;
    for (int i = tid; i < kInPad * kHid; i += 128) s.W1[i] = W1b[i];
    for (int i = tid; i < kHid * kHid; i += 128) s.W2[i] = W2b[i];
    for (int i = tid; i < kPts * kInPad; i += 128) {
        const int p = i / kInPad, c = i % kInPad;
        const int64_t r = r0 + p;
        float v = 0.0f;
        if (c < 8 && r < rows) v = X[(perm ? int64_t(perm[r]) : r) * 8 + c];
        s.X[i] = __float2bfloat16_rn(v);
    }
    __syncthreads();

    const int wr = warp * 16;  // this warp's 16 points
    // h1 = relu(x W1 + b1), bf16
    {
        wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, wmma::row_major> a;
        wmma::load_matrix_sync(a, s.X + wr * kInPad, kInPad);
        for (int j = 0; j < 4; ++j) {
            wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16, wmma::row_major> b;
            wmma::fragment<wmma::accumulator, 16, 16, 16, float> c;
            wmma::fill_fragment(c, 0.0f);
            wmma::load_matrix_sync(b, s.W1 + j * 16, kHid);
            wmma::mma_sync(c, a, b, c);
            wmma::store_matrix_sync(s.Acc + wr * kHid + j * 16, c, kHid, wmma::mem_row_major);
        }
        __syncwarp();
        for (int i = lane; i < 16 * kHid; i += 32) {
            const int idx = wr * kHid + i;
            s.H1[idx] = __float2bfloat16_rn(fmaxf(s.Acc[idx] + theta[kMlpB1 + (i % kHid)], 0.0f));
        }
        __syncwarp();
    }
    // h2 = relu(h1 W2 + b2), fp32
    {
        wmma::fragment<wmma::accumulator, 16, 16, 16, float> c[4];
        for (int j = 0; j < 4; ++j) wmma::fill_fragment(c[j], 0.0f);
        for (int k = 0; k < 4; ++k) {
            wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, wmma::row_major> a;
            wmma::load_matrix_sync(a, s.H1 + wr * kHid + k * 16, kHid);
            for (int j = 0; j < 4; ++j) {
                wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16, wmma::row_major> b;
                wmma::load_matrix_sync(b, s.W2 + (k * 16) * kHid + j * 16, kHid);
                wmma::mma_sync(c[j], a, b, c[j]);
            }
        }
        for (int j = 0; j < 4; ++j) wmma::store_matrix_sync(s.Acc + wr * kHid + j * 16, c[j], kHid, wmma::mem_row_major);
        __syncwarp();
        for (int i = lane; i < 16 * kHid; i += 32) {
            const int idx = wr * kHid + i;
            s.H2[idx] = fmaxf(s.Acc[idx] + theta[kMlpB2 + (i % kHid)], 0.0f);
        }
        __syncwarp();
    }
    // y = h2 . W3 + b3: lanes l and l+16 share point l
    const int p = lane & 15, half = lane >> 4;
    float part = 0.0f;
    for (int c = half * 32; c < half * 32 + 32; ++c) part += s.H2[(wr + p) * kHid + c] * theta[kMlpW3 + c];
    part += __shfl_xor_sync(0xffffffffu, part, 16);
    const float y = part + theta[kMlpB3];
    const int64_t r = r0 + wr + p;
    const bool valid = r < rows;
    if (!TRAIN) {
        if (half == 0 && valid) y_out[r] = y;
        return;
    }
    if (half == 0) {
        const float e = valid ? y - t[perm ? perm[r] : r] : 0.0f;
        s.dy[wr + p] = inv_batch * e;
        float sq = e * e;
        for (int sh = 8; sh > 0; sh >>= 1) sq += __shfl_down_sync(0x0000ffffu, sq, sh);
        if (p == 0) atomicAdd(loss, sq);
    }
    __syncthreads();

    // output layer and dh2 = dy W3 (h2 > 0), bf16
    if (tid < kHid) {
        float g = 0.0f;
        for (int q = 0; q < kPts; ++q) g += s.dy[q] * s.H2[q * kHid + tid];
        atomicAdd(grad + kMlpW3 + tid, g);
    } else if (tid == kHid) {
        float g = 0.0f;
        for (int q = 0; q < kPts; ++q) g += s.dy[q];
        atomicAdd(grad + kMlpB3, g);
    }
    for (int i = tid; i < kPts * kHid; i += 128) {
        const int q = i / kHid, c = i % kHid;
        const float v = s.H2[i] > 0.0f ? s.dy[q] * theta[kMlpW3 + c] : 0.0f;
        s.D2[i] = __float2bfloat16_rn(v);
    }
    __syncthreads();
    if (tid < kHid) {
        float g = 0.0f;
        for (int q = 0; q < kPts; ++q) g += __bfloat162float(s.D2[q * kHid + tid]);
        atomicAdd(grad + kMlpB2 + tid, g);
    }
    // dW2 = h1^T dh2 (this warp: input rows wr..wr+15)
    {
        wmma::fragment<wmma::accumulator, 16, 16, 16, float> c[4];
        for (int j = 0; j < 4; ++j) wmma::fill_fragment(c[j], 0.0f);
        for (int k = 0; k < 4; ++k) {
            wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, wmma::col_major> a;
            wmma::load_matrix_sync(a, s.H1 + (k * 16) * kHid + wr, kHid);
            for (int j = 0; j < 4; ++j) {
                wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16, wmma::row_major> b;
                wmma::load_matrix_sync(b, s.D2 + (k * 16) * kHid + j * 16, kHid);
                wmma::mma_sync(c[j], a, b, c[j]);
            }
        }
        __syncthreads();  // Acc is reused: every warp is done reading it
        for (int j = 0; j < 4; ++j) wmma::store_matrix_sync(s.Acc + wr * kHid + j * 16, c[j], kHid, wmma::mem_row_major);
        __syncwarp();
        for (int i = lane; i < 16 * kHid; i += 32) atomicAdd(grad + kMlpW2 + wr * kHid + i, s.Acc[wr * kHid + i]);
        __syncwarp();
    }
    // dh1 = dh2 W2^T (h1 > 0), bf16 (this warp: points wr..wr+15)
    {
        wmma::fragment<wmma::accumulator, 16, 16, 16, float> c[4];
        for (int j = 0; j < 4; ++j) wmma::fill_fragment(c[j], 0.0f);
        for (int k = 0; k < 4; ++k) {
            wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, wmma::row_major> a;
            wmma::load_matrix_sync(a, s.D2 + wr * kHid + k * 16, kHid);
            for (int j = 0; j < 4; ++j) {
                wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16, wmma::col_major> b;
                wmma::load_matrix_sync(b, s.W2 + (j * 16) * kHid + k * 16, kHid);
                wmma::mma_sync(c[j], a, b, c[j]);
            }
        }
        for (int j = 0; j < 4; ++j) wmma::store_matrix_sync(s.Acc + wr * kHid + j * 16, c[j], kHid, wmma::mem_row_major);
        __syncwarp();
        for (int i = lane; i < 16 * kHid; i += 32) {
            const int idx = wr * kHid + i;
            const float v = __bfloat162float(s.H1[idx]) > 0.0f ? s.Acc[idx] : 0.0f;
            s.D1[idx] = __float2bfloat16_rn(v);
        }
        __syncwarp();
        for (int c2 = lane; c2 < kHid; c2 += 32) {
            float g = 0.0f;
            for (int q = 0; q < 16; ++q) g += __bfloat162float(s.D1[(wr + q) * kHid + c2]);
            s.red[warp][c2] = g;
        }
    }
    __syncthreads();
    if (tid < kHid) atomicAdd(grad + kMlpB1 + tid, s.red[0][tid] + s.red[1][tid] + s.red[2][tid] + s.red[3][tid]);
    // dW1 = x^T dh1 (this warp: hidden columns warp*16..+15)
    {
        wmma::fragment<wmma::accumulator, 16, 16, 16, float> c;
        wmma::fill_fragment(c, 0.0f);
        for (int k = 0; k < 4; ++k) {
            wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, wmma::col_major> a;
            wmma::load_matrix_sync(a, s.X + (k * 16) * kInPad, kInPad);
            wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16, wmma::row_major> b;
            wmma::load_matrix_sync(b, s.D1 + (k * 16) * kHid + warp * 16, kHid);
            wmma::mma_sync(c, a, b, c);
        }
        __syncthreads();
        wmma::store_matrix_sync(s.Acc + warp * 16, c, kHid, wmma::mem_row_major);
        __syncwarp();
        for (int i = lane; i < 8 * 16; i += 32) {
            const int row = i / 16, col = warp * 16 + i % 16;
            atomicAdd(grad + kMlpW1 + row * kHid + col, s.Acc[row * kHid + col]);
        }
    }
}

// Adam (Kingma & Ba 2015) on the FP32 master parameters; refreshes the bf16
// copies and clears the gradient accumulator.
__global__ void k_mlp_adam(float *__restrict__ theta, float *__restrict__ m, float *__restrict__ v,
                           float *__restrict__ grad, float lr, float b1, float b2, float eps, float c1, float c2,
                           bf16 *__restrict__ W1b, bf16 *__restrict__ W2b) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpN) return;
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.0f - b1) * g;
    const float vi = b2 * v[i] + (1.0f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float th = theta[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    theta[i] = th;
    grad[i] = 0.0f;
    if (i >= kMlpW1 && i < kMlpW1 + 8 * kHid) W1b[i - kMlpW1] = __float2bfloat16_rn(th);
    if (i >= kMlpW2 && i < kMlpW2 + kHid * kHid) W2b[i - kMlpW2] = __float2bfloat16_rn(th);
}

// Eight per-point features of the reduction network (Section 2.2.2 inputs):
// log density, the largest log-density contrast to a neighbour, the largest
// velocity change to a neighbour in local Doppler widths, log temperature,
// log mean neighbour distance (Eq. 8's L), neighbour count, log distance from
// the coordinate origin, log line-centre optical depth across an element.
__global__ void k_mlp_features(DevMesh m, const float *__restrict__ chi0, int32_t L, const float *__restrict__ dvw,
                               const double *__restrict__ rho, const double *__restrict__ T, float *__restrict__ X) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= m.n) return;
    const double xi = m.x[i], yi = m.y[i], zi = m.z[i];
    const double lr = log(rho[i]);
    double dmax = 0.0, vmax = 0.0, sum = 0.0;
    const int32_t e0 = m.off[i], e1 = m.off[i + 1];
    for (int32_t e = e0; e < e1; ++e) {
        const int32_t j = m.nbr[e];
        dmax = fmax(dmax, fabs(log(rho[j]) - lr));
        const double ux = m.vx[j] - m.vx[i], uy = m.vy[j] - m.vy[i], uz = m.vz[j] - m.vz[i];
        vmax = fmax(vmax, sqrt(ux * ux + uy * uy + uz * uz));
        const double dx = m.x[j] - xi, dy = m.y[j] - yi, dz = m.z[j] - zi;
        sum += sqrt(dx * dx + dy * dy + dz * dz);
    }
    const int32_t deg = e1 - e0;
    const double Li = deg > 0 ? sum / deg : 0.0;
    const double tiny = 1e-30;
    float *o = X + i * 8;
    o[0] = float(lr);
    o[1] = float(dmax);
    o[2] = float(vmax / double(dvw[i]));
    o[3] = float(log(T[i]));
    o[4] = float(log(Li + tiny));
    o[5] = float(deg);
    o[6] = float(log(sqrt(xi * xi + yi * yi + zi * zi) + tiny));
    o[7] = float(log(double(chi0[i * L]) * Li + tiny));
}

__global__ void k_iota(int32_t *ids, int64_t n) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i < n) ids[i] = int32_t(i);
}

__global__ void k_mark_top(const int32_t *__restrict__ ids_sorted, int64_t n, int64_t k, uint8_t *__restrict__ keep) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i < n) keep[ids_sorted[i]] = i < k ? 1 : 0;
}

}  // namespace

// keep[i] = 1 for the k points with the largest score (ties: smaller index first)
void launch_select_top(const float *score, int64_t n, int64_t k, int32_t *ids, float *score_sorted,
                       int32_t *ids_sorted, uint8_t *keep, cudaStream_t st) {
    const int tb = 256;
    const unsigned grid = unsigned((n + tb - 1) / tb);
    k_iota<<<grid, tb, 0, st>>>(ids, n);
    size_t bytes = 0;
    cub::DeviceRadixSort::SortPairsDescending(nullptr, bytes, score, score_sorted, ids, ids_sorted, n, 0, 32, st);
    void *tmp = nullptr;
    cudaMallocAsync(&tmp, bytes ? bytes : 1, st);
    cub::DeviceRadixSort::SortPairsDescending(tmp, bytes, score, score_sorted, ids, ids_sorted, n, 0, 32, st);
    cudaFreeAsync(tmp, st);
    k_mark_top<<<grid, tb, 0, st>>>(ids_sorted, n, k, keep);
}

size_t mlp_smem_bytes() { return sizeof(Smem); }

void launch_mlp_convert(const float *theta, void *W1b, void *W2b, cudaStream_t st) {
    k_mlp_convert<<<(kHid * kHid + 255) / 256, 256, 0, st>>>(theta, static_cast<bf16 *>(W1b), static_cast<bf16 *>(W2b));
}

void launch_mlp(bool train, const float *X, const float *t, const int32_t *perm, int64_t rows, const void *W1b,
                const void *W2b, const float *theta, float *y, float *grad, float *loss, float inv_batch,
                cudaStream_t st) {
    if (rows <= 0) return;
    const size_t smem = sizeof(Smem);
    const unsigned grid = unsigned((rows + kPts - 1) / kPts);
    if (train) {
        cudaFuncSetAttribute(k_mlp<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        k_mlp<true><<<grid, 128, smem, st>>>(X, t, perm, rows, static_cast<const bf16 *>(W1b),
                                             static_cast<const bf16 *>(W2b), theta, y, grad, loss, inv_batch);
    } else {
        cudaFuncSetAttribute(k_mlp<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        k_mlp<false><<<grid, 128, smem, st>>>(X, t, perm, rows, static_cast<const bf16 *>(W1b),
                                              static_cast<const bf16 *>(W2b), theta, y, grad, loss, inv_batch);
    }
}

void launch_mlp_adam(float *theta, float *m, float *v, float *grad, float lr, float b1, float b2, float eps, float c1,
                     float c2, void *W1b, void *W2b, cudaStream_t st) {
    k_mlp_adam<<<(kMlpN + 255) / 256, 256, 0, st>>>(theta, m, v, grad, lr, b1, b2, eps, c1, c2,
                                                    static_cast<bf16 *>(W1b), static_cast<bf16 *>(W2b));
}

void launch_mlp_features(const DevMesh &m, const float *chi0, int32_t L, const float *dvw, const double *rho,
                         const double *T, float *X, cudaStream_t st) {
    const int tb = 256;
    k_mlp_features<<<unsigned((m.n + tb - 1) / tb), tb, 0, st>>>(m, chi0, L, dvw, rho, T, X);
}

}  // namespace mgx
