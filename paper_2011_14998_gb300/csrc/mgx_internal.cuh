// mgx_internal.cuh -- device-side views and launch entry points shared by the
// CUDA translation units of libmgx.  Nothing here is part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mgx.h"

namespace mgx {

constexpr double kC = 299792.458;  // speed of light, km/s

// First error wins; kernels report through a device status word.
enum DevErr : int {
    kDevOk = 0,
    kDevBadCsr = 1,        // neighbour index out of range / offsets not monotone
    kDevNonFinite = 2,     // NaN or inf in an input array
    kDevTraceGuard = 3,    // a half-ray exceeded n points (cannot happen for valid input)
    kDevTraceMismatch = 4, // emit pass disagrees with the count pass
    kDevSubdivLimit = 5,   // more than kMaxSubdiv optical-depth sub-intervals in one step
    kDevBadInput = 6,      // value outside its documented range
    kDevArenaOverflow = 7, // traced lists longer than the arena planned for them
};

constexpr int kMaxSubdiv = 1 << 20;

__device__ __forceinline__ void dev_fail(int *status, int code) {
    atomicCAS(status, 0, code);
}

// HEALPix direction tables of levels 0..lmax are concatenated; level l starts at
// pixel offset 4 (4^l - 1) (= sum of 12 4^k for k < l).
__host__ __device__ __forceinline__ int64_t level_offset(int l) {
    return 4 * ((int64_t(1) << (2 * l)) - 1);
}

struct DevMesh {
    int32_t n;
    const double *x, *y, *z;     // positions, structure of arrays
    const double *vx, *vy, *vz;  // velocities km/s
    const float *vxf, *vyf, *vzf;
    const int32_t *off;  // [n+1]
    const int32_t *nbr;  // [E]
    const float4 *phi;        // positions rounded to float; w: the largest |x_n - x|_1 over the neighbours (float)
    const float4 *nrec;       // [E + 1] neighbour records: fl32 position of nbr[e] minus that of its point, id in w (int bits)
    float g0;                 // 32 u^2 max_n (|x|+|y|+|z|) + 1e-37: floor of the screen's error bounds
};

struct DevLines {
    int32_t L, F;
    double x_span;
    double ratio[MGX_MAX_LINES * MGX_MAX_LINES];  // nu0[l] / nu0[lp] at [l*MAX + lp]
    const double *chi0, *eta0;  // [n][L]
    const double *dvw, *chic, *etac;
    const float *chi0f, *eta0f;
    const float *dvwf, *chicf, *etacf;
};

struct DevRays {
    int32_t lmin, lmax, npairs;
    const uint32_t *rays;  // [n][npairs], (level << 28) | pixel
    const double *dir;     // [level_offset(lmax+1)][3] pixel-centre unit vectors
    const float4 *dirf;    // the same vectors rounded to float (w = 0)
};

struct SolveArgs {
    double dtau_max, dv_max, I_bdy;
    int32_t o_begin, o_end;   // origins of this chunk
    int32_t n_tiles;          // frequency tiles per origin (32 x bins-per-lane bins each)
    // Traced lists.  Packed (pad == 0): the ids of half-ray h are
    // idx[offs[h] - base .. offs[h+1] - base).  Padded (pad > 0): its length is
    // lens[h], entries k < pad are idx[h pad + k] and entries k >= pad are
    // tail[offs[h] - base + k - pad].
    const int64_t *offs;      // [2 npairs (o_end - o_begin) + 1] arena (or tail) offsets (absolute)
    int64_t base;             // offs[first half-ray of the chunk]
    const int32_t *idx;       // arena point ids (relative to base), or the padded rows
    int32_t pad = 0;
    const int64_t *lens = nullptr;  // padded: half-ray lengths
    const int32_t *tail = nullptr;  // padded: entries beyond the row
    double *u_out = nullptr;        // optional: u per (origin - o_begin, pair, bin)
    double *J;                // [n][L*F]
    int *status;
    unsigned long long *counters;  // nullable: [0] elimination updates, [1] optics samples,
                                   // [2] tracer steps, [3] tracer steps redone in double
    double w2[MGX_MAX_LEVEL + 1];  // 2 w_l = 2 / (12 4^l), pair weight of level l (Eq. 4)
};

// Fill SolveArgs::w2 (host).
inline void fill_pair_weights(SolveArgs &a) {
    for (int l = 0; l <= MGX_MAX_LEVEL; ++l) a.w2[l] = 2.0 / double(int64_t(12) << (2 * l));
}

// ---- ingest (k_mesh.cu)
void launch_ingest_mesh(int32_t n, const double *pos_aos, const double *vel_aos, const int64_t *off64,
                        int64_t E, double *x, double *y, double *z, double *vx, double *vy,
                        double *vz, float *vxf, float *vyf, float *vzf, int32_t *off32,
                        const int32_t *nbr, float4 *phi, unsigned int *xmax_bits, int *status,
                        cudaStream_t st);
void launch_pack_neighbours(int32_t n, const int32_t *off, const int32_t *nbr, float4 *phi,
                            float4 *nrec, cudaStream_t st);
void launch_ingest_lines(int32_t n, int32_t L, const double *chi0, const double *eta0,
                         const double *dvw, const double *chic, const double *etac, float *chi0f,
                         float *eta0f, float *dvwf, float *chicf, float *etacf, int *status,
                         cudaStream_t st);

// ---- ray sets (k_rays.cu)
void launch_rays_fixed(int32_t n, int32_t level, int32_t npairs, const uint32_t *pairs,
                       uint32_t *rays, cudaStream_t st);
void launch_rays_adaptive(const DevMesh &m, int32_t lmin, int32_t lmax, int32_t npairs,
                          int64_t n_sample, const int32_t *sample, const int32_t *anti,
                          const uint32_t *pairs_lmin, int32_t n_pairs_lmin, uint32_t *rays,
                          int *status, cudaStream_t st);

// ---- tracing (k_trace.cu)
// o_stride > 1: only every o_stride-th origin from o_begin (a sample), each length at its own index.
void launch_trace_count(const DevMesh &m, const DevRays &R, int32_t o_begin, int32_t o_end,
                        int64_t *lens, int *status, unsigned long long *counters, cudaStream_t st,
                        int32_t o_stride = 1);
// Z == nullptr: ids only (the solver's arena); otherwise also exact Z (and delta if given).
// Entries beyond cap (relative to base) are refused with kDevArenaOverflow.
void launch_trace_emit(const DevMesh &m, const DevRays &R, int32_t o_begin, int32_t o_end,
                       const int64_t *offs, int64_t base, int64_t cap, int32_t *idx, double *Z, double *delta,
                       int *status, cudaStream_t st);
// padded layout (see k_trace.cu): rows [n_half][pad], lengths, excess over
// pad, walk state after the row for the half-rays longer than it
void launch_trace_pad(const DevMesh &m, const DevRays &R, int32_t o_begin, int32_t o_end, int32_t pad,
                      int64_t *lens, int64_t *excess, int4 *resume, int32_t *rows, int *status,
                      unsigned long long *counters, cudaStream_t st, int ctas_per_sm = 0);
void launch_trace_tail(const DevMesh &m, const DevRays &R, int32_t o_begin, int32_t o_end, int32_t pad,
                       const int64_t *lens, const int4 *resume, const int64_t *offs, int64_t base, int64_t cap,
                       int32_t *tail, int *status, cudaStream_t st, int ctas_per_sm = 0);

// One model of a batched solve (device-resident descriptor).
struct BatchSlot {
    DevMesh m;
    DevLines Ln;
    DevRays R;
    SolveArgs a;  // o_begin = 0, o_end = n; offsets into the batch's shared arena
};

// Geometry of one model of a batch: its half-rays start at half_base in the
// batch's offset array, 2 npairs per origin, n_tiles frequency tiles.
struct BatchGeom {
    int64_t half_base;
    int32_t npairs2;
    int32_t n_tiles;
    int64_t work_base;  // first work item of the model in plain order
};

// ---- batched work list (k_batch.cu)
// Work list from the half-ray lengths lens (all models' half-rays, in order).
// Buffers of the cost-binned work list: sort keys and values [n_origins] (in
// and out), item counts and their inclusive prefix sums [n_origins], CUB
// temporary storage of batch_worklist_temp_bytes(n_origins) bytes.
struct WorkListBufs {
    uint8_t *key_in = nullptr, *key_out = nullptr;
    int32_t *val_in = nullptr, *val_out = nullptr;
    int64_t *tiles = nullptr, *toff = nullptr;
    void *tmp = nullptr;
    size_t tmp_bytes = 0;
};
size_t batch_worklist_temp_bytes(int64_t n_origins);
// (natural: plain (model, origin, tile) order instead of the cost bins)
void launch_batch_worklist(const BatchGeom *geo, const int64_t *origin_base, int32_t n_models, int64_t n_origins,
                           const int64_t *lens, const WorkListBufs &b, uint2 *work, bool natural, cudaStream_t st);
// Row widths 2^j (j < kPadCandidates) considered for the padded layout:
// out[j] = sum over half-rays of max(0, len - 2^j), out[kPadCandidates] = sum of len.
constexpr int kPadCandidates = 11;
void launch_excess_totals(const int64_t *lens, int64_t n, unsigned long long *out, cudaStream_t st);

// ---- formal solution (k_solve.cu)
// frequency bins per lane of the solve kernel; a chunk has
// ceil(n_bins / (32 * bins_per_lane)) tiles per origin
int solve_bins_per_lane(int precision, int32_t n_bins);
// order: 2 (second-order scheme) or 4 (Hermitian scheme)
void launch_solve(const DevMesh &m, const DevLines &Ln, const DevRays &R, const SolveArgs &a,
                  int precision, int order, cudaStream_t st);
// persistent launch over a work list (x = model << 16 | tile, y = origin); next: zeroed counter
void launch_solve_queue(int precision, int order, int bins_per_lane, int max_lines, const BatchSlot *slots,
                        const uint2 *work, int64_t n_work, unsigned long long *next, cudaStream_t st);
// the single-precision form with double-precision increments and pivots
// (MGX_FP32_DT64, second-order scheme; k_solve_mix.cu)
void launch_solve_dt64(const DevMesh &m, const DevLines &Ln, const DevRays &R, const SolveArgs &a, int bins_per_lane,
                       cudaStream_t st);
void launch_solve_queue_dt64(int bins_per_lane, int max_lines, const BatchSlot *slots, const uint2 *work,
                             int64_t n_work, unsigned long long *next, cudaStream_t st);
// the two instantiations (k_solve.cu, k_solve_herm.cu)
template <int ORD>
void launch_solve_ord(const DevMesh &m, const DevLines &Ln, const DevRays &R, const SolveArgs &a, int precision,
                      cudaStream_t st);
template <int ORD>
void launch_solve_queue_ord(int precision, int bins_per_lane, int max_lines, const BatchSlot *slots,
                            const uint2 *work, int64_t n_work, unsigned long long *next, cudaStream_t st);

// SplitMix64 (Steele, Lea & Flood 2014) started at seed + (i+1) * golden gamma,
// its top 53 bits as a uniform in [0, 1): the thinning coin of point i.
__device__ __forceinline__ double splitmix_uniform(uint64_t seed, int64_t i) {
    uint64_t z = seed + uint64_t(i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return __dmul_rn(double(z >> 11), 1.0 / 9007199254740992.0);
}

// ---- element-size field of an analytic model (k_analytic.cu); mm[0], mm[1]:
// bits of the smallest and largest Gf (non-negative doubles order as integers),
// kept: number of kept points
void launch_size_field(int32_t nx, int32_t ny, int32_t nz, const double *f, double h, double *Gf,
                       unsigned long long *mm, cudaStream_t st);
void launch_size_map(int64_t n, const double *Gf, const unsigned long long *mm, double h, double ell_min,
                     double ell_max, uint64_t seed, double *ell, uint8_t *keep, unsigned long long *kept,
                     cudaStream_t st);

// ---- score-weighted thinning (k_thin.cu): w = 10^(alpha y); expected kept
// count for a scale c; the coin flips
void launch_thin_weights(const float *y, int64_t n, float alpha, float *w, cudaStream_t st);
void launch_thin_expected(const float *w, int64_t n, double c, double *sum, cudaStream_t st);
void launch_thin_mark(const float *w, int64_t n, double c, uint64_t seed, uint8_t *keep, unsigned long long *kept,
                      cudaStream_t st);

// ---- reduction criterion (k_reduce.cu)
void launch_reduce(const DevMesh &m, const double *f, double f_small, double f_large,
                   double G_thres, uint64_t seed, double *Gf, double *L, double *ell,
                   uint8_t *keep, cudaStream_t st);

// ---- allocation-free solve with a fixed scratch array (noalloc.cu)
int noalloc_solve(int device, const DevMesh &m, const DevLines &Ln, const DevRays &R, double dtau_max,
                  double dv_max, double I_bdy, int precision, int order, double *J, int *status, cudaStream_t st,
                  char *err, size_t errlen);

// ---- learned reduction network (k_mlp.cu); parameter offsets in theta
constexpr int kMlpW1 = 0, kMlpB1 = 512, kMlpW2 = 576, kMlpB2 = 4672, kMlpW3 = 4736, kMlpB3 = 4800, kMlpN = 4801;
size_t mlp_smem_bytes();
void launch_mlp_convert(const float *theta, void *W1b, void *W2b, cudaStream_t st);
// train == false: y[r] = network(X[perm[r]]); train == true: adds the gradient of
// sum_r (y - t)^2 * inv_batch / 2 ... scaled so that inv_batch = 2 / B gives the MSE gradient
void launch_mlp(bool train, const float *X, const float *t, const int32_t *perm, int64_t rows, const void *W1b,
                const void *W2b, const float *theta, float *y, float *grad, float *loss, float inv_batch,
                cudaStream_t st);
void launch_mlp_adam(float *theta, float *m, float *v, float *grad, float lr, float b1, float b2, float eps, float c1,
                     float c2, void *W1b, void *W2b, cudaStream_t st);
void launch_mlp_features(const DevMesh &m, const float *chi0, int32_t L, const float *dvw, const double *rho,
                         const double *T, float *X, cudaStream_t st);
void launch_select_top(const float *score, int64_t n, int64_t k, int32_t *ids, float *score_sorted,
                       int32_t *ids_sorted, uint8_t *keep, cudaStream_t st);

// ---- approximate single-precision functions of the solve (k_approx.cu):
// kind 0: 2^x (ex2.approx.ftz.f32), kind 1: 1/x (rcp.approx.ftz.f32); and the
// relative error bound the solve's decisions take for each
void launch_eval_approx(int kind, const float *x, int64_t n, float *y, cudaStream_t st);
float approx_bound(int kind);
void launch_eval_atan2(const float *x, int64_t n, float *y, cudaStream_t st);  // k_rays.cu
float atan2_bound();

// ---- arithmetic-pipe throughput microbenchmarks (k_peaks.cu)
cudaError_t alu_peaks(cudaStream_t st, int reps, double out[4]);

// ---- host HEALPix tables (hpx_host.cpp)
int64_t hpx_npix(int l);
void hpx_pix2vec(int l, int64_t p, double v[3]);
int64_t hpx_vec2pix(int l, const double d[3]);
int64_t rayset_npairs(int lmin, int lmax);

}  // namespace mgx
