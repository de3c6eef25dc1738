/*
 * mgx.h -- C ABI of the GB300 radiation-field library (libmgx.so).
 *
 * The library computes, for every point of a 3-D point-cloud mesh, the mean
 * intensity J of a set of spectral lines, following De Ceuster et al. (2020),
 * "Magritte II: adaptive ray-tracing, mesh construction and reduction":
 *   ray set    -- hierarchical, mesh-adaptive HEALPix directions (Section 2.1.3, Eq. 4)
 *   trace      -- point-to-point long characteristics (Section 2.1, Fig. 2)
 *   line data  -- Doppler-shifted opacity/emissivity with adaptive velocity and
 *                 optical-depth sampling (Sections 2.1.1-2.1.2, Eq. 2)
 *   solve      -- second-order Feautrier transfer equation per ray pair and
 *                 frequency bin (Eq. 1)
 *   J          -- direction-weighted mean intensity (Eq. 3)
 *   reduction  -- the re-meshing criterion of Section 2.2.2 (Eqs. 6-8, Table 1)
 *
 * Conventions for every call:
 *   - Every function returns an mgx_status; 0 is success, negative is an error.
 *     A failing call leaves outputs undefined and stores a message retrievable
 *     with mgx_last_error().  No function throws or aborts.
 *   - Arguments are validated on the host before anything is launched.
 *   - Input arrays are host pointers unless stated otherwise; the library copies
 *     them, the caller keeps ownership.  Device memory allocated by the library
 *     belongs to the context and is released by mgx_free_model / mgx_destroy.
 *   - All work is enqueued on the CUDA stream given to mgx_create.  Calls that
 *     return host results synchronise that stream; calls with device outputs do
 *     not (the caller orders further work on the same stream).
 *   - A context is not thread-safe: use one context per host thread.
 *   - Array layouts are C order; [n][3] means 3 consecutive values per point.
 */
#ifndef MGX_H
#define MGX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mgx_ctx mgx_ctx;
typedef int32_t mgx_status;

enum {
    MGX_OK = 0,
    MGX_EINVAL = -1, /* bad argument (null pointer, size, index out of range, NaN) */
    MGX_ENOMEM = -2, /* device allocation failed                                   */
    MGX_ECUDA = -3,  /* CUDA runtime error (message has the CUDA error string)     */
    MGX_ESTATE = -4, /* call out of order (e.g. solve before set_lines)            */
    MGX_ERANGE = -6  /* a size limit was exceeded (message says which)             */
};

/* arithmetic forms of the formal solution */
enum {
    MGX_FP64 = 0, /* plain form: every step in double precision                    */
    MGX_FP32 = 1, /* single-precision bulk; double for the distance increments along
                     the ray and the compensated J sum.  The integer decisions (the
                     velocity-sample count of Section 2.1.1, Eq. 2's n_inter) are
                     the double-precision definition's: taken in single precision
                     under a rigorous error bound, redone in double precision
                     where the bound leaves the integer open                        */
    MGX_FP32_DT64 = 2 /* MGX_FP32 with the optical-depth increments and the pivot
                     recurrence of the elimination (Fh and D of the scaled 1+B form)
                     also in double precision, z and S in single precision; second-
                     order scheme only (order 4 gives MGX_EINVAL)                    */
};

/* Limits. */
#define MGX_MAX_LINES 8      /* spectral lines per model                          */
#define MGX_MAX_LEVEL 8      /* HEALPix level of a fixed ray set (nside 256)      */
#define MGX_MAX_ADAPT_LEVEL 5 /* finest level of an adaptive ray set (nside 32)   */

typedef struct {
    double dtau_max;       /* Eq. 2: largest optical-depth increment (> 0)              */
    double dv_max;         /* Section 2.1.1: largest change of projected velocity between
                              consecutive samples, in units of the smaller of their two
                              Doppler widths; <= 0 disables velocity sampling             */
    double I_bdy;          /* intensity entering both ends of every ray                  */
    int32_t precision;     /* MGX_FP64 or MGX_FP32                                       */
    int32_t out_on_device; /* nonzero: J_out is a device pointer on the context's device */
    int32_t order;         /* discretisation of Eq. 1 (Section 2.1): 0 or 2, the second-order
                              scheme with second-order boundary conditions; 4, the Hermitian
                              fourth-order scheme of Auer (1976) with third-order boundary
                              conditions; anything else gives MGX_EINVAL                  */
    int32_t reserved;      /* 0 */
} mgx_solve_params;

/* Create a context on CUDA device `device`, enqueuing on `stream` (a cudaStream_t;
 * NULL selects the legacy default stream).  Library lifecycle: no counterpart in
 * the paper. */
mgx_status mgx_create(int device, void *stream, mgx_ctx **out);

/* Release the context and every model in it.  NULL is allowed.  Library
 * lifecycle: no counterpart in the paper. */
void mgx_destroy(mgx_ctx *ctx);

/* Message of the last failing call on this context ("" if none).  The pointer
 * stays valid until the next call on the context. */
const char *mgx_last_error(const mgx_ctx *ctx);

/* Number of ray pairs of a ray set spanning levels l_min..l_max (Section 2.1.3):
 * 6*4^l for a fixed level; otherwise the top half of the candidate pairs is
 * refined at each level, e.g. 276 pairs (552 rays) for l_min = 1, l_max = 4.
 * Returns -1 for invalid levels. */
int64_t mgx_rayset_npairs(int32_t l_min, int32_t l_max);

/* HEALPix nested scheme (Gorski et al. 2005), host only: the unit vector of the
 * centre of pixel p of level l (v [3]), and the pixel containing -v (its
 * antipode).  Return 0 / the antipode, or -1 for l outside 0..MGX_MAX_LEVEL or
 * p outside 0..12*4^l-1 (or a null v). */
int32_t mgx_pix2vec(int32_t l, int64_t p, double *v);
int64_t mgx_antipode(int32_t l, int64_t p);

/* Load a point cloud with its neighbour graph (Section 2.2: "a point cloud and
 * nearest neighbour information").
 *   n        number of points, 1 <= n < 2^31
 *   pos      [n][3] positions, |coordinate| <= 1e30 (any length unit; opacities are per
 *            that unit)
 *   vel      [n][3] velocities in km/s
 *   nbr_off  [n+1] CSR row offsets, nbr_off[0] = 0, non-decreasing, total < 2^31
 *   nbr_idx  [nbr_off[n]] neighbour indices in [0, n), no self references
 * On success *model_id receives the model handle (>= 0). */
mgx_status mgx_load_mesh(mgx_ctx *ctx, int64_t n, const double *pos, const double *vel,
                         const int64_t *nbr_off, const int32_t *nbr_idx, int32_t *model_id);

/* Release a model's device memory.  The handle becomes invalid. */
mgx_status mgx_free_model(mgx_ctx *ctx, int32_t model);

/* Line data of a model (Sections 2.1.1-2.1.2; the profile is the Gaussian of
 * Magritte I with its normalisation folded into chi0 and eta0).
 *   n_lines   1..MGX_MAX_LINES
 *   nu0       [n_lines] line-centre frequencies (> 0)
 *   chi0      [n][n_lines] line-centre opacities (>= 0)
 *   eta0      [n][n_lines] line-centre emissivities (>= 0)
 *   dvw       [n] Doppler widths in km/s (> 0)
 *   chi_c     [n] continuum opacities (> 0; keeps every optical depth positive)
 *   eta_c     [n] continuum emissivities (>= 0)
 *   n_freq    bins per line (>= 1): bin k of line l sits at
 *             nu = nu0[l] (1 + x_k dvw[o] / c) in the comoving frame of the origin o,
 *             x_k uniform on [-x_span, x_span] (x_0 = 0 if n_freq == 1)
 *   x_span    >= 0
 * J has n_lines*n_freq values per point, index l*n_freq + k. */
mgx_status mgx_set_lines(mgx_ctx *ctx, int32_t model, int32_t n_lines, const double *nu0,
                         const double *chi0, const double *eta0, const double *dvw,
                         const double *chi_c, const double *eta_c, int32_t n_freq, double x_span);

/* Build the ray set of every point (Section 2.1.3, Eq. 4, Fig. 1).
 * l_min == l_max selects the fixed HEALPix set of that level (0..MGX_MAX_LEVEL).
 * l_min < l_max (l_max <= MGX_MAX_ADAPT_LEVEL) builds the adaptive set: the
 * directions from the point to the sample points are counted per pixel, and at
 * each level the top half of the candidate antipodal pairs (by count, ties to
 * the smaller nested index) is refined.  `sample` [n_sample] holds the indices
 * of the global sample of points (the paper draws 10 000); the point itself and
 * coincident points are skipped.  sample may be NULL when l_min == l_max.
 * Each ray pair is stored as (level << 28) | nested pixel of the member with
 * the smaller index; the pair's rays point along +r and -r, r = that pixel's
 * centre; its weight is 2/(12 * 4^level). */
mgx_status mgx_set_rays(mgx_ctx *ctx, int32_t model, int32_t l_min, int32_t l_max,
                        int64_t n_sample, const int32_t *sample);

/* Copy the ray sets to the host: out [n][mgx_rayset_npairs(l_min, l_max)],
 * pairs of each point sorted ascending. */
mgx_status mgx_get_rays(mgx_ctx *ctx, int32_t model, uint32_t *out);

/* Trace the ray pairs of origins [o_begin, o_end) (Section 2.1, Fig. 2): from
 * the current point, step to the neighbour that lies strictly further along the
 * ray and closest to it (ties to the smaller index), until there is none.
 * Half-ray h = ((o - o_begin) * npairs + p) * 2 + s, s = 0 along -r, 1 along +r.
 *   off_out    [2*npairs*(o_end-o_begin) + 1] host: entries of half-ray h are
 *              [off_out[h], off_out[h+1]) in the arrays below (always written)
 *   idx_out    [capacity] point indices in trace order (may be NULL)
 *   Z_out      [capacity] projected distances (x_n - x_o).d, bit-exact double
 *   delta_out  [capacity] projected velocity differences (v_n - v_o).d in km/s
 *              (double; may be NULL)
 * If idx_out is NULL only off_out is filled.  If capacity < off_out[last] the
 * call fails with MGX_ERANGE after filling off_out. */
mgx_status mgx_trace(mgx_ctx *ctx, int32_t model, int64_t o_begin, int64_t o_end,
                     int64_t *off_out, int32_t *idx_out, double *Z_out, double *delta_out,
                     int64_t capacity);

/* Mean intensity of every point of a model (Eqs. 1-3): traces all ray pairs,
 * samples velocities and optical depths, solves the Feautrier equation for
 * every bin, and sums 2 w u over the pairs in ascending pair order with
 * compensated (Neumaier) double-precision summation.
 *   J_out  [n][n_lines*n_freq] doubles, host or device per params->out_on_device
 * The call synchronises the stream (the tracer's total length sizes the
 * point-list arena; device-side checks are reported before returning).  Origins
 * are processed in chunks whose traced point ids fit a 16 GiB arena.  The first
 * call on a model counts the traced length of every half-ray and keeps the
 * prefix sums with the model ((2 n npairs + 1) x 8 bytes of device memory)
 * until mgx_set_rays or mgx_free_model; later calls trace and solve without
 * the counting pass. */
mgx_status mgx_solve_J(mgx_ctx *ctx, int32_t model, const mgx_solve_params *params, void *J_out);

/* Mesh-reduction criterion of Section 2.2.2 with tracer f (Eqs. 6-8):
 *   Gf_i  = max over neighbours n of |(f_i - f_n)/(f_i + f_n)|  (0 if f_i + f_n = 0)
 *   L_i   = mean distance to the neighbours (0 without neighbours)
 *   ell_i = L_i * (f_small if Gf_i >= G_thres else f_large)
 * The Gmsh re-meshing of the paper is replaced by thinning: point i is kept if
 * u_i < min(1, (L_i/ell_i)^3) with u_i the SplitMix64 uniform of (seed, i)
 * (state seed + (i+1)*0x9E3779B97F4A7C15, top 53 bits), or if it has no
 * neighbours.  f [n] host; outputs [n] host (any may be NULL except keep);
 * *n_kept receives the number of kept points. */
mgx_status mgx_reduce_mesh(mgx_ctx *ctx, int32_t model, const double *f, double f_small,
                           double f_large, double G_thres, uint64_t seed, double *Gf, double *L,
                           double *ell, uint8_t *keep, int64_t *n_kept);

/* u at the origin of every pair line (Eq. 1 solved per ray pair and bin, the
 * quantity that Eq. 3-4 weight into J), for origins [o_begin, o_end):
 * u_out [o_end - o_begin][n_pairs][n_lines*n_freq], host or device as
 * params->out_on_device says.  Same parameters and errors as mgx_solve_J; the
 * traced lists of the range must fit the context's arena (16 GiB), else
 * MGX_ERANGE (split the range). */
mgx_status mgx_solve_u(mgx_ctx *ctx, int32_t model, const mgx_solve_params *params, int64_t o_begin,
                       int64_t o_end, double *u_out);

/* Learned reduction by weighted thinning (the learned variant of Section
 * 2.2.2's random thinning; no counterpart in the paper).  With y_i the network's
 * prediction for the features X [n][8] (as in mgx_reduce_mesh_learned), point i
 * is kept when u_i < min(1, c 10^(alpha y_i)), u_i the SplitMix64 uniform of
 * (seed, i) as in mgx_reduce_mesh, and c the scale at which the expected kept
 * count sum_i min(1, c 10^(alpha y_i)) equals keep_fraction * n (bisection on
 * log2 c).  alpha = 0 is uniform thinning.  keep [n] host; *n_kept and *scale
 * (c) may be NULL.  Requires 0 <= keep_fraction <= 1, alpha finite and >= 0,
 * and parameters set (mgx_mlp_set_params) else MGX_ESTATE. */
mgx_status mgx_reduce_mesh_learned_weighted(mgx_ctx *ctx, int32_t model, const float *X, double keep_fraction,
                                            double alpha, uint64_t seed, uint8_t *keep, int64_t *n_kept,
                                            double *scale);

/* Element-size field of an analytic model and its mesh (Section 2.2.1, Eq. 5).
 * f [nx][ny][nz] (index (i*ny + j)*nz + k, host, every value finite and > 0)
 * is the tracer at the points of a regular Cartesian background mesh of
 * spacing h.  For every point:
 *   Gf = ||grad f|| / f  (the maximal relative change of Eq. 5), the gradient by
 *        central differences, first differences on the faces, 0 along an axis
 *        with a single point;
 *   ell = ell_max - (Gf - min Gf)(ell_max - ell_min) / (max Gf - min Gf), the
 *        linear map of [max Gf, min Gf] onto [ell_min, ell_max] (ell_max
 *        everywhere when Gf is constant);
 *   keep = u < (h / ell)^3, u the SplitMix64 uniform of (seed, point index) as
 *        in mgx_reduce_mesh: the background mesh (point density h^-3) thinned to
 *        the density ell^-3, in place of the paper's Gmsh meshing.
 * Requires nx, ny, nz >= 1 and 0 < h <= ell_min <= ell_max (the background
 * resolves the smallest desired element).  Gf, ell [n] (may be NULL) and keep [n] are host outputs;
 * *n_kept (may be NULL) receives the number kept.  Every operation is
 * explicitly rounded: the outputs are reproducible bit for bit. */
mgx_status mgx_analytic_mesh(mgx_ctx *ctx, int32_t nx, int32_t ny, int32_t nz, const double *f, double h,
                             double ell_min, double ell_max, uint64_t seed, double *Gf, double *ell,
                             uint8_t *keep, int64_t *n_kept);

/* Flags of mgx_solve_J_batch. */
enum {
    MGX_BATCH_GRAPH = 1, /* capture the step in a CUDA graph and replay it on later calls */
    MGX_BATCH_RAYS = 2   /* rebuild every model's ray set first (its last levels and sample) */
};

/* Mean intensity of several models in one launch (the batched form of
 * mgx_solve_J, Eqs. 1-3 of Section 2.1, same results; the batching itself has no
 * counterpart in the paper).  All models' half-rays are traced together into
 * fixed-width rows (the width chosen from the length distribution when the
 * call plans) plus a packed overflow for the longer ones; each (model, origin,
 * frequency tile) item's cost is the number of points on its traced lines,
 * items are binned by log2 of that cost and laid out longest bin first, and
 * one persistent kernel (one warp per item, items taken from a global counter)
 * solves them all, so very uneven ray lengths and model sizes share the GPU
 * without a long tail.  Launch parameters come from the context's tuning
 * (mgx_set_tuning / mgx_autotune).
 *   models  [n_models] distinct model handles (1..65535), lines and rays set
 *   J_out   [n_models] outputs, J_out[k] of size [n_k][n_lines_k*n_freq_k]: device
 *           memory of the context's device, or host memory (pageable or pinned),
 *           which the call stages in device memory that the plan owns and
 *           copies back (one copy per model, on the context's stream) after
 *           each step; a graph replay then copies too
 *   flags   MGX_BATCH_RAYS: the step starts by rebuilding the ray sets;
 *           MGX_BATCH_GRAPH: the first call plans the layout (the row width
 *           from the traced lengths of a sample of the origins, the tail from
 *           the first step's own padded trace: two host synchronisations),
 *           runs the step and captures it as a CUDA graph;
 *           later calls with the same models, parameters, outputs, flags and
 *           tuning replay the graph without host work.  A replay whose traced
 *           lists no longer fit the planned layout fails with MGX_ERANGE and
 *           drops the plan.  Freeing a model drops the plan.
 * The call synchronises the stream before returning. */
mgx_status mgx_solve_J_batch(mgx_ctx *ctx, const int32_t *models, int32_t n_models, const mgx_solve_params *params,
                             double *const *J_out, int32_t flags);

/* Launch parameters of the batched solve (no counterpart in the paper).  The
 * tracer grid and the row width change only the speed of mgx_solve_J_batch;
 * the bins per lane select a differently compiled single-precision kernel,
 * whose J may differ from the other's in its rounding (about 1e-8 relative:
 * the compilers' fused multiply-adds differ), never beyond that. */
typedef struct {
    int32_t bins_per_lane;     /* single-precision frequency bins per lane: 0 automatic (2 above 32 bins), 1, 2 */
    int32_t trace_ctas_per_sm; /* resident tracer CTAs of 128 threads per SM: 0 = 7, else 1..32 (capped at
                                  what fits) */
    int32_t tail_permille;     /* row width of the traced lists: the narrowest power of two leaving at most this
                                  share of the points (per mille) to the overflow pass; 0 = 20, else 1..1000 */
    int32_t schedule;          /* order of the persistent solve's work list: 0, items binned by log2 of
                                  their traced length, longest bin first; 1, plain (model, origin,
                                  tile) order (for comparison) */
} mgx_tuning;

/* Set (NULL: reset to automatic) or read the context's tuning; out-of-range
 * fields give MGX_EINVAL.  Setting it drops a planned batch.  Launch tuning of
 * the batched solve: no counterpart in the paper. */
mgx_status mgx_set_tuning(mgx_ctx *ctx, const mgx_tuning *tuning);
mgx_status mgx_get_tuning(mgx_ctx *ctx, mgx_tuning *tuning);

/* One timed candidate of mgx_autotune. */
typedef struct {
    mgx_tuning tuning;
    double step_ms; /* median device time of one step (CUDA events on the context's stream) */
} mgx_tune_trial;

/* Autotuner of the batched solve (no counterpart in the paper): times candidate tunings of
 * mgx_solve_J_batch(ctx, models, n_models, params, J_out, flags) by coordinate
 * descent (bins per lane 1/2 in single precision, tracer CTAs per SM 4/6/8,
 * tail share 5/20/80 per mille, work-list schedule 0/1), each candidate planned once and then run
 * `reps` times (1..100), and leaves the fastest as the context's tuning.
 * J_out receives the solution of the chosen tuning.  trials
 * [max_trials] (may be NULL) receives the timed candidates in order, *n_trials
 * their number.  Same argument rules and errors as mgx_solve_J_batch. */
mgx_status mgx_autotune(mgx_ctx *ctx, const int32_t *models, int32_t n_models, const mgx_solve_params *params,
                        double *const *J_out, int32_t flags, int32_t reps, mgx_tune_trial *trials,
                        int32_t max_trials, int32_t *n_trials);

/* Allocation-free variant of mgx_solve_J, for callers that must not allocate
 * device memory during their step: code running while a framework owns every
 * device byte and forbids third-party allocations, or code that may not enqueue
 * allocations at all.  The paper has no counterpart; this is a property of the
 * library.  Same inputs and result as mgx_solve_J, but J_out must be a device
 * pointer ([n][n_lines*n_freq] doubles; params->out_on_device is ignored), and
 * the working memory (half-ray lengths and offsets, traced point lists) comes
 * from one fixed 64 MiB device array compiled into the library instead of an
 * allocation.  Origins are processed in chunks that fit it; the call fails with
 * MGX_ERANGE when the ray set has too many pairs for the array or when one
 * origin's traced point lists alone do not fit (more than about 14 million
 * points).  No cudaMalloc, cudaFree or allocating library routine is called.
 * The first call on a device looks up the array's device address (set-up);
 * make that first call before any stream capture.  For every chunk the call
 * reads the traced total back to the host and synchronises the stream.  Every call
 * shares the array: calls that overlap on the GPU (other streams or contexts
 * on the same device) race on it. */
mgx_status mgx_solve_J_noalloc(mgx_ctx *ctx, int32_t model, const mgx_solve_params *params,
                               double *J_out);

/* Learned mesh reduction (a learned companion to the criterion of Section
 * 2.2.2; the paper has no network).  A small MLP, 8 -> 64 -> 64 -> 1 with ReLU,
 * predicts from eight per-point features how much J error dropping a point
 * causes; mgx_reduce_mesh_learned keeps the points with the largest
 * prediction.  Parameters are one FP32 vector of MGX_MLP_NPARAM values:
 * W1 [8][64], b1 [64], W2 [64][64], b2 [64], W3 [64], b3 [1]
 * (h1 = relu(x W1 + b1), h2 = relu(h1 W2 + b2), y = h2 . W3 + b3).
 * The kernels compute the two hidden products on the tensor cores in bfloat16
 * (inputs, W1, W2, h1 and the back-propagated hidden gradients rounded to
 * bfloat16) with FP32 accumulation; everything else is FP32.  The loss is the
 * mean squared error; training uses Adam (beta1 0.9, beta2 0.999, eps 1e-8)
 * on the FP32 master parameters. */
#define MGX_MLP_NPARAM 4801

/* Set the parameters (host [MGX_MLP_NPARAM]); resets the optimiser state. */
mgx_status mgx_mlp_set_params(mgx_ctx *ctx, const float *theta);
/* Copy the current parameters to the host. */
mgx_status mgx_mlp_get_params(mgx_ctx *ctx, float *theta);
/* y [n] = network(X [n][8]) (host arrays): the learned reduction's network,
 * which the paper does not have. */
mgx_status mgx_mlp_forward(mgx_ctx *ctx, const float *X, int64_t n, float *y);
/* Training of the learned reduction's network (no counterpart in the paper).
 * Gradient of the mean squared error over all n rows (one batch), host
 * [MGX_MLP_NPARAM]; *loss (may be NULL) receives the loss.  No update. */
mgx_status mgx_mlp_grad(mgx_ctx *ctx, const float *X, const float *t, int64_t n, float *grad, float *loss);
/* Training of the learned reduction's network (no counterpart in the paper):
 * Adam for `epochs` passes in shuffled mini-batches of `batch` rows
 * (shuffles from SplitMix64 seeded with `seed`); loss_per_epoch [epochs]
 * (may be NULL) receives each epoch's mean loss. */
mgx_status mgx_mlp_train(mgx_ctx *ctx, const float *X, const float *t, int64_t n, int32_t epochs, int32_t batch,
                         float lr, uint64_t seed, float *loss_per_epoch);
/* Per-point features X [n][8] (host output) of a model with lines set, from
 * its density rho [n] and temperature T [n] (host, > 0): log rho, the largest
 * |log rho contrast| to a neighbour, the largest neighbour velocity difference
 * in local Doppler widths, log T, log of the mean neighbour distance L (Eq. 8),
 * neighbour count, log distance from the coordinate origin, and log of the
 * first line's centre opacity times L. */
mgx_status mgx_mlp_features(mgx_ctx *ctx, int32_t model, const double *rho, const double *T, float *X);
/* Keep the round(keep_fraction * n) points with the largest network output
 * for standardised features X [n][8] (host): keep [n] (host) receives 1/0,
 * *n_kept the count.  Ties go to the smaller index. */
mgx_status mgx_reduce_mesh_learned(mgx_ctx *ctx, int32_t model, const float *X, double keep_fraction, uint8_t *keep,
                                   int64_t *n_kept);

/* The approximate single-precision functions of the single-precision solve and
 * ray-set screen, for tests of the error bounds their integer decisions
 * (velocity-sample counts, Eq. 2 sub-interval counts, HEALPix pixels) are
 * certified with; no counterpart in the paper.  kind 0: y = 2^x as the solve
 * evaluates exp(-a^2); kind 1: y = 1/x; kind 2: y[i] = atan2f(x[n + i], x[i])
 * as the ray set's single-precision vec2pix evaluates the azimuth (x holds 2n
 * values: the n x-components, then the n y-components).  x, y are device
 * pointers on the context's device; the work is enqueued on the context's
 * stream (no synchronisation).  *bound (may be NULL) receives the largest
 * error the certification assumes for that function: relative for kinds 0 and
 * 1, absolute (radians) for kind 2.  MGX_EINVAL for another kind, n < 0, or
 * null arrays with n > 0. */
mgx_status mgx_eval_approx(mgx_ctx *ctx, int32_t kind, const float *x, int64_t n, float *y, float *bound);

/* Measured throughput of the arithmetic pipes the formal solution runs on (no
 * counterpart in the paper; the denominators of its roofline): out[0] FP32
 * fused multiply-add TFLOP/s (two flops each), out[1] FP64 fused multiply-add
 * TFLOP/s, out[2] approximate exp2 and out[3] approximate reciprocal, each in
 * Gop/s; every figure is the best of `reps` (1..100) timed launches of eight
 * independent dependency chains per thread on every SM (CUDA events on the
 * context's stream).  Allocates and frees a small device buffer; synchronises
 * the stream.  Takes about a second. */
mgx_status mgx_alu_peaks(mgx_ctx *ctx, int32_t reps, double *out);

/* Kernel-level profiling.  While enabled, every kernel launch of the context is
 * bracketed by CUDA events on the context's stream and the work counters below
 * are accumulated on the device; mgx_profile_read synchronises the stream and
 * returns the totals since the last mgx_profile_enable(ctx, 1). */
enum {
    MGX_K_RAYS = 0,        /* ray-set construction                          */
    MGX_K_TRACE_COUNT = 1, /* tracer, counting pass                          */
    MGX_K_SCAN = 2,        /* prefix sum of half-ray lengths                 */
    MGX_K_TRACE_EMIT = 3,  /* tracer, emitting pass                          */
    MGX_K_SOLVE = 4,       /* formal solution and J                          */
    MGX_K_OTHER = 5,       /* ingest, reduction                              */
    MGX_K_COUNT = 6
};

typedef struct {
    double ms[MGX_K_COUNT];        /* summed device time per kernel class (ms)      */
    int64_t launches[MGX_K_COUNT]; /* kernel launches per class                      */
    int64_t trace_points;          /* points emitted by the tracer (emit pass)       */
    int64_t solves;                /* (origin, ray pair, bin) Feautrier solutions     */
    int64_t updates;               /* (bin, optical-depth sub-interval) elimination steps */
    int64_t samples;               /* (bin, velocity sample) line-optics evaluations  */
    int64_t trace_steps;           /* tracer steps of the counting pass               */
    int64_t trace_exact_steps;     /* of those, steps the single-precision screen could
                                      not decide, redone in double precision          */
    int64_t decisions_redone;      /* integer decisions of the single-precision solve (velocity-
                                      sample counts, Eq. 2 sub-interval counts) that its error
                                      bound left open, redone in double precision     */
} mgx_profile;

/* enable != 0 starts (and resets) profiling; 0 stops it. */
mgx_status mgx_profile_enable(mgx_ctx *ctx, int32_t enable);

/* Totals since profiling was enabled (synchronises the stream). */
mgx_status mgx_profile_read(mgx_ctx *ctx, mgx_profile *out);

#ifdef __cplusplus
}
#endif

#endif /* MGX_H */
