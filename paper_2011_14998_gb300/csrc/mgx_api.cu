// mgx_api.cu -- host side of the C ABI declared in include/mgx.h.
//
// Owns the per-context device state (models, HEALPix tables, status word),
// validates arguments, moves data, sequences the kernels of k_*.cu and maps
// device-side error codes to mgx_status values.  No arithmetic of the method
// runs here except building the constant HEALPix direction/antipode tables.
#include <cub/device/device_scan.cuh>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "mgx_internal.cuh"

using namespace mgx;

namespace {

constexpr int kCounters = 8;  // device work counters of a context (see mgx_ctx::d_counters)

struct Model {
    bool live = false;
    int32_t n = 0;
    int64_t E = 0;
    // mesh
    double *x = nullptr, *y = nullptr, *z = nullptr, *vx = nullptr, *vy = nullptr, *vz = nullptr;
    float *vxf = nullptr, *vyf = nullptr, *vzf = nullptr;
    int32_t *off = nullptr, *nbr = nullptr;
    float4 *phi = nullptr, *nrec = nullptr;
    float g0 = 0.0f;
    // lines
    bool has_lines = false;
    int32_t L = 0, F = 0;
    double x_span = 0.0;
    double nu0[MGX_MAX_LINES] = {};
    double *chi0 = nullptr, *eta0 = nullptr, *dvw = nullptr, *chic = nullptr, *etac = nullptr;
    float *chi0f = nullptr, *eta0f = nullptr, *dvwf = nullptr, *chicf = nullptr, *etacf = nullptr;
    // rays
    bool has_rays = false;
    int32_t lmin = 0, lmax = 0, npairs = 0;
    uint32_t *rays = nullptr;
    int32_t *sample = nullptr;  // device copy of the ray-set sample (adaptive sets)
    int64_t n_sample = 0;
    // half-ray offsets of every origin, [2 n npairs + 1] on the device, and
    // their values at origin boundaries, [n + 1] on the host: made by the first
    // mgx_solve_J and kept until the ray set changes (the mesh never does)
    int64_t *offs_all = nullptr;
    std::vector<int64_t> obound;
};

// A batched solve kept for replay: its buffers and, in graph mode, the
// instantiated CUDA graph of the whole step.  Traced lists use the padded
// layout (k_trace.cu): rows of `pad` ids per half-ray plus a tail arena for
// the entries beyond the row, at the prefix sums (offs) of the excesses.
struct BatchPlan {
    bool valid = false;
    std::vector<int32_t> models;
    std::vector<double *> J;
    std::vector<double *> Jdev;   // device staging of an output in host memory (null: J[k] is device memory)
    std::vector<size_t> Jbytes;
    mgx_solve_params p{};
    int32_t flags = 0;
    int64_t total_half = 0, n_origins = 0, n_work = 0, tail_cap = 0, total_points = 0;
    int32_t pad = 0;
    int bpl = 1, max_lines = 1;
    mgx_tuning tune{};
    int64_t *lens = nullptr, *excess = nullptr, *offs = nullptr, *obase = nullptr;
    int32_t *rows = nullptr, *tail = nullptr;
    int4 *resume = nullptr;
    BatchGeom *geo = nullptr;
    BatchSlot *slots = nullptr;
    uint2 *work = nullptr;
    unsigned long long *scratch = nullptr;  // the queue counter, row-width totals
    WorkListBufs wl;
    void *cub_tmp = nullptr;
    size_t cub_bytes = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

}  // namespace

struct mgx_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    std::vector<Model> models;
    int *d_status = nullptr;
    int *h_status = nullptr;
    // HEALPix tables of levels 0..tab_level
    int tab_level = -1;
    double *dir = nullptr;    // [level_offset(tab_level+1)][3]
    float4 *dirf = nullptr;   // [level_offset(tab_level+1)], dir rounded to float
    int32_t *anti = nullptr;  // [level_offset(tab_level+1)]
    std::vector<std::vector<uint32_t>> pair_lists;  // per level, host
    std::vector<uint32_t *> pair_lists_dev;         // per level, device
    size_t arena_budget = size_t(16) << 30;
    // profiling
    bool prof = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[MGX_K_COUNT];
    int64_t launches[MGX_K_COUNT] = {};
    std::vector<cudaEvent_t> event_pool;
    unsigned long long *d_counters = nullptr;  // [0] updates, [1] samples, [2] trace steps, [3] redone,
                                               // [4] solve decisions redone in double, [5..7] spare
    int64_t trace_points = 0, solves = 0;
    BatchPlan plan;
    mgx_tuning tune{};  // launch parameters of the batched solve (zero: automatic)
    cudaStream_t capture_stream = nullptr;
    // learned reduction network: FP32 master parameters, Adam moments, gradient
    // accumulator, loss accumulator, bf16 copies of W1 (padded) and W2
    float *mlp_theta = nullptr, *mlp_m = nullptr, *mlp_v = nullptr, *mlp_grad = nullptr, *mlp_loss = nullptr;
    void *mlp_W1b = nullptr, *mlp_W2b = nullptr;
    int64_t mlp_step = 0;  // graphs are captured here (the caller's may be the legacy stream)
};

namespace {

struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess) ok = true;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

mgx_status fail(mgx_ctx *c, mgx_status code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

#define CK(call)                                                                                       \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) {                                                                       \
            cudaGetLastError();                                                                        \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? MGX_ENOMEM : MGX_ECUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                            \
        }                                                                                              \
    } while (0)

template <typename T>
cudaError_t dalloc(mgx_ctx *ctx, T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMallocAsync(reinterpret_cast<void **>(p), count * sizeof(T), ctx->stream);
}

template <typename T>
void dfree(mgx_ctx *ctx, T *&p) {
    if (p) cudaFreeAsync(p, ctx->stream);
    p = nullptr;
}

const char *dev_err_text(int code) {
    switch (code) {
        case kDevBadCsr: return "neighbour graph invalid (offsets not monotone or index out of range/self)";
        case kDevNonFinite: return "non-finite position or velocity, or a coordinate beyond 1e30";
        case kDevTraceGuard: return "tracer step guard hit";
        case kDevTraceMismatch: return "trace emit pass disagrees with count pass";
        case kDevSubdivLimit: return "more than 2^20 optical-depth sub-intervals in one step (dtau_max too small?)";
        case kDevBadInput: return "line data out of range (chi0, eta0 >= 0; dvw, chi_c > 0; eta_c >= 0; finite)";
        case kDevArenaOverflow: return "traced point lists longer than planned (mesh or rays changed since the plan?)";
        default: return "unknown device error";
    }
}

// Synchronise the stream and turn a device status into an mgx_status.
mgx_status sync_status(mgx_ctx *ctx) {
    CK(cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const int code = *ctx->h_status;
    if (code != 0) {
        const mgx_status s = (code == kDevSubdivLimit || code == kDevTraceGuard || code == kDevArenaOverflow) ? MGX_ERANGE : MGX_EINVAL;
        cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream);
        cudaStreamSynchronize(ctx->stream);
        return fail(ctx, s, "device check failed: %s", dev_err_text(code));
    }
    return MGX_OK;
}

cudaEvent_t take_event(mgx_ctx *c) {
    if (!c->event_pool.empty()) {
        cudaEvent_t e = c->event_pool.back();
        c->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// Counts a kernel launch of class `slot` and, while profiling, brackets it
// with CUDA events on the context's stream.
struct Timed {
    mgx_ctx *c;
    int slot;
    cudaEvent_t a = nullptr, b = nullptr;
    Timed(mgx_ctx *c_, int slot_) : c(c_), slot(slot_) {  // slot < 0: not recorded
        if (slot < 0) return;
        c->launches[slot] += 1;
        if (c->prof) {
            a = take_event(c);
            b = take_event(c);
            if (a && b) cudaEventRecord(a, c->stream);
        }
    }
    ~Timed() {
        if (a && b) {
            cudaEventRecord(b, c->stream);
            c->ev[slot].emplace_back(a, b);
        }
    }
};

void reset_profile(mgx_ctx *c) {
    for (auto &v : c->ev) {
        for (auto &pr : v) {
            c->event_pool.push_back(pr.first);
            c->event_pool.push_back(pr.second);
        }
        v.clear();
    }
    for (auto &l : c->launches) l = 0;
    c->trace_points = 0;
    c->solves = 0;
    if (c->d_counters) cudaMemsetAsync(c->d_counters, 0, kCounters * sizeof(unsigned long long), c->stream);
}

Model *get_model(mgx_ctx *ctx, int32_t id) {
    if (id < 0 || size_t(id) >= ctx->models.size() || !ctx->models[id].live) return nullptr;
    return &ctx->models[id];
}

DevMesh mesh_view(const Model &m) {
    DevMesh d;
    d.n = m.n;
    d.x = m.x; d.y = m.y; d.z = m.z;
    d.vx = m.vx; d.vy = m.vy; d.vz = m.vz;
    d.vxf = m.vxf; d.vyf = m.vyf; d.vzf = m.vzf;
    d.off = m.off;
    d.nbr = m.nbr;
    d.phi = m.phi;
    d.nrec = m.nrec;
    d.g0 = m.g0;
    return d;
}

DevLines lines_view(const Model &m) {
    DevLines d;
    d.L = m.L;
    d.F = m.F;
    d.x_span = m.x_span;
    for (int i = 0; i < MGX_MAX_LINES * MGX_MAX_LINES; ++i) d.ratio[i] = 1.0;
    for (int l = 0; l < m.L; ++l)
        for (int lp = 0; lp < m.L; ++lp) d.ratio[l * MGX_MAX_LINES + lp] = m.nu0[l] / m.nu0[lp];
    d.chi0 = m.chi0; d.eta0 = m.eta0; d.dvw = m.dvw; d.chic = m.chic; d.etac = m.etac;
    d.chi0f = m.chi0f; d.eta0f = m.eta0f; d.dvwf = m.dvwf; d.chicf = m.chicf; d.etacf = m.etacf;
    return d;
}

DevRays rays_view(const mgx_ctx *ctx, const Model &m) {
    DevRays r;
    r.lmin = m.lmin;
    r.lmax = m.lmax;
    r.npairs = m.npairs;
    r.rays = m.rays;
    r.dir = ctx->dir;
    r.dirf = ctx->dirf;
    return r;
}

// HEALPix direction and antipode tables up to `level`, plus the sorted list of
// pair representatives (the member with the smaller index) of every level.
mgx_status ensure_tables(mgx_ctx *ctx, int level) {
    if (level <= ctx->tab_level) return MGX_OK;
    const int64_t total = level_offset(level + 1);
    std::vector<double> dir(size_t(total) * 3);
    std::vector<float4> dirf(static_cast<size_t>(total));
    std::vector<int32_t> anti(static_cast<size_t>(total));
    std::vector<std::vector<uint32_t>> lists(size_t(level) + 1);
    for (int l = 0; l <= level; ++l) {
        const int64_t np = hpx_npix(l), base = level_offset(l);
        for (int64_t p = 0; p < np; ++p) {
            double v[3];
            hpx_pix2vec(l, p, v);
            dir[size_t(base + p) * 3 + 0] = v[0];
            dir[size_t(base + p) * 3 + 1] = v[1];
            dir[size_t(base + p) * 3 + 2] = v[2];
            dirf[size_t(base + p)] = make_float4(float(v[0]), float(v[1]), float(v[2]), 0.0f);  // round to nearest
            const double w[3] = {-v[0], -v[1], -v[2]};
            anti[size_t(base + p)] = int32_t(hpx_vec2pix(l, w));
        }
        for (int64_t p = 0; p < np; ++p) {
            const int64_t a = anti[size_t(base + p)];
            if (a == p || anti[size_t(base + a)] != p)
                return fail(ctx, MGX_ECUDA, "internal: HEALPix antipode table inconsistent at level %d", l);
            if (p < a) lists[size_t(l)].push_back(uint32_t(p));
        }
    }
    double *ddir = nullptr;
    float4 *ddirf = nullptr;
    int32_t *danti = nullptr;
    CK(dalloc(ctx, &ddir, dir.size()));
    CK(dalloc(ctx, &ddirf, dirf.size()));
    CK(cudaMemcpyAsync(ddirf, dirf.data(), dirf.size() * sizeof(float4), cudaMemcpyHostToDevice, ctx->stream));
    CK(dalloc(ctx, &danti, anti.size()));
    CK(cudaMemcpyAsync(ddir, dir.data(), dir.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(danti, anti.data(), anti.size() * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
    std::vector<uint32_t *> dl(size_t(level) + 1, nullptr);
    for (int l = 0; l <= level; ++l) {
        CK(dalloc(ctx, &dl[size_t(l)], lists[size_t(l)].size()));
        CK(cudaMemcpyAsync(dl[size_t(l)], lists[size_t(l)].data(), lists[size_t(l)].size() * sizeof(uint32_t),
                           cudaMemcpyHostToDevice, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    dfree(ctx, ctx->dir);
    dfree(ctx, ctx->dirf);
    dfree(ctx, ctx->anti);
    for (auto *p : ctx->pair_lists_dev) dfree(ctx, p);
    ctx->dir = ddir;
    ctx->dirf = ddirf;
    ctx->anti = danti;
    ctx->pair_lists = std::move(lists);
    ctx->pair_lists_dev = std::move(dl);
    ctx->tab_level = level;
    return MGX_OK;
}

void free_lines(mgx_ctx *ctx, Model &m) {
    dfree(ctx, m.chi0); dfree(ctx, m.eta0); dfree(ctx, m.dvw); dfree(ctx, m.chic); dfree(ctx, m.etac);
    dfree(ctx, m.chi0f); dfree(ctx, m.eta0f); dfree(ctx, m.dvwf); dfree(ctx, m.chicf); dfree(ctx, m.etacf);
    m.has_lines = false;
}

void drop_offsets(mgx_ctx *ctx, Model &m) {
    dfree(ctx, m.offs_all);
    m.obound.clear();
    m.obound.shrink_to_fit();
}

void free_model(mgx_ctx *ctx, Model &m) {
    dfree(ctx, m.x); dfree(ctx, m.y); dfree(ctx, m.z);
    dfree(ctx, m.vx); dfree(ctx, m.vy); dfree(ctx, m.vz);
    dfree(ctx, m.vxf); dfree(ctx, m.vyf); dfree(ctx, m.vzf);
    dfree(ctx, m.off); dfree(ctx, m.nbr);
    dfree(ctx, m.phi); dfree(ctx, m.nrec);
    free_lines(ctx, m);
    dfree(ctx, m.rays);
    dfree(ctx, m.sample);
    drop_offsets(ctx, m);
    m.has_rays = false;
    m.live = false;
}

// inclusive prefix sum of n int64 values: out[i] = sum in[0..i]
mgx_status scan_i64(mgx_ctx *ctx, const int64_t *in, int64_t *out, int64_t n) {
    size_t tmp_bytes = 0;
    CK(cub::DeviceScan::InclusiveSum(nullptr, tmp_bytes, in, out, n, ctx->stream));
    void *tmp = nullptr;
    CK(cudaMallocAsync(&tmp, tmp_bytes ? tmp_bytes : 1, ctx->stream));
    CK(cub::DeviceScan::InclusiveSum(tmp, tmp_bytes, in, out, n, ctx->stream));
    CK(cudaFreeAsync(tmp, ctx->stream));
    return MGX_OK;
}

// Trace lengths of every half-ray of origins [o0, o1) and their offsets:
// offs[0] = 0, offs[h+1] = offs[h] + length(h).
mgx_status trace_offsets(mgx_ctx *ctx, Model &m, int32_t o0, int32_t o1, int64_t **offs_out) {
    const int64_t n_half = int64_t(o1 - o0) * m.npairs * 2;
    int64_t *lens = nullptr, *offs = nullptr;
    CK(dalloc(ctx, &lens, size_t(n_half)));
    CK(dalloc(ctx, &offs, size_t(n_half + 1)));
    CK(cudaMemsetAsync(offs, 0, sizeof(int64_t), ctx->stream));
    {
        Timed t(ctx, MGX_K_TRACE_COUNT);
        launch_trace_count(mesh_view(m), rays_view(ctx, m), o0, o1, lens, ctx->d_status,
                           ctx->prof ? ctx->d_counters : nullptr, ctx->stream);
    }
    CK(cudaGetLastError());
    if (n_half > 0) {
        Timed t(ctx, MGX_K_SCAN);
        const mgx_status s = scan_i64(ctx, lens, offs + 1, n_half);
        if (s != MGX_OK) {
            dfree(ctx, lens);
            dfree(ctx, offs);
            return s;
        }
    }
    dfree(ctx, lens);
    *offs_out = offs;
    return MGX_OK;
}


void free_plan(mgx_ctx *ctx, BatchPlan &pl) {
    if (pl.exec) cudaGraphExecDestroy(pl.exec);
    if (pl.graph) cudaGraphDestroy(pl.graph);
    pl.exec = nullptr;
    pl.graph = nullptr;
    for (double *&q : pl.Jdev) dfree(ctx, q);
    pl.Jdev.clear();
    pl.Jbytes.clear();
    dfree(ctx, pl.lens);
    dfree(ctx, pl.excess);
    dfree(ctx, pl.offs);
    dfree(ctx, pl.rows);
    dfree(ctx, pl.tail);
    dfree(ctx, pl.resume);
    dfree(ctx, pl.obase);
    dfree(ctx, pl.geo);
    dfree(ctx, pl.slots);
    dfree(ctx, pl.work);
    dfree(ctx, pl.scratch);
    dfree(ctx, pl.wl.key_in);
    dfree(ctx, pl.wl.key_out);
    dfree(ctx, pl.wl.val_in);
    dfree(ctx, pl.wl.val_out);
    dfree(ctx, pl.wl.tiles);
    dfree(ctx, pl.wl.toff);
    if (pl.wl.tmp) cudaFreeAsync(pl.wl.tmp, ctx->stream);
    pl.wl = WorkListBufs{};
    if (pl.cub_tmp) cudaFreeAsync(pl.cub_tmp, ctx->stream);
    pl.cub_tmp = nullptr;
    pl.valid = false;
}

// Rebuild the ray set of a model with its current levels and sample (enqueue only).
void enqueue_rays(mgx_ctx *ctx, Model &m, bool timed = true) {
    Timed t(ctx, timed ? MGX_K_RAYS : -1);
    if (m.lmin == m.lmax) {
        launch_rays_fixed(m.n, m.lmin, m.npairs, ctx->pair_lists_dev[size_t(m.lmin)], m.rays, ctx->stream);
    } else {
        launch_rays_adaptive(mesh_view(m), m.lmin, m.lmax, m.npairs, m.n_sample, m.sample, ctx->anti,
                             ctx->pair_lists_dev[size_t(m.lmin)], int32_t(ctx->pair_lists[size_t(m.lmin)].size()),
                             m.rays, ctx->d_status, ctx->stream);
    }
}

constexpr int kScratchQueue = 0;   // the persistent solve's work counter
constexpr int kScratchTotals = 8;  // kPadCandidates + 1 row-width totals
constexpr int kScratchSize = kScratchTotals + kPadCandidates + 1;

// One step of a batched solve: (ray sets,) padded trace, tail offsets, tail
// trace, work list, persistent solve.
// The first part of a batched step: ray sets (when asked for), the padded
// trace and the prefix sums of the excesses that place the tail.
mgx_status enqueue_batch_front(mgx_ctx *ctx, BatchPlan &pl, std::vector<Model *> &ms) {
    if (pl.flags & MGX_BATCH_RAYS)
        for (Model *m : ms) enqueue_rays(ctx, *m);
    int64_t hb = 0;
    for (Model *m : ms) {
        Timed t(ctx, MGX_K_TRACE_COUNT);
        launch_trace_pad(mesh_view(*m), rays_view(ctx, *m), 0, m->n, pl.pad, pl.lens + hb, pl.excess + hb,
                         pl.resume + hb, pl.rows + hb * pl.pad, ctx->d_status,
                         ctx->prof ? ctx->d_counters : nullptr, ctx->stream, pl.tune.trace_ctas_per_sm);
        hb += int64_t(m->n) * m->npairs * 2;
    }
    CK(cudaMemsetAsync(pl.offs, 0, sizeof(int64_t), ctx->stream));
    {
        Timed t(ctx, MGX_K_SCAN);
        CK(cub::DeviceScan::InclusiveSum(pl.cub_tmp, pl.cub_bytes, pl.excess, pl.offs + 1, pl.total_half,
                                         ctx->stream));
    }
    CK(cudaGetLastError());
    return MGX_OK;
}

// The rest: the tail trace, the work list and the persistent solve.
mgx_status enqueue_batch_back(mgx_ctx *ctx, BatchPlan &pl, std::vector<Model *> &ms) {
    int64_t hb = 0;
    if (pl.tail_cap > 0) {
        for (Model *m : ms) {
            Timed t(ctx, MGX_K_TRACE_EMIT);
            launch_trace_tail(mesh_view(*m), rays_view(ctx, *m), 0, m->n, pl.pad, pl.lens + hb, pl.resume + hb,
                              pl.offs + hb, 0, pl.tail_cap, pl.tail, ctx->d_status, ctx->stream,
                              pl.tune.trace_ctas_per_sm);
            hb += int64_t(m->n) * m->npairs * 2;
        }
    }
    {
        Timed t(ctx, MGX_K_OTHER);
        launch_batch_worklist(pl.geo, pl.obase, int32_t(ms.size()), pl.n_origins, pl.lens, pl.wl, pl.work,
                              pl.tune.schedule == 1, ctx->stream);
    }
    CK(cudaMemsetAsync(pl.scratch + kScratchQueue, 0, sizeof(unsigned long long), ctx->stream));
    {
        Timed t(ctx, MGX_K_SOLVE);
        launch_solve_queue(pl.p.precision, pl.p.order == 4 ? 4 : 2, pl.bpl, pl.max_lines, pl.slots, pl.work, pl.n_work,
                           pl.scratch + kScratchQueue, ctx->stream);
    }
    CK(cudaGetLastError());
    return MGX_OK;
}

mgx_status enqueue_batch_step(mgx_ctx *ctx, BatchPlan &pl, std::vector<Model *> &ms) {
    const mgx_status s = enqueue_batch_front(ctx, pl, ms);
    return s != MGX_OK ? s : enqueue_batch_back(ctx, pl, ms);
}

// Copy the staged outputs of a batched step to their host buffers (one copy
// per model, after the step on the same stream) and wait for the stream.
mgx_status finish_batch_step(mgx_ctx *ctx, BatchPlan &pl) {
    for (size_t k = 0; k < pl.Jdev.size(); ++k)
        if (pl.Jdev[k]) CK(cudaMemcpyAsync(pl.J[k], pl.Jdev[k], pl.Jbytes[k], cudaMemcpyDeviceToHost, ctx->stream));
    return sync_status(ctx);
}

// Device memory the fixed-width rows of a batched plan may take.
constexpr size_t kRowsBudget = size_t(96) << 30;
// The planning sample of half-ray lengths: every kSampleShare-th origin of a
// model with more than kSampleAll origins (all of a smaller one), counted by
// one launch per model.
constexpr int32_t kSampleShare = 32, kSampleAll = 1024;

// Row width of the padded layout: the narrowest power of two that leaves at
// most `permille` / 1000 of the traced points to the tail pass, within the
// memory budget for the rows (else the widest that fits).
int32_t choose_pad(const unsigned long long *tot, int64_t total_half, size_t budget_bytes, int32_t permille) {
    const unsigned long long all = tot[kPadCandidates];
    int best = -1;
    for (int j = 0; j < kPadCandidates; ++j) {
        if (size_t(total_half) * (size_t(1) << j) * sizeof(int32_t) > budget_bytes) break;
        best = j;
        if (double(tot[j]) * 1000.0 <= double(permille) * double(all)) break;
    }
    return best < 0 ? 1 : int32_t(1) << best;
}

bool same_tuning(const mgx_tuning &a, const mgx_tuning &b) {
    return a.bins_per_lane == b.bins_per_lane && a.trace_ctas_per_sm == b.trace_ctas_per_sm &&
           a.tail_permille == b.tail_permille && a.schedule == b.schedule;
}

bool valid_tuning(const mgx_tuning &t) {
    return t.bins_per_lane >= 0 && t.bins_per_lane <= 2 && t.trace_ctas_per_sm >= 0 && t.trace_ctas_per_sm <= 32 &&
           t.tail_permille >= 0 && t.tail_permille <= 1000 && (t.schedule == 0 || t.schedule == 1);
}

bool plan_matches(const BatchPlan &pl, const int32_t *models, int32_t n, const mgx_solve_params *p,
                  double *const *J, int32_t flags, const mgx_tuning &tune) {
    if (!pl.valid || int32_t(pl.models.size()) != n || pl.flags != flags || !same_tuning(pl.tune, tune)) return false;
    for (int32_t k = 0; k < n; ++k)
        if (pl.models[size_t(k)] != models[k] || pl.J[size_t(k)] != J[k]) return false;
    return pl.p.dtau_max == p->dtau_max && pl.p.dv_max == p->dv_max && pl.p.I_bdy == p->I_bdy &&
           pl.p.precision == p->precision && pl.p.order == p->order;
}

}  // namespace

extern "C" {

mgx_status mgx_create(int device, void *stream, mgx_ctx **out) {
    if (!out) return MGX_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return MGX_EINVAL;
    }
    std::unique_ptr<mgx_ctx> c(new mgx_ctx());
    c->device = device;
    c->stream = static_cast<cudaStream_t>(stream);
    mgx_ctx *ctx = c.get();
    DeviceGuard g(device);
    if (!g.ok) return MGX_ECUDA;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;  // keep freed stream-ordered memory cached in the process
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    CK(cudaMalloc(&c->d_status, sizeof(int)));
    CK(cudaMemset(c->d_status, 0, sizeof(int)));
    CK(cudaMallocHost(&c->h_status, sizeof(int)));
    CK(cudaMalloc(&c->d_counters, kCounters * sizeof(unsigned long long)));
    CK(cudaMemset(c->d_counters, 0, kCounters * sizeof(unsigned long long)));
    *out = c.release();
    return MGX_OK;
}

void mgx_destroy(mgx_ctx *ctx) {
    if (!ctx) return;
    {
        DeviceGuard g(ctx->device);
        free_plan(ctx, ctx->plan);
        dfree(ctx, ctx->mlp_theta); dfree(ctx, ctx->mlp_m); dfree(ctx, ctx->mlp_v);
        dfree(ctx, ctx->mlp_grad); dfree(ctx, ctx->mlp_loss);
        if (ctx->mlp_W1b) cudaFreeAsync(ctx->mlp_W1b, ctx->stream);
        if (ctx->mlp_W2b) cudaFreeAsync(ctx->mlp_W2b, ctx->stream);
        for (auto &m : ctx->models)
            if (m.live) free_model(ctx, m);
        dfree(ctx, ctx->dirf);
        dfree(ctx, ctx->dir);
        dfree(ctx, ctx->anti);
        for (auto *p : ctx->pair_lists_dev) dfree(ctx, p);
        reset_profile(ctx);  // before the counters are freed: it clears them on the stream
        cudaStreamSynchronize(ctx->stream);
        if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
        ctx->capture_stream = nullptr;
        for (auto e : ctx->event_pool) cudaEventDestroy(e);
        ctx->event_pool.clear();
        cudaFree(ctx->d_status);
        ctx->d_status = nullptr;
        cudaFreeHost(ctx->h_status);
        ctx->h_status = nullptr;
        cudaFree(ctx->d_counters);
        ctx->d_counters = nullptr;
        cudaGetLastError();
    }
    delete ctx;
}

const char *mgx_last_error(const mgx_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int32_t mgx_pix2vec(int32_t l, int64_t p, double *v) {
    if (!v || l < 0 || l > MGX_MAX_LEVEL || p < 0 || p >= hpx_npix(l)) return -1;
    hpx_pix2vec(l, p, v);
    return 0;
}

int64_t mgx_antipode(int32_t l, int64_t p) {
    if (l < 0 || l > MGX_MAX_LEVEL || p < 0 || p >= hpx_npix(l)) return -1;
    double v[3];
    hpx_pix2vec(l, p, v);
    const double w[3] = {-v[0], -v[1], -v[2]};
    return hpx_vec2pix(l, w);
}

int64_t mgx_rayset_npairs(int32_t l_min, int32_t l_max) {
    if (l_min < 0 || l_max < l_min || l_max > MGX_MAX_LEVEL) return -1;
    if (l_min < l_max && l_max > MGX_MAX_ADAPT_LEVEL) return -1;
    return rayset_npairs(l_min, l_max);
}

mgx_status mgx_load_mesh(mgx_ctx *ctx, int64_t n, const double *pos, const double *vel,
                         const int64_t *nbr_off, const int32_t *nbr_idx, int32_t *model_id) {
    if (!ctx) return MGX_EINVAL;
    ctx->err.clear();
    if (!pos || !vel || !nbr_off || !model_id) return fail(ctx, MGX_EINVAL, "load_mesh: null pointer");
    if (n < 1 || n >= (int64_t(1) << 31)) return fail(ctx, MGX_EINVAL, "load_mesh: n = %lld out of range", (long long)n);
    if (nbr_off[0] != 0) return fail(ctx, MGX_EINVAL, "load_mesh: nbr_off[0] must be 0");
    const int64_t E = nbr_off[n];
    if (E < 0 || E >= (int64_t(1) << 31)) return fail(ctx, MGX_EINVAL, "load_mesh: edge count %lld out of range", (long long)E);
    if (E > 0 && !nbr_idx) return fail(ctx, MGX_EINVAL, "load_mesh: null nbr_idx");
    DeviceGuard g(ctx->device);
    Model m;
    m.n = int32_t(n);
    m.E = E;
    double *pos_d = nullptr, *vel_d = nullptr;
    int64_t *off64 = nullptr;
    CK(dalloc(ctx, &pos_d, size_t(3 * n)));
    CK(dalloc(ctx, &vel_d, size_t(3 * n)));
    CK(dalloc(ctx, &off64, size_t(n + 1)));
    CK(dalloc(ctx, &m.x, size_t(n))); CK(dalloc(ctx, &m.y, size_t(n))); CK(dalloc(ctx, &m.z, size_t(n)));
    CK(dalloc(ctx, &m.vx, size_t(n))); CK(dalloc(ctx, &m.vy, size_t(n))); CK(dalloc(ctx, &m.vz, size_t(n)));
    CK(dalloc(ctx, &m.vxf, size_t(n))); CK(dalloc(ctx, &m.vyf, size_t(n))); CK(dalloc(ctx, &m.vzf, size_t(n)));
    CK(dalloc(ctx, &m.off, size_t(n + 1)));
    CK(dalloc(ctx, &m.nbr, size_t(E)));
    CK(dalloc(ctx, &m.phi, size_t(n)));
    // one spare record after the last: the tracer reads the records in aligned pairs
    CK(dalloc(ctx, &m.nrec, size_t(E) + 1));
    CK(cudaMemsetAsync(m.nrec, 0, (size_t(E) + 1) * sizeof(float4), ctx->stream));
    if (reinterpret_cast<uintptr_t>(m.nrec) % 32 != 0) {  // the pair loads need 32-byte alignment
        dfree(ctx, pos_d);
        dfree(ctx, vel_d);
        dfree(ctx, off64);
        free_model(ctx, m);
        return fail(ctx, MGX_ECUDA, "load_mesh: neighbour records not 32-byte aligned");
    }
    unsigned int *xmax = nullptr;
    CK(dalloc(ctx, &xmax, 1));
    CK(cudaMemsetAsync(xmax, 0, sizeof(unsigned int), ctx->stream));
    CK(cudaMemcpyAsync(pos_d, pos, size_t(3 * n) * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(vel_d, vel, size_t(3 * n) * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(off64, nbr_off, size_t(n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, ctx->stream));
    if (E > 0)
        CK(cudaMemcpyAsync(m.nbr, nbr_idx, size_t(E) * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
    {
        Timed t(ctx, MGX_K_OTHER);
        launch_ingest_mesh(m.n, pos_d, vel_d, off64, E, m.x, m.y, m.z, m.vx, m.vy, m.vz, m.vxf, m.vyf,
                           m.vzf, m.off, m.nbr, m.phi, xmax, ctx->d_status, ctx->stream);
        launch_pack_neighbours(m.n, m.off, m.nbr, m.phi, m.nrec, ctx->stream);
    }
    CK(cudaGetLastError());
    unsigned int xmax_h = 0;
    CK(cudaMemcpyAsync(&xmax_h, xmax, sizeof xmax_h, cudaMemcpyDeviceToHost, ctx->stream));
    dfree(ctx, xmax);
    dfree(ctx, pos_d);
    dfree(ctx, vel_d);
    dfree(ctx, off64);
    m.live = true;
    const mgx_status s = sync_status(ctx);
    if (s != MGX_OK) {
        free_model(ctx, m);
        return s;
    }
    {
        float xm;
        std::memcpy(&xm, &xmax_h, sizeof xm);
        const double u = 1.0 / 16777216.0;  // 2^-24
        m.g0 = float(32.0 * u * u * double(xm) * (1.0 + 1e-6)) + 1e-37f;
    }
    ctx->models.push_back(m);
    *model_id = int32_t(ctx->models.size() - 1);
    return MGX_OK;
}

mgx_status mgx_free_model(mgx_ctx *ctx, int32_t model) {
    if (!ctx) return MGX_EINVAL;
    Model *m = get_model(ctx, model);
    if (!m) return fail(ctx, MGX_EINVAL, "free_model: no model %d", model);
    DeviceGuard g(ctx->device);
    free_plan(ctx, ctx->plan);
    free_model(ctx, *m);
    return MGX_OK;
}

mgx_status mgx_set_lines(mgx_ctx *ctx, int32_t model, int32_t n_lines, const double *nu0,
                         const double *chi0, const double *eta0, const double *dvw,
                         const double *chi_c, const double *eta_c, int32_t n_freq, double x_span) {
    if (!ctx) return MGX_EINVAL;
    ctx->err.clear();
    Model *m = get_model(ctx, model);
    if (!m) return fail(ctx, MGX_EINVAL, "set_lines: no model %d", model);
    if (n_lines < 1 || n_lines > MGX_MAX_LINES) return fail(ctx, MGX_EINVAL, "set_lines: n_lines = %d not in 1..%d", n_lines, MGX_MAX_LINES);
    if (!nu0 || !chi0 || !eta0 || !dvw || !chi_c || !eta_c) return fail(ctx, MGX_EINVAL, "set_lines: null pointer");
    if (n_freq < 1 || int64_t(n_freq) * n_lines > (int64_t(1) << 20)) return fail(ctx, MGX_EINVAL, "set_lines: n_freq = %d out of range", n_freq);
    if (!std::isfinite(x_span) || x_span < 0.0) return fail(ctx, MGX_EINVAL, "set_lines: x_span must be finite and >= 0");
    for (int l = 0; l < n_lines; ++l)
        if (!std::isfinite(nu0[l]) || !(nu0[l] > 0.0)) return fail(ctx, MGX_EINVAL, "set_lines: nu0[%d] must be > 0", l);
    DeviceGuard g(ctx->device);
    free_lines(ctx, *m);
    const size_t n = size_t(m->n), nl = n * size_t(n_lines);
    CK(dalloc(ctx, &m->chi0, nl)); CK(dalloc(ctx, &m->eta0, nl));
    CK(dalloc(ctx, &m->dvw, n)); CK(dalloc(ctx, &m->chic, n)); CK(dalloc(ctx, &m->etac, n));
    CK(dalloc(ctx, &m->chi0f, nl)); CK(dalloc(ctx, &m->eta0f, nl));
    CK(dalloc(ctx, &m->dvwf, n)); CK(dalloc(ctx, &m->chicf, n)); CK(dalloc(ctx, &m->etacf, n));
    CK(cudaMemcpyAsync(m->chi0, chi0, nl * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(m->eta0, eta0, nl * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(m->dvw, dvw, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(m->chic, chi_c, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(m->etac, eta_c, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    {
        Timed t(ctx, MGX_K_OTHER);
        launch_ingest_lines(m->n, n_lines, m->chi0, m->eta0, m->dvw, m->chic, m->etac, m->chi0f, m->eta0f,
                            m->dvwf, m->chicf, m->etacf, ctx->d_status, ctx->stream);
    }
    CK(cudaGetLastError());
    m->L = n_lines;
    m->F = n_freq;
    m->x_span = x_span;
    for (int l = 0; l < n_lines; ++l) m->nu0[l] = nu0[l];
    const mgx_status s = sync_status(ctx);
    if (s != MGX_OK) {
        free_lines(ctx, *m);
        return s;
    }
    m->has_lines = true;
    return MGX_OK;
}

mgx_status mgx_set_rays(mgx_ctx *ctx, int32_t model, int32_t l_min, int32_t l_max, int64_t n_sample,
                        const int32_t *sample) {
    if (!ctx) return MGX_EINVAL;
    ctx->err.clear();
    Model *m = get_model(ctx, model);
    if (!m) return fail(ctx, MGX_EINVAL, "set_rays: no model %d", model);
    const int64_t np = mgx_rayset_npairs(l_min, l_max);
    if (np < 0) return fail(ctx, MGX_EINVAL, "set_rays: levels %d..%d invalid (fixed <= %d, adaptive <= %d)", l_min, l_max, MGX_MAX_LEVEL, MGX_MAX_ADAPT_LEVEL);
    if (int64_t(m->n) * np >= (int64_t(1) << 40)) return fail(ctx, MGX_ERANGE, "set_rays: too many rays");
    const bool adaptive = l_min < l_max;
    if (adaptive) {
        if (n_sample < 0 || (n_sample > 0 && !sample)) return fail(ctx, MGX_EINVAL, "set_rays: bad sample");
        for (int64_t s = 0; s < n_sample; ++s)
            if (sample[s] < 0 || sample[s] >= m->n) return fail(ctx, MGX_EINVAL, "set_rays: sample[%lld] out of range", (long long)s);
    }
    DeviceGuard g(ctx->device);
    mgx_status s = ensure_tables(ctx, l_max);
    if (s != MGX_OK) return s;
    drop_offsets(ctx, *m);
    if (!m->rays || m->npairs != np) {
        dfree(ctx, m->rays);
        CK(dalloc(ctx, &m->rays, size_t(m->n) * size_t(np)));
    }
    m->lmin = l_min;
    m->lmax = l_max;
    m->npairs = int32_t(np);
    if (!adaptive) {
        Timed t(ctx, MGX_K_RAYS);
        launch_rays_fixed(m->n, l_min, m->npairs, ctx->pair_lists_dev[size_t(l_min)], m->rays, ctx->stream);
        CK(cudaGetLastError());
    } else {
        dfree(ctx, m->sample);
        CK(dalloc(ctx, &m->sample, size_t(n_sample)));
        m->n_sample = n_sample;
        if (n_sample > 0)
            CK(cudaMemcpyAsync(m->sample, sample, size_t(n_sample) * sizeof(int32_t), cudaMemcpyHostToDevice,
                               ctx->stream));
        Timed t(ctx, MGX_K_RAYS);
        launch_rays_adaptive(mesh_view(*m), l_min, l_max, m->npairs, n_sample, m->sample, ctx->anti,
                             ctx->pair_lists_dev[size_t(l_min)], int32_t(ctx->pair_lists[size_t(l_min)].size()),
                             m->rays, ctx->d_status, ctx->stream);
        CK(cudaGetLastError());
    }
    s = sync_status(ctx);
    m->has_rays = (s == MGX_OK);
    return s;
}

mgx_status mgx_get_rays(mgx_ctx *ctx, int32_t model, uint32_t *out) {
    if (!ctx) return MGX_EINVAL;
    ctx->err.clear();
    Model *m = get_model(ctx, model);
    if (!m || !out) return fail(ctx, MGX_EINVAL, "get_rays: bad model or null output");
    if (!m->has_rays) return fail(ctx, MGX_ESTATE, "get_rays: set_rays not called");
    DeviceGuard g(ctx->device);
    CK(cudaMemcpyAsync(out, m->rays, size_t(m->n) * m->npairs * sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return MGX_OK;
}

mgx_status mgx_trace(mgx_ctx *ctx, int32_t model, int64_t o_begin, int64_t o_end, int64_t *off_out,
                     int32_t *idx_out, double *Z_out, double *delta_out, int64_t capacity) {
    if (!ctx) return MGX_EINVAL;
    ctx->err.clear();
    Model *m = get_model(ctx, model);
    if (!m) return fail(ctx, MGX_EINVAL, "trace: no model %d", model);
    if (!m->has_rays) return fail(ctx, MGX_ESTATE, "trace: set_rays not called");
    if (o_begin < 0 || o_end > m->n || o_begin > o_end) return fail(ctx, MGX_EINVAL, "trace: origin range invalid");
    if (!off_out) return fail(ctx, MGX_EINVAL, "trace: null off_out");
    if (idx_out && !Z_out) return fail(ctx, MGX_EINVAL, "trace: Z_out required with idx_out");
    DeviceGuard g(ctx->device);
    const int64_t n_half = (o_end - o_begin) * m->npairs * 2;
    int64_t *offs = nullptr;
    mgx_status s = trace_offsets(ctx, *m, int32_t(o_begin), int32_t(o_end), &offs);
    if (s != MGX_OK) return s;
    CK(cudaMemcpyAsync(off_out, offs, size_t(n_half + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    s = sync_status(ctx);
    if (s != MGX_OK || !idx_out) {
        dfree(ctx, offs);
        return s;
    }
    const int64_t total = off_out[n_half];
    if (capacity < total) {
        dfree(ctx, offs);
        return fail(ctx, MGX_ERANGE, "trace: capacity %lld < %lld entries", (long long)capacity, (long long)total);
    }
    int32_t *idx = nullptr;
    double *Z = nullptr, *de = nullptr;
    CK(dalloc(ctx, &idx, size_t(total)));
    CK(dalloc(ctx, &Z, size_t(total)));
    if (delta_out) CK(dalloc(ctx, &de, size_t(total)));
    {
        Timed t(ctx, MGX_K_TRACE_EMIT);
        launch_trace_emit(mesh_view(*m), rays_view(ctx, *m), int32_t(o_begin), int32_t(o_end), offs, 0, total, idx,
                          Z, de, ctx->d_status, ctx->stream);
    }
    CK(cudaGetLastError());
    if (total > 0) {
        CK(cudaMemcpyAsync(idx_out, idx, size_t(total) * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(Z_out, Z, size_t(total) * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        if (delta_out)
            CK(cudaMemcpyAsync(delta_out, de, size_t(total) * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    }
    dfree(ctx, idx);
    dfree(ctx, Z);
    dfree(ctx, de);
    dfree(ctx, offs);
    return sync_status(ctx);
}

mgx_status mgx_solve_J(mgx_ctx *ctx, int32_t model, const mgx_solve_params *p, void *J_out) {
    if (!ctx) return MGX_EINVAL;
    ctx->err.clear();
    Model *m = get_model(ctx, model);
    if (!m) return fail(ctx, MGX_EINVAL, "solve_J: no model %d", model);
    if (!p || !J_out) return fail(ctx, MGX_EINVAL, "solve_J: null params or output");
    if (!m->has_lines) return fail(ctx, MGX_ESTATE, "solve_J: set_lines not called");
    if (!m->has_rays) return fail(ctx, MGX_ESTATE, "solve_J: set_rays not called");
    if (!std::isfinite(p->dtau_max) || !(p->dtau_max > 0.0)) return fail(ctx, MGX_EINVAL, "solve_J: dtau_max must be > 0");
    if (!std::isfinite(p->dv_max)) return fail(ctx, MGX_EINVAL, "solve_J: dv_max must be finite");
    if (!std::isfinite(p->I_bdy)) return fail(ctx, MGX_EINVAL, "solve_J: I_bdy must be finite");
    if (p->precision != MGX_FP64 && p->precision != MGX_FP32 && p->precision != MGX_FP32_DT64)
        return fail(ctx, MGX_EINVAL, "solve_J: unknown precision");
    if (p->precision == MGX_FP32_DT64 && p->order == 4)
        return fail(ctx, MGX_EINVAL, "solve_J: MGX_FP32_DT64 exists for the second-order scheme only");
    if ((p->order != 0 && p->order != 2 && p->order != 4) || p->reserved != 0)
        return fail(ctx, MGX_EINVAL, "solve_J: order must be 0, 2 or 4 (reserved 0)");
    DeviceGuard g(ctx->device);
    const int32_t n = m->n, np = m->npairs;
    if (!m->offs_all) {
        int64_t *offs = nullptr;
        mgx_status s = trace_offsets(ctx, *m, 0, n, &offs);
        if (s != MGX_OK) return s;
        // half-ray offsets at origin boundaries decide the chunks
        m->obound.assign(size_t(n) + 1, 0);
        CK(cudaMemcpy2DAsync(m->obound.data(), sizeof(int64_t), offs, size_t(2 * np) * sizeof(int64_t),
                             sizeof(int64_t), size_t(n) + 1, cudaMemcpyDeviceToHost, ctx->stream));
        s = sync_status(ctx);
        if (s != MGX_OK) {
            dfree(ctx, offs);
            m->obound.clear();
            return s;
        }
        m->offs_all = offs;
    }
    const int64_t *offs = m->offs_all;
    const std::vector<int64_t> &obound = m->obound;
    const int64_t total = obound[size_t(n)];
    const int64_t budget = int64_t(ctx->arena_budget / sizeof(int32_t));
    std::vector<int32_t> cuts{0};
    int64_t chunk_max = 0;
    while (cuts.back() < n) {
        const int32_t a = cuts.back();
        int32_t b = a + 1;
        while (b < n && obound[size_t(b) + 1] - obound[size_t(a)] <= budget) ++b;
        chunk_max = std::max(chunk_max, obound[size_t(b)] - obound[size_t(a)]);
        cuts.push_back(b);
    }
    ctx->trace_points += total;
    ctx->solves += int64_t(n) * np * int64_t(m->L) * m->F;
    int32_t *aidx = nullptr;
    CK(dalloc(ctx, &aidx, size_t(chunk_max)));
    const int64_t NB = int64_t(m->L) * m->F;
    double *J = nullptr;
    if (p->out_on_device) {
        J = static_cast<double *>(J_out);
    } else {
        CK(dalloc(ctx, &J, size_t(n) * size_t(NB)));
    }
    const DevMesh dm = mesh_view(*m);
    const DevLines dl = lines_view(*m);
    const DevRays dr = rays_view(ctx, *m);
    for (size_t c = 0; c + 1 < cuts.size(); ++c) {
        const int32_t o0 = cuts[c], o1 = cuts[c + 1];
        const int64_t h0 = int64_t(o0) * np * 2;
        const int64_t base = obound[size_t(o0)];
        {
            Timed t(ctx, MGX_K_TRACE_EMIT);
            launch_trace_emit(dm, dr, o0, o1, offs + h0, base, chunk_max, aidx, nullptr, nullptr, ctx->d_status,
                              ctx->stream);
        }
        CK(cudaGetLastError());
        SolveArgs a;
        a.dtau_max = p->dtau_max;
        a.dv_max = p->dv_max;
        a.I_bdy = p->I_bdy;
        a.o_begin = o0;
        a.o_end = o1;
        {
            const int64_t per = 32 * solve_bins_per_lane(p->precision, int32_t(NB));
            a.n_tiles = int32_t((NB + per - 1) / per);
        }
        a.offs = offs + h0;
        a.base = base;
        a.idx = aidx;
        a.J = J;
        a.status = ctx->d_status;
        a.counters = ctx->prof ? ctx->d_counters : nullptr;
        fill_pair_weights(a);
        {
            Timed t(ctx, MGX_K_SOLVE);
            launch_solve(dm, dl, dr, a, p->precision, p->order == 4 ? 4 : 2, ctx->stream);
        }
        CK(cudaGetLastError());
    }
    if (!p->out_on_device)
        CK(cudaMemcpyAsync(J_out, J, size_t(n) * size_t(NB) * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    dfree(ctx, aidx);
    if (!p->out_on_device) dfree(ctx, J);
    return sync_status(ctx);
}

mgx_status mgx_reduce_mesh(mgx_ctx *ctx, int32_t model, const double *f, double f_small, double f_large,
                           double G_thres, uint64_t seed, double *Gf, double *L, double *ell, uint8_t *keep,
                           int64_t *n_kept) {
    if (!ctx) return MGX_EINVAL;
    ctx->err.clear();
    Model *m = get_model(ctx, model);
    if (!m) return fail(ctx, MGX_EINVAL, "reduce_mesh: no model %d", model);
    if (!f || !keep) return fail(ctx, MGX_EINVAL, "reduce_mesh: null f or keep");
    if (!(f_small > 0.0) || !(f_large > 0.0) || !std::isfinite(f_small) || !std::isfinite(f_large) ||
        !std::isfinite(G_thres))
        return fail(ctx, MGX_EINVAL, "reduce_mesh: f_small, f_large must be > 0 and finite");
    DeviceGuard g(ctx->device);
    const size_t n = size_t(m->n);
    double *fd = nullptr, *gd = nullptr, *ld = nullptr, *ed = nullptr;
    uint8_t *kd = nullptr;
    CK(dalloc(ctx, &fd, n));
    CK(dalloc(ctx, &kd, n));
    if (Gf) CK(dalloc(ctx, &gd, n));
    if (L) CK(dalloc(ctx, &ld, n));
    if (ell) CK(dalloc(ctx, &ed, n));
    CK(cudaMemcpyAsync(fd, f, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    {
        Timed t(ctx, MGX_K_OTHER);
        launch_reduce(mesh_view(*m), fd, f_small, f_large, G_thres, seed, gd, ld, ed, kd, ctx->stream);
    }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(keep, kd, n, cudaMemcpyDeviceToHost, ctx->stream));
    if (Gf) CK(cudaMemcpyAsync(Gf, gd, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (L) CK(cudaMemcpyAsync(L, ld, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (ell) CK(cudaMemcpyAsync(ell, ed, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    dfree(ctx, fd); dfree(ctx, kd); dfree(ctx, gd); dfree(ctx, ld); dfree(ctx, ed);
    const mgx_status s = sync_status(ctx);
    if (s != MGX_OK) return s;
    if (n_kept) {
        int64_t k = 0;
        for (size_t i = 0; i < n; ++i) k += keep[i] != 0;
        *n_kept = k;
    }
    return MGX_OK;
}

mgx_status mgx_solve_u(mgx_ctx *ctx, int32_t model, const mgx_solve_params *p, int64_t o_begin, int64_t o_end,
                       double *u_out) {
    if (!ctx) return MGX_EINVAL;
    ctx->err.clear();
    Model *m = get_model(ctx, model);
    if (!m) return fail(ctx, MGX_EINVAL, "solve_u: no model %d", model);
    if (!p || !u_out) return fail(ctx, MGX_EINVAL, "solve_u: null params or output");
    if (!m->has_lines || !m->has_rays) return fail(ctx, MGX_ESTATE, "solve_u: set_lines / set_rays not called");
    if (!std::isfinite(p->dtau_max) || !(p->dtau_max > 0.0) || !std::isfinite(p->dv_max) || !std::isfinite(p->I_bdy))
        return fail(ctx, MGX_EINVAL, "solve_u: dtau_max must be > 0, dv_max and I_bdy finite");
    if (p->precision != MGX_FP64 && p->precision != MGX_FP32 && p->precision != MGX_FP32_DT64)
        return fail(ctx, MGX_EINVAL, "solve_u: unknown precision");
    if (p->precision == MGX_FP32_DT64 && p->order == 4)
        return fail(ctx, MGX_EINVAL, "solve_u: MGX_FP32_DT64 exists for the second-order scheme only");
    if ((p->order != 0 && p->order != 2 && p->order != 4) || p->reserved != 0)
        return fail(ctx, MGX_EINVAL, "solve_u: order must be 0, 2 or 4 (reserved 0)");
    if (o_begin < 0 || o_end > m->n || o_begin > o_end) return fail(ctx, MGX_EINVAL, "solve_u: bad origin range");
    if (o_begin == o_end) return MGX_OK;
    DeviceGuard g(ctx->device);
    const int32_t o0 = int32_t(o_begin), o1 = int32_t(o_end), np = m->npairs;
    const int64_t n_half = int64_t(o1 - o0) * np * 2, NB = int64_t(m->L) * m->F;
    int64_t *offs = nullptr;
    mgx_status s = trace_offsets(ctx, *m, o0, o1, &offs);
    if (s != MGX_OK) return s;
    int64_t total = 0;
    CK(cudaMemcpyAsync(&total, offs + n_half, sizeof total, cudaMemcpyDeviceToHost, ctx->stream));
    s = sync_status(ctx);
    if (s != MGX_OK || total > int64_t(ctx->arena_budget / sizeof(int32_t))) {
        dfree(ctx, offs);
        return s != MGX_OK ? s : fail(ctx, MGX_ERANGE, "solve_u: traced lists of the range exceed the arena");
    }
    const size_t n_u = size_t(o1 - o0) * size_t(np) * size_t(NB);
    int32_t *aidx = nullptr;
    double *J = nullptr, *u = nullptr;
    CK(dalloc(ctx, &aidx, size_t(std::max<int64_t>(total, 1))));
    CK(dalloc(ctx, &J, size_t(m->n) * size_t(NB)));  // the kernel indexes J by absolute origin
    if (p->out_on_device) u = u_out;
    else CK(dalloc(ctx, &u, n_u));
    const DevMesh dm = mesh_view(*m);
    const DevRays dr = rays_view(ctx, *m);
    launch_trace_emit(dm, dr, o0, o1, offs, 0, total, aidx, nullptr, nullptr, ctx->d_status, ctx->stream);
    SolveArgs a;
    a.dtau_max = p->dtau_max;
    a.dv_max = p->dv_max;
    a.I_bdy = p->I_bdy;
    a.o_begin = o0;
    a.o_end = o1;
    {
        const int64_t per = 32 * solve_bins_per_lane(p->precision, int32_t(NB));
        a.n_tiles = int32_t((NB + per - 1) / per);
    }
    a.offs = offs;
    a.base = 0;
    a.idx = aidx;
    a.J = J;
    a.u_out = u;
    a.status = ctx->d_status;
    a.counters = ctx->prof ? ctx->d_counters : nullptr;
    fill_pair_weights(a);
    {
        Timed t(ctx, MGX_K_SOLVE);
        launch_solve(dm, lines_view(*m), dr, a, p->precision, p->order == 4 ? 4 : 2, ctx->stream);
    }
    CK(cudaGetLastError());
    if (!p->out_on_device) CK(cudaMemcpyAsync(u_out, u, n_u * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    dfree(ctx, aidx);
    dfree(ctx, J);
    dfree(ctx, offs);
    if (!p->out_on_device) dfree(ctx, u);
    return sync_status(ctx);
}

mgx_status mgx_analytic_mesh(mgx_ctx *ctx, int32_t nx, int32_t ny, int32_t nz, const double *f, double h,
                             double ell_min, double ell_max, uint64_t seed, double *Gf, double *ell,
                             uint8_t *keep, int64_t *n_kept) {
    if (!ctx) return MGX_EINVAL;
    ctx->err.clear();
    if (nx < 1 || ny < 1 || nz < 1 || !f || !keep) return fail(ctx, MGX_EINVAL, "analytic_mesh: bad sizes or null f/keep");
    if (!(h > 0.0) || !std::isfinite(h) || !(ell_min >= h) || !(ell_max >= ell_min) || !std::isfinite(ell_max))
        return fail(ctx, MGX_EINVAL, "analytic_mesh: need 0 < h <= ell_min <= ell_max, finite");
    const int64_t n = int64_t(nx) * ny * nz;
    for (int64_t q = 0; q < n; ++q)
        if (!(f[q] > 0.0) || !std::isfinite(f[q])) return fail(ctx, MGX_EINVAL, "analytic_mesh: f[%lld] is not finite and > 0", (long long)q);
    DeviceGuard g(ctx->device);
    double *fd = nullptr, *gd = nullptr, *ed = nullptr;
    uint8_t *kd = nullptr;
    unsigned long long *cnt = nullptr;  // [0] min bits, [1] max bits, [2] kept
    CK(dalloc(ctx, &fd, size_t(n)));
    CK(dalloc(ctx, &gd, size_t(n)));
    CK(dalloc(ctx, &kd, size_t(n)));
    if (ell) CK(dalloc(ctx, &ed, size_t(n)));
    CK(dalloc(ctx, &cnt, 3));
    const unsigned long long init[3] = {~0ull, 0ull, 0ull};
    CK(cudaMemcpyAsync(cnt, init, sizeof init, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(fd, f, size_t(n) * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    {
        Timed t(ctx, MGX_K_OTHER);
        launch_size_field(nx, ny, nz, fd, h, gd, cnt, ctx->stream);
        launch_size_map(n, gd, cnt, h, ell_min, ell_max, seed, ed, kd, cnt + 2, ctx->stream);
    }
    CK(cudaGetLastError());
    unsigned long long kept = 0;
    CK(cudaMemcpyAsync(keep, kd, size_t(n), cudaMemcpyDeviceToHost, ctx->stream));
    if (Gf) CK(cudaMemcpyAsync(Gf, gd, size_t(n) * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (ell) CK(cudaMemcpyAsync(ell, ed, size_t(n) * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(&kept, cnt + 2, sizeof kept, cudaMemcpyDeviceToHost, ctx->stream));
    dfree(ctx, fd); dfree(ctx, gd); dfree(ctx, kd); dfree(ctx, ed); dfree(ctx, cnt);
    const mgx_status s = sync_status(ctx);
    if (s != MGX_OK) return s;
    if (n_kept) *n_kept = int64_t(kept);
    return MGX_OK;
}

mgx_status mgx_solve_J_noalloc(mgx_ctx *ctx, int32_t model, const mgx_solve_params *p, double *J_out) {
    if (!ctx) return MGX_EINVAL;
    ctx->err.clear();
    Model *m = get_model(ctx, model);
    if (!m) return fail(ctx, MGX_EINVAL, "solve_J_noalloc: no model %d", model);
    if (!p || !J_out) return fail(ctx, MGX_EINVAL, "solve_J_noalloc: null params or output");
    if (!m->has_lines) return fail(ctx, MGX_ESTATE, "solve_J_noalloc: set_lines not called");
    if (!m->has_rays) return fail(ctx, MGX_ESTATE, "solve_J_noalloc: set_rays not called");
    if (!std::isfinite(p->dtau_max) || !(p->dtau_max > 0.0)) return fail(ctx, MGX_EINVAL, "solve_J_noalloc: dtau_max must be > 0");
    if (!std::isfinite(p->dv_max)) return fail(ctx, MGX_EINVAL, "solve_J_noalloc: dv_max must be finite");
    if (!std::isfinite(p->I_bdy)) return fail(ctx, MGX_EINVAL, "solve_J_noalloc: I_bdy must be finite");
    if (p->precision != MGX_FP64 && p->precision != MGX_FP32 && p->precision != MGX_FP32_DT64)
        return fail(ctx, MGX_EINVAL, "solve_J_noalloc: unknown precision");
    if (p->precision == MGX_FP32_DT64 && p->order == 4)
        return fail(ctx, MGX_EINVAL, "solve_J_noalloc: MGX_FP32_DT64 exists for the second-order scheme only");
    if ((p->order != 0 && p->order != 2 && p->order != 4) || p->reserved != 0)
        return fail(ctx, MGX_EINVAL, "solve_J_noalloc: order must be 0, 2 or 4 (reserved 0)");
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, J_out) != cudaSuccess || attr.type != cudaMemoryTypeDevice ||
        attr.device != ctx->device) {
        cudaGetLastError();
        return fail(ctx, MGX_EINVAL, "solve_J_noalloc: J_out must be device memory of device %d", ctx->device);
    }
    DeviceGuard g(ctx->device);
    char msg[256] = {0};
    const int rc = noalloc_solve(ctx->device, mesh_view(*m), lines_view(*m), rays_view(ctx, *m), p->dtau_max,
                                 p->dv_max, p->I_bdy, p->precision, p->order == 4 ? 4 : 2, J_out, ctx->d_status,
                                 ctx->stream, msg,
                                 sizeof msg);
    if (rc != MGX_OK) {
        cudaGetLastError();
        return fail(ctx, rc, "solve_J_noalloc: %s", msg);
    }
    return sync_status(ctx);
}


mgx_status mgx_solve_J_batch(mgx_ctx *ctx, const int32_t *models, int32_t n_models, const mgx_solve_params *p,
                             double *const *J_out, int32_t flags) {
    if (!ctx) return MGX_EINVAL;
    ctx->err.clear();
    if (!models || !p || !J_out || n_models < 1 || n_models > 65535)
        return fail(ctx, MGX_EINVAL, "solve_J_batch: bad model list, params or outputs");
    if (!std::isfinite(p->dtau_max) || !(p->dtau_max > 0.0)) return fail(ctx, MGX_EINVAL, "solve_J_batch: dtau_max must be > 0");
    if (!std::isfinite(p->dv_max) || !std::isfinite(p->I_bdy)) return fail(ctx, MGX_EINVAL, "solve_J_batch: dv_max, I_bdy must be finite");
    if (p->precision != MGX_FP64 && p->precision != MGX_FP32 && p->precision != MGX_FP32_DT64)
        return fail(ctx, MGX_EINVAL, "solve_J_batch: unknown precision");
    if (p->precision == MGX_FP32_DT64 && p->order == 4)
        return fail(ctx, MGX_EINVAL, "solve_J_batch: MGX_FP32_DT64 exists for the second-order scheme only");
    if ((p->order != 0 && p->order != 2 && p->order != 4) || p->reserved != 0)
        return fail(ctx, MGX_EINVAL, "solve_J_batch: order must be 0, 2 or 4 (reserved 0)");
    if (flags & ~(MGX_BATCH_GRAPH | MGX_BATCH_RAYS)) return fail(ctx, MGX_EINVAL, "solve_J_batch: unknown flags");
    std::vector<Model *> ms;
    for (int32_t k = 0; k < n_models; ++k) {
        Model *m = get_model(ctx, models[k]);
        if (!m) return fail(ctx, MGX_EINVAL, "solve_J_batch: no model %d", models[k]);
        if (!m->has_lines || !m->has_rays) return fail(ctx, MGX_ESTATE, "solve_J_batch: model %d lacks lines or rays", models[k]);
        for (int32_t j = 0; j < k; ++j)
            if (models[j] == models[k]) return fail(ctx, MGX_EINVAL, "solve_J_batch: model %d listed twice", models[k]);
        cudaPointerAttributes attr;
        if (!J_out[k] || cudaPointerGetAttributes(&attr, J_out[k]) != cudaSuccess ||
            (attr.type == cudaMemoryTypeDevice && attr.device != ctx->device)) {
            cudaGetLastError();
            return fail(ctx, MGX_EINVAL, "solve_J_batch: J_out[%d] must be host memory or device memory of device %d",
                        k, ctx->device);
        }
        ms.push_back(m);
    }
    DeviceGuard g(ctx->device);
    BatchPlan &pl = ctx->plan;
    const bool graph = (flags & MGX_BATCH_GRAPH) != 0;
    if (graph && plan_matches(pl, models, n_models, p, J_out, flags, ctx->tune) && pl.exec) {
        CK(cudaGraphLaunch(pl.exec, ctx->stream));
        ctx->launches[MGX_K_SOLVE] += 1;
        const mgx_status s = finish_batch_step(ctx, pl);
        if (s != MGX_OK) free_plan(ctx, pl);
        return s;
    }
    free_plan(ctx, pl);
    pl.models.assign(models, models + n_models);
    pl.J.assign(J_out, J_out + n_models);
    pl.p = *p;
    pl.flags = flags;
    pl.tune = ctx->tune;
    int64_t max_nb = 1;
    pl.max_lines = 1;
    for (Model *m : ms) {
        max_nb = std::max<int64_t>(max_nb, int64_t(m->L) * m->F);
        pl.max_lines = std::max(pl.max_lines, int(m->L));
    }
    pl.bpl = solve_bins_per_lane(p->precision, int32_t(max_nb));
    if (p->precision != MGX_FP64 && pl.tune.bins_per_lane > 0) pl.bpl = pl.tune.bins_per_lane;
    std::vector<BatchGeom> geo(static_cast<size_t>(n_models));
    std::vector<int64_t> obase(static_cast<size_t>(n_models));
    pl.total_half = pl.n_origins = pl.n_work = 0;
    for (int32_t k = 0; k < n_models; ++k) {
        const Model &m = *ms[size_t(k)];
        const int64_t nb = int64_t(m.L) * m.F;
        geo[size_t(k)].half_base = pl.total_half;
        geo[size_t(k)].npairs2 = 2 * m.npairs;
        geo[size_t(k)].n_tiles = int32_t((nb + 32 * pl.bpl - 1) / (32 * pl.bpl));
        obase[size_t(k)] = pl.n_origins;
        pl.total_half += int64_t(m.n) * m.npairs * 2;
        pl.n_origins += m.n;
        geo[size_t(k)].work_base = pl.n_work;
        pl.n_work += int64_t(m.n) * geo[size_t(k)].n_tiles;
        if (geo[size_t(k)].n_tiles > 65535) return fail(ctx, MGX_ERANGE, "solve_J_batch: too many frequency tiles");
    }
    // outputs in host memory are staged on the device and copied back after each step
    pl.Jdev.assign(size_t(n_models), nullptr);
    pl.Jbytes.assign(size_t(n_models), 0);
    for (int32_t k = 0; k < n_models; ++k) {
        cudaPointerAttributes attr;
        CK(cudaPointerGetAttributes(&attr, J_out[k]));
        if (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged) continue;
        const Model &m = *ms[size_t(k)];
        pl.Jbytes[size_t(k)] = size_t(m.n) * size_t(m.L) * size_t(m.F) * sizeof(double);
        CK(dalloc(ctx, &pl.Jdev[size_t(k)], size_t(m.n) * size_t(m.L) * size_t(m.F)));
    }
    CK(dalloc(ctx, &pl.lens, size_t(pl.total_half)));
    CK(dalloc(ctx, &pl.excess, size_t(pl.total_half)));
    CK(dalloc(ctx, &pl.resume, size_t(pl.total_half)));
    CK(dalloc(ctx, &pl.offs, size_t(pl.total_half + 1)));
    CK(dalloc(ctx, &pl.obase, size_t(n_models)));
    CK(dalloc(ctx, &pl.geo, size_t(n_models)));
    CK(dalloc(ctx, &pl.slots, size_t(n_models)));
    CK(dalloc(ctx, &pl.work, size_t(pl.n_work)));
    CK(dalloc(ctx, &pl.scratch, kScratchSize));
    if (pl.n_origins > int64_t(INT32_MAX)) return fail(ctx, MGX_ERANGE, "solve_J_batch: more than 2^31 origins");
    CK(dalloc(ctx, &pl.wl.key_in, size_t(pl.n_origins)));
    CK(dalloc(ctx, &pl.wl.key_out, size_t(pl.n_origins)));
    CK(dalloc(ctx, &pl.wl.val_in, size_t(pl.n_origins)));
    CK(dalloc(ctx, &pl.wl.val_out, size_t(pl.n_origins)));
    CK(dalloc(ctx, &pl.wl.tiles, size_t(pl.n_origins)));
    CK(dalloc(ctx, &pl.wl.toff, size_t(pl.n_origins)));
    pl.wl.tmp_bytes = batch_worklist_temp_bytes(pl.n_origins);
    CK(cudaMallocAsync(&pl.wl.tmp, pl.wl.tmp_bytes ? pl.wl.tmp_bytes : 1, ctx->stream));
    CK(cub::DeviceScan::InclusiveSum(nullptr, pl.cub_bytes, pl.excess, pl.offs + 1, pl.total_half, ctx->stream));
    CK(cudaMallocAsync(&pl.cub_tmp, pl.cub_bytes ? pl.cub_bytes : 1, ctx->stream));
    CK(cudaMemcpyAsync(pl.geo, geo.data(), geo.size() * sizeof(BatchGeom), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(pl.obase, obase.data(), obase.size() * sizeof(int64_t), cudaMemcpyHostToDevice, ctx->stream));
    // the row width from the lengths of a sample of the half-rays: every kSampleShare-th origin
    // of each model (all of a small model), one launch per model; the rest of the lengths stay
    // 0 and add nothing to the totals, whose ratios pick the width
    if (flags & MGX_BATCH_RAYS)
        for (Model *m : ms) enqueue_rays(ctx, *m, false);  // planning is not part of a step's profile
    CK(cudaMemsetAsync(pl.lens, 0, size_t(pl.total_half) * sizeof(int64_t), ctx->stream));
    {
        int64_t hb = 0;
        for (Model *m : ms) {
            const int32_t n = m->n, np2 = 2 * m->npairs;
            launch_trace_count(mesh_view(*m), rays_view(ctx, *m), 0, n, pl.lens + hb, ctx->d_status, nullptr,
                               ctx->stream, n <= kSampleAll ? 1 : kSampleShare);
            hb += int64_t(n) * np2;
        }
    }
    launch_excess_totals(pl.lens, pl.total_half, pl.scratch + kScratchTotals, ctx->stream);
    unsigned long long tot[kPadCandidates + 1] = {};
    CK(cudaMemcpyAsync(tot, pl.scratch + kScratchTotals, sizeof tot, cudaMemcpyDeviceToHost, ctx->stream));
    mgx_status s = sync_status(ctx);
    if (s != MGX_OK) {
        free_plan(ctx, pl);
        return s;
    }
    size_t free_b = 0, total_b = 0;
    CK(cudaMemGetInfo(&free_b, &total_b));
    // the rows may take up to a third of free device memory (at most kRowsBudget): every point
    // they do not hold is walked a second time by the tail pass
    pl.pad = choose_pad(tot, pl.total_half, std::min(kRowsBudget, free_b / 3),
                        pl.tune.tail_permille > 0 ? pl.tune.tail_permille : 20);
    int j = 0;
    while ((int32_t(1) << j) < pl.pad) ++j;
    CK(dalloc(ctx, &pl.rows, size_t(pl.total_half) * size_t(pl.pad)));
    // the first step's padded trace gives every length: the exact tail, then the rest of the step
    s = enqueue_batch_front(ctx, pl, ms);
    if (s != MGX_OK) {
        free_plan(ctx, pl);
        return s;
    }
    launch_excess_totals(pl.lens, pl.total_half, pl.scratch + kScratchTotals, ctx->stream);
    CK(cudaMemcpyAsync(tot, pl.scratch + kScratchTotals, sizeof tot, cudaMemcpyDeviceToHost, ctx->stream));
    s = sync_status(ctx);
    if (s != MGX_OK) {
        free_plan(ctx, pl);
        return s;
    }
    pl.tail_cap = int64_t(tot[j]);
    pl.total_points = int64_t(tot[kPadCandidates]);
    CK(dalloc(ctx, &pl.tail, size_t(std::max<int64_t>(pl.tail_cap, 1))));
    std::vector<BatchSlot> slots(static_cast<size_t>(n_models));
    for (int32_t k = 0; k < n_models; ++k) {
        Model &m = *ms[size_t(k)];
        BatchSlot &b = slots[size_t(k)];
        b.m = mesh_view(m);
        b.Ln = lines_view(m);
        b.R = rays_view(ctx, m);
        SolveArgs &a = b.a;
        a.dtau_max = p->dtau_max;
        a.dv_max = p->dv_max;
        a.I_bdy = p->I_bdy;
        a.o_begin = 0;
        a.o_end = m.n;
        a.n_tiles = geo[size_t(k)].n_tiles;
        a.offs = pl.offs + geo[size_t(k)].half_base;
        a.base = 0;
        a.idx = pl.rows + geo[size_t(k)].half_base * pl.pad;
        a.pad = pl.pad;
        a.lens = pl.lens + geo[size_t(k)].half_base;
        a.tail = pl.tail;
        a.J = pl.Jdev[size_t(k)] ? pl.Jdev[size_t(k)] : J_out[k];
        a.status = ctx->d_status;
        a.counters = ctx->prof ? ctx->d_counters : nullptr;
        fill_pair_weights(a);
        ctx->solves += int64_t(m.n) * m.npairs * int64_t(m.L) * m.F;
    }
    ctx->trace_points += pl.total_points;
    CK(cudaMemcpyAsync(pl.slots, slots.data(), slots.size() * sizeof(BatchSlot), cudaMemcpyHostToDevice, ctx->stream));
    s = enqueue_batch_back(ctx, pl, ms);
    if (s != MGX_OK) {
        free_plan(ctx, pl);
        return s;
    }
    s = finish_batch_step(ctx, pl);
    if (s != MGX_OK) {
        free_plan(ctx, pl);
        return s;
    }
    pl.valid = true;
    if (graph) {
        // capture the whole step for replay; kernels only, no profiling events
        const bool prof = ctx->prof;
        ctx->prof = false;
        for (auto &sl : slots) sl.a.counters = nullptr;
        CK(cudaMemcpyAsync(pl.slots, slots.data(), slots.size() * sizeof(BatchSlot), cudaMemcpyHostToDevice,
                           ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        if (!ctx->capture_stream) CK(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
        cudaStream_t user = ctx->stream;
        ctx->stream = ctx->capture_stream;
        cudaError_t ce = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
        mgx_status s2 = MGX_ECUDA;
        cudaGraph_t gr = nullptr;
        if (ce == cudaSuccess) {
            s2 = enqueue_batch_step(ctx, pl, ms);
            ce = cudaStreamEndCapture(ctx->stream, &gr);
        }
        ctx->stream = user;
        ctx->prof = prof;
        if (s2 != MGX_OK || ce != cudaSuccess) {
            if (gr) cudaGraphDestroy(gr);
            cudaGetLastError();
            free_plan(ctx, pl);
            return s2 != MGX_OK ? s2 : fail(ctx, MGX_ECUDA, "solve_J_batch: graph capture failed: %s", cudaGetErrorString(ce));
        }
        pl.graph = gr;
        CK(cudaGraphInstantiate(&pl.exec, gr, 0));
    }
    return MGX_OK;
}


mgx_status mgx_set_tuning(mgx_ctx *ctx, const mgx_tuning *t) {
    if (!ctx) return MGX_EINVAL;
    ctx->err.clear();
    mgx_tuning v{};
    if (t) {
        v = *t;
        if (!valid_tuning(v)) return fail(ctx, MGX_EINVAL, "set_tuning: a field is out of range");
    }
    if (!same_tuning(v, ctx->tune)) {
        DeviceGuard g(ctx->device);
        free_plan(ctx, ctx->plan);
    }
    ctx->tune = v;
    return MGX_OK;
}

mgx_status mgx_get_tuning(mgx_ctx *ctx, mgx_tuning *t) {
    if (!ctx || !t) return MGX_EINVAL;
    *t = ctx->tune;
    return MGX_OK;
}

mgx_status mgx_autotune(mgx_ctx *ctx, const int32_t *models, int32_t n_models, const mgx_solve_params *p,
                        double *const *J_out, int32_t flags, int32_t reps, mgx_tune_trial *trials,
                        int32_t max_trials, int32_t *n_trials) {
    if (!ctx) return MGX_EINVAL;
    ctx->err.clear();
    if (n_trials) *n_trials = 0;
    if (reps < 1 || reps > 100) return fail(ctx, MGX_EINVAL, "autotune: reps must be in 1..100");
    if (max_trials < 0 || (max_trials > 0 && !trials)) return fail(ctx, MGX_EINVAL, "autotune: bad trial buffer");
    if (!models || !p || n_models < 1) return fail(ctx, MGX_EINVAL, "autotune: bad model list or params");
    int64_t max_nb = 1;
    for (int32_t k = 0; k < n_models; ++k) {
        const Model *m = get_model(ctx, models[k]);
        if (!m) return fail(ctx, MGX_EINVAL, "autotune: no model %d", models[k]);
        max_nb = std::max<int64_t>(max_nb, int64_t(m->L) * m->F);
    }
    DeviceGuard g(ctx->device);
    const mgx_tuning saved = ctx->tune;
    const bool prof = ctx->prof;
    ctx->prof = false;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int32_t count = 0;
    // candidate -> median step time; the plan (and graph) is built by an untimed first call
    auto time_one = [&](const mgx_tuning &t, double *ms) -> mgx_status {
        ctx->tune = t;
        mgx_status s = mgx_solve_J_batch(ctx, models, n_models, p, J_out, flags);
        if (s != MGX_OK) return s;
        std::vector<float> v;
        for (int32_t r = 0; r < reps; ++r) {
            if (cudaEventRecord(e0, ctx->stream) != cudaSuccess) return fail(ctx, MGX_ECUDA, "autotune: event");
            s = mgx_solve_J_batch(ctx, models, n_models, p, J_out, flags);
            if (s != MGX_OK) return s;
            if (cudaEventRecord(e1, ctx->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
                return fail(ctx, MGX_ECUDA, "autotune: event");
            float x = 0.0f;
            cudaEventElapsedTime(&x, e0, e1);
            v.push_back(x);
        }
        std::sort(v.begin(), v.end());
        *ms = double(v[v.size() / 2]);
        if (count < max_trials) trials[count] = mgx_tune_trial{t, *ms};
        ++count;
        return MGX_OK;
    };
    // start from the current tuning with its automatic fields made explicit
    mgx_tuning best = saved;
    if (best.bins_per_lane == 0 && p->precision != MGX_FP64) best.bins_per_lane = solve_bins_per_lane(MGX_FP32, int32_t(max_nb));
    if (best.trace_ctas_per_sm == 0) best.trace_ctas_per_sm = 7;
    if (best.tail_permille == 0) best.tail_permille = 20;
    double best_ms = 0.0;
    mgx_status s = time_one(best, &best_ms);
    const int32_t bpl_c[] = {1, 2}, trace_c[] = {4, 5, 7}, tail_c[] = {5, 20, 80}, sched_c[] = {0, 1};
    for (int dim = 0; dim < 4 && s == MGX_OK; ++dim) {
        if (dim == 0 && p->precision == MGX_FP64) continue;
        const int32_t *cand = dim == 0 ? bpl_c : dim == 1 ? trace_c : dim == 2 ? tail_c : sched_c;
        const int nc = (dim == 0 || dim == 3) ? 2 : 3;
        const mgx_tuning base = best;
        for (int c = 0; c < nc && s == MGX_OK; ++c) {
            mgx_tuning t = base;
            int32_t &field = dim == 0 ? t.bins_per_lane : dim == 1 ? t.trace_ctas_per_sm
                           : dim == 2 ? t.tail_permille : t.schedule;
            if (field == cand[c]) continue;
            field = cand[c];
            double ms = 0.0;
            s = time_one(t, &ms);
            if (s == MGX_OK && ms < best_ms) {
                best = t;
                best_ms = ms;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->prof = prof;
    if (n_trials) *n_trials = count;
    if (s != MGX_OK) {
        ctx->tune = saved;
        free_plan(ctx, ctx->plan);
        return s;
    }
    ctx->tune = best;
    return mgx_solve_J_batch(ctx, models, n_models, p, J_out, flags);  // leaves the fastest plan in place
}

mgx_status mgx_mlp_set_params(mgx_ctx *ctx, const float *theta) {
    if (!ctx) return MGX_EINVAL;
    ctx->err.clear();
    if (!theta) return fail(ctx, MGX_EINVAL, "mlp_set_params: null parameters");
    for (int i = 0; i < kMlpN; ++i)
        if (!std::isfinite(theta[i])) return fail(ctx, MGX_EINVAL, "mlp_set_params: non-finite parameter %d", i);
    DeviceGuard g(ctx->device);
    if (!ctx->mlp_theta) {
        CK(dalloc(ctx, &ctx->mlp_theta, kMlpN));
        CK(dalloc(ctx, &ctx->mlp_m, kMlpN));
        CK(dalloc(ctx, &ctx->mlp_v, kMlpN));
        CK(dalloc(ctx, &ctx->mlp_grad, kMlpN));
        CK(dalloc(ctx, &ctx->mlp_loss, 1));
        CK(cudaMallocAsync(&ctx->mlp_W1b, 16 * 64 * 2, ctx->stream));
        CK(cudaMallocAsync(&ctx->mlp_W2b, 64 * 64 * 2, ctx->stream));
    }
    CK(cudaMemcpyAsync(ctx->mlp_theta, theta, kMlpN * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemsetAsync(ctx->mlp_m, 0, kMlpN * sizeof(float), ctx->stream));
    CK(cudaMemsetAsync(ctx->mlp_v, 0, kMlpN * sizeof(float), ctx->stream));
    CK(cudaMemsetAsync(ctx->mlp_grad, 0, kMlpN * sizeof(float), ctx->stream));
    {
        Timed t(ctx, MGX_K_OTHER);
        launch_mlp_convert(ctx->mlp_theta, ctx->mlp_W1b, ctx->mlp_W2b, ctx->stream);
    }
    ctx->mlp_step = 0;
    return sync_status(ctx);
}

mgx_status mgx_mlp_get_params(mgx_ctx *ctx, float *theta) {
    if (!ctx) return MGX_EINVAL;
    ctx->err.clear();
    if (!theta) return fail(ctx, MGX_EINVAL, "mlp_get_params: null output");
    if (!ctx->mlp_theta) return fail(ctx, MGX_ESTATE, "mlp_get_params: mgx_mlp_set_params not called");
    DeviceGuard g(ctx->device);
    CK(cudaMemcpyAsync(theta, ctx->mlp_theta, kMlpN * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return MGX_OK;
}

mgx_status mgx_mlp_forward(mgx_ctx *ctx, const float *X, int64_t n, float *y) {
    if (!ctx) return MGX_EINVAL;
    ctx->err.clear();
    if (!X || !y || n < 1 || n >= (int64_t(1) << 31)) return fail(ctx, MGX_EINVAL, "mlp_forward: bad arguments");
    if (!ctx->mlp_theta) return fail(ctx, MGX_ESTATE, "mlp_forward: mgx_mlp_set_params not called");
    DeviceGuard g(ctx->device);
    float *Xd = nullptr, *yd = nullptr;
    CK(dalloc(ctx, &Xd, size_t(n) * 8));
    CK(dalloc(ctx, &yd, size_t(n)));
    CK(cudaMemcpyAsync(Xd, X, size_t(n) * 8 * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    {
        Timed t(ctx, MGX_K_OTHER);
        launch_mlp(false, Xd, nullptr, nullptr, n, ctx->mlp_W1b, ctx->mlp_W2b, ctx->mlp_theta, yd, nullptr, nullptr,
                   0.0f, ctx->stream);
    }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(y, yd, size_t(n) * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    dfree(ctx, Xd);
    dfree(ctx, yd);
    return sync_status(ctx);
}

mgx_status mgx_mlp_grad(mgx_ctx *ctx, const float *X, const float *t, int64_t n, float *grad, float *loss) {
    if (!ctx) return MGX_EINVAL;
    ctx->err.clear();
    if (!X || !t || !grad || n < 1 || n >= (int64_t(1) << 31)) return fail(ctx, MGX_EINVAL, "mlp_grad: bad arguments");
    if (!ctx->mlp_theta) return fail(ctx, MGX_ESTATE, "mlp_grad: mgx_mlp_set_params not called");
    DeviceGuard g(ctx->device);
    float *Xd = nullptr, *td = nullptr;
    CK(dalloc(ctx, &Xd, size_t(n) * 8));
    CK(dalloc(ctx, &td, size_t(n)));
    CK(cudaMemcpyAsync(Xd, X, size_t(n) * 8 * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(td, t, size_t(n) * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemsetAsync(ctx->mlp_grad, 0, kMlpN * sizeof(float), ctx->stream));
    CK(cudaMemsetAsync(ctx->mlp_loss, 0, sizeof(float), ctx->stream));
    {
        Timed tm(ctx, MGX_K_OTHER);
        launch_mlp(true, Xd, td, nullptr, n, ctx->mlp_W1b, ctx->mlp_W2b, ctx->mlp_theta, nullptr, ctx->mlp_grad,
                   ctx->mlp_loss, float(2.0 / double(n)), ctx->stream);
    }
    CK(cudaGetLastError());
    float lsum = 0.0f;
    CK(cudaMemcpyAsync(grad, ctx->mlp_grad, kMlpN * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(&lsum, ctx->mlp_loss, sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemsetAsync(ctx->mlp_grad, 0, kMlpN * sizeof(float), ctx->stream));
    dfree(ctx, Xd);
    dfree(ctx, td);
    const mgx_status s = sync_status(ctx);
    if (loss) *loss = lsum / float(n);
    return s;
}

mgx_status mgx_mlp_train(mgx_ctx *ctx, const float *X, const float *t, int64_t n, int32_t epochs, int32_t batch,
                         float lr, uint64_t seed, float *loss_per_epoch) {
    if (!ctx) return MGX_EINVAL;
    ctx->err.clear();
    if (!X || !t || n < 1 || n >= (int64_t(1) << 31) || epochs < 1 || batch < 1 || !(lr > 0.0f) || !std::isfinite(lr))
        return fail(ctx, MGX_EINVAL, "mlp_train: bad arguments");
    if (!ctx->mlp_theta) return fail(ctx, MGX_ESTATE, "mlp_train: mgx_mlp_set_params not called");
    DeviceGuard g(ctx->device);
    float *Xd = nullptr, *td = nullptr;
    int32_t *perm = nullptr;
    CK(dalloc(ctx, &Xd, size_t(n) * 8));
    CK(dalloc(ctx, &td, size_t(n)));
    CK(dalloc(ctx, &perm, size_t(n)));
    CK(cudaMemcpyAsync(Xd, X, size_t(n) * 8 * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(td, t, size_t(n) * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    std::vector<int32_t> order(static_cast<size_t>(n));
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    uint64_t state = seed;
    auto next_u64 = [&state]() {  // SplitMix64 (Steele, Lea & Flood 2014) for the shuffles
        uint64_t z = (state += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    for (int32_t ep = 0; ep < epochs; ++ep) {
        for (int64_t i = 0; i < n; ++i) order[size_t(i)] = int32_t(i);
        for (int64_t i = n - 1; i > 0; --i) std::swap(order[size_t(i)], order[size_t(next_u64() % uint64_t(i + 1))]);
        CK(cudaMemcpyAsync(perm, order.data(), size_t(n) * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemsetAsync(ctx->mlp_loss, 0, sizeof(float), ctx->stream));
        for (int64_t b0 = 0; b0 < n; b0 += batch) {
            const int64_t rows = std::min<int64_t>(batch, n - b0);
            {
                Timed tm(ctx, MGX_K_OTHER);
                launch_mlp(true, Xd, td, perm + b0, rows, ctx->mlp_W1b, ctx->mlp_W2b, ctx->mlp_theta, nullptr,
                           ctx->mlp_grad, ctx->mlp_loss, float(2.0 / double(rows)), ctx->stream);
            }
            ctx->mlp_step += 1;
            const float c1 = float(1.0 / (1.0 - std::pow(double(b1), double(ctx->mlp_step))));
            const float c2 = float(1.0 / (1.0 - std::pow(double(b2), double(ctx->mlp_step))));
            {
                Timed tm(ctx, MGX_K_OTHER);
                launch_mlp_adam(ctx->mlp_theta, ctx->mlp_m, ctx->mlp_v, ctx->mlp_grad, lr, b1, b2, eps, c1, c2,
                                ctx->mlp_W1b, ctx->mlp_W2b, ctx->stream);
            }
        }
        CK(cudaGetLastError());
        if (loss_per_epoch) {
            float lsum = 0.0f;
            CK(cudaMemcpyAsync(&lsum, ctx->mlp_loss, sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
            loss_per_epoch[ep] = lsum / float(n);
        }
    }
    dfree(ctx, Xd);
    dfree(ctx, td);
    dfree(ctx, perm);
    return sync_status(ctx);
}

mgx_status mgx_mlp_features(mgx_ctx *ctx, int32_t model, const double *rho, const double *T, float *X) {
    if (!ctx) return MGX_EINVAL;
    ctx->err.clear();
    Model *m = get_model(ctx, model);
    if (!m) return fail(ctx, MGX_EINVAL, "mlp_features: no model %d", model);
    if (!m->has_lines) return fail(ctx, MGX_ESTATE, "mlp_features: set_lines not called");
    if (!rho || !T || !X) return fail(ctx, MGX_EINVAL, "mlp_features: null pointer");
    for (int64_t i = 0; i < m->n; ++i)
        if (!(rho[i] > 0.0) || !(T[i] > 0.0) || !std::isfinite(rho[i]) || !std::isfinite(T[i]))
            return fail(ctx, MGX_EINVAL, "mlp_features: rho and T must be positive and finite (point %lld)", (long long)i);
    DeviceGuard g(ctx->device);
    const size_t n = size_t(m->n);
    double *rd = nullptr, *Td = nullptr;
    float *Xd = nullptr;
    CK(dalloc(ctx, &rd, n));
    CK(dalloc(ctx, &Td, n));
    CK(dalloc(ctx, &Xd, n * 8));
    CK(cudaMemcpyAsync(rd, rho, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(Td, T, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    {
        Timed t(ctx, MGX_K_OTHER);
        launch_mlp_features(mesh_view(*m), m->chi0f, m->L, m->dvwf, rd, Td, Xd, ctx->stream);
    }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(X, Xd, n * 8 * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    dfree(ctx, rd);
    dfree(ctx, Td);
    dfree(ctx, Xd);
    return sync_status(ctx);
}

mgx_status mgx_reduce_mesh_learned(mgx_ctx *ctx, int32_t model, const float *X, double keep_fraction, uint8_t *keep,
                                   int64_t *n_kept) {
    if (!ctx) return MGX_EINVAL;
    ctx->err.clear();
    Model *m = get_model(ctx, model);
    if (!m) return fail(ctx, MGX_EINVAL, "reduce_mesh_learned: no model %d", model);
    if (!X || !keep || !(keep_fraction >= 0.0) || !(keep_fraction <= 1.0))
        return fail(ctx, MGX_EINVAL, "reduce_mesh_learned: bad arguments");
    if (!ctx->mlp_theta) return fail(ctx, MGX_ESTATE, "reduce_mesh_learned: mgx_mlp_set_params not called");
    DeviceGuard g(ctx->device);
    const int64_t n = m->n;
    const int64_t k = std::llround(keep_fraction * double(n));
    float *Xd = nullptr, *yd = nullptr, *ys = nullptr;
    int32_t *ids = nullptr, *ids_s = nullptr;
    uint8_t *kd = nullptr;
    CK(dalloc(ctx, &Xd, size_t(n) * 8));
    CK(dalloc(ctx, &yd, size_t(n)));
    CK(dalloc(ctx, &ys, size_t(n)));
    CK(dalloc(ctx, &ids, size_t(n)));
    CK(dalloc(ctx, &ids_s, size_t(n)));
    CK(dalloc(ctx, &kd, size_t(n)));
    CK(cudaMemcpyAsync(Xd, X, size_t(n) * 8 * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    {
        Timed t(ctx, MGX_K_OTHER);
        launch_mlp(false, Xd, nullptr, nullptr, n, ctx->mlp_W1b, ctx->mlp_W2b, ctx->mlp_theta, yd, nullptr, nullptr,
                   0.0f, ctx->stream);
        launch_select_top(yd, n, k, ids, ys, ids_s, kd, ctx->stream);
    }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(keep, kd, size_t(n), cudaMemcpyDeviceToHost, ctx->stream));
    dfree(ctx, Xd); dfree(ctx, yd); dfree(ctx, ys); dfree(ctx, ids); dfree(ctx, ids_s); dfree(ctx, kd);
    const mgx_status s = sync_status(ctx);
    if (n_kept) *n_kept = k;
    return s;
}

mgx_status mgx_reduce_mesh_learned_weighted(mgx_ctx *ctx, int32_t model, const float *X, double keep_fraction,
                                            double alpha, uint64_t seed, uint8_t *keep, int64_t *n_kept,
                                            double *scale) {
    if (!ctx) return MGX_EINVAL;
    ctx->err.clear();
    Model *m = get_model(ctx, model);
    if (!m) return fail(ctx, MGX_EINVAL, "reduce_mesh_learned_weighted: no model %d", model);
    if (!X || !keep || !(keep_fraction >= 0.0) || !(keep_fraction <= 1.0) || !(alpha >= 0.0) || !std::isfinite(alpha))
        return fail(ctx, MGX_EINVAL, "reduce_mesh_learned_weighted: bad arguments");
    if (!ctx->mlp_theta) return fail(ctx, MGX_ESTATE, "reduce_mesh_learned_weighted: mgx_mlp_set_params not called");
    DeviceGuard g(ctx->device);
    const int64_t n = m->n;
    const double target = keep_fraction * double(n);
    float *Xd = nullptr, *yd = nullptr, *wd = nullptr;
    double *sd = nullptr;
    unsigned long long *cnt = nullptr;
    uint8_t *kd = nullptr;
    CK(dalloc(ctx, &Xd, size_t(n) * 8));
    CK(dalloc(ctx, &yd, size_t(n)));
    CK(dalloc(ctx, &wd, size_t(n)));
    CK(dalloc(ctx, &sd, 1));
    CK(dalloc(ctx, &cnt, 1));
    CK(dalloc(ctx, &kd, size_t(n)));
    CK(cudaMemcpyAsync(Xd, X, size_t(n) * 8 * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    double c = 0.0;
    {
        Timed t(ctx, MGX_K_OTHER);
        launch_mlp(false, Xd, nullptr, nullptr, n, ctx->mlp_W1b, ctx->mlp_W2b, ctx->mlp_theta, yd, nullptr, nullptr,
                   0.0f, ctx->stream);
        launch_thin_weights(yd, n, float(alpha), wd, ctx->stream);
        // bisection on log2 c: the expected kept count grows with c
        double lo = -400.0, hi = 400.0;
        for (int it = 0; it < 80 && keep_fraction > 0.0 && keep_fraction < 1.0; ++it) {
            const double mid = 0.5 * (lo + hi);
            double sum = 0.0;
            launch_thin_expected(wd, n, std::exp2(mid), sd, ctx->stream);
            CK(cudaMemcpyAsync(&sum, sd, sizeof sum, cudaMemcpyDeviceToHost, ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
            if (sum < target) lo = mid;
            else hi = mid;
        }
        c = keep_fraction <= 0.0 ? 0.0 : keep_fraction >= 1.0 ? 1e300 : std::exp2(0.5 * (lo + hi));
        launch_thin_mark(wd, n, c, seed, kd, cnt, ctx->stream);
    }
    CK(cudaGetLastError());
    unsigned long long kept = 0;
    CK(cudaMemcpyAsync(keep, kd, size_t(n), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(&kept, cnt, sizeof kept, cudaMemcpyDeviceToHost, ctx->stream));
    const mgx_status s = sync_status(ctx);
    dfree(ctx, Xd); dfree(ctx, yd); dfree(ctx, wd); dfree(ctx, sd); dfree(ctx, cnt); dfree(ctx, kd);
    if (s != MGX_OK) return s;
    if (n_kept) *n_kept = int64_t(kept);
    if (scale) *scale = c;
    return MGX_OK;
}

mgx_status mgx_eval_approx(mgx_ctx *ctx, int32_t kind, const float *x, int64_t n, float *y, float *bound) {
    if (!ctx) return MGX_EINVAL;
    ctx->err.clear();
    if (kind < 0 || kind > 2) return fail(ctx, MGX_EINVAL, "eval_approx: kind must be 0, 1 or 2");
    if (n < 0 || (n > 0 && (!x || !y))) return fail(ctx, MGX_EINVAL, "eval_approx: bad arrays");
    if (bound) *bound = kind == 2 ? atan2_bound() : approx_bound(kind);
    DeviceGuard g(ctx->device);
    if (kind == 2) launch_eval_atan2(x, n, y, ctx->stream);
    else launch_eval_approx(kind, x, n, y, ctx->stream);
    CK(cudaGetLastError());
    return MGX_OK;
}

mgx_status mgx_alu_peaks(mgx_ctx *ctx, int32_t reps, double *out) {
    if (!ctx) return MGX_EINVAL;
    ctx->err.clear();
    if (!out || reps < 1 || reps > 100) return fail(ctx, MGX_EINVAL, "alu_peaks: null output or reps outside 1..100");
    DeviceGuard g(ctx->device);
    CK(alu_peaks(ctx->stream, reps, out));
    return MGX_OK;
}

mgx_status mgx_profile_enable(mgx_ctx *ctx, int32_t enable) {
    if (!ctx) return MGX_EINVAL;
    ctx->err.clear();
    DeviceGuard g(ctx->device);
    reset_profile(ctx);
    ctx->prof = enable != 0;
    CK(cudaGetLastError());
    return MGX_OK;
}

mgx_status mgx_profile_read(mgx_ctx *ctx, mgx_profile *out) {
    if (!ctx || !out) return MGX_EINVAL;
    ctx->err.clear();
    DeviceGuard g(ctx->device);
    unsigned long long cnt[kCounters] = {};
    CK(cudaMemcpyAsync(cnt, ctx->d_counters, sizeof cnt, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    std::memset(out, 0, sizeof *out);
    for (int k = 0; k < MGX_K_COUNT; ++k) {
        double ms = 0.0;
        for (auto &pr : ctx->ev[k]) {
            float t = 0.0f;
            CK(cudaEventElapsedTime(&t, pr.first, pr.second));
            ms += double(t);
        }
        out->ms[k] = ms;
        out->launches[k] = ctx->launches[k];
    }
    out->trace_points = ctx->trace_points;
    out->solves = ctx->solves;
    out->updates = int64_t(cnt[1] + cnt[0]);  // one row per sample and bin, plus the extra sub-intervals
    out->samples = int64_t(cnt[1]);
    out->trace_steps = int64_t(cnt[2]);
    out->trace_exact_steps = int64_t(cnt[3]);
    out->decisions_redone = int64_t(cnt[4]);
    return MGX_OK;
}

}  // extern "C"
