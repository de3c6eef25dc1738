// k_solve.cu -- formal solution along ray pairs and the mean intensity J
// (Eqs. 1-3, Sections 2.1.1-2.1.2).
//
// One warp per (origin, 32-bin frequency tile); lane = frequency bin.  The warp
// walks every ray pair of its origin in ascending pair order.  For each half of
// the pair it starts at the far end of the traced point list and eliminates
// towards the origin:
//   * adaptive velocity sampling (Section 2.1.1): between consecutive points
//     whose projected velocities differ by more than dv_max times the smaller
//     Doppler width, equally spaced samples with linearly interpolated data;
//   * line optics: chi = chi_c + sum_l chi0_l exp(-a_l^2), eta likewise, a_l the
//     Doppler-shifted profile argument of line l at this lane's frequency;
//   * adaptive optical-depth increments (Eq. 2): each sample interval is split
//     into n_inter = ceil(max(chi) ds / dtau_max) equal parts with chi and eta
//     linear, trapezoidal dtau;
//   * Gaussian elimination of the Feautrier system (Eq. 1, second-order
//     boundary condition) in the scaled form of Rybicki & Hummer (1991):
//         boundary row:  Fh = 1 + dt/2,            D = 1/(1 + dt Fh), zh = D (S dt/2 + I)
//         interior row:  Fh = dtbar + D Fh,        D = 1/(1 + dt Fh), zh = D (dtbar S + zh)
//     with Fh = F_i / dtau_i and zh = z_i / dtau_i of the textbook 1+B form, so
//     no quantity overflows for small dtau and no difference of nearly equal
//     numbers is formed.  The boundary row is the interior row applied to the
//     state (Fh, D, zh, dtbar) = (1, 1, I, dt/2), and one reciprocal
//     1 / (chi (1 + dt Fh)) per row yields both D and D S = D eta / chi.
// The two half-sweeps meet at the origin row, which gives u without back
// substitution:  u_o = (dtbar S_o + zh- + zh+) / (dtbar + D- Fh- + D+ Fh+),
// an empty half contributing (zh, D Fh) = (I, 1).  J accumulates 2 w u in
// double precision with Neumaier's compensated sum.
//
// Template R selects the arithmetic: double (plain form) or float (the distance
// increments come from double Z differences; J is summed in double).
#include "mgx_internal.cuh"

namespace mgx {

namespace {

template <typename R>
struct Ar;

// Double precision (plain form): the Gaussian exp(-a^2) and Eq. 2's n_inter
// exactly as defined, with IEEE divisions.
template <>
struct Ar<double> {
    static constexpr double kArgScale = 1.0;
    static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
    static __device__ __forceinline__ double gauss(double a) { return exp(-(a * a)); }
    static __device__ __forceinline__ double ninter(double cm, double hs, double dtau_max, double) {
        return ceil(cm * hs / dtau_max);
    }
};

// Single precision: the profile constants are prescaled by sqrt(log2 e), so
// exp(-a^2) = 2^(-a'^2) is one ex2.approx; reciprocals are rcp.approx; Eq. 2's
// ratio is formed as (chi_max * ds) * fl32(1 / dtau_max).
template <>
struct Ar<float> {
    static constexpr double kArgScale = 1.2011224087864498;  // sqrt(log2(e))
    static __device__ __forceinline__ float rcp(float x) {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
    static __device__ __forceinline__ float gauss(float a) {
        float r;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(-(a * a)));
        return r;
    }
    static __device__ __forceinline__ float ninter(float cm, float hs, float, float inv_dtau_max) {
        return ceilf((cm * hs) * inv_dtau_max);
    }
};

template <typename R, int NL>
struct Sample {
    R delta, dv, chic, etac;
    R chi0[NL], eta0[NL];
};

template <typename R>
struct Data;

template <>
struct Data<double> {
    const double *vx, *vy, *vz, *chi0, *eta0, *dvw, *chic, *etac;
    __device__ Data(const DevMesh &m, const DevLines &Ln)
        : vx(m.vx), vy(m.vy), vz(m.vz), chi0(Ln.chi0), eta0(Ln.eta0), dvw(Ln.dvw), chic(Ln.chic),
          etac(Ln.etac) {}
};

template <>
struct Data<float> {
    const float *vx, *vy, *vz, *chi0, *eta0, *dvw, *chic, *etac;
    __device__ Data(const DevMesh &m, const DevLines &Ln)
        : vx(m.vxf), vy(m.vyf), vz(m.vzf), chi0(Ln.chi0f), eta0(Ln.eta0f), dvw(Ln.dvwf),
          chic(Ln.chicf), etac(Ln.etacf) {}
};

template <typename R, int NL>
__device__ __forceinline__ void load_sample(const Data<R> &D, int32_t L, int32_t id, R vox, R voy, R voz,
                                            R d0, R d1, R d2, Sample<R, NL> &s) {
    const R ux = __ldg(D.vx + id) - vox, uy = __ldg(D.vy + id) - voy, uz = __ldg(D.vz + id) - voz;
    s.delta = (ux * d0 + uy * d1) + uz * d2;
    s.dv = __ldg(D.dvw + id);
    s.chic = __ldg(D.chic + id);
    s.etac = __ldg(D.etac + id);
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        if (l < L) {
            s.chi0[l] = __ldg(D.chi0 + int64_t(id) * L + l);
            s.eta0[l] = __ldg(D.eta0 + int64_t(id) * L + l);
        } else {
            s.chi0[l] = R(0);
            s.eta0[l] = R(0);
        }
    }
}

// Total opacity and emissivity of a sample for this lane's bin.  Lines past
// the model's count have chi0 = eta0 = 0 and contribute nothing.
template <typename R, int NL>
__device__ __forceinline__ void optics(const Sample<R, NL> &s, const R (&A)[NL], const R (&B)[NL], R &chi,
                                       R &eta) {
    chi = s.chic;
    eta = s.etac;
    const R rdv = Ar<R>::rcp(s.dv);
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        const R g = Ar<R>::gauss((A[l] + B[l] * s.delta) * rdv);
        chi += s.chi0[l] * g;
        eta += s.eta0[l] * g;
    }
}

template <typename R, int NL>
__device__ __forceinline__ void shfl_sample(const Sample<R, NL> &s, int j, Sample<R, NL> &o) {
    o.delta = __shfl_sync(0xffffffffu, s.delta, j);
    o.dv = __shfl_sync(0xffffffffu, s.dv, j);
    o.chic = __shfl_sync(0xffffffffu, s.chic, j);
    o.etac = __shfl_sync(0xffffffffu, s.etac, j);
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        o.chi0[l] = __shfl_sync(0xffffffffu, s.chi0[l], j);
        o.eta0[l] = __shfl_sync(0xffffffffu, s.eta0[l], j);
    }
}

// State of the elimination along one half of a pair line.  Starting from
// (Fh, D, zh, dtp) = (1, 1, I, 0) the interior row below reproduces the
// second-order boundary row (Fh = 1 + dt/2, zh = D (S dt/2 + I)), and a half
// without points leaves exactly the empty-half coupling (D Fh, zh) = (1, I).
template <typename R>
struct Sweep {
    R Fh, Dm, zh, dtp;  // scaled 1+B quantities of the last eliminated row, its dtau
    R chi_c, eta_c;     // optics of the current (not yet eliminated) sub-point
    R chi_p, eta_p;     // optics of the current velocity sample
};

// Eliminate the row of the current sub-point once the increment dt beyond it
// is known.  One reciprocal R = 1 / (chi (1 + dt Fh)) gives D = chi R and
// D S = eta R.
template <typename R>
__device__ __forceinline__ void row(Sweep<R> &w, R dt) {
    const R dtb = (w.dtp + dt) * R(0.5);
    w.Fh = dtb + w.Dm * w.Fh;
    const R rr = Ar<R>::rcp(w.chi_c * (R(1) + dt * w.Fh));
    w.Dm = w.chi_c * rr;
    w.zh = w.Dm * w.zh + dtb * (w.eta_c * rr);
    w.dtp = dt;
}

// One velocity sample q at distance hs beyond the previous one: line optics,
// Eq. 2 sub-intervals with linear chi and eta, elimination rows.
template <typename R, int NL>
__device__ __forceinline__ void sample_step(const Sample<R, NL> &q, R hs, R dtau_max, R inv_dtau_max,
                                            const R (&A)[NL], const R (&B)[NL], Sweep<R> &w, int *status,
                                            unsigned &n_upd) {
    R chi_q, eta_q;
    optics<R, NL>(q, A, B, chi_q, eta_q);
    const R nr = Ar<R>::ninter(fmax(w.chi_p, chi_q), hs, dtau_max, inv_dtau_max);
    if (nr <= R(1)) {
        row(w, hs * (w.chi_p + chi_q) * R(0.5));
        w.chi_c = chi_q;
        w.eta_c = eta_q;
        ++n_upd;
    } else {
        int ni = int(fmin(nr, R(kMaxSubdiv)));
        if (nr > R(kMaxSubdiv)) dev_fail(status, kDevSubdivLimit);
        const R rni = R(1) / R(ni);
        const R hh = hs * rni * R(0.5);
        const R dchi = (chi_q - w.chi_p) * rni, deta = (eta_q - w.eta_p) * rni;
        R cprev = w.chi_p;
        for (int i = 1; i < ni; ++i) {
            const R ci = w.chi_p + dchi * R(i);
            row(w, hh * (cprev + ci));
            w.chi_c = ci;
            w.eta_c = w.eta_p + deta * R(i);
            cprev = ci;
        }
        row(w, hh * (cprev + chi_q));
        w.chi_c = chi_q;
        w.eta_c = eta_q;
        n_upd += unsigned(ni);
    }
    w.chi_p = chi_q;
    w.eta_p = eta_q;
}

// One interval between consecutive traced points (far -> near): adaptive
// velocity sampling (Section 2.1.1), then each sample's optics and rows.
template <typename R, int NL>
__device__ __forceinline__ void interval(const Sample<R, NL> &cur, const Sample<R, NL> &nxt, R ds,
                                         const SolveArgs &a, R dtau_max, R inv_dtau_max, R dv_max,
                                         const R (&A)[NL], const R (&B)[NL], Sweep<R> &w, unsigned &n_upd,
                                         unsigned &n_smp) {
    int nv = 1;
    if (dv_max > R(0)) {
        const R jump = fabs(nxt.delta - cur.delta);
        const R lim = dv_max * fmin(cur.dv, nxt.dv);
        if (jump > lim) {
            const R nvr = ceil(jump / lim);
            if (nvr > R(kMaxSubdiv)) {
                dev_fail(a.status, kDevSubdivLimit);
                nv = kMaxSubdiv;
            } else {
                nv = int(nvr);
            }
        }
    }
    n_smp += unsigned(nv);
    if (nv == 1) {
        sample_step<R, NL>(nxt, ds, dtau_max, inv_dtau_max, A, B, w, a.status, n_upd);
        return;
    }
    const R rnv = Ar<R>::rcp(R(nv));
    const R hs = ds * rnv;
    Sample<R, NL> q = cur, st;
    st.delta = (nxt.delta - cur.delta) * rnv;
    st.dv = (nxt.dv - cur.dv) * rnv;
    st.chic = (nxt.chic - cur.chic) * rnv;
    st.etac = (nxt.etac - cur.etac) * rnv;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        st.chi0[l] = (nxt.chi0[l] - cur.chi0[l]) * rnv;
        st.eta0[l] = (nxt.eta0[l] - cur.eta0[l]) * rnv;
    }
    for (int j = 1; j < nv; ++j) {
        const R t = R(j);
        q.delta = cur.delta + st.delta * t;
        q.dv = cur.dv + st.dv * t;
        q.chic = cur.chic + st.chic * t;
        q.etac = cur.etac + st.etac * t;
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            q.chi0[l] = cur.chi0[l] + st.chi0[l] * t;
            q.eta0[l] = cur.eta0[l] + st.eta0[l] * t;
        }
        sample_step<R, NL>(q, hs, dtau_max, inv_dtau_max, A, B, w, a.status, n_upd);
    }
    sample_step<R, NL>(nxt, hs, dtau_max, inv_dtau_max, A, B, w, a.status, n_upd);
}

// Eliminate one half of a pair line from its far end up to (excluding) the
// origin row.  The warp stages 32 traced points at a time: lane j loads entry
// kb - j (coalesced ids and distances, gathered point data, its projected
// velocity and its distance to the farther neighbour), then the warp walks the
// chunk, broadcasting each point with shuffles.  Returns the origin row's
// coupling (P = D Fh, Q = zh) and the last optical-depth increment.
// Projected distance Z = (x_n - x_o).d exactly as the tracer and its
// definition form it (explicitly rounded double operations in fixed order).
__device__ __forceinline__ double exact_Z(const DevMesh &m, int32_t id, double xo, double yo, double zo, double d0,
                                          double d1, double d2) {
    const double dx = __dsub_rn(__ldg(m.x + id), xo);
    const double dy = __dsub_rn(__ldg(m.y + id), yo);
    const double dz = __dsub_rn(__ldg(m.z + id), zo);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, d0), __dmul_rn(dy, d1)), __dmul_rn(dz, d2));
}

// Eliminate one half of a pair line from its far end up to (excluding) the
// origin row.  The warp stages 32 traced points at a time: lane j takes entry
// kb - j (coalesced ids, gathered point data), forms its exact Z and projected
// velocity, and gets the distance to the farther entry from its neighbour lane;
// then the warp walks the chunk, broadcasting each point with shuffles.
// Returns the origin row's coupling (P = D Fh, Q = zh) and the last
// optical-depth increment.
template <typename R, int NL>
__device__ void half_sweep(const DevMesh &m, const Data<R> &D, const SolveArgs &a, int32_t L, int lane,
                           int64_t beg, int32_t cnt, double xo, double yo, double zo, double e0, double e1,
                           double e2, R vox, R voy, R voz, const Sample<R, NL> &origin, const R (&A)[NL],
                           const R (&B)[NL], R &P, R &Q, R &dtl, unsigned &n_upd, unsigned &n_smp) {
    Sweep<R> w;
    w.Fh = R(1);
    w.Dm = R(1);
    w.zh = R(a.I_bdy);
    w.dtp = R(0);
    if (cnt > 0) {
        const R dtau_max = R(a.dtau_max), inv_dtau_max = R(1.0 / a.dtau_max), dv_max = R(a.dv_max);
        const R d0 = R(e0), d1 = R(e1), d2 = R(e2);
        Sample<R, NL> cur, nxt, st;
        double zcarry = 0.0;  // Z of the entry just beyond the current chunk (farther)
        for (int32_t kb = cnt - 1; kb >= 0; kb -= 32) {
            const int32_t nch = kb + 1 < 32 ? kb + 1 : 32;
            double zk = 0.0;
            if (lane < nch) {
                const int32_t id = __ldg(a.idx + beg + kb - lane);
                zk = exact_Z(m, id, xo, yo, zo, e0, e1, e2);
                load_sample<R, NL>(D, L, id, vox, voy, voz, d0, d1, d2, st);
            } else {
                st = origin;
            }
            double zf = __shfl_up_sync(0xffffffffu, zk, 1);
            if (lane == 0) zf = (kb == cnt - 1) ? zk : zcarry;
            const R sds = R(zf - zk);  // distance increment, differenced in double
            zcarry = __shfl_sync(0xffffffffu, zk, nch - 1);
            for (int j = 0; j < nch; ++j) {
                shfl_sample<R, NL>(st, j, nxt);
                const R ds = __shfl_sync(0xffffffffu, sds, j);
                if (kb == cnt - 1 && j == 0) {  // the far end: its row follows with the first increment
                    cur = nxt;
                    optics<R, NL>(cur, A, B, w.chi_p, w.eta_p);
                    w.chi_c = w.chi_p;
                    w.eta_c = w.eta_p;
                    continue;
                }
                interval<R, NL>(cur, nxt, ds, a, dtau_max, inv_dtau_max, dv_max, A, B, w, n_upd, n_smp);
                cur = nxt;
            }
        }
        interval<R, NL>(cur, origin, R(zcarry), a, dtau_max, inv_dtau_max, dv_max, A, B, w, n_upd, n_smp);
    }
    P = w.Dm * w.Fh;
    Q = w.zh;
    dtl = w.dtp;
}

template <typename R>
struct Occ {
    static constexpr int kMinBlocks = 1;
};
template <>
struct Occ<float> {
    static constexpr int kMinBlocks = 2;  // 16 warps per SM without spills
};

template <typename R, int NL>
__global__ void __launch_bounds__(256, Occ<R>::kMinBlocks)
k_solve(DevMesh m, DevLines Ln, DevRays Rs, SolveArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t item = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
    const int64_t n_items = int64_t(a.o_end - a.o_begin) * a.n_tiles;
    if (item >= n_items) return;
    const int32_t oc = int32_t(item / a.n_tiles);
    const int32_t o = a.o_begin + oc;
    const int32_t tile = int32_t(item % a.n_tiles);
    const int32_t L = Ln.L, F = Ln.F, NB = L * F;
    const int32_t b = tile * 32 + lane;
    const bool active = b < NB;
    const int32_t bb = active ? b : NB - 1;
    const int32_t l = bb / F, k = bb % F;

    const Data<R> D(m, Ln);
    // frequency of this lane and the profile constants of every line
    const double x = (F == 1) ? 0.0 : -Ln.x_span + 2.0 * Ln.x_span * double(k) / double(F - 1);
    const double dvo = Ln.dvw[o];
    const double ub = x * dvo;
    R A[NL], B[NL];
#pragma unroll
    for (int lp = 0; lp < NL; ++lp) {
        const double r = (lp < L) ? Ln.ratio[l * MGX_MAX_LINES + lp] : 1.0;
        A[lp] = R((kC * (r - 1.0) + r * ub) * Ar<R>::kArgScale);
        B[lp] = R(r * (1.0 + ub / kC) * Ar<R>::kArgScale);
    }
    const R vox = __ldg(D.vx + o), voy = __ldg(D.vy + o), voz = __ldg(D.vz + o);
    const double xo = m.x[o], yo = m.y[o], zo = m.z[o];
    Sample<R, NL> org;
    load_sample<R, NL>(D, L, o, vox, voy, voz, R(0), R(0), R(0), org);
    org.delta = R(0);
    R chi_o, eta_o;
    optics<R, NL>(org, A, B, chi_o, eta_o);
    const R S_o = eta_o / chi_o;

    double sum = 0.0, comp = 0.0;
    unsigned n_upd = 0, n_smp = 0;
    const int64_t h0 = int64_t(oc) * Rs.npairs * 2;
    for (int32_t p = 0; p < Rs.npairs; ++p) {
        const uint32_t ray = __ldg(Rs.rays + int64_t(o) * Rs.npairs + p);
        const int lev = int(ray >> 28);
        const double *rv = Rs.dir + 3 * (level_offset(lev) + (ray & 0x0FFFFFFFu));
        const double r0 = rv[0], r1 = rv[1], r2 = rv[2];
        R P0, Q0, t0, P1, Q1, t1;
        const int64_t hb = h0 + 2 * int64_t(p);
        {
            const int64_t beg = a.offs[hb] - a.base;
            const int32_t cnt = int32_t(a.offs[hb + 1] - a.offs[hb]);
            half_sweep<R, NL>(m, D, a, L, lane, beg, cnt, xo, yo, zo, -r0, -r1, -r2, vox, voy, voz, org, A, B,
                              P0, Q0, t0, n_upd, n_smp);
        }
        {
            const int64_t beg = a.offs[hb + 1] - a.base;
            const int32_t cnt = int32_t(a.offs[hb + 2] - a.offs[hb + 1]);
            half_sweep<R, NL>(m, D, a, L, lane, beg, cnt, xo, yo, zo, r0, r1, r2, vox, voy, voz, org, A, B,
                              P1, Q1, t1, n_upd, n_smp);
        }
        const R dtb = (t0 + t1) * R(0.5);
        const R u = (dtb * S_o + Q0 + Q1) / (dtb + P0 + P1);
        const double xv = a.w2[lev] * double(u);
        const double t = sum + xv;  // Neumaier compensated sum
        if (fabs(sum) >= fabs(xv)) comp += (sum - t) + xv;
        else comp += (xv - t) + sum;
        sum = t;
    }
    if (active) a.J[int64_t(o) * NB + b] = sum + comp;
    if (a.counters) {
        unsigned long long u = active ? n_upd : 0, s = active ? n_smp : 0;
#pragma unroll
        for (int sh = 16; sh > 0; sh >>= 1) {
            u += __shfl_down_sync(0xffffffffu, u, sh);
            s += __shfl_down_sync(0xffffffffu, s, sh);
        }
        if (lane == 0) {
            atomicAdd(a.counters, u);
            atomicAdd(a.counters + 1, s);
        }
    }
}

template <typename R>
void launch_R(const DevMesh &m, const DevLines &Ln, const DevRays &R_, const SolveArgs &a, cudaStream_t st) {
    const int64_t n_items = int64_t(a.o_end - a.o_begin) * a.n_tiles;
    if (n_items == 0) return;
    const int tb = 256;
    const unsigned grid = unsigned((n_items * 32 + tb - 1) / tb);
    if (Ln.L <= 1) k_solve<R, 1><<<grid, tb, 0, st>>>(m, Ln, R_, a);
    else if (Ln.L <= 2) k_solve<R, 2><<<grid, tb, 0, st>>>(m, Ln, R_, a);
    else if (Ln.L <= 4) k_solve<R, 4><<<grid, tb, 0, st>>>(m, Ln, R_, a);
    else k_solve<R, 8><<<grid, tb, 0, st>>>(m, Ln, R_, a);
}

}  // namespace

void launch_solve(const DevMesh &m, const DevLines &Ln, const DevRays &R, const SolveArgs &a,
                  int precision, cudaStream_t st) {
    if (precision == MGX_FP64) launch_R<double>(m, Ln, R, a, st);
    else launch_R<float>(m, Ln, R, a, st);
}

}  // namespace mgx
