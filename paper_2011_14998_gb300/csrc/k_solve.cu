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
//     numbers is formed.
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

template <>
struct Ar<double> {
    static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
    static __device__ __forceinline__ double div(double a, double b) { return a / b; }
    static __device__ __forceinline__ double gauss(double a) { return exp(-(a * a)); }
    static __device__ __forceinline__ double arg(double A, double B, double de, double dv) {
        return (A + B * de) / dv;
    }
};

template <>
struct Ar<float> {
    static __device__ __forceinline__ float rcp(float x) {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
    static __device__ __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
    static __device__ __forceinline__ float gauss(float a) { return __expf(-(a * a)); }
    static __device__ __forceinline__ float arg(float A, float B, float de, float dv) {
        return (A + B * de) * rcp(dv);
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

template <typename R, int NL>
__device__ __forceinline__ void lerp_sample(const Sample<R, NL> &a, const Sample<R, NL> &b, R t,
                                            Sample<R, NL> &s) {
    s.delta = a.delta + (b.delta - a.delta) * t;
    s.dv = a.dv + (b.dv - a.dv) * t;
    s.chic = a.chic + (b.chic - a.chic) * t;
    s.etac = a.etac + (b.etac - a.etac) * t;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        s.chi0[l] = a.chi0[l] + (b.chi0[l] - a.chi0[l]) * t;
        s.eta0[l] = a.eta0[l] + (b.eta0[l] - a.eta0[l]) * t;
    }
}

template <typename R, int NL>
__device__ __forceinline__ void optics(const Sample<R, NL> &s, const R (&A)[NL], const R (&B)[NL],
                                       int32_t L, R &chi, R &eta) {
    chi = s.chic;
    eta = s.etac;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        if (l < L) {
            const R g = Ar<R>::gauss(Ar<R>::arg(A[l], B[l], s.delta, s.dv));
            chi += s.chi0[l] * g;
            eta += s.eta0[l] * g;
        }
    }
}

// Eliminate one half of a pair line from its far end up to (excluding) the
// origin row.  Returns the origin row's coupling (P = D Fh, Q = zh) and the
// last optical-depth increment.
template <typename R, int NL>
__device__ void half_sweep(const Data<R> &D, const SolveArgs &a, int32_t L, int64_t beg, int32_t cnt,
                           R vox, R voy, R voz, R d0, R d1, R d2, const Sample<R, NL> &origin,
                           const R (&A)[NL], const R (&B)[NL], R &P, R &Q, R &dtl,
                           unsigned &n_upd, unsigned &n_smp) {
    const R I = R(a.I_bdy);
    if (cnt == 0) {
        P = R(1);
        Q = I;
        dtl = R(0);
        return;
    }
    const R dtau_max = R(a.dtau_max), dv_max = R(a.dv_max);
    Sample<R, NL> cur, nxt, q;
    int64_t e = beg + cnt - 1;
    load_sample<R, NL>(D, L, __ldg(a.idx + e), vox, voy, voz, d0, d1, d2, cur);
    double zcur = __ldg(a.Z + e);
    R chi_p, eta_p;
    optics<R, NL>(cur, A, B, L, chi_p, eta_p);
    R S_c = Ar<R>::div(eta_p, chi_p);
    bool first = true;
    R Fh = R(0), Dm = R(1), zh = R(0), dtp = R(0);
    for (int32_t k = cnt - 1; k >= 0; --k) {
        double znext;
        if (k > 0) {
            load_sample<R, NL>(D, L, __ldg(a.idx + beg + k - 1), vox, voy, voz, d0, d1, d2, nxt);
            znext = __ldg(a.Z + beg + k - 1);
        } else {
            nxt = origin;
            znext = 0.0;
        }
        const R ds = R(zcur - znext);  // distance increment, differenced in double
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
        const R hs = ds / R(nv);
        for (int j = 1; j <= nv; ++j) {
            if (j == nv) {
                q = nxt;
            } else {
                lerp_sample<R, NL>(cur, nxt, R(j) / R(nv), q);
            }
            R chi_q, eta_q;
            optics<R, NL>(q, A, B, L, chi_q, eta_q);
            ++n_smp;
            const R cm = fmax(chi_p, chi_q);
            R nr = ceil(cm * hs / dtau_max);
            int ni = nr < R(1) ? 1 : (nr > R(kMaxSubdiv) ? kMaxSubdiv + 1 : int(nr));
            if (ni > kMaxSubdiv) {
                dev_fail(a.status, kDevSubdivLimit);
                ni = kMaxSubdiv;
            }
            const R hh = hs / R(ni);
            n_upd += unsigned(ni);
            R cprev = chi_p;
            for (int i = 1; i <= ni; ++i) {
                R ci, ei;
                if (i == ni) {
                    ci = chi_q;
                    ei = eta_q;
                } else {
                    const R t = R(i) / R(ni);
                    ci = chi_p + (chi_q - chi_p) * t;
                    ei = eta_p + (eta_q - eta_p) * t;
                }
                const R dt = hh * (cprev + ci) * R(0.5);
                if (first) {
                    Fh = R(1) + dt * R(0.5);
                    Dm = Ar<R>::rcp(R(1) + dt * Fh);
                    zh = Dm * (S_c * dt * R(0.5) + I);
                    first = false;
                } else {
                    const R dtb = (dtp + dt) * R(0.5);
                    Fh = dtb + Dm * Fh;
                    Dm = Ar<R>::rcp(R(1) + dt * Fh);
                    zh = Dm * (dtb * S_c + zh);
                }
                dtp = dt;
                S_c = Ar<R>::div(ei, ci);
                cprev = ci;
            }
            chi_p = chi_q;
            eta_p = eta_q;
        }
        cur = nxt;
        zcur = znext;
    }
    P = Dm * Fh;
    Q = zh;
    dtl = dtp;
}

template <typename R, int NL>
__global__ void __launch_bounds__(256)
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
        A[lp] = R(kC * (r - 1.0) + r * ub);
        B[lp] = R(r * (1.0 + ub / kC));
    }
    const R vox = __ldg(D.vx + o), voy = __ldg(D.vy + o), voz = __ldg(D.vz + o);
    Sample<R, NL> org;
    load_sample<R, NL>(D, L, o, vox, voy, voz, R(0), R(0), R(0), org);
    org.delta = R(0);
    R chi_o, eta_o;
    optics<R, NL>(org, A, B, L, chi_o, eta_o);
    const R S_o = Ar<R>::div(eta_o, chi_o);

    double sum = 0.0, comp = 0.0;
    unsigned n_upd = 0, n_smp = 0;
    const int64_t h0 = int64_t(oc) * Rs.npairs * 2;
    for (int32_t p = 0; p < Rs.npairs; ++p) {
        const uint32_t ray = __ldg(Rs.rays + int64_t(o) * Rs.npairs + p);
        const int lev = int(ray >> 28);
        const double *rv = Rs.dir + 3 * (level_offset(lev) + (ray & 0x0FFFFFFFu));
        const R r0 = R(rv[0]), r1 = R(rv[1]), r2 = R(rv[2]);
        R P0, Q0, t0, P1, Q1, t1;
        const int64_t hb = h0 + 2 * int64_t(p);
        {
            const int64_t beg = a.offs[hb] - a.base;
            const int32_t cnt = int32_t(a.offs[hb + 1] - a.offs[hb]);
            half_sweep<R, NL>(D, a, L, beg, cnt, vox, voy, voz, -r0, -r1, -r2, org, A, B, P0, Q0, t0, n_upd,
                              n_smp);
        }
        {
            const int64_t beg = a.offs[hb + 1] - a.base;
            const int32_t cnt = int32_t(a.offs[hb + 2] - a.offs[hb + 1]);
            half_sweep<R, NL>(D, a, L, beg, cnt, vox, voy, voz, r0, r1, r2, org, A, B, P1, Q1, t1, n_upd,
                              n_smp);
        }
        const R dtb = (t0 + t1) * R(0.5);
        const R u = Ar<R>::div(dtb * S_o + Q0 + Q1, dtb + P0 + P1);
        const double w2 = 2.0 / double(int64_t(12) << (2 * lev));
        const double xv = w2 * double(u);
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
