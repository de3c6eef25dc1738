// k_solve_impl.cuh -- formal solution along ray pairs and the mean intensity J
// (Eqs. 1-3, Sections 2.1.1-2.1.2).
//
// One warp per (origin, frequency tile); each lane carries BPL frequency bins
// (bin tile*32*BPL + lane + 32 i, i < BPL).  The warp walks every ray pair of
// its origin in ascending pair order.  For each half of the pair it starts at
// the far end of the traced point list and eliminates towards the origin:
//   * adaptive velocity sampling (Section 2.1.1): between consecutive points
//     whose projected velocities differ by more than dv_max times the smaller
//     Doppler width, equally spaced samples with linearly interpolated data;
//   * line optics: chi = chi_c + sum_l chi0_l exp(-a_l^2), eta likewise, a_l the
//     Doppler-shifted profile argument of line l at the bin's frequency;
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
// The frequency-independent work of a line point (staging, exact Z, projected
// velocity, velocity sampling, interpolation, the width's reciprocal) is done
// once per warp and shared by the lane's BPL bins.
//
// Template R selects the arithmetic: double (plain form) or float (the distance
// increments come from double Z differences; J is summed in double).
#pragma once

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
    static __device__ __forceinline__ double ratio(double cm, double hs, double dtau_max, double) {
        return cm * hs / dtau_max;
    }
    static __device__ __forceinline__ double src(double eta, double chi) { return eta / chi; }
    // projected velocity (x + y) + z, every product and sum rounded (no contraction)
    static __device__ __forceinline__ double proj(double ux, double uy, double uz, double d0, double d1, double d2) {
        return __dadd_rn(__dadd_rn(__dmul_rn(ux, d0), __dmul_rn(uy, d1)), __dmul_rn(uz, d2));
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
    static __device__ __forceinline__ float ratio(float cm, float hs, float, float inv_dtau_max) {
        return (cm * hs) * inv_dtau_max;
    }
    static __device__ __forceinline__ float src(float eta, float chi) { return eta * rcp(chi); }
    // projected velocity (x + y) + z, every product and sum rounded (no
    // contraction): the velocity-sample count of an interval is decided on it
    static __device__ __forceinline__ float proj(float ux, float uy, float uz, float d0, float d1, float d2) {
        return __fadd_rn(__fadd_rn(__fmul_rn(ux, d0), __fmul_rn(uy, d1)), __fmul_rn(uz, d2));
    }
};

// Frequency-independent data of one line sample.
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
    s.delta = Ar<R>::proj(ux, uy, uz, d0, d1, d2);
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

// Per-bin constants: the Doppler-shifted profile argument of line l at this
// bin is (A[l] + B[l] delta) / dv (prescaled for the single-precision ex2).
template <typename R, int NL>
struct Bin {
    R A[NL], B[NL];
};

// Total opacity and emissivity of a sample for one bin (rdv = 1 / dv).  Lines
// past the model's count have chi0 = eta0 = 0 and contribute nothing.
template <typename R, int NL>
__device__ __forceinline__ void optics(const Sample<R, NL> &s, R rdv, const Bin<R, NL> &f, R &chi, R &eta) {
    chi = s.chic;
    eta = s.etac;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        const R g = Ar<R>::gauss((f.A[l] + f.B[l] * s.delta) * rdv);
        chi += s.chi0[l] * g;
        eta += s.eta0[l] * g;
    }
}

// State of the elimination of one bin along one half of a pair line.
// Starting from (Fh, D, zh, dtp) = (1, 1, I, 0) the interior row reproduces
// the second-order boundary row, and a half without points leaves exactly the
// empty-half coupling (D Fh, zh) = (1, I).
//
// The Hermitian scheme (ORD 4) also carries the source function of the last
// eliminated row (Sp) and of the current sample (Sc), the last increment (hp,
// negative before the first row) and its reciprocal (rh).
template <typename R>
struct Sweep {
    R Fh, Dm, zh, dtp;  // scaled 1+B quantities of the last eliminated row, half its dtau
    R chi, eta;         // optics of the current (not yet eliminated) sample
    R Sp, Sc, hp, rh;   // Hermitian scheme only
};

// Eliminate the row of the current sub-point (optics chi, eta) once the
// increment dt beyond it is known.  One reciprocal R = 1 / (chi (1 + dt Fh))
// gives D = chi R and D S = eta R.  The state carries half the previous
// increment, so dtbar = (dt_prev + dt) / 2 is one fused operation (the
// halvings are exact, so the rounding is that of the plain expression).
//
// ORD 4: the Hermitian row of Auer (1976) (Section 2.1) in the same scaled
// form.  With h- the previous and h+ the current increment, hbar their mean,
//   1 - lambda = (h-^2 + h- h+ - h+^2) / 12,  mu = (h+^2 + h- h+ - h-^2) / 12,
//   Fh = (hbar + lambda D Fh_prev) / (1 - mu),   D = 1 / (1 + h+ Fh),
//   zh = D (hbar r + lambda zh_prev) / (1 - mu),
//   hbar r = hbar S_i + ((1 - lambda) / h-) (S_{i-1} - S_i) + (mu / h+) (S_{i+1} - S_i),
// which is the textbook elimination with the compact weights
// a = (1 - lambda) / (h- hbar), g = mu / (h+ hbar), b = 1 - a - g, scaled by
// the increment beyond each row (F = h+ Fh, z = h+ zh).  A row whose two
// increments differ by more than a factor kHermRatio takes the second-order
// weights (lambda = 1, mu = 0): the compact weights grow like the ratio and
// would amplify the rounding of S next to a vanishing increment.  The first
// row of a half is the third-order boundary row (Auer 1967):
//   Fh = (1 + h/2) / (1 - h^2/6),  zh = D (h S_i / 3 + h S_{i+1} / 6 + I) / (1 - h^2/6).
constexpr double kHermRatio = 64.0;

template <int ORD, typename R>
__device__ __forceinline__ void row(Sweep<R> &w, R chi, R eta, R dt, R Si, R Sn) {
    if constexpr (ORD == 2) {
        const R dtb = fma(dt, R(0.5), w.dtp);
        w.Fh = dtb + w.Dm * w.Fh;
        const R rr = Ar<R>::rcp(chi * (R(1) + dt * w.Fh));
        w.Dm = chi * rr;
        w.zh = w.Dm * w.zh + dtb * (eta * rr);
        w.dtp = dt * R(0.5);
    } else {
        const R rh = Ar<R>::rcp(dt);
        if (w.hp < R(0)) {  // boundary row
            const R k = Ar<R>::rcp(R(1) - dt * dt * R(1.0 / 6.0));
            w.Fh = fma(dt, R(0.5), R(1)) * k;
            const R D = Ar<R>::rcp(fma(dt, w.Fh, R(1)));
            w.zh = D * k * (dt * (Si * R(1.0 / 3.0) + Sn * R(1.0 / 6.0)) + w.zh);
            w.Dm = D;
        } else {
            const R hm = w.hp, p = hm * dt;
            const bool compact = !(dt > R(kHermRatio) * hm || hm > R(kHermRatio) * dt);
            const R oml = compact ? (hm * hm + p - dt * dt) * R(1.0 / 12.0) : R(0);  // 1 - lambda
            const R mu = compact ? (dt * dt + p - hm * hm) * R(1.0 / 12.0) : R(0);
            const R k = Ar<R>::rcp(R(1) - mu);
            const R hb = (hm + dt) * R(0.5);
            const R hr = hb * Si + oml * w.rh * (w.Sp - Si) + mu * rh * (Sn - Si);
            const R lam = R(1) - oml;
            w.Fh = k * (hb + lam * w.Dm * w.Fh);
            const R D = Ar<R>::rcp(fma(dt, w.Fh, R(1)));
            w.zh = D * k * (hr + lam * w.zh);
            w.Dm = D;
        }
        w.rh = rh;
        w.hp = dt;
        w.Sp = Si;
    }
}

// One velocity sample q at distance hs beyond the previous one, for every bin
// of the lane: line optics, Eq. 2 sub-intervals with linear chi and eta,
// elimination rows.  When no bin of the warp needs sub-intervals (the common
// case) the rows run as straight-line code, so the bins' chains interleave.
//
// Single precision decides "more than one sub-interval" as chi_max > thr with
// thr = fl32(dtau_max / hs) (the same inequality as Eq. 2's ceiling exceeding
// one), on the lane's running maximum of chi over its bins (cmax: the previous
// sample's, updated here), and only then forms the ceiling; double precision
// evaluates Eq. 2 as written.
template <typename R, int NL, int BPL, int ORD>
__device__ __forceinline__ void sample_step(const Sample<R, NL> &q, R hs, R thr, R &cmax, R dtau_max,
                                            R inv_dtau_max, const Bin<R, NL> (&f)[BPL], const bool (&act)[BPL],
                                            Sweep<R> (&w)[BPL], int *status, unsigned &n_extra) {
    const R rdv = Ar<R>::rcp(q.dv);
    R chi_q[BPL], eta_q[BPL];
#pragma unroll
    for (int i = 0; i < BPL; ++i) optics<R, NL>(q, rdv, f[i], chi_q[i], eta_q[i]);
    bool split = false;
    if constexpr (sizeof(R) == 4) {
        R cq = chi_q[0];
#pragma unroll
        for (int i = 1; i < BPL; ++i) cq = fmax(cq, chi_q[i]);
        split = fmax(cmax, cq) > thr;
        cmax = cq;
    } else {
#pragma unroll
        for (int i = 0; i < BPL; ++i)
            split |= Ar<R>::ratio(fmax(w[i].chi, chi_q[i]), hs, dtau_max, inv_dtau_max) > R(1);
    }
    if (!__any_sync(0xffffffffu, split)) {
        const R hh = hs * R(0.5);
#pragma unroll
        for (int i = 0; i < BPL; ++i) {
            R Sq = R(0);
            if constexpr (ORD == 4) Sq = Ar<R>::src(eta_q[i], chi_q[i]);
            row<ORD>(w[i], w[i].chi, w[i].eta, hh * (w[i].chi + chi_q[i]), w[i].Sc, Sq);
            w[i].chi = chi_q[i];
            w[i].eta = eta_q[i];
            w[i].Sc = Sq;
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < BPL; ++i) {
        const R cm = fmax(w[i].chi, chi_q[i]);
        int ni = 1;
        if (sizeof(R) == 8 || cm > thr) {
            const R nr = ceil(Ar<R>::ratio(cm, hs, dtau_max, inv_dtau_max));  // Eq. 2
            ni = nr <= R(1) ? 1 : int(fmin(nr, R(kMaxSubdiv)));
            if (nr > R(kMaxSubdiv)) dev_fail(status, kDevSubdivLimit);
        }
        const R rni = R(1) / R(ni);
        const R hh = hs * rni * R(0.5);
        const R c0 = w[i].chi, e0 = w[i].eta;
        const R dchi = (chi_q[i] - c0) * rni, deta = (eta_q[i] - e0) * rni;
        R cprev = c0, eprev = e0, Sprev = w[i].Sc;
        for (int k = 1; k < ni; ++k) {
            const R ck = c0 + dchi * R(k), ek = e0 + deta * R(k);
            R Sk = R(0);
            if constexpr (ORD == 4) Sk = Ar<R>::src(ek, ck);
            row<ORD>(w[i], cprev, eprev, hh * (cprev + ck), Sprev, Sk);
            cprev = ck;
            eprev = ek;
            Sprev = Sk;
        }
        R Sq = R(0);
        if constexpr (ORD == 4) Sq = Ar<R>::src(eta_q[i], chi_q[i]);
        row<ORD>(w[i], cprev, eprev, hh * (cprev + chi_q[i]), Sprev, Sq);
        w[i].chi = chi_q[i];
        w[i].eta = eta_q[i];
        w[i].Sc = Sq;
        n_extra += act[i] ? unsigned(ni - 1) : 0u;
    }
}

// Velocity samples of the interval between consecutive points a (farther)
// and b (Section 2.1.1): ceil(|delta_b - delta_a| / (dv_max min(dv_a, dv_b)))
// when that exceeds one, else 1.
template <typename R>
__device__ __forceinline__ int velocity_samples(R da, R wa, R db, R wb, R dv_max, int *status) {
    if (!(dv_max > R(0))) return 1;
    const R jump = fabs(db - da);
    const R lim = dv_max * fmin(wa, wb);
    if (!(jump > lim)) return 1;
    const R nvr = ceil(jump / lim);
    if (nvr > R(kMaxSubdiv)) {
        dev_fail(status, kDevSubdivLimit);
        return kMaxSubdiv;
    }
    return int(nvr);
}

// One interval from the current point (cur, modified in place) to nxt with nv
// velocity samples: interpolated samples, then nxt itself.  The code layout was
// chosen by measurement on GB300: one line inlines the sample step at three
// sites (the common one-sample path stays separate); several lines share the
// final sample's site with the one-sample case, whose smaller code was 16 %
// (two lines) to 33 % (four lines) faster.
template <typename R, int NL, int BPL, int ORD>
__device__ __forceinline__ void interval(Sample<R, NL> &cur, const Sample<R, NL> &nxt, R ds, R thr, int nv,
                                         R &cmax, const SolveArgs &a, R dtau_max, R inv_dtau_max,
                                         const Bin<R, NL> (&f)[BPL], const bool (&act)[BPL], Sweep<R> (&w)[BPL],
                                         unsigned &n_extra) {
    if constexpr (NL == 1) {
        if (nv > 1) {
            const R rnv = Ar<R>::rcp(R(nv));
            const R hs = ds * rnv;
            const R ths = thr * R(nv);  // dtau_max / hs
            Sample<R, NL> st;
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
                cur.delta += st.delta;
                cur.dv += st.dv;
                cur.chic += st.chic;
                cur.etac += st.etac;
#pragma unroll
                for (int l = 0; l < NL; ++l) {
                    cur.chi0[l] += st.chi0[l];
                    cur.eta0[l] += st.eta0[l];
                }
                sample_step<R, NL, BPL, ORD>(cur, hs, ths, cmax, dtau_max, inv_dtau_max, f, act, w, a.status, n_extra);
            }
            sample_step<R, NL, BPL, ORD>(nxt, hs, ths, cmax, dtau_max, inv_dtau_max, f, act, w, a.status, n_extra);
        } else {
            sample_step<R, NL, BPL, ORD>(nxt, ds, thr, cmax, dtau_max, inv_dtau_max, f, act, w, a.status, n_extra);
        }
    } else {
        // several lines: two call sites (the nv = 1 case shares the final sample's);
        // measured faster when the per-sample optics are longer
        R hs = ds, ths = thr;
        if (nv > 1) {
            const R rnv = Ar<R>::rcp(R(nv));
            hs = ds * rnv;
            ths = thr * R(nv);  // dtau_max / hs
            Sample<R, NL> st;
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
                cur.delta += st.delta;
                cur.dv += st.dv;
                cur.chic += st.chic;
                cur.etac += st.etac;
#pragma unroll
                for (int l = 0; l < NL; ++l) {
                    cur.chi0[l] += st.chi0[l];
                    cur.eta0[l] += st.eta0[l];
                }
                sample_step<R, NL, BPL, ORD>(cur, hs, ths, cmax, dtau_max, inv_dtau_max, f, act, w, a.status, n_extra);
            }
        }
        sample_step<R, NL, BPL, ORD>(nxt, hs, ths, cmax, dtau_max, inv_dtau_max, f, act, w, a.status, n_extra);
    }
    cur = nxt;
}

// Projected distance Z = (x_n - x_o).d exactly as the tracer and its
// definition form it (explicitly rounded double operations in fixed order).
__device__ __forceinline__ double exact_Z(const DevMesh &m, int32_t id, double xo, double yo, double zo, double d0,
                                          double d1, double d2) {
    const double dx = __dsub_rn(__ldg(m.x + id), xo);
    const double dy = __dsub_rn(__ldg(m.y + id), yo);
    const double dz = __dsub_rn(__ldg(m.z + id), zo);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, d0), __dmul_rn(dy, d1)), __dmul_rn(dz, d2));
}

// u at the origin row from the two half-sweeps (the origin row couples the
// last eliminated rows of both halves; no back substitution is needed).
// Second order: u_o = (dtbar S_o + zh- + zh+) / (dtbar + D- Fh- + D+ Fh+), an
// empty half contributing (D Fh, zh) = (1, I) through its initial state.
template <typename R>
__device__ __forceinline__ R origin_u2(const Sweep<R> &b, const Sweep<R> &f, R So) {
    const R dtb = b.dtp + f.dtp;  // the halves of the two last increments
    return (dtb * So + b.zh + f.zh) / (dtb + b.Dm * b.Fh + f.Dm * f.Fh);
}

// Hermitian scheme: with h- (h+) the last increment of the backward (forward)
// half and lambda- = 1 - (h-^2 + h- h+ - h+^2)/12, lambda+ = 1 - (h+^2 + h- h+ - h-^2)/12,
//   u_o = (hbar r_o + lambda- zh- + lambda+ zh+) / (hbar + lambda- D- Fh- + lambda+ D+ Fh+);
// with one half empty the origin row is the third-order boundary row,
//   u_o = (h S_o/3 + h S_1/6 + I + (1 - h^2/6) zh) / (1 + h/2 + (1 - h^2/6) D Fh);
// with both empty u_o = I.
template <typename R>
__device__ __forceinline__ R origin_u4(const Sweep<R> &b, const Sweep<R> &f, R So, R I) {
    if (b.hp < R(0) && f.hp < R(0)) return I;
    if (b.hp < R(0) || f.hp < R(0)) {
        const Sweep<R> &w = b.hp < R(0) ? f : b;
        const R h = w.hp, k1 = R(1) - h * h * R(1.0 / 6.0);
        return (h * (So * R(1.0 / 3.0) + w.Sp * R(1.0 / 6.0)) + I + k1 * w.zh) / (fma(h, R(0.5), R(1)) + k1 * w.Dm * w.Fh);
    }
    const R hm = b.hp, hp = f.hp, p = hm * hp;
    const bool compact = !(hp > R(kHermRatio) * hm || hm > R(kHermRatio) * hp);
    const R oml = compact ? (hm * hm + p - hp * hp) * R(1.0 / 12.0) : R(0);  // 1 - lambda-
    const R mu = compact ? (hp * hp + p - hm * hm) * R(1.0 / 12.0) : R(0);   // 1 - lambda+
    const R hb = (hm + hp) * R(0.5);
    const R hr = hb * So + oml * b.rh * (b.Sp - So) + mu * f.rh * (f.Sp - So);
    return (hr + (R(1) - oml) * b.zh + (R(1) - mu) * f.zh) /
           (hb + (R(1) - oml) * b.Dm * b.Fh + (R(1) - mu) * f.Dm * f.Fh);
}

// Where the ids of one half-ray are: entries k < n_main at main[k], the rest
// at tail[tail_off + k] (padded layout); cnt entries in all.
struct HalfList {
    const int32_t *main;
    const int32_t *tail;
    int64_t tail_off;
    int32_t n_main, cnt;
};

__device__ __forceinline__ HalfList half_list(const SolveArgs &a, int64_t h) {
    HalfList l;
    if (a.pad == 0) {
        l.main = a.idx + (a.offs[h] - a.base);
        l.cnt = l.n_main = int32_t(a.offs[h + 1] - a.offs[h]);
        l.tail = a.idx;
        l.tail_off = 0;
    } else {
        l.cnt = int32_t(a.lens[h]);
        l.main = a.idx + h * a.pad;
        l.n_main = l.cnt < a.pad ? l.cnt : a.pad;
        l.tail = a.tail;
        l.tail_off = a.offs[h] - a.base - a.pad;
    }
    return l;
}

// Per-warp staging area of 32 line points in shared memory.
template <typename R, int NL>
struct Stage {
    R delta[32], dv[32], chic[32], etac[32], ds[32], thr[32];
    R chi0[NL][32], eta0[NL][32];
    int nv[32];
};

// Eliminate one half of a pair line from its far end up to (excluding) the
// origin row.  The warp stages 32 traced points at a time: lane j takes entry
// kb - j (coalesced ids, gathered point data), forms its exact Z, projected
// velocity, the distance to the farther entry and that interval's number of
// velocity samples (its neighbour lane holds the farther entry), and writes
// them to the warp's shared staging area; then the warp walks the chunk.
// Leaves the origin row's coupling (P = D Fh, Q = zh) and the last
// optical-depth increment in w.
template <typename R, int NL, int BPL, int ORD>
__device__ void half_sweep(const DevMesh &m, const Data<R> &D, const SolveArgs &a, int32_t L, int lane,
                           Stage<R, NL> &sg, const HalfList &hl, double xo, double yo, double zo,
                           double e0, double e1, double e2, R vox, R voy, R voz, int32_t o,
                           const Bin<R, NL> (&f)[BPL], const bool (&act)[BPL], Sweep<R> (&w)[BPL],
                           unsigned &n_extra, unsigned &n_smp) {
#pragma unroll
    for (int i = 0; i < BPL; ++i) {
        w[i].Fh = R(1);
        w[i].Dm = R(1);
        w[i].zh = R(a.I_bdy);
        w[i].dtp = R(0);
        w[i].hp = R(-1);  // no row yet (Hermitian scheme)
        w[i].Sp = w[i].Sc = w[i].rh = R(0);
    }
    const int32_t cnt = hl.cnt;
    if (cnt == 0) return;
    const R dtau_max = R(a.dtau_max), inv_dtau_max = R(1.0 / a.dtau_max), dv_max = R(a.dv_max);
    const R d0 = R(e0), d1 = R(e1), d2 = R(e2);
    Sample<R, NL> cur, nxt;
    R cmax = R(0);  // running maximum of chi over the lane's bins at the current sample
    double zcarry = 0.0;          // Z of the entry just beyond the current chunk (farther)
    R dcarry = R(0), wcarry = R(1);  // its projected velocity and width
    for (int32_t kb = cnt - 1; kb >= 0; kb -= 32) {
        const int32_t nch = kb + 1 < 32 ? kb + 1 : 32;
        double zk = 0.0;
        Sample<R, NL> st;
        st.delta = st.dv = R(1);
        if (lane < nch) {
            const int32_t k = kb - lane;
            const int32_t id = k < hl.n_main ? __ldg(hl.main + k) : __ldg(hl.tail + (hl.tail_off + k));
            zk = exact_Z(m, id, xo, yo, zo, e0, e1, e2);
            load_sample<R, NL>(D, L, id, vox, voy, voz, d0, d1, d2, st);
        }
        double zf = __shfl_up_sync(0xffffffffu, zk, 1);
        R df = __shfl_up_sync(0xffffffffu, st.delta, 1), wf = __shfl_up_sync(0xffffffffu, st.dv, 1);
        const bool far_end = kb == cnt - 1 && lane == 0;
        if (lane == 0) {
            zf = far_end ? zk : zcarry;
            df = far_end ? st.delta : dcarry;
            wf = far_end ? st.dv : wcarry;
        }
        zcarry = __shfl_sync(0xffffffffu, zk, nch - 1);
        dcarry = __shfl_sync(0xffffffffu, st.delta, nch - 1);
        wcarry = __shfl_sync(0xffffffffu, st.dv, nch - 1);
        __syncwarp();
        if (lane < nch) {
            sg.delta[lane] = st.delta;
            sg.dv[lane] = st.dv;
            sg.chic[lane] = st.chic;
            sg.etac[lane] = st.etac;
#pragma unroll
            for (int l = 0; l < NL; ++l) {
                sg.chi0[l][lane] = st.chi0[l];
                sg.eta0[l][lane] = st.eta0[l];
            }
            sg.ds[lane] = R(zf - zk);  // distance increment, differenced in double
            sg.thr[lane] = dtau_max / sg.ds[lane];  // Eq. 2 threshold on chi (single precision)
            sg.nv[lane] = far_end ? 0 : velocity_samples<R>(df, wf, st.delta, st.dv, dv_max, a.status);
        }
        __syncwarp();
        for (int j = 0; j < nch; ++j) {
            nxt.delta = sg.delta[j];
            nxt.dv = sg.dv[j];
            nxt.chic = sg.chic[j];
            nxt.etac = sg.etac[j];
#pragma unroll
            for (int l = 0; l < NL; ++l) {
                nxt.chi0[l] = sg.chi0[l][j];
                nxt.eta0[l] = sg.eta0[l][j];
            }
            const int nv = sg.nv[j];
            if (nv == 0) {  // the far end: its row follows with the first increment
                cur = nxt;
                const R rdv = Ar<R>::rcp(cur.dv);
#pragma unroll
                for (int i = 0; i < BPL; ++i) {
                    optics<R, NL>(cur, rdv, f[i], w[i].chi, w[i].eta);
                    if constexpr (ORD == 4) w[i].Sc = Ar<R>::src(w[i].eta, w[i].chi);
                }
                cmax = w[0].chi;
#pragma unroll
                for (int i = 1; i < BPL; ++i) cmax = fmax(cmax, w[i].chi);
                continue;
            }
            n_smp += unsigned(nv);
            interval<R, NL, BPL, ORD>(cur, nxt, sg.ds[j], sg.thr[j], nv, cmax, a, dtau_max, inv_dtau_max, f, act, w,
                                 n_extra);
        }
    }
    Sample<R, NL> origin;
    load_sample<R, NL>(D, L, o, vox, voy, voz, R(0), R(0), R(0), origin);
    origin.delta = R(0);
    const int nv = velocity_samples<R>(cur.delta, cur.dv, origin.delta, origin.dv, dv_max, a.status);
    n_smp += unsigned(nv);
    const R ds_o = R(zcarry);
    interval<R, NL, BPL, ORD>(cur, origin, ds_o, dtau_max / ds_o, nv, cmax, a, dtau_max, inv_dtau_max, f, act, w,
                         n_extra);
}

// CTAs of 128 threads; the minimum resident CTAs per SM caps the registers
// (65536 / (128 x CTAs)).  Measured on GB300 with the persistent solve: more
// resident warps beat the spills they cost down to 80 registers for one line
// (6 CTAs: 15 % faster than 4); two and four lines run best at 128 registers
// (4 CTAs) and eight at 168 (3), where the per-line sample data need them.
template <typename R, int NL, int BPL>
struct Occ {
    static constexpr int kMinBlocks = sizeof(R) == 8 ? 1 : (NL == 1 ? 6 : NL <= 4 ? 4 : 3);
};

// J of origin a.o_begin + oc for the bins of frequency tile `tile`, by one warp.
template <typename R, int NL, int BPL, int ORD>
__device__ __forceinline__ void solve_item(const DevMesh &m, const DevLines &Ln, const DevRays &Rs,
                                           const SolveArgs &a, int32_t oc, int32_t tile, Stage<R, NL> &sg,
                                           int lane) {
    const int32_t o = a.o_begin + oc;
    const int32_t L = Ln.L, F = Ln.F, NB = L * F;
    const Data<R> D(m, Ln);
    const double dvo = Ln.dvw[o];
    const R vox = __ldg(D.vx + o), voy = __ldg(D.vy + o), voz = __ldg(D.vz + o);
    const double xo = m.x[o], yo = m.y[o], zo = m.z[o];
    Sample<R, NL> org;
    load_sample<R, NL>(D, L, o, vox, voy, voz, R(0), R(0), R(0), org);
    org.delta = R(0);
    (void)sizeof(org);
    const R rdvo = Ar<R>::rcp(org.dv);

    // frequency of each bin of this lane and its profile constants
    Bin<R, NL> f[BPL];
    int32_t bin[BPL];
    bool act[BPL];
    R S_o[BPL];
#pragma unroll
    for (int i = 0; i < BPL; ++i) {
        const int32_t b = tile * 32 * BPL + lane + 32 * i;
        bin[i] = b;
        act[i] = b < NB;
        const int32_t bb = b < NB ? b : NB - 1;
        const int32_t l = bb / F, k = bb % F;
        const double x = (F == 1) ? 0.0 : -Ln.x_span + 2.0 * Ln.x_span * double(k) / double(F - 1);
        const double ub = x * dvo;
#pragma unroll
        for (int lp = 0; lp < NL; ++lp) {
            const double r = (lp < L) ? Ln.ratio[l * MGX_MAX_LINES + lp] : 1.0;
            f[i].A[lp] = R((kC * (r - 1.0) + r * ub) * Ar<R>::kArgScale);
            f[i].B[lp] = R(r * (1.0 + ub / kC) * Ar<R>::kArgScale);
        }
        R chi_o, eta_o;
        optics<R, NL>(org, rdvo, f[i], chi_o, eta_o);
        S_o[i] = eta_o / chi_o;
    }

    double sum[BPL], comp[BPL];
#pragma unroll
    for (int i = 0; i < BPL; ++i) sum[i] = comp[i] = 0.0;
    unsigned n_extra = 0, n_smp = 0;
    const int64_t h0 = int64_t(oc) * Rs.npairs * 2;
    Sweep<R> wb[BPL], wf[BPL];
    for (int32_t p = 0; p < Rs.npairs; ++p) {
        const uint32_t ray = __ldg(Rs.rays + int64_t(o) * Rs.npairs + p);
        const int lev = int(ray >> 28);
        const double *rv = Rs.dir + 3 * (level_offset(lev) + (ray & 0x0FFFFFFFu));
        const double r0 = rv[0], r1 = rv[1], r2 = rv[2];
        const int64_t hb = h0 + 2 * int64_t(p);
        half_sweep<R, NL, BPL, ORD>(m, D, a, L, lane, sg, half_list(a, hb), xo, yo, zo, -r0, -r1, -r2, vox, voy, voz, o,
                               f, act, wb, n_extra, n_smp);
        half_sweep<R, NL, BPL, ORD>(m, D, a, L, lane, sg, half_list(a, hb + 1), xo, yo, zo, r0, r1, r2, vox, voy, voz, o,
                               f, act, wf, n_extra, n_smp);
        const double w2 = a.w2[lev];
#pragma unroll
        for (int i = 0; i < BPL; ++i) {
            const R u = ORD == 4 ? origin_u4(wb[i], wf[i], S_o[i], R(a.I_bdy)) : origin_u2(wb[i], wf[i], S_o[i]);
            if (a.u_out && act[i]) a.u_out[(int64_t(oc) * Rs.npairs + p) * NB + bin[i]] = double(u);
            const double xv = w2 * double(u);
            const double t = sum[i] + xv;  // Neumaier compensated sum
            if (fabs(sum[i]) >= fabs(xv)) comp[i] += (sum[i] - t) + xv;
            else comp[i] += (xv - t) + sum[i];
            sum[i] = t;
        }
    }
    unsigned n_act = 0;
#pragma unroll
    for (int i = 0; i < BPL; ++i) {
        if (act[i]) {
            a.J[int64_t(o) * NB + bin[i]] = sum[i] + comp[i];
            ++n_act;
        }
    }
    if (a.counters) {
        // [0]: sub-intervals beyond one per sample (active bins); [1]: samples x active bins
        unsigned long long u = n_extra;
        unsigned long long s = (unsigned long long)n_smp * n_act;
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

// Grid-mapped launch: warp w of the grid solves item w = oc * n_tiles + tile.
template <typename R, int NL, int BPL, int ORD>
__global__ void __launch_bounds__(128, (Occ<R, NL, BPL>::kMinBlocks))
k_solve(DevMesh m, DevLines Ln, DevRays Rs, SolveArgs a) {
    __shared__ Stage<R, NL> stage[4];  // one per warp of the 128-thread CTA
    const int lane = threadIdx.x & 31;
    const int64_t item = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
    const int64_t n_items = int64_t(a.o_end - a.o_begin) * a.n_tiles;
    if (item >= n_items) return;
    solve_item<R, NL, BPL, ORD>(m, Ln, Rs, a, int32_t(item / a.n_tiles), int32_t(item % a.n_tiles),
                           stage[threadIdx.x >> 5], lane);
}

// Persistent launch over a work list of (model, origin, tile) items of many
// models, sorted by decreasing traced length: each warp takes the next item
// from a global counter until the list is exhausted, so the longest lines
// start first and the tail is short.
template <typename R, int NL, int BPL, int ORD>
__global__ void __launch_bounds__(128, (Occ<R, NL, BPL>::kMinBlocks))
k_solve_queue(const BatchSlot *__restrict__ slots, const uint2 *__restrict__ work, int64_t n_work,
              unsigned long long *__restrict__ next) {
    __shared__ Stage<R, NL> stage[4];
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(next, 1ull);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= (unsigned long long)n_work) return;
        const uint2 w = work[it];  // x = model << 16 | tile, y = origin
        const BatchSlot &s = slots[w.x >> 16];
        solve_item<R, NL, BPL, ORD>(s.m, s.Ln, s.R, s.a, int32_t(w.y), int32_t(w.x & 0xffffu), stage[threadIdx.x >> 5],
                               lane);
    }
}

template <typename R, int BPL, int ORD>
void launch_RB(const DevMesh &m, const DevLines &Ln, const DevRays &R_, const SolveArgs &a, cudaStream_t st) {
    const int64_t n_items = int64_t(a.o_end - a.o_begin) * a.n_tiles;
    if (n_items == 0) return;
    const int tb = 128;
    const unsigned grid = unsigned((n_items * 32 + tb - 1) / tb);
    if (Ln.L <= 1) k_solve<R, 1, BPL, ORD><<<grid, tb, 0, st>>>(m, Ln, R_, a);
    else if (Ln.L <= 2) k_solve<R, 2, BPL, ORD><<<grid, tb, 0, st>>>(m, Ln, R_, a);
    else if (Ln.L <= 4) k_solve<R, 4, BPL, ORD><<<grid, tb, 0, st>>>(m, Ln, R_, a);
    else k_solve<R, 8, BPL, ORD><<<grid, tb, 0, st>>>(m, Ln, R_, a);
}

template <typename R, int BPL, int NL, int ORD>
void launch_queue_NL(const BatchSlot *slots, const uint2 *work, int64_t n_work, unsigned long long *next,
                     cudaStream_t st) {
    int dev = 0, sms = 152, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve_queue<R, NL, BPL, ORD>, 128, 0);
    if (per_sm < 1) per_sm = 1;
    int64_t grid = int64_t(sms) * per_sm;
    const int64_t need = (n_work + 3) / 4;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    k_solve_queue<R, NL, BPL, ORD><<<unsigned(grid), 128, 0, st>>>(slots, work, n_work, next);
}

template <typename R, int BPL, int ORD>
void launch_queue_RB(int max_lines, const BatchSlot *slots, const uint2 *work, int64_t n_work,
                     unsigned long long *next, cudaStream_t st) {
    if (max_lines <= 1) launch_queue_NL<R, BPL, 1, ORD>(slots, work, n_work, next, st);
    else if (max_lines <= 2) launch_queue_NL<R, BPL, 2, ORD>(slots, work, n_work, next, st);
    else if (max_lines <= 4) launch_queue_NL<R, BPL, 4, ORD>(slots, work, n_work, next, st);
    else launch_queue_NL<R, BPL, 8, ORD>(slots, work, n_work, next, st);
}

}  // namespace

template <int ORD>
void launch_solve_ord(const DevMesh &m, const DevLines &Ln, const DevRays &R, const SolveArgs &a, int precision,
                      cudaStream_t st) {
    const int bpl = solve_bins_per_lane(precision, Ln.L * Ln.F);
    if (precision == MGX_FP64) launch_RB<double, 1, ORD>(m, Ln, R, a, st);
    else if (bpl == 2) launch_RB<float, 2, ORD>(m, Ln, R, a, st);
    else launch_RB<float, 1, ORD>(m, Ln, R, a, st);
}

template <int ORD>
void launch_solve_queue_ord(int precision, int bins_per_lane, int max_lines, const BatchSlot *slots,
                            const uint2 *work, int64_t n_work, unsigned long long *next, cudaStream_t st) {
    if (n_work == 0) return;
    if (precision == MGX_FP64) launch_queue_RB<double, 1, ORD>(max_lines, slots, work, n_work, next, st);
    else if (bins_per_lane == 2) launch_queue_RB<float, 2, ORD>(max_lines, slots, work, n_work, next, st);
    else launch_queue_RB<float, 1, ORD>(max_lines, slots, work, n_work, next, st);
}

}  // namespace mgx
