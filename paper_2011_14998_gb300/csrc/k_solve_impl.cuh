// k_solve_impl.cuh -- formal solution along ray pairs and the mean intensity J
// (Eqs. 1-3, Sections 2.1.1-2.1.2).
//
// One warp per (origin, frequency tile); each lane carries BPL frequency bins
// (bin tile*32*BPL + lane + 32 i, i < BPL).  The warp walks every ray pair of
// its origin in ascending pair order.  Each half of the pair runs from the far
// end of its traced point list to the origin, in chunks of 32 points:
//   1. staging: lane j takes one point of the chunk -- its exact projected
//      distance Z (double), projected velocity difference delta = (v - v_o).d
//      and line data -- and, for the interval to the farther point, the number
//      of velocity samples (Section 2.1.1) and the constants of Eq. 2;
//   2. sample generation: the chunk's velocity samples (data linear in
//      distance between consecutive points, Section 2.1.1) are written to
//      shared memory as one record per sample, the lanes generating them in
//      parallel, so the frequency-independent work of a sample is done once
//      per warp instead of once per lane;
//   3. elimination: every lane reads each record (a broadcast) and, for each
//      of its bins,
//        * line optics: chi = chi_c + sum_l chi0_l exp(-a_l^2), eta likewise,
//          a_l the Doppler-shifted profile argument of line l at the bin;
//        * Eq. 2: the sample interval is split into
//          n_inter = ceil(max(chi) ds / dtau_max) equal parts, chi and eta
//          linear, trapezoidal dtau;
//        * Gaussian elimination of the Feautrier system (Eq. 1, second-order
//          boundary condition) in the scaled form of Rybicki & Hummer (1991):
//            boundary row:  Fh = 1 + dt/2,       D = 1/(1 + dt Fh), zh = D (S dt/2 + I)
//            interior row:  Fh = dtbar + D Fh,   D = 1/(1 + dt Fh), zh = D (dtbar S + zh)
//          with Fh = F_i / dtau_i and zh = z_i / dtau_i of the textbook 1+B
//          form, so no quantity overflows for small dtau and no difference of
//          nearly equal numbers is formed.  The boundary row is the interior row
//          applied to the state (Fh, D, zh, dtbar) = (1, 1, I, dt/2), and one
//          reciprocal 1 / (chi (1 + dt Fh)) per row yields both D and D S.
// The two half-sweeps meet at the origin row, which gives u without back
// substitution:  u_o = (dtbar S_o + zh- + zh+) / (dtbar + D- Fh- + D+ Fh+),
// an empty half contributing (zh, D Fh) = (I, 1).  J accumulates 2 w u in
// double precision with Neumaier's compensated sum.
//
// Template R selects the arithmetic: double (plain form: the samples are laid
// out exactly as the definition interpolates them, and Eq. 2 is evaluated as
// written) or float (single-precision bulk; Z and its differences and the J
// sum in double).
//
// Integer decisions of the single-precision form.  The velocity-sample count
// and Eq. 2's n_inter are the integers the double-precision definition gives.
// Each is first taken on the single-precision values together with a rigorous
// bound on their distance from the double-precision ones (the rounding of every
// operand and operation, the approximate reciprocal and exp2 at the error
// bounds below); where the bound does not separate the decision from the next
// integer it is redone in double precision from the double-precision point
// data, in the definition's order of operations.  The bound of Eq. 2 is folded
// into the per-interval threshold on chi, so the common case (no sub-interval
// anywhere in the warp) costs nothing extra.
#pragma once

#include "mgx_internal.cuh"

namespace mgx {

namespace {

constexpr unsigned kFull = 0xffffffffu;

template <typename R>
struct Ar;

// Double precision (plain form): the Gaussian exp(-a^2) and IEEE divisions.
template <>
struct Ar<double> {
    static constexpr double kArgScale = 1.0;
    static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
    static __device__ __forceinline__ double gauss(double a) { return exp(-(a * a)); }
    static __device__ __forceinline__ double src(double eta, double chi) { return eta / chi; }
};

// Single precision: the profile constants are prescaled by sqrt(log2 e), so
// exp(-a^2) = 2^(-a'^2) is one ex2.approx; reciprocals are rcp.approx.
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
    static __device__ __forceinline__ float src(float eta, float chi) { return eta * rcp(chi); }
};

// Error constants of the single-precision decisions: the unit roundoff and the
// relative errors taken for rcp.approx.ftz.f32 (documented at 1 ulp; 2 ulp
// taken) and ex2.approx.ftz.f32 (2^-20, well above what GB300 gives; a GPU
// test checks both bounds against double-precision references).
constexpr float kU = 5.9604644775390625e-8f;    // 2^-24
constexpr float kERcp = 2.384185791015625e-7f;  // 2^-22
constexpr float kEEx2 = 9.5367431640625e-7f;    // 2^-20
// |delta32 - delta64| <= kDeltaErr sum_i (|v_i| + |v_o,i|) |d_i| for the
// single-precision projection (operands rounded to single, then three
// products and two sums)
constexpr float kDeltaErr = 6.5f * kU;

// The point arrays of the form's precision, read from the mesh and line
// descriptors at each use (the descriptors live in constant or global memory,
// so no registers hold the pointers across the elimination loop).
template <typename R>
struct Pts;

template <>
struct Pts<double> {
    static __device__ __forceinline__ const double *vx(const DevMesh &m) { return m.vx; }
    static __device__ __forceinline__ const double *vy(const DevMesh &m) { return m.vy; }
    static __device__ __forceinline__ const double *vz(const DevMesh &m) { return m.vz; }
    static __device__ __forceinline__ const double *chi0(const DevLines &L) { return L.chi0; }
    static __device__ __forceinline__ const double *eta0(const DevLines &L) { return L.eta0; }
    static __device__ __forceinline__ const double *dvw(const DevLines &L) { return L.dvw; }
    static __device__ __forceinline__ const double *chic(const DevLines &L) { return L.chic; }
    static __device__ __forceinline__ const double *etac(const DevLines &L) { return L.etac; }
};

template <>
struct Pts<float> {
    static __device__ __forceinline__ const float *vx(const DevMesh &m) { return m.vxf; }
    static __device__ __forceinline__ const float *vy(const DevMesh &m) { return m.vyf; }
    static __device__ __forceinline__ const float *vz(const DevMesh &m) { return m.vzf; }
    static __device__ __forceinline__ const float *chi0(const DevLines &L) { return L.chi0f; }
    static __device__ __forceinline__ const float *eta0(const DevLines &L) { return L.eta0f; }
    static __device__ __forceinline__ const float *dvw(const DevLines &L) { return L.dvwf; }
    static __device__ __forceinline__ const float *chic(const DevLines &L) { return L.chicf; }
    static __device__ __forceinline__ const float *etac(const DevLines &L) { return L.etacf; }
};

// Per-bin constants: the Doppler-shifted profile argument of line l at this
// bin is (A[l] + B[l] delta) / dv (prescaled for the single-precision ex2).
template <typename R, int NL>
struct Bin {
    R A[NL], B[NL];
};

// Total opacity and emissivity of a sample for one bin: delta, rdv = 1/dv,
// continuum (cc, ec) and line-centre values ce[2l] = chi0_l, ce[2l+1] = eta0_l.
// Lines past the model's count have chi0 = eta0 = 0 and contribute nothing.
template <typename R, int NL>
__device__ __forceinline__ void optics(R delta, R rdv, R cc, R ec, const R *ce, const Bin<R, NL> &f, R &chi,
                                       R &eta) {
    chi = cc;
    eta = ec;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        const R g = Ar<R>::gauss(fma(f.B[l], delta, f.A[l]) * rdv);
        chi = fma(ce[2 * l], g, chi);
        eta = fma(ce[2 * l + 1], g, eta);
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
//
// P is the precision of the pivot recurrence (Fh, D and the increments dt):
// R, or double with R = float (the form with double-precision optical-depth
// increments and pivots, second-order scheme only).
template <typename R, typename P = R>
struct Sweep {
    P Fh, Dm, dtp;  // scaled 1+B quantities of the last eliminated row, half its dtau
    R zh;
    R chi, eta;     // optics of the current (not yet eliminated) sample
    R Sp, Sc, hp, rh;  // Hermitian scheme only
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

template <int ORD, typename R, typename P>
__device__ __forceinline__ void row(Sweep<R, P> &w, R chi, R eta, P dt, R Si, R Sn) {
    if constexpr (ORD == 2) {
        const P dtb = fma(dt, P(0.5), w.dtp);
        w.Fh = dtb + w.Dm * w.Fh;
        if constexpr (sizeof(P) == sizeof(R)) {
            const R rr = Ar<R>::rcp(chi * (R(1) + dt * w.Fh));
            w.Dm = chi * rr;
            w.zh = w.Dm * w.zh + dtb * (eta * rr);
        } else {
            // pivots in double precision: D = 1 / (1 + dt Fh); z in single
            // precision from D and S = eta / chi
            const P D = P(1) / (P(1) + dt * w.Fh);
            w.Dm = D;
            w.zh = R(D) * w.zh + R(dtb * D) * (eta * Ar<R>::rcp(chi));
        }
        w.dtp = dt * P(0.5);
    } else {
        static_assert(sizeof(P) == sizeof(R), "the Hermitian scheme keeps its pivots in the form's precision");
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

// u at the origin row from the two half-sweeps (the origin row couples the
// last eliminated rows of both halves; no back substitution is needed).
// Second order: u_o = (dtbar S_o + zh- + zh+) / (dtbar + D- Fh- + D+ Fh+), an
// empty half contributing (D Fh, zh) = (1, I) through its initial state.
template <typename R, typename P>
__device__ __forceinline__ R origin_u2(const Sweep<R, P> &b, const Sweep<R, P> &f, R So) {
    const P dtb = b.dtp + f.dtp;  // the halves of the two last increments
    return R((dtb * P(So) + P(b.zh) + P(f.zh)) / (dtb + b.Dm * b.Fh + f.Dm * f.Fh));
}

// Hermitian scheme: with h- (h+) the last increment of the backward (forward)
// half and lambda- = 1 - (h-^2 + h- h+ - h+^2)/12, lambda+ = 1 - (h+^2 + h- h+ - h-^2)/12,
//   u_o = (hbar r_o + lambda- zh- + lambda+ zh+) / (hbar + lambda- D- Fh- + lambda+ D+ Fh+);
// with one half empty the origin row is the third-order boundary row,
//   u_o = (h S_o/3 + h S_1/6 + I + (1 - h^2/6) zh) / (1 + h/2 + (1 - h^2/6) D Fh);
// with both empty u_o = I.
template <typename R, typename P>
__device__ __forceinline__ R origin_u4(const Sweep<R, P> &b, const Sweep<R, P> &f, R So, R I) {
    if (b.hp < R(0) && f.hp < R(0)) return I;
    if (b.hp < R(0) || f.hp < R(0)) {
        const Sweep<R, P> &w = b.hp < R(0) ? f : b;
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

// Layout of one velocity-sample record, as the bins read it: delta, 1/dv,
// continuum opacity and emissivity, half the distance to the previous sample,
// the Eq. 2 threshold on chi, then chi0 and eta0 of each line; padded to whole
// 16-byte words so that each word is one shared-memory load.  In single
// precision with one line, a negative 1/dv marks a sample in the far wing of
// every bin of the tile (the optics are the continuum's) and an infinite
// threshold an interval on which no bin can need a split.
template <typename R, int NL>
struct Rec {
    static constexpr int kVals = 6 + 2 * NL;
    static constexpr int kPer16 = int(16 / sizeof(R));
    static constexpr int kStride = (kVals + kPer16 - 1) / kPer16 * kPer16;
};

// Per-warp shared staging: the sample records of the chunk being eliminated
// (kCap at a time), the chunk's points (slot 0 holds the point just farther
// than the chunk, slots 1..32 the chunk, far to near) with the constants of
// the interval from the farther point, and the warp's item.
template <typename R, int NL>
struct Stage {
    static constexpr int kCap = sizeof(R) == 4 ? 32 : (NL <= 4 ? 32 : 16);
    static constexpr int kS = Rec<R, NL>::kStride;
    static constexpr int kF = sizeof(R) == 4 ? 33 : 1;  // arrays of the single-precision decisions
    alignas(16) R rec[kCap * kS];
    int sk[kCap];                           // slot | (sample index j << 6) of each record
    R d[33], w[33], cc[33], ec[33];         // delta, Doppler width, continuum
    R ce[2 * NL][33];                       // chi0 and eta0 per line
    R hq[33], thr[33];                      // half the sample spacing, Eq. 2 threshold
    R E[kF], qlo[kF], qhi[kF];              // bound of |chi - chi64|, Eq. 2 ratio factors
    R de0;                                  // single precision: bound of |delta - delta64| of the carried point
    double z[sizeof(R) == 8 ? 33 : 1];      // exact Z (single precision: the carried point's only)
    int id[33], nv[33], so[33];             // point (-1: the origin), velocity samples, their offset
    R Am[NL], Bm[NL];                       // largest |A|, |B| of each line over the warp's bins
    double r[3], xo[3], vo[3];              // pair direction, origin position and velocity (double)
    R vor[3];                               // origin velocity in the form's precision
    int o, NB, tile;                        // origin, bins of the model, the warp's frequency tile
    HalfList hl;                            // traced list of the half being eliminated
    unsigned n_smp, n_extra, n_redo;        // work counters of the item (samples, extra sub-intervals, redone decisions)
    int fix[2][32];                         // Eq. 2 counts of a sample whose single-precision decision was
                                            // left open (-1: to redo in double precision; 0: not open)
    R fA[NL][2][32], fB[NL][2][32];         // profile constants of each lane's bins (Bin)
    float wa[2], wb[2];                     // single precision, one line: A, B of the tile's first and last bin
    int wing;                               // the far-wing test of the records is on
};

// Bin i of the lane in the warp's tile (>= NB: beyond the last, inactive).
template <int BPL, typename St>
__device__ __forceinline__ int32_t lane_bin(const St &sg, int i, int lane) {
    return sg.tile * 32 * BPL + lane + 32 * i;
}

// Per-lane state that lives across chunks of samples, kept in shared memory
// so that no register holds it across the out-of-line staging calls: the
// elimination state of each of the lane's (at most two) bins (D and Fh enter
// every step only as their product, which is what is kept) and the running
// maximum of chi.  The pivot quantities (D Fh, dtb/2) are kept in the pivot
// precision P.  What is needed only once per pair (the J sums, the origin's
// source function, the backward half's coupling to the origin row) stays in
// the item loop's registers, so that 9 CTAs fit the shared memory.
template <typename R, int ORD, typename P = R>
struct Lane {
    static constexpr int kWR = ORD == 4 ? 6 : 3;  // zh, chi, eta (Hermitian: + Sp, Sc, hp; rh = 1/hp re-formed)
    P wp[2][2][32];                              // D Fh, dtb/2
    R wr[kWR][2][32];
    R cm[32];
};

// Projected distance Z = (x_n - x_o).d exactly as the tracer and its
// definition form it (explicitly rounded double operations in fixed order).
__device__ __forceinline__ double exact_Z(const DevMesh &m, int32_t id, double xo, double yo, double zo, double d0,
                                          double d1, double d2) {
    const double dx = __dsub_rn(__ldg(m.x + id), xo);
    const double dy = __dsub_rn(__ldg(m.y + id), yo);
    const double dz = __dsub_rn(__ldg(m.z + id), zo);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, d0), __dmul_rn(dy, d1)), __dmul_rn(dz, d2));
}

// Projected velocity difference (v_n - v_o).d in double precision, (x + y) + z
// with every product and sum rounded (the definition's order).
__device__ __forceinline__ double proj64(const DevMesh &m, int32_t id, const double *vo, double d0, double d1,
                                         double d2) {
    const double ux = __dsub_rn(__ldg(m.vx + id), vo[0]);
    const double uy = __dsub_rn(__ldg(m.vy + id), vo[1]);
    const double uz = __dsub_rn(__ldg(m.vz + id), vo[2]);
    return __dadd_rn(__dadd_rn(__dmul_rn(ux, d0), __dmul_rn(uy, d1)), __dmul_rn(uz, d2));
}

// ---- double-precision redo of the single-precision form's decisions ------
// (rare: only where the single-precision bound leaves the integer open)

// Velocity samples of the interval between points ia and ib (-1: the origin)
// on the half along sgn r (Section 2.1.1): ceil(|delta_b - delta_a| /
// (dv_max min(dv_a, dv_b))) when the jump exceeds the limit, else 1.
__device__ __noinline__ int redo_velocity_samples(const DevMesh &m, const DevLines &Ln, const double *r,
                                                  const double *vo, int32_t o, double sgn, int32_t ia, int32_t ib,
                                                  double dv_max) {
    const double e0 = sgn * r[0], e1 = sgn * r[1], e2 = sgn * r[2];
    const double da = ia < 0 ? 0.0 : proj64(m, ia, vo, e0, e1, e2);
    const double db = ib < 0 ? 0.0 : proj64(m, ib, vo, e0, e1, e2);
    const double wa = Ln.dvw[ia < 0 ? o : ia], wb = Ln.dvw[ib < 0 ? o : ib];
    const double jump = fabs(__dsub_rn(db, da));
    const double lim = __dmul_rn(dv_max, fmin(wa, wb));
    if (!(jump > lim)) return 1;
    const double n = ceil(__ddiv_rn(jump, lim));
    return n > double(kMaxSubdiv) ? kMaxSubdiv + 1 : int(n);
}

// Eq. 2's n_inter for bin `bin` on the sub-interval between the velocity
// samples j-1 and j (counted from the farther point a, 0 = a, nv = b) of the
// interval from point ia to point ib, -1 being the origin.  The two samples are formed as the definition lays out the pair
// line: ordered along +r (the backward half from its far end, the forward half
// from the origin), each quantity interpolated linearly from the earlier point
// with t = i / nv; the opacity is the line optics of Magritte I evaluated in
// that order; n_inter = ceil(max(chi) ds / dtau_max), at least 1.
__device__ __noinline__ int redo_n_inter(const DevMesh &m, const DevLines &Ln, const double *r, const double *vo,
                                         int32_t o, double sgn, int32_t ia, int32_t ib, int nv, int j, int32_t bin,
                                         double dtau_max) {
    const bool bwd = sgn < 0.0;
    const double e0 = sgn * r[0], e1 = sgn * r[1], e2 = sgn * r[2];
    // the exact Z of the two points (0 at the origin, id -1)
    const double xo = m.x[o], yo = m.y[o], zo = m.z[o];
    const double za = ia < 0 ? 0.0 : exact_Z(m, ia, xo, yo, zo, e0, e1, e2);
    const double zb = ib < 0 ? 0.0 : exact_Z(m, ib, xo, yo, zo, e0, e1, e2);
    const int32_t p0 = bwd ? ia : ib, p1 = bwd ? ib : ia;  // base points in the definition's order
    const double z0 = bwd ? za : zb, z1 = bwd ? zb : za;
    const int ilo = bwd ? j - 1 : nv - j;  // indices of the two samples from p0
    const int32_t L = Ln.L, F = Ln.F, l = bin / F, k = bin - l * F;
    const double x = F == 1 ? 0.0
                            : __dadd_rn(-Ln.x_span, __ddiv_rn(__dmul_rn(2.0 * Ln.x_span, double(k)), double(F - 1)));
    const double ub = __dmul_rn(x, Ln.dvw[o]);
    const int32_t q0 = p0 < 0 ? o : p0, q1 = p1 < 0 ? o : p1;
    const double d0 = p0 < 0 ? 0.0 : proj64(m, p0, vo, e0, e1, e2);
    const double d1 = p1 < 0 ? 0.0 : proj64(m, p1, vo, e0, e1, e2);
    const double s0 = p0 < 0 ? 0.0 : sgn * z0, s1 = p1 < 0 ? 0.0 : sgn * z1;
    double chi[2], s[2];
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
        const int i = ilo + h;
        const bool at0 = i == 0, at1 = i == nv;
        const double t = __ddiv_rn(double(i), double(nv));
        auto lerp = [&](double a0, double a1) -> double {
            return at0 ? a0 : at1 ? a1 : __dadd_rn(a0, __dmul_rn(__dsub_rn(a1, a0), t));
        };
        s[h] = lerp(s0, s1);
        const double dl = lerp(d0, d1);
        const double dv = lerp(Ln.dvw[q0], Ln.dvw[q1]);
        double c = lerp(Ln.chic[q0], Ln.chic[q1]);
        for (int lp = 0; lp < L; ++lp) {
            const double c0 = lerp(Ln.chi0[int64_t(q0) * L + lp], Ln.chi0[int64_t(q1) * L + lp]);
            const double rr = Ln.ratio[l * MGX_MAX_LINES + lp];
            const double num = __dadd_rn(__dadd_rn(__dmul_rn(kC, __dsub_rn(rr, 1.0)), __dmul_rn(rr, ub)),
                                         __dmul_rn(__dmul_rn(rr, __dadd_rn(1.0, __ddiv_rn(ub, kC))), dl));
            const double arg = __ddiv_rn(num, dv);
            const double g = exp(-__dmul_rn(arg, arg));
            c = __dadd_rn(c, __dmul_rn(c0, g));
        }
        chi[h] = c;
    }
    const double n = ceil(__ddiv_rn(__dmul_rn(fmax(chi[0], chi[1]), __dsub_rn(s[1], s[0])), dtau_max));
    if (n > double(kMaxSubdiv)) return kMaxSubdiv + 1;
    return n < 1.0 ? 1 : int(n);
}

// ---- staging ----------------------------------------------------------------

// Point q of the half (q < cnt: traced entry cnt-1-q, far end first; q == cnt:
// the origin) into `slot`; its exact Z and (single precision) the bound of
// its delta's error are also returned, for the interval to it.
template <typename R, int NL>
__device__ __forceinline__ void stage_point(const DevMesh &m, const DevLines &Ln, Stage<R, NL> &sg, int32_t q,
                                            int32_t cnt, int slot, int sign, double &zq, R &deq) {
    const HalfList &hl = sg.hl;
    const double sgn = double(sign);
    const int32_t L = Ln.L;
    const double e0 = sgn * sg.r[0], e1 = sgn * sg.r[1], e2 = sgn * sg.r[2];
    int32_t id = sg.o;
    double z = 0.0;
    R d = R(0), de = R(0);
    if (q < cnt) {
        const int32_t k = cnt - 1 - q;
        // the traced ids stream through once: evict-first, so that they do not push the
        // mesh and the spilled item state out of L2
        id = k < hl.n_main ? __ldcs(hl.main + k) : __ldcs(hl.tail + (hl.tail_off + k));
        z = exact_Z(m, id, sg.xo[0], sg.xo[1], sg.xo[2], e0, e1, e2);
        if constexpr (sizeof(R) == 8) {
            d = proj64(m, id, sg.vo, e0, e1, e2);
        } else {
            const float f0 = float(e0), f1 = float(e1), f2 = float(e2);
            const float vx = __ldg(Pts<R>::vx(m) + id), vy = __ldg(Pts<R>::vy(m) + id), vz = __ldg(Pts<R>::vz(m) + id);
            const float ux = vx - sg.vor[0], uy = vy - sg.vor[1], uz = vz - sg.vor[2];
            d = fmaf(uz, f2, fmaf(uy, f1, ux * f0));
            de = kDeltaErr * ((fabsf(vx) + fabsf(sg.vor[0])) * fabsf(f0) + (fabsf(vy) + fabsf(sg.vor[1])) * fabsf(f1) +
                              (fabsf(vz) + fabsf(sg.vor[2])) * fabsf(f2));
        }
    }
    sg.id[slot] = q < cnt ? id : -1;
    if constexpr (sizeof(R) == 8) sg.z[slot] = z;
    zq = z;
    deq = de;
    sg.d[slot] = d;
    sg.w[slot] = __ldg(Pts<R>::dvw(Ln) + id);
    sg.cc[slot] = __ldg(Pts<R>::chic(Ln) + id);
    sg.ec[slot] = __ldg(Pts<R>::etac(Ln) + id);
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        sg.ce[2 * l][slot] = l < L ? __ldg(Pts<R>::chi0(Ln) + int64_t(id) * L + l) : R(0);
        sg.ce[2 * l + 1][slot] = l < L ? __ldg(Pts<R>::eta0(Ln) + int64_t(id) * L + l) : R(0);
    }
}

// The interval from the point in slot-1 (farther) to the point in `slot`:
// its number of velocity samples (Section 2.1.1) and, in single precision,
// the constants of Eq. 2 with the bound on the opacity's error.  za, zb are
// the exact Z of the farther and the nearer point, dea, deb the bounds of
// their deltas' errors (single precision).
template <typename R, int NL>
__device__ __forceinline__ int stage_interval(const DevMesh &m, const DevLines &Ln, const SolveArgs &a,
                                              Stage<R, NL> &sg, int slot, int sign, double za, double zb, R dea,
                                              R deb) {
    const int pa = slot - 1;
    if constexpr (sizeof(R) == 8) {
        // as defined: ceil(|delta_b - delta_a| / (dv_max min(dv_a, dv_b))) when that exceeds one
        int nv = 1;
        if (a.dv_max > 0.0) {
            const double jump = fabs(sg.d[slot] - sg.d[pa]);
            const double lim = a.dv_max * fmin(sg.w[pa], sg.w[slot]);
            if (jump > lim) {
                const double n = ceil(jump / lim);
                nv = n > double(kMaxSubdiv) ? kMaxSubdiv + 1 : int(n);
            }
        }
        if (nv > kMaxSubdiv) {
            dev_fail(a.status, kDevSubdivLimit);
            nv = kMaxSubdiv;
        }
        return nv;
    } else {
        const float da = sg.d[pa], db = sg.d[slot], wa = sg.w[pa], wb = sg.w[slot];
        int nv = 1;
        if (a.dv_max > 0.0) {
            // q64 = jump64 / lim64 lies in [(jump - ej) / lim (1 - k), (jump + ej) / lim (1 + k)]
            const float jump = fabsf(db - da);
            const float ej = dea + deb + 2.f * kU * jump;
            const float rl = 1.f / (float(a.dv_max) * fminf(wa, wb));
            const float nhi = ceilf((jump + ej) * rl * (1.f + 16.f * kU));
            if (nhi > 1.f) {
                const float nlo = ceilf((jump - ej) * rl * (1.f - 16.f * kU));
                if (nlo == nhi) {
                    nv = nhi > float(kMaxSubdiv) ? kMaxSubdiv + 1 : int(nhi);
                } else {
                    nv = redo_velocity_samples(m, Ln, sg.r, sg.vo, sg.o, double(sign), sg.id[pa], sg.id[slot],
                                               a.dv_max);
                    atomicAdd(&sg.n_redo, 1u);
                }
                if (nv > kMaxSubdiv) {
                    dev_fail(a.status, kDevSubdivLimit);
                    nv = kMaxSubdiv;
                }
            }
        }
        const float ds = float(za - zb);  // distance increment, differenced in double
        const float rn = 1.f / float(nv);
        const float hs = ds * rn;
        // Bound E of |chi32 - chi64| at every sample of the interval (both
        // ends included), from the errors of delta (de, interpolation), dv,
        // the profile constants, the profile argument, ex2 and the sums:
        //   |g32 - g64| <= 0.7142 |da'| + 0.7358 rho + u/e + eps_ex2
        // (0.7142 = max |d/da 2^(-a^2)|, 0.7358 = max |a d/da 2^(-a^2)|).
        const float k6 = 6.f * kU + kERcp;  // interpolation in single precision
        const float ada = fabsf(da), adb = fabsf(db);
        const float dmax = fmaxf(ada, adb);
        const float edi = dea + deb + k6 * (ada + adb);
        const float rdvmin = 1.f / fminf(wa, wb);
        const float rho = kERcp + k6 * (wa + wb) * rdvmin + 4.f * kU;
        float E = 0.f, csum = fmaxf(sg.cc[pa], sg.cc[slot]);
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            const float dA = (3.f * kU * (sg.Am[l] + sg.Bm[l] * dmax) + sg.Bm[l] * edi) * rdvmin * (1.f + rho);
            const float Eg = 0.7142f * dA + 0.7358f * rho * 1.001f + 0.3679f * kU + kEEx2 + 2.f * dA * dA;
            const float c0a = sg.ce[2 * l][pa], c0b = sg.ce[2 * l][slot], c0m = fmaxf(c0a, c0b);
            E += c0m * Eg + k6 * (c0a + c0b) + kU * c0m;
            csum += c0m;
        }
        E += k6 * (sg.cc[pa] + sg.cc[slot]) + kU * fmaxf(sg.cc[pa], sg.cc[slot]) + float(NL + 1) * kU * csum;
        E *= 1.0625f;
        // Eq. 2: n_inter = max(1, ceil(fl(fl(chi64 ds64) / dtau_max))); ds64, the
        // definition's sample spacing, is within (3u + rho_s) of hs, rho_s the
        // rounding of its interpolated distances (8 u64 max|Z| / hs)
        const float zmax = float(fmax(za, zb));
        const float kap = 15.f * kU + 9.0e-16f * zmax / hs + 1e-15f;
        const float dtm = float(a.dtau_max);
        const float qs = hs * float(1.0 / a.dtau_max);
        sg.hq[slot] = 0.5f * hs;
        sg.thr[slot] = (dtm / hs) * (1.f - kap) - E * (1.f + 4.f * kU);
        sg.qlo[slot] = qs * (1.f - kap);
        sg.qhi[slot] = qs * (1.f + kap);
        sg.E[slot] = E;
        return nv;
    }
}

// Record of sample s_abs of the chunk (relative to its first) into record s_rec.
template <typename R, int NL>
__device__ __forceinline__ void gen_sample(Stage<R, NL> &sg, int s_abs, int s_rec, int nch, int sign,
                                           double dtau_max) {
    constexpr int kS = Stage<R, NL>::kS;
    int lo = 1, hi = nch;  // the last slot whose samples start at or before s_abs
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sg.so[mid] <= s_abs) lo = mid;
        else hi = mid - 1;
    }
    const int k = lo, nv = sg.nv[k], j = s_abs - sg.so[k] + 1;
    R *o = sg.rec + s_rec * kS;
    sg.sk[s_rec] = k | (j << 6);
    if constexpr (sizeof(R) == 4) {
        const int pa = k - 1;
        float wv;
        if (j == nv) {
            o[0] = sg.d[k];
            wv = sg.w[k];
            o[2] = sg.cc[k];
            o[3] = sg.ec[k];
#pragma unroll
            for (int c = 0; c < 2 * NL; ++c) o[6 + c] = sg.ce[c][k];
        } else {
            const float t = float(j) * (1.f / float(nv));  // rn of the interval, formed again
            o[0] = fmaf(sg.d[k] - sg.d[pa], t, sg.d[pa]);
            wv = fmaf(sg.w[k] - sg.w[pa], t, sg.w[pa]);
            o[2] = fmaf(sg.cc[k] - sg.cc[pa], t, sg.cc[pa]);
            o[3] = fmaf(sg.ec[k] - sg.ec[pa], t, sg.ec[pa]);
#pragma unroll
            for (int c = 0; c < 2 * NL; ++c) o[6 + c] = fmaf(sg.ce[c][k] - sg.ce[c][pa], t, sg.ce[c][pa]);
        }
        o[1] = Ar<float>::rcp(wv);
        if constexpr (NL == 1) {
            // far wing: when every bin's profile argument a = fl(fl(B delta + A) rdv)
            // has a^2 >= 128, ex2.approx.ftz(-a^2) is exactly 0 and the optics are
            // the continuum's (bit for bit).  A and B rise with the bin, so over the
            // tile B delta + A lies in [min(tf, tl) - W, max(tf, tl) + W] with
            // W = (B_last - B_first) |delta|; |a| >= 12.1 leaves margin for every
            // rounding.  The record carries the outcome as a negative 1/dv.
            if (sg.wing) {
                const float dl = o[0];
                const float tf = fmaf(sg.wb[0], dl, sg.wa[0]), tl = fmaf(sg.wb[1], dl, sg.wa[1]);
                const float W = 1.01f * (sg.wb[1] - sg.wb[0]) * fabsf(dl);
                const float lo = (fminf(tf, tl) - W) * o[1], hi = (fmaxf(tf, tl) + W) * o[1];
                if (lo >= 12.1f || hi <= -12.1f) o[1] = -o[1];
            }
        }
        o[4] = sg.hq[k];
        o[5] = sg.thr[k];
        if constexpr (NL == 1) {
            // no bin can split anywhere on the interval when the largest opacity any
            // sample of it (or the point before it) can reach, continuum plus line
            // centre (the profile is at most 1; interpolation and the fused sums
            // round within 4u), stays below the threshold: the record says so
            // with an infinite threshold and the step skips the vote
            const float cb = fmaxf(sg.cc[pa], sg.cc[k]) + fmaxf(sg.ce[0][pa], sg.ce[0][k]);
            if (cb * (1.f + 8.f * kU) <= o[5]) o[5] = INFINITY;
        }
    } else {
        // the definition's layout: samples interpolated from the earlier point
        // along +r with t = i / nv, exact end points; ds between consecutive samples
        const bool bwd = sign < 0;
        const double sgn = double(sign);
        const int b0 = bwd ? k - 1 : k, b1 = bwd ? k : k - 1;
        const int i = bwd ? j : nv - j, ip = bwd ? j - 1 : nv - j + 1;
        auto at = [&](double x0, double x1, int ii) -> double {
            if (ii == 0) return x0;
            if (ii == nv) return x1;
            const double t = __ddiv_rn(double(ii), double(nv));
            return __dadd_rn(x0, __dmul_rn(__dsub_rn(x1, x0), t));
        };
        const double s0 = sgn * sg.z[b0], s1 = sgn * sg.z[b1];
        const double si = at(s0, s1, i), sp = at(s0, s1, ip);
        const double ds = bwd ? __dsub_rn(si, sp) : __dsub_rn(sp, si);
        o[0] = at(sg.d[b0], sg.d[b1], i);
        o[1] = 1.0 / at(sg.w[b0], sg.w[b1], i);
        o[2] = at(sg.cc[b0], sg.cc[b1], i);
        o[3] = at(sg.ec[b0], sg.ec[b1], i);
#pragma unroll
        for (int c = 0; c < 2 * NL; ++c) o[6 + c] = at(sg.ce[c][b0], sg.ce[c][b1], i);
        o[4] = 0.5 * ds;
        o[5] = (dtau_max / ds) * (1.0 - 0x1p-40);  // chi below this gives n_inter = 1
    }
}

template <typename R, int NL>
__device__ __forceinline__ void load_rec(const R *src, R (&v)[Stage<R, NL>::kS]) {
    constexpr int kS = Stage<R, NL>::kS;
    if constexpr (sizeof(R) == 4) {
#pragma unroll
        for (int c = 0; c < kS / 4; ++c) {
            const float4 t = reinterpret_cast<const float4 *>(src)[c];
            v[4 * c] = t.x;
            v[4 * c + 1] = t.y;
            v[4 * c + 2] = t.z;
            v[4 * c + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int c = 0; c < kS / 2; ++c) {
            const double2 t = reinterpret_cast<const double2 *>(src)[c];
            v[2 * c] = t.x;
            v[2 * c + 1] = t.y;
        }
    }
}

// Eq. 2's n_inter of one bin whose larger opacity cm may exceed the sample's
// threshold.  Double precision: as defined.  Single precision: certified from
// the bound E; 0 when the bound leaves the integer open (the caller has it
// redone in double precision).
template <typename R, int NL>
__device__ __forceinline__ int n_inter(R cm, R hq, int s, const Stage<R, NL> &sg, const SolveArgs &a) {
    int n;
    if constexpr (sizeof(R) == 8) {
        const double nr = ceil((cm * (hq + hq)) / a.dtau_max);
        n = nr > double(kMaxSubdiv) ? kMaxSubdiv + 1 : nr <= 1.0 ? 1 : int(nr);
    } else {
        const int k = sg.sk[s] & 63;
        const float E = sg.E[k];
        const float nhi = ceilf((cm + E) * sg.qhi[k]);
        if (nhi <= 1.f) return 1;
        const float nlo = ceilf((cm - E) * sg.qlo[k]);
        if (nlo != nhi) return 0;
        n = nhi > float(kMaxSubdiv) ? kMaxSubdiv + 1 : int(nhi);
    }
    if (n > kMaxSubdiv) {
        dev_fail(a.status, kDevSubdivLimit);
        n = kMaxSubdiv;
    }
    return n;
}

// The Eq. 2 counts of sample s that its single-precision bound left open
// (sg.fix[i][lane] == -1), redone in double precision into sg.fix.  Out of
// line and outside the elimination loop, which it interrupts only for such a
// sample: a call inside the loop would cost the loop its registers.
template <typename R, int NL>
__device__ __noinline__ void resolve_n_inter(Stage<R, NL> &sg, const DevMesh &m, const DevLines &Ln,
                                             const SolveArgs &a, int sign, int s, int32_t bin0, int32_t bin1) {
    const int lane = threadIdx.x & 31;
    const int sk = sg.sk[s], k = sk & 63, j = sk >> 6;
#pragma unroll 1
    for (int i = 0; i < 2; ++i) {
        if (sg.fix[i][lane] >= 0) continue;
        const int32_t b = i == 0 ? bin0 : bin1;
        int n = redo_n_inter(m, Ln, sg.r, sg.vo, sg.o, double(sign), sg.id[k - 1], sg.id[k], sg.nv[k], j,
                             b < sg.NB ? b : sg.NB - 1, a.dtau_max);
        if (n > kMaxSubdiv) {
            dev_fail(a.status, kDevSubdivLimit);
            n = kMaxSubdiv;
        }
        sg.fix[i][lane] = n;
        atomicAdd(&sg.n_redo, 1u);
    }
    __syncwarp();
}

// One velocity sample (record v, index s of the round) for every bin of the
// lane: line optics, Eq. 2 sub-intervals with linear chi and eta, elimination
// rows.  When no bin of the warp can need sub-intervals (the common case) the
// rows run as straight-line code, so the bins' chains interleave.  Single
// precision tests "possibly more than one sub-interval" on the lane's running
// maximum of chi over its bins (cmax: the previous sample's, updated here)
// against the certified threshold; double precision per bin.  Returns false,
// with nothing changed, when a single-precision count is left open somewhere
// in the warp (sg.fix marks it); once it has been redone the sample is
// stepped again with `fixed` set, taking the counts from sg.fix.
template <typename R, int NL, int BPL, int ORD, typename P>
__device__ __forceinline__ bool sample_step(const R (&v)[Stage<R, NL>::kS], int s, bool fixed, Stage<R, NL> &sg,
                                            const SolveArgs &a, R &cmax, const Bin<R, NL> (&f)[BPL],
                                            const bool (&act)[BPL], Sweep<R, P> (&w)[BPL]) {
    const R dl = v[0], rdv = v[1], hq = v[4], thr = v[5];
    R chi_q[BPL], eta_q[BPL];
    if (sizeof(R) == 4 && NL == 1 && rdv < R(0)) {  // far wing of every bin: the continuum (as ex2 gives 0)
#pragma unroll
        for (int i = 0; i < BPL; ++i) {
            chi_q[i] = v[2];
            eta_q[i] = v[3];
        }
    } else {
#pragma unroll
        for (int i = 0; i < BPL; ++i) optics<R, NL>(dl, rdv, v[2], v[3], v + 6, f[i], chi_q[i], eta_q[i]);
    }
    bool go;  // no bin needs a split (n_inter = 1 for all)
    R cq = chi_q[0];
    if constexpr (sizeof(R) == 4) {
#pragma unroll
        for (int i = 1; i < BPL; ++i) cq = fmax(cq, chi_q[i]);
        // an infinite threshold (uniform: the warp's record) means no bin of the interval can split
        go = (NL == 1 && thr == R(INFINITY)) || !__any_sync(kFull, fmax(cmax, cq) > thr);
    } else {
        bool split = false;
#pragma unroll
        for (int i = 0; i < BPL; ++i) split |= fmax(w[i].chi, chi_q[i]) > thr;
        go = !__any_sync(kFull, split);
    }
    if (go) {
#pragma unroll
        for (int i = 0; i < BPL; ++i) {
            R Sq = R(0);
            if constexpr (ORD == 4) Sq = Ar<R>::src(eta_q[i], chi_q[i]);
            row<ORD>(w[i], w[i].chi, w[i].eta, P(hq) * (P(w[i].chi) + P(chi_q[i])), w[i].Sc, Sq);
            w[i].chi = chi_q[i];
            w[i].eta = eta_q[i];
            w[i].Sc = Sq;
        }
        cmax = cq;
        return true;
    }
    const int lane = threadIdx.x & 31;
    int nis[BPL];
    bool open = false;
#pragma unroll
    for (int i = 0; i < BPL; ++i) {
        const R cm = fmax(w[i].chi, chi_q[i]);
        int n = 1;
        if (cm > thr) {
            n = (fixed && sg.fix[i][lane] > 0) ? sg.fix[i][lane] : n_inter<R, NL>(cm, hq, s, sg, a);
            open |= n == 0;
        }
        nis[i] = n;
    }
    if constexpr (sizeof(R) == 4) {
        if (__any_sync(kFull, open)) {
#pragma unroll
            for (int i = 0; i < 2; ++i) sg.fix[i][lane] = (i < BPL && nis[i < BPL ? i : 0] == 0) ? -1 : 0;
            __syncwarp();
            return false;
        }
    }
#pragma unroll
    for (int i = 0; i < BPL; ++i) {
        const int ni = nis[i];
        const R rni = R(1) / R(ni);
        const R hh = hq * rni;
        const R c0 = w[i].chi, e0 = w[i].eta;
        const R dchi = (chi_q[i] - c0) * rni, deta = (eta_q[i] - e0) * rni;
        R cprev = c0, eprev = e0, Sprev = w[i].Sc;
#pragma unroll 1
        for (int k = 1; k < ni; ++k) {
            const R ck = c0 + dchi * R(k), ek = e0 + deta * R(k);
            R Sk = R(0);
            if constexpr (ORD == 4) Sk = Ar<R>::src(ek, ck);
            row<ORD>(w[i], cprev, eprev, P(hh) * (P(cprev) + P(ck)), Sprev, Sk);
            cprev = ck;
            eprev = ek;
            Sprev = Sk;
        }
        R Sq = R(0);
        if constexpr (ORD == 4) Sq = Ar<R>::src(eta_q[i], chi_q[i]);
        row<ORD>(w[i], cprev, eprev, P(hh) * (P(cprev) + P(chi_q[i])), Sprev, Sq);
        w[i].chi = chi_q[i];
        w[i].eta = eta_q[i];
        w[i].Sc = Sq;
        if (act[i] && ni > 1) atomicAdd(&sg.n_extra, unsigned(ni - 1));
    }
    cmax = cq;
    return true;
}

// The lane's sweep state to and from shared memory (D Fh kept as one value,
// read back as Fh = D Fh, D = 1).
template <typename R, int BPL, int ORD, typename P>
__device__ __forceinline__ void put_sweep(Lane<R, ORD, P> &ln, const Sweep<R, P> (&w)[BPL], int lane) {
#pragma unroll
    for (int i = 0; i < BPL; ++i) {
        ln.wp[0][i][lane] = w[i].Dm * w[i].Fh;
        ln.wp[1][i][lane] = w[i].dtp;
        ln.wr[0][i][lane] = w[i].zh;
        ln.wr[1][i][lane] = w[i].chi;
        ln.wr[2][i][lane] = w[i].eta;
        if constexpr (ORD == 4) {
            ln.wr[3][i][lane] = w[i].Sp;
            ln.wr[4][i][lane] = w[i].Sc;
            ln.wr[5][i][lane] = w[i].hp;
        }
    }
}

template <typename R, int BPL, int ORD, typename P>
__device__ __forceinline__ void get_sweep(const Lane<R, ORD, P> &ln, Sweep<R, P> (&w)[BPL], int lane) {
#pragma unroll
    for (int i = 0; i < BPL; ++i) {
        w[i].Fh = ln.wp[0][i][lane];
        w[i].Dm = P(1);
        w[i].dtp = ln.wp[1][i][lane];
        w[i].zh = ln.wr[0][i][lane];
        w[i].chi = ln.wr[1][i][lane];
        w[i].eta = ln.wr[2][i][lane];
        if constexpr (ORD == 4) {
            w[i].Sp = ln.wr[3][i][lane];
            w[i].Sc = ln.wr[4][i][lane];
            w[i].hp = ln.wr[5][i][lane];
            // the reciprocal of the last increment, formed again as the row formed it
            w[i].rh = w[i].hp < R(0) ? R(0) : Ar<R>::rcp(w[i].hp);
        } else {
            w[i].Sp = w[i].Sc = w[i].hp = w[i].rh = R(0);
        }
    }
}

template <typename R, int NL, int BPL>
__device__ __forceinline__ void get_bins(const Stage<R, NL> &sg, Bin<R, NL> (&f)[BPL], bool (&act)[BPL], int lane) {
#pragma unroll
    for (int i = 0; i < BPL; ++i) {
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            f[i].A[l] = sg.fA[l][i][lane];
            f[i].B[l] = sg.fB[l][i][lane];
        }
        act[i] = lane_bin<BPL>(sg, i, lane) < sg.NB;
    }
}

// Eliminate the samples of a staged chunk from sample `pos` on, generating the
// records kCap at a time (the round holding `pos` is already generated unless
// `fresh`).  The lane's state comes from and goes back to shared memory, so
// the registers hold it only here.  Returns the first sample not stepped
// (total when the chunk is done; else a sample whose single-precision Eq. 2
// count was left open, whose record round stays in place).  Kept out of line
// (one call per chunk): its loop then gets a register allocation of its own,
// unaffected by the calls of the code around it.  pend: a sample whose open
// counts have been redone into sg.fix (-1: none).
template <typename R, int NL, int BPL, int ORD, typename P>
__device__ __noinline__ int consume_chunk(Stage<R, NL> &sg, Lane<R, ORD, P> &ln, const SolveArgs &a, int total,
                                          int nch, int sign, int pos, int pend, bool fresh) {
    constexpr int kS = Stage<R, NL>::kS, kCap = Stage<R, NL>::kCap;
    const int lane = threadIdx.x & 31;
    Sweep<R, P> w[BPL];
    Bin<R, NL> f[BPL];
    bool act[BPL];
    get_sweep<R, BPL, ORD, P>(ln, w, lane);
    get_bins<R, NL, BPL>(sg, f, act, lane);
    R cmax = ln.cm[lane];
    int r0 = pos / kCap * kCap, s = pos - r0;
#pragma unroll 1
    for (; r0 < total; r0 += kCap, s = 0, fresh = true) {
        const int nr = total - r0 < kCap ? total - r0 : kCap;
        if (fresh) {
#pragma unroll 1
            for (int q = lane; q < nr; q += 32) gen_sample<R, NL>(sg, r0 + q, q, nch, sign, a.dtau_max);
            __syncwarp();
        }
#pragma unroll 2
        for (; s < nr; ++s) {
            R v[kS];
            load_rec<R, NL>(sg.rec + s * kS, v);
            if (!sample_step<R, NL, BPL, ORD, P>(v, s, r0 + s == pend, sg, a, cmax, f, act, w)) break;
        }
        if (s < nr) break;
        __syncwarp();
    }
    put_sweep<R, BPL, ORD, P>(ln, w, lane);
    ln.cm[lane] = cmax;
    __syncwarp();
    return r0 < total ? r0 + s : total;
}

// Copy the point data of slot `from` into slot 0 (the next chunk's farther point).
template <typename R, int NL>
__device__ __forceinline__ void carry_slot(Stage<R, NL> &sg, int from) {
    sg.d[0] = sg.d[from];
    sg.w[0] = sg.w[from];
    sg.cc[0] = sg.cc[from];
    sg.ec[0] = sg.ec[from];
#pragma unroll
    for (int c = 0; c < 2 * NL; ++c) sg.ce[c][0] = sg.ce[c][from];
    if constexpr (sizeof(R) == 8) sg.z[0] = sg.z[from];  // single precision: carried by stage_chunk
    sg.id[0] = sg.id[from];
}

// Stage the chunk of points qb .. qb+nch-1 of the half (slot 0 already holds
// the point farther than the chunk): points, intervals, and the offsets of
// their velocity samples.  Returns the chunk's number of samples.  Called once
// per 32 points and kept out of line, so that its double-precision and bound
// arithmetic does not add to the registers of the elimination loop.
template <typename R, int NL>
__device__ __noinline__ int stage_chunk(const DevMesh &m, const DevLines &Ln, const SolveArgs &a, Stage<R, NL> &sg,
                                        int32_t qb, int32_t cnt, int sign) {
    const int lane = threadIdx.x & 31;
    const int32_t npt = cnt + 1;
    const int nch = npt - qb < 32 ? int(npt - qb) : 32;
    const int slot = lane + 1;
    const int32_t q = qb + lane;
    double zq = 0.0;
    R deq = R(0);
    if (lane < nch) stage_point<R, NL>(m, Ln, sg, q, cnt, slot, sign, zq, deq);
    // the farther point's Z and delta bound: the previous lane's, or the carried point's for lane 0
    double zf = __shfl_up_sync(kFull, zq, 1);
    R def = __shfl_up_sync(kFull, deq, 1);
    if (lane == 0) {
        zf = sg.z[0];
        if constexpr (sizeof(R) == 4) def = sg.de0;
    }
    __syncwarp();
    if constexpr (sizeof(R) == 4) {
        if (lane == nch - 1) {  // the next chunk's farther point
            sg.z[0] = zq;
            sg.de0 = deq;
        }
    }
    int nvk = 0;  // the far end (q = 0) starts the line: no interval
    if (lane < nch && q > 0) nvk = stage_interval<R, NL>(m, Ln, a, sg, slot, sign, zf, zq, def, deq);
    int incl = nvk;
#pragma unroll
    for (int sh = 1; sh < 32; sh <<= 1) {
        const int t = __shfl_up_sync(kFull, incl, sh);
        if (lane >= sh) incl += t;
    }
    const int total = __shfl_sync(kFull, incl, 31);
    if (lane < nch) {
        sg.nv[slot] = nvk;
        sg.so[slot] = incl - nvk;
    }
    if (lane == 0) sg.n_smp += unsigned(total);
    __syncwarp();
    return total;
}

// Eliminate one half of a pair line (direction sign r) from its far end up to
// (excluding) the origin row.  Leaves the origin row's coupling (D Fh, zh)
// and the last optical-depth increment in the lane's sweep state.
template <typename R, int NL, int BPL, int ORD, typename P>
__device__ void half_sweep(const DevMesh &m, const DevLines &Ln, const SolveArgs &a, Stage<R, NL> &sg,
                           Lane<R, ORD, P> &ln, int sign) {
    constexpr int kCap = Stage<R, NL>::kCap;
    const int lane = threadIdx.x & 31;
    {
        Sweep<R, P> w[BPL];
#pragma unroll
        for (int i = 0; i < BPL; ++i) {
            w[i].Fh = P(1);
            w[i].Dm = P(1);
            w[i].zh = R(a.I_bdy);
            w[i].dtp = P(0);
            w[i].hp = R(-1);  // no row yet (Hermitian scheme)
            w[i].Sp = w[i].Sc = w[i].rh = w[i].chi = w[i].eta = R(0);
        }
        put_sweep<R, BPL, ORD, P>(ln, w, lane);
    }
    const int32_t cnt = sg.hl.cnt;
    __syncwarp();
    if (cnt == 0) return;
#pragma unroll 1
    for (int32_t qb = 0; qb <= cnt; qb += 32) {
        const int total = stage_chunk<R, NL>(m, Ln, a, sg, qb, cnt, sign);
        const int nch = cnt + 1 - qb < 32 ? int(cnt + 1 - qb) : 32;
        if (qb == 0) {  // the far end: its optics; its row follows with the first increment
            Bin<R, NL> f[BPL];
            bool act[BPL];
            get_bins<R, NL, BPL>(sg, f, act, lane);
            R ce[2 * NL];
#pragma unroll
            for (int c = 0; c < 2 * NL; ++c) ce[c] = sg.ce[c][1];
            const R rdv = Ar<R>::rcp(sg.w[1]);
            R cmax = R(0);
#pragma unroll
            for (int i = 0; i < BPL; ++i) {
                R chi, eta;
                optics<R, NL>(sg.d[1], rdv, sg.cc[1], sg.ec[1], ce, f[i], chi, eta);
                ln.wr[1][i][lane] = chi;
                ln.wr[2][i][lane] = eta;
                if constexpr (ORD == 4) ln.wr[4][i][lane] = Ar<R>::src(eta, chi);
                cmax = i == 0 ? chi : fmax(cmax, chi);
            }
            ln.cm[lane] = cmax;
            __syncwarp();
        }
        int pos = 0, pend = -1;
        bool fresh = true;
#pragma unroll 1
        for (;;) {
            pos = consume_chunk<R, NL, BPL, ORD, P>(sg, ln, a, total, nch, sign, pos, pend, fresh);
            if (pos >= total) break;
            resolve_n_inter<R, NL>(sg, m, Ln, a, sign, pos % kCap, lane_bin<BPL>(sg, 0, lane),
                                   lane_bin<BPL>(sg, BPL - 1, lane));
            pend = pos;
            fresh = false;
        }
        if (lane == 0) carry_slot<R, NL>(sg, nch);
        __syncwarp();
    }
}

// CTAs of 4 warps (2 in double precision, whose per-warp stage is twice as
// large); the minimum resident CTAs per SM caps the registers
// (65536 / (threads x CTAs)).  One line, second order: 9 CTAs (56 registers;
// the shared staging of 9 CTAs, 24.5 KB each plus 1 KB reserved, fits 228 KB),
// measured 4 % faster than 8 and 10 % faster than 7 on GB300 (the Hermitian
// scheme: 3 % faster than 8).  Two lines: 8 CTAs (64 registers; 18 % faster
// than 4 on the clump octree); three and four: 6 (80 registers; 11 % faster
// than 4 on a four-line wind).
template <typename R, int NL, int BPL, typename P = R>
struct Occ {
    static constexpr int kWarps = sizeof(R) == 8 ? 2 : 4;
    static constexpr int kThreads = 32 * kWarps;
    static constexpr int kMinBlocks =
        sizeof(R) == 8 ? 1
        : sizeof(P) == 8 ? (NL == 1 ? 4 : 2)
        : (NL == 1 ? 9 : NL == 2 ? 8 : NL <= 4 ? 6 : 3);
};

// J of origin a.o_begin + oc for the bins of frequency tile `tile`, by one warp.
template <typename R, int NL, int BPL, int ORD, typename P>
__device__ __forceinline__ void solve_item(const DevMesh &m, const DevLines &Ln, const DevRays &Rs,
                                           const SolveArgs &a, int32_t oc, int32_t tile, Stage<R, NL> &sg,
                                           Lane<R, ORD, P> &ln, int lane) {
    static_assert(BPL <= 2, "the shared per-lane state holds two bins");
    const int32_t o = a.o_begin + oc;
    const int32_t L = Ln.L, F = Ln.F, NB = L * F;
    const double dvo = Ln.dvw[o];
    if (lane == 0) {
        sg.o = o;
        sg.NB = NB;
        sg.tile = tile;
        sg.xo[0] = m.x[o];
        sg.xo[1] = m.y[o];
        sg.xo[2] = m.z[o];
        sg.vo[0] = m.vx[o];
        sg.vo[1] = m.vy[o];
        sg.vo[2] = m.vz[o];
        sg.vor[0] = Pts<R>::vx(m)[o];
        sg.vor[1] = Pts<R>::vy(m)[o];
        sg.vor[2] = Pts<R>::vz(m)[o];
        sg.n_smp = sg.n_extra = sg.n_redo = 0u;
    }
    // the origin's own optics give S_o
    R oce[2 * NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        oce[2 * l] = l < L ? __ldg(Pts<R>::chi0(Ln) + int64_t(o) * L + l) : R(0);
        oce[2 * l + 1] = l < L ? __ldg(Pts<R>::eta0(Ln) + int64_t(o) * L + l) : R(0);
    }
    const R rdvo = Ar<R>::rcp(__ldg(Pts<R>::dvw(Ln) + o));

    // frequency of each bin of this lane and its profile constants
    float am[NL], bm[NL];
    R So_[BPL];  // the source function at the origin of each bin
#pragma unroll
    for (int l = 0; l < NL; ++l) am[l] = bm[l] = 0.f;
#pragma unroll
    for (int i = 0; i < BPL; ++i) {
        const int32_t b = tile * 32 * BPL + lane + 32 * i;
        const int32_t bb = b < NB ? b : NB - 1;
        const int32_t l = bb / F, k = bb % F;
        const double x = (F == 1) ? 0.0 : -Ln.x_span + 2.0 * Ln.x_span * double(k) / double(F - 1);
        const double ub = x * dvo;
        Bin<R, NL> f;
#pragma unroll
        for (int lp = 0; lp < NL; ++lp) {
            const double r = (lp < L) ? Ln.ratio[l * MGX_MAX_LINES + lp] : 1.0;
            f.A[lp] = R((kC * (r - 1.0) + r * ub) * Ar<R>::kArgScale);
            f.B[lp] = R(r * (1.0 + ub / kC) * Ar<R>::kArgScale);
            sg.fA[lp][i][lane] = f.A[lp];
            sg.fB[lp][i][lane] = f.B[lp];
            am[lp] = fmaxf(am[lp], fabsf(float(f.A[lp])));
            bm[lp] = fmaxf(bm[lp], fabsf(float(f.B[lp])));
        }
        R chi_o, eta_o;
        optics<R, NL>(R(0), rdvo, __ldg(Pts<R>::chic(Ln) + o), __ldg(Pts<R>::etac(Ln) + o), oce, f, chi_o, eta_o);
        So_[i] = eta_o / chi_o;
    }
    if constexpr (sizeof(R) == 4 && NL == 1) {
        // the profile constants of the tile's first and last bin (the far-wing test of gen_sample)
        __syncwarp();
        if (lane == 0) {
            const int32_t jl = (NB - 1 - tile * 32 * BPL) < 32 * BPL - 1 ? NB - 1 - tile * 32 * BPL : 32 * BPL - 1;
            sg.wa[0] = sg.fA[0][0][0];
            sg.wb[0] = sg.fB[0][0][0];
            sg.wa[1] = sg.fA[0][jl / 32][jl % 32];
            sg.wb[1] = sg.fB[0][jl / 32][jl % 32];
            sg.wing = L == 1;
        }
    }
    if constexpr (sizeof(R) == 4) {
        // largest |A|, |B| of each line over the warp's bins (the opacity bound of Eq. 2)
#pragma unroll
        for (int lp = 0; lp < NL; ++lp) {
#pragma unroll
            for (int sh = 16; sh > 0; sh >>= 1) {
                am[lp] = fmaxf(am[lp], __shfl_xor_sync(kFull, am[lp], sh));
                bm[lp] = fmaxf(bm[lp], __shfl_xor_sync(kFull, bm[lp], sh));
            }
            if (lane == 0) {
                sg.Am[lp] = am[lp];
                sg.Bm[lp] = bm[lp];
            }
        }
    }

    const int64_t h0 = int64_t(oc) * Rs.npairs * 2;
    double js[BPL], jc[BPL];  // each bin's J: Neumaier sum and compensation
    P cpD[BPL], cpT[BPL];     // the backward half's coupling to the origin row: D Fh, dtb / 2,
    R cpZ[BPL], cpH[BPL], cpS[BPL];  // zh (Hermitian: + the last increment and S)
#pragma unroll
    for (int i = 0; i < BPL; ++i) js[i] = jc[i] = 0.0;
#pragma unroll 1
    for (int32_t p = 0; p < Rs.npairs; ++p) {
        const uint32_t ray = __ldg(Rs.rays + int64_t(o) * Rs.npairs + p);
        const int lev = int(ray >> 28);
        const int64_t hb = h0 + 2 * int64_t(p);
        if (lane < 3) sg.r[lane] = Rs.dir[3 * (level_offset(lev) + (ray & 0x0FFFFFFFu)) + lane];
        if (lane == 0) sg.hl = half_list(a, hb);
        __syncwarp();
        half_sweep<R, NL, BPL, ORD, P>(m, Ln, a, sg, ln, -1);
#pragma unroll
        for (int i = 0; i < BPL; ++i) {  // the backward half's coupling to the origin row
            cpD[i] = ln.wp[0][i][lane];  // D Fh
            cpT[i] = ln.wp[1][i][lane];  // dtb / 2
            cpZ[i] = ln.wr[0][i][lane];  // zh
            if constexpr (ORD == 4) {
                cpH[i] = ln.wr[5][i][lane];  // hp
                cpS[i] = ln.wr[3][i][lane];  // Sp
            }
        }
        if (lane == 0) sg.hl = half_list(a, hb + 1);
        __syncwarp();
        half_sweep<R, NL, BPL, ORD, P>(m, Ln, a, sg, ln, 1);
        const double w2 = a.w2[lev];
        Sweep<R, P> wf[BPL];
        get_sweep<R, BPL, ORD, P>(ln, wf, lane);
#pragma unroll
        for (int i = 0; i < BPL; ++i) {
            Sweep<R, P> wb;
            wb.Fh = cpD[i];
            wb.Dm = P(1);
            wb.dtp = cpT[i];
            wb.zh = cpZ[i];
            if constexpr (ORD == 4) {
                wb.hp = cpH[i];
                wb.Sp = cpS[i];
                wb.rh = wb.hp < R(0) ? R(0) : Ar<R>::rcp(wb.hp);
            }
            const R So = So_[i];
            const R u = ORD == 4 ? origin_u4(wb, wf[i], So, R(a.I_bdy)) : origin_u2(wb, wf[i], So);
            const int32_t b = lane_bin<BPL>(sg, i, lane);
            if (a.u_out && b < NB) a.u_out[(int64_t(oc) * Rs.npairs + p) * NB + b] = double(u);
            const double xv = w2 * double(u);
            const double sum = js[i];
            const double t = sum + xv;  // Neumaier compensated sum
            if (fabs(sum) >= fabs(xv)) jc[i] += (sum - t) + xv;
            else jc[i] += (xv - t) + sum;
            js[i] = t;
        }
        __syncwarp();
    }
    unsigned n_act = 0;
#pragma unroll
    for (int i = 0; i < BPL; ++i) {
        const int32_t b = lane_bin<BPL>(sg, i, lane);
        if (b < NB) {
            a.J[int64_t(o) * NB + b] = js[i] + jc[i];
            ++n_act;
        }
    }
    if (a.counters) {
        // [0]: sub-intervals beyond one per sample (active bins); [1]: samples x active bins;
        // [4]: integer decisions redone in double precision
        unsigned long long na = n_act;
#pragma unroll
        for (int sh = 16; sh > 0; sh >>= 1) na += __shfl_down_sync(kFull, na, sh);
        __syncwarp();
        if (lane == 0) {
            atomicAdd(a.counters, (unsigned long long)sg.n_extra);
            atomicAdd(a.counters + 1, (unsigned long long)sg.n_smp * na);
            atomicAdd(a.counters + 4, (unsigned long long)sg.n_redo);
        }
    }
}

// Grid-mapped launch: warp w of the grid solves item w = oc * n_tiles + tile.
template <typename R, int NL, int BPL, int ORD, typename P>
__global__ void __launch_bounds__(Occ<R, NL, BPL, P>::kThreads, (Occ<R, NL, BPL, P>::kMinBlocks))
k_solve(const __grid_constant__ DevMesh m, const __grid_constant__ DevLines Ln, const __grid_constant__ DevRays Rs,
        const __grid_constant__ SolveArgs a) {
    __shared__ Stage<R, NL> stage[Occ<R, NL, BPL, P>::kWarps];  // one per warp
    __shared__ Lane<R, ORD, P> lanes[Occ<R, NL, BPL, P>::kWarps];
    const int lane = threadIdx.x & 31;
    const int64_t item = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
    const int64_t n_items = int64_t(a.o_end - a.o_begin) * a.n_tiles;
    if (item >= n_items) return;
    solve_item<R, NL, BPL, ORD, P>(m, Ln, Rs, a, int32_t(item / a.n_tiles), int32_t(item % a.n_tiles),
                                stage[threadIdx.x >> 5], lanes[threadIdx.x >> 5], lane);
}

// Persistent launch over a work list of (model, origin, tile) items of many
// models: each warp takes the next item from a global counter until the list
// is exhausted.
template <typename R, int NL, int BPL, int ORD, typename P>
__global__ void __launch_bounds__(Occ<R, NL, BPL, P>::kThreads, (Occ<R, NL, BPL, P>::kMinBlocks))
k_solve_queue(const BatchSlot *__restrict__ slots, const uint2 *__restrict__ work, int64_t n_work,
              unsigned long long *__restrict__ next) {
    __shared__ Stage<R, NL> stage[Occ<R, NL, BPL, P>::kWarps];
    __shared__ Lane<R, ORD, P> lanes[Occ<R, NL, BPL, P>::kWarps];
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(next, 1ull);
        it = __shfl_sync(kFull, it, 0);
        if (it >= (unsigned long long)n_work) return;
        const uint2 w = work[it];  // x = model << 16 | tile, y = origin
        const BatchSlot &s = slots[w.x >> 16];
        solve_item<R, NL, BPL, ORD, P>(s.m, s.Ln, s.R, s.a, int32_t(w.y), int32_t(w.x & 0xffffu), stage[threadIdx.x >> 5],
                                    lanes[threadIdx.x >> 5], lane);
        __syncwarp();
    }
}

// Prefer the largest shared-memory carveout for a solve kernel (its resident
// CTAs are bounded by their per-warp staging), once per kernel and process.
template <typename K>
void prefer_shared(K kernel) {
    static bool done = false;
    if (!done) {
        cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        done = true;
    }
}

template <typename R, int BPL, int ORD, typename P = R>
void launch_RB(const DevMesh &m, const DevLines &Ln, const DevRays &R_, const SolveArgs &a, cudaStream_t st) {
    const int64_t n_items = int64_t(a.o_end - a.o_begin) * a.n_tiles;
    if (n_items == 0) return;
    constexpr int tb = Occ<R, 1, BPL, P>::kThreads;
    const unsigned grid = unsigned((n_items * 32 + tb - 1) / tb);
    if (Ln.L <= 1) {
        prefer_shared(k_solve<R, 1, BPL, ORD, P>);
        k_solve<R, 1, BPL, ORD, P><<<grid, tb, 0, st>>>(m, Ln, R_, a);
    } else if (Ln.L <= 2) {
        prefer_shared(k_solve<R, 2, BPL, ORD, P>);
        k_solve<R, 2, BPL, ORD, P><<<grid, tb, 0, st>>>(m, Ln, R_, a);
    } else if (Ln.L <= 4) {
        prefer_shared(k_solve<R, 4, BPL, ORD, P>);
        k_solve<R, 4, BPL, ORD, P><<<grid, tb, 0, st>>>(m, Ln, R_, a);
    } else {
        prefer_shared(k_solve<R, 8, BPL, ORD, P>);
        k_solve<R, 8, BPL, ORD, P><<<grid, tb, 0, st>>>(m, Ln, R_, a);
    }
}

template <typename R, int BPL, int NL, int ORD, typename P = R>
void launch_queue_NL(const BatchSlot *slots, const uint2 *work, int64_t n_work, unsigned long long *next,
                     cudaStream_t st) {
    int dev = 0, sms = 152, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    constexpr int tb = Occ<R, NL, BPL, P>::kThreads, nw = Occ<R, NL, BPL, P>::kWarps;
    prefer_shared(k_solve_queue<R, NL, BPL, ORD, P>);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve_queue<R, NL, BPL, ORD, P>, tb, 0);
    if (per_sm < 1) per_sm = 1;
    int64_t grid = int64_t(sms) * per_sm;
    const int64_t need = (n_work + nw - 1) / nw;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    k_solve_queue<R, NL, BPL, ORD, P><<<unsigned(grid), tb, 0, st>>>(slots, work, n_work, next);
}

template <typename R, int BPL, int ORD, typename P = R>
void launch_queue_RB(int max_lines, const BatchSlot *slots, const uint2 *work, int64_t n_work,
                     unsigned long long *next, cudaStream_t st) {
    if (max_lines <= 1) launch_queue_NL<R, BPL, 1, ORD, P>(slots, work, n_work, next, st);
    else if (max_lines <= 2) launch_queue_NL<R, BPL, 2, ORD, P>(slots, work, n_work, next, st);
    else if (max_lines <= 4) launch_queue_NL<R, BPL, 4, ORD, P>(slots, work, n_work, next, st);
    else launch_queue_NL<R, BPL, 8, ORD, P>(slots, work, n_work, next, st);
}

}  // namespace

template <int ORD>
void launch_solve_ord(const DevMesh &m, const DevLines &Ln, const DevRays &R, const SolveArgs &a, int precision,
                      cudaStream_t st) {
    const int bpl = solve_bins_per_lane(precision, Ln.L * Ln.F);
    if (precision == MGX_FP64) launch_RB<double, 1, ORD>(m, Ln, R, a, st);
    else if (precision == MGX_FP32_DT64) launch_solve_dt64(m, Ln, R, a, bpl, st);
    else if (bpl == 2) launch_RB<float, 2, ORD>(m, Ln, R, a, st);
    else launch_RB<float, 1, ORD>(m, Ln, R, a, st);
}

template <int ORD>
void launch_solve_queue_ord(int precision, int bins_per_lane, int max_lines, const BatchSlot *slots,
                            const uint2 *work, int64_t n_work, unsigned long long *next, cudaStream_t st) {
    if (n_work == 0) return;
    if (precision == MGX_FP64) launch_queue_RB<double, 1, ORD>(max_lines, slots, work, n_work, next, st);
    else if (precision == MGX_FP32_DT64)
        launch_solve_queue_dt64(bins_per_lane, max_lines, slots, work, n_work, next, st);
    else if (bins_per_lane == 2) launch_queue_RB<float, 2, ORD>(max_lines, slots, work, n_work, next, st);
    else launch_queue_RB<float, 1, ORD>(max_lines, slots, work, n_work, next, st);
}

}  // namespace mgx
