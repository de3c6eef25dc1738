// k_trace.cu -- long-characteristic tracer (Section 2.1, Fig. 2).
//
// One thread per half-ray.  From the current point c the next point is the
// neighbour of c that lies strictly further along the ray (Z_n > Z_c with
// Z = (x_n - x_o).d) and closest to it (smallest q = |(x_n - x_o) - Z d|^2),
// ties to the smaller index; the half-ray ends when c has no such neighbour.
// The decisions are those of the double-precision definition, with every
// product and sum explicitly rounded in a fixed order, so the traced point
// lists and distances are bit-reproducible.
//
// GB300 executes double precision at a small fraction of its single-precision
// rate, so each step first screens the neighbours in single precision: each
// CSR edge carries the difference of the float-rounded positions of its
// neighbour and its own point, Delta32 = fl(x_n32 - x_c32), next to the
// neighbour's id; the records are read two at a time (one 32-byte load per
// lane, which halves the load instructions of the walk).  The screen
// works relative to the current point c rather than to the origin: with
// Delta = x_n - x_c, the increment Z_n - Z_c = Delta.d and the lateral offset
// e_n = e_c + Delta - (Delta.d) d (q_n = |e_n|^2) involve only differences of
// neighbouring points, so their rounding scales with the spacing of the mesh
// and the positions' own rounding, not with the distance from the origin.  The
// walk carries e_c in float with a rigorous bound on its error; each quantity
// gets such a bound (from the unit roundoff u = 2^-24; see step_screen).
// A neighbour is surely (not) forward when Delta.d clears its bound; the step
// is decided in single precision when one surely forward neighbour's interval
// [q32 - eq, q32 + eq] lies strictly below the intervals of every other
// candidate.  Otherwise (near-ties, exact ties of lattice meshes, ambiguous
// forward tests) the step is redone exactly in double precision.
//
// An undecided step is decided by the whole warp at once (step_exact_warp):
// every neighbour of the current point is evaluated in double precision, one
// per lane, and a warp reduction applies the defining rule.  Lanes wait for
// one another only at these steps, and for a few tens of cycles rather than a
// serial double-precision pass over the neighbour list.
//
// The fast path carries the winner's lateral offset and position into the
// next step, so it executes no double-precision operation at all; exact values
// are formed only on undecided steps, when a tail walk resumes (its lateral
// offset), and for the inspection output of mgx_trace.
//
// The walk serves three layouts of the traced lists (the solver re-forms each
// point's exact Z from its position, so only point ids are stored):
//   * packed: a count pass stores the half-ray lengths, which are prefix-summed
//     into arena offsets, and an emit pass writes the ids at those offsets;
//   * padded (batched solves): one pass writes the first `pad` ids of each
//     half-ray into a fixed-width row h * pad, stores the full length and its
//     excess over the row, and for a half-ray longer than the row the walk's
//     state after its pad-th point; a tail pass resumes those walks from
//     their states and writes the remaining ids into a packed overflow arena
//     at the prefix sums of the excesses.  Every step is walked once by the
//     padded pass and the tail steps once more, so the lists cost about one
//     walk instead of two.
#include "mgx_internal.cuh"

namespace mgx {

namespace {

constexpr float kU = 5.9604644775390625e-8f;  // 2^-24

struct Step {
    int32_t next;  // -1: the half-ray ends
    double Z;
};

__device__ __forceinline__ double exact_Z(const DevMesh &m, int32_t c, double xo, double yo, double zo, double d0,
                                          double d1, double d2) {
    const double dx = __dsub_rn(__ldg(m.x + c), xo);
    const double dy = __dsub_rn(__ldg(m.y + c), yo);
    const double dz = __dsub_rn(__ldg(m.z + c), zo);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, d0), __dmul_rn(dy, d1)), __dmul_rn(dz, d2));
}

// State of one lane's current walk (the half-ray index h is the walking
// loop's own variable).  It holds the direction in float only (the rounded
// table entry, negated for a backward half, which equals the rounded
// negation); the origin and the double direction are formed again from h on
// the rare steps that need them, so the walk keeps few registers and setting
// it up executes no double-precision operation.
struct Walk {
    int64_t w;                // write base of the entries (not kept by the padded pass: h * pad)
    float f0, f1, f2;         // direction (float)
    float ecx, ecy, ecz, eec; // lateral offset of the current point from the ray (float) and its bound
    int32_t c, k, expect;
};


// Single-precision screen of one step over the neighbour records of c (the
// difference Delta32 of the float positions, neighbour minus c, stored next to
// the neighbour's id, read in aligned pairs; the mesh stores one spare record
// after the last so that a pair never leaves the array).  hc is c's float
// position, loaded with c's largest neighbour distance; the walk holds (ecx, ecy, ecz)
// approximating c's lateral offset e_c = (x_c - x_o) - Z_c d componentwise
// within eec, and the direction f rounded to float.  Bounds, with a_i = |hn_i| + |hc_i|,
// S = |Delta32|_1, X = |hn|_1 + |hc|_1 <= 2 Xc + 1.01 S (Xc = |hc|_1) and
// E1 = |e32|_1 (positions round to float within u |x|, d to f within u |d|):
//   |Delta32_i - Delta_i| <= u (|Delta32_i| + a_i) (1 + 2u)
//   |dZ32 - dZ| <= 5.01u S + 1.01u X <= 6.04u S + 2.02u Xc       (used: 8u S + 4u Xc)
//   |e32_i - e_i| <= eec + 1.01 |dZ32 - dZ| + 1.01u (4.1 S + X + E1)
//                 <= eec + u (13.4 S + 6.2 Xc + 1.01 E1)   (used: de = eec + u (15 S + 8 Xc + 2 E1))
//   |q32 - q| <= 2 E1 de + 3 de^2 + 3.01u q32     (used: 2.02 E1 de + 3.03 de^2 + 6u q32,
//                                                  the margin covering the rounding of the bounds)
// The definition's own double rounding adds at most g0 to a Z difference
// (16 u64 max|x|_1 against g0 = 32 u^2 max|x|_1) and g0 (E1 + de) + g0^2 to q
// (16.2 u64 |x_n - x_o|_1 |e|_1 + 3.01 u64 q + 197 u64^2 |x_n - x_o|_1^2).
// In the loop the S-dependent parts of edZ and de take the largest S over the
// point's neighbours (stored with the mesh), so that per neighbour only dZ, e,
// |e|_1, q and eq are formed, and only the two smallest lower bounds and the
// leader's record are kept; the leader's upper bound and forward test, and the
// winner's own de for the next step, are formed again from its record.
// Returns the next point (-1: the half-ray ends; -2: undecided); when it
// decides a next point it moves the walk's lateral offset to it.
__device__ __forceinline__ int32_t step_screen(const DevMesh &m, Walk &wk) {
    const int32_t c = wk.c;
    // hc: c's float position (only Xc = |hc|_1 enters the bounds) and its largest neighbour distance
    const float4 pc = m.phi[c];
    const float hcw = fabsf(pc.x) + fabsf(pc.y) + fabsf(pc.z);
    const float f0 = wk.f0, f1 = wk.f1, f2 = wk.f2, ecx = wk.ecx, ecy = wk.ecy, ecz = wk.ecz, eec = wk.eec;
    int32_t be = -1;  // record of the candidate with the smallest lower bound (-1: none yet)
    float lo1 = INFINITY, lo2 = INFINITY;  // the smallest lower bound, and the smallest of the others
    const float g02 = m.g0 * m.g0;
    const int32_t e1 = m.off[c + 1];
    // the screen of neighbour record e (the same arithmetic for the loop and the winner)
    const float bz = fmaf(4.0f * kU, hcw, m.g0), be0 = fmaf(8.0f * kU, hcw, eec);
    // bounds shared by every neighbour of c, from Smax = max_n S (the mesh
    // stores it in phi[c].w, formed as S is below): edZ <= edZs, and de <= des
    // through |e|_1 <= E1max (|w|_1 <= S (1 + |f|_1) <= 2.74 S), each raised by
    // 16u for its own rounding; the q-interval keeps each neighbour's own |e|_1
    const float smax = pc.w;
    const float edZs = fmaf(8.0f * kU, smax, bz) * (1.0f + 16.0f * kU);
    const float E1max = (fabsf(ecx) + fabsf(ecy) + fabsf(ecz) + 2.74f * smax) * (1.0f + 16.0f * kU);
    const float des = fmaf(15.0f * kU, smax, fmaf(2.0f * kU, E1max, be0)) * (1.0f + 16.0f * kU);
    // eq = (2.02 E1 + 3.03 de) de + 6u q + g0 (E1 + de) + g0^2 regrouped around E1 and q
    const float k1 = fmaf(2.02f, des, m.g0), k0 = fmaf(fmaf(3.03f, des, m.g0), des, g02);
    auto screen = [&](const float4 &rec, float &dZ, float &edZ, float &ex, float &ey, float &ez, float &S) {
        const float dx = rec.x, dy = rec.y, dz = rec.z;  // the record holds x_n - x_c in float
        S = fabsf(dx) + fabsf(dy) + fabsf(dz);
        dZ = fmaf(dz, f2, fmaf(dy, f1, dx * f0));
        edZ = fmaf(8.0f * kU, S, bz);
        ex = ecx + fmaf(-dZ, f0, dx);
        ey = ecy + fmaf(-dZ, f1, dy);
        ez = ecz + fmaf(-dZ, f2, dz);
    };
    auto bound = [&](float S, float E1) { return fmaf(15.0f * kU, S, fmaf(2.0f * kU, E1, be0)); };
    // the neighbour records two at a time (one 32-byte load per lane; the records
    // before off[c] and from off[c + 1] on in a pair take no part)
    auto consider = [&](const float4 &rec, int32_t e, bool valid) {
        const float dx = rec.x, dy = rec.y, dz = rec.z;  // the record holds x_n - x_c in float
        const float dZ = fmaf(dz, f2, fmaf(dy, f1, dx * f0));
        const float ex = ecx + fmaf(-dZ, f0, dx), ey = ecy + fmaf(-dZ, f1, dy), ez = ecz + fmaf(-dZ, f2, dz);
        const float q = fmaf(ez, ez, fmaf(ey, ey, ex * ex));
        const float E1 = fabsf(ex) + fabsf(ey) + fabsf(ez);
        const float eq = fmaf(k1, E1, fmaf(6.0f * kU, q, k0));
        // surely not forward, or not a neighbour of c: no part in the decision
        const float lo = (valid && !(dZ < -edZs)) ? q - eq : INFINITY;
        // the candidate with the smallest lower bound decides the step when it is surely
        // forward and its whole interval lies below every other candidate's (ascending
        // record order, as one record at a time would take them); its upper bound and
        // forward test are formed again from its record after the loop
        const bool lead = lo < lo1;
        lo2 = lead ? lo1 : fminf(lo2, lo);
        lo1 = lead ? lo : lo1;
        be = lead ? e : be;
    };
    const int32_t eb = m.off[c];
    for (int32_t e = eb & ~1; e < e1; e += 2) {
        float4 ra, rb;  // records e and e + 1: one 256-bit read-only load (32-byte aligned, e even)
        asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
            : "=f"(ra.x), "=f"(ra.y), "=f"(ra.z), "=f"(ra.w), "=f"(rb.x), "=f"(rb.y), "=f"(rb.z), "=f"(rb.w)
            : "l"(m.nrec + e));
        consider(ra, e, e >= eb);
        consider(rb, e + 1, e + 1 < e1);
    }
    if (be < 0) return -1;  // no neighbour can be forward: the half-ray ends
    // the leading candidate's interval and forward test, formed again from its record
    // with the loop's arithmetic (so bit for bit the loop's values)
    const float4 rec = __ldg(m.nrec + be);
    float dZ, edZ, ex, ey, ez, S;
    screen(rec, dZ, edZ, ex, ey, ez, S);
    const float q = fmaf(ez, ez, fmaf(ey, ey, ex * ex));
    const float E1 = fabsf(ex) + fabsf(ey) + fabsf(ez);
    const float hi1 = q + fmaf(k1, E1, fmaf(6.0f * kU, q, k0));
    if (!(dZ > edZs) || !(hi1 < lo2)) return -2;
    const int32_t best = __float_as_int(rec.w);
    // the winner's offset and bound for the next step
    wk.eec = bound(S, E1) * (1.0f + 8.0f * kU);  // with the rounding of the bound itself
    wk.ecx = ex;
    wk.ecy = ey;
    wk.ecz = ez;
    return best;
}

// Origin of half-ray h (two halves per pair, npairs pairs per origin).
__device__ __forceinline__ int32_t walk_origin(const DevRays &R, int32_t o_begin, int64_t h) {
    const int64_t pr = h >> 1;  // pair index from o_begin's first pair
    // a 32-bit division whenever the index fits (always, short of 2^32 pairs in one call)
    return o_begin + (pr < (int64_t(1) << 32) ? int32_t(uint32_t(pr) / uint32_t(R.npairs)) : int32_t(pr / R.npairs));
}

// Table index of half-ray h's pair direction.
__device__ __forceinline__ int32_t walk_pix(const DevRays &R, int32_t o_begin, int64_t h) {
    // the rays of origin o_begin + pr / npairs, entry pr % npairs: entry pr from o_begin's row
    const uint32_t ray = R.rays[int64_t(o_begin) * R.npairs + (h >> 1)];
    return int32_t(level_offset(int(ray >> 28)) + (ray & 0x0FFFFFFFu));
}

// The double direction of half-ray h (a backward half, h even, negated).
__device__ __forceinline__ void walk_dir(const DevRays &R, int32_t o_begin, int64_t h, double &d0, double &d1,
                                         double &d2) {
    const double *r = R.dir + 3 * int64_t(walk_pix(R, o_begin, h));
    const bool back = (h & 1) == 0;
    d0 = back ? -r[0] : r[0];
    d1 = back ? -r[1] : r[1];
    d2 = back ? -r[2] : r[2];
}

// Half-ray of launch position h.  The counting pass (MODE 0) given a stride
// > 1 (the `pad` argument, unused otherwise by that pass) counts a planning
// sample: every stride-th origin from o_begin, position h standing for the
// half-ray h % (2 npairs) of origin o_begin + (h / (2 npairs)) stride, whose
// length it stores at that half-ray's own index.  Every other pass: h itself.
template <int MODE>
__device__ __forceinline__ int64_t sampled(const DevRays &R, int32_t stride, int64_t h) {
    if (MODE != 0 || stride <= 1) return h;
    const int64_t np2 = 2 * int64_t(R.npairs);
    return (h / np2) * stride * np2 + h % np2;
}

// The lateral offset of the walk's current point c (exact Z given) in
// double, rounded to float, with its error bound (the float rounding plus g0).
__device__ __forceinline__ void lateral(const DevMesh &m, Walk &wk, double Z, double d0, double d1, double d2,
                                        double xo, double yo, double zo) {
    const int32_t c = wk.c;
    wk.ecx = __double2float_rn(__dsub_rn(__dsub_rn(m.x[c], xo), __dmul_rn(Z, d0)));
    wk.ecy = __double2float_rn(__dsub_rn(__dsub_rn(m.y[c], yo), __dmul_rn(Z, d1)));
    wk.ecz = __double2float_rn(__dsub_rn(__dsub_rn(m.z[c], zo), __dmul_rn(Z, d2)));
    wk.eec = fmaf(1.01f * kU, fmaxf(fabsf(wk.ecx), fmaxf(fabsf(wk.ecy), fabsf(wk.ecz))), m.g0);
}

// Set up the walk of half-ray h; false when h needs no walk (MODE 4: no
// tail) or its output range is inconsistent (reported through status).
template <int MODE>
__device__ __forceinline__ bool begin_walk(const DevMesh &m, const DevRays &R, int32_t o_begin, int64_t h,
                                           const int64_t *__restrict__ lens, const int64_t *__restrict__ offs,
                                           int64_t base, int64_t cap, int32_t pad, const int4 *__restrict__ resume,
                                           int *status, Walk &wk) {
    int64_t expect_len = 0;
    if (MODE == 4) {  // only the half-rays longer than their row
        expect_len = lens[h];
        if (expect_len <= pad) return false;
    }
    const int64_t hs = sampled<MODE>(R, pad, h);
    const int32_t o = walk_origin(R, o_begin, hs);
    const float4 df = R.dirf[walk_pix(R, o_begin, hs)];
    const bool back = (hs & 1) == 0;  // backward half: exact negation of the pair direction
    wk.f0 = back ? -df.x : df.x;
    wk.f1 = back ? -df.y : df.y;
    wk.f2 = back ? -df.z : df.z;
    wk.w = 0;
    wk.expect = 0;
    if (MODE == 1 || MODE == 2) {
        wk.w = offs[h] - base;
        wk.expect = int32_t(offs[h + 1] - offs[h]);
        if (wk.w < 0 || offs[h + 1] - base > cap) {
            dev_fail(status, kDevArenaOverflow);
            return false;
        }
    } else if (MODE == 4) {
        wk.w = offs[h] - base - pad;  // entry k >= pad goes to w + k
        wk.expect = int32_t(expect_len);
        if (offs[h] - base < 0 || offs[h + 1] - base > cap || offs[h + 1] - offs[h] != expect_len - pad) {
            dev_fail(status, kDevArenaOverflow);
            return false;
        }
    }
    wk.c = o;
    wk.k = 0;
    wk.ecx = wk.ecy = wk.ecz = wk.eec = 0.0f;  // the origin lies on the ray
    if (MODE == 4) {  // resume after the row's last entry
        wk.c = resume[h].x;
        wk.k = pad;
        if (wk.c < 0 || wk.c >= m.n) {
            dev_fail(status, kDevTraceMismatch);
            return false;
        }
        // the lateral offset of the current point, formed in double: each
        // component within 8.1 u64 |x_c - x_o|_1 (<= g0) of the exact value
        double d0, d1, d2;
        walk_dir(R, o_begin, h, d0, d1, d2);
        const double xo = m.x[o], yo = m.y[o], zo = m.z[o];
        const double Z = exact_Z(m, wk.c, xo, yo, zo, d0, d1, d2);
        lateral(m, wk, Z, d0, d1, d2, xo, yo, zo);
    }
    return true;
}

// A step of lane L's walk decided exactly by the whole warp: lane j takes the
// neighbours off[c] + j, off[c] + j + 32, ... of the current point c, forms
// their exact Z and q in double precision (the defining rule, on every
// neighbour, so no screen is needed), and a warp reduction picks the smallest
// q among the forward ones, ties to the smaller index.  All lanes return the
// same step.
__device__ Step step_exact_warp(const DevMesh &m, int32_t c, int32_t o, double d0, double d1, double d2,
                                int lane) {
    const double xo = m.x[o], yo = m.y[o], zo = m.z[o];
    const double zc = (c == o) ? 0.0 : exact_Z(m, c, xo, yo, zo, d0, d1, d2);
    int32_t best = -1;
    double qbest = 0.0, zbest = 0.0;
    const int32_t e1 = m.off[c + 1];
    for (int32_t e = m.off[c] + lane; e < e1; e += 32) {
        const int32_t nb = __ldg(m.nbr + e);
        const double ddx = __dsub_rn(__ldg(m.x + nb), xo);
        const double ddy = __dsub_rn(__ldg(m.y + nb), yo);
        const double ddz = __dsub_rn(__ldg(m.z + nb), zo);
        const double zn = __dadd_rn(__dadd_rn(__dmul_rn(ddx, d0), __dmul_rn(ddy, d1)), __dmul_rn(ddz, d2));
        if (!(zn > zc)) continue;
        const double qx = __dsub_rn(ddx, __dmul_rn(zn, d0));
        const double qy = __dsub_rn(ddy, __dmul_rn(zn, d1));
        const double qz = __dsub_rn(ddz, __dmul_rn(zn, d2));
        const double qd = __dadd_rn(__dadd_rn(__dmul_rn(qx, qx), __dmul_rn(qy, qy)), __dmul_rn(qz, qz));
        if (best < 0 || qd < qbest || (qd == qbest && nb < best)) {
            best = nb;
            qbest = qd;
            zbest = zn;
        }
    }
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) {
        const int32_t b2 = __shfl_xor_sync(0xffffffffu, best, sh);
        const double q2 = __shfl_xor_sync(0xffffffffu, qbest, sh);
        const double z2 = __shfl_xor_sync(0xffffffffu, zbest, sh);
        if (b2 >= 0 && (best < 0 || q2 < qbest || (q2 == qbest && b2 < best))) {
            best = b2;
            qbest = q2;
            zbest = z2;
        }
    }
    return Step{best, zbest};
}

// MODE 0: count the points of each half-ray (with pad > 1: of every pad-th
// origin only, see sampled); MODE 1: write their ids;
// MODE 2: write ids, exact double Z and (optionally) projected velocities;
// MODE 3: padded pass (ids k < pad to row h, length to lens[h], excess over
// the row to excess[h], the walk state after entry pad - 1 to resume[h] when
// the half-ray is longer); MODE 4: tail pass (ids k >= pad of the half-rays
// longer than the row, at offs[h] - base + k - pad, resumed from resume[h]).
//
// Lane t walks half-rays t, t + T, t + 2T, ... (T = all threads).  The loop
// advances every lane by one step per iteration, and a lane whose walk ends
// sets up its next half-ray inside the iteration, so the lanes of a warp stay
// busy although the half-rays they trace differ widely in length.
template <int MODE>
__global__ void __launch_bounds__(128, 7)
k_trace(DevMesh m, DevRays R, int32_t o_begin, int64_t n_half, int64_t *__restrict__ lens,
        const int64_t *__restrict__ offs, int64_t base, int64_t cap, int32_t *__restrict__ idx_out,
        double *__restrict__ Z_out, double *__restrict__ delta_out, int *status,
        unsigned long long *__restrict__ counters, int32_t pad, int64_t *__restrict__ excess,
        int4 *__restrict__ resume) {
    const int64_t T = int64_t(gridDim.x) * blockDim.x;
    unsigned n_steps = 0, n_exact = 0;
    Walk wk;
    // h: the lane's current half-ray while live
    int64_t h = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    bool live = false;
    for (; h < n_half; h += T)
        if ((live = begin_walk<MODE>(m, R, o_begin, h, lens, offs, base, cap, pad, resume, status, wk))) break;
    const int lane = threadIdx.x & 31;
    // every lane stays in the loop until the whole warp is done, so that undecided
    // steps can be resolved by the warp together
    while (__any_sync(0xffffffffu, live)) {
        int32_t next = -1;
        if (live) {
            next = step_screen(m, wk);
            ++n_steps;
        }
        double zexact = 0.0;
        bool have_exact = false;
        unsigned todo = __ballot_sync(0xffffffffu, live && next == -2);
        while (todo) {  // undecided in single precision: decided exactly, one lane's step at a time
            const int L = __ffs(todo) - 1;
            todo &= todo - 1;
            const int32_t c = __shfl_sync(0xffffffffu, wk.c, L);
            const int64_t hL = sampled<MODE>(R, pad, __shfl_sync(0xffffffffu, h, L));
            const int32_t o = walk_origin(R, o_begin, hL);
            double d0 = 0.0, d1 = 0.0, d2 = 0.0;
            if (lane == L) walk_dir(R, o_begin, hL, d0, d1, d2);
            d0 = __shfl_sync(0xffffffffu, d0, L);
            d1 = __shfl_sync(0xffffffffu, d1, L);
            d2 = __shfl_sync(0xffffffffu, d2, L);
            const Step x = step_exact_warp(m, c, o, d0, d1, d2, lane);
            if (lane == L) {
                next = x.next;
                zexact = x.Z;
                ++n_exact;
                have_exact = true;
                if (x.next >= 0) {
                    // the next point's position and lateral offset (exact Z known)
                    wk.c = x.next;
                    lateral(m, wk, x.Z, d0, d1, d2, m.x[o], m.y[o], m.z[o]);
                    wk.c = c;
                }
            }
        }
        if (!live) continue;
        bool ended = next < 0, failed = false;
        if (!ended) {
            const int32_t k = wk.k;
            if (MODE == 3) {
                if (k < pad) idx_out[h * int64_t(pad) + k] = next;
            } else if (MODE == 4) {
                if (k >= wk.expect) failed = true;
                else idx_out[wk.w + k] = next;  // k >= pad here
            } else if (MODE > 0) {
                if (k >= wk.expect) {
                    failed = true;
                } else {
                    idx_out[wk.w + k] = next;
                    if (MODE == 2) {
                        const int32_t o = walk_origin(R, o_begin, h);
                        const double xo = m.x[o], yo = m.y[o], zo = m.z[o];
                        double d0, d1, d2;
                        walk_dir(R, o_begin, h, d0, d1, d2);
                        Z_out[wk.w + k] = have_exact ? zexact : exact_Z(m, next, xo, yo, zo, d0, d1, d2);
                        if (delta_out) {
                            const double ux = __dsub_rn(m.vx[next], m.vx[o]);
                            const double uy = __dsub_rn(m.vy[next], m.vy[o]);
                            const double uz = __dsub_rn(m.vz[next], m.vz[o]);
                            delta_out[wk.w + k] =
                                __dadd_rn(__dadd_rn(__dmul_rn(ux, d0), __dmul_rn(uy, d1)), __dmul_rn(uz, d2));
                        }
                    }
                }
            }
            if (failed) {
                dev_fail(status, kDevTraceMismatch);
                ended = true;
            } else {
                wk.k = k + 1;
                wk.c = next;
                if (MODE == 3 && wk.k == pad) resume[h] = make_int4(wk.c, 0, 0, 0);
                if (wk.k > m.n) {  // Z increases strictly, so this cannot happen
                    dev_fail(status, kDevTraceGuard);
                    ended = true;
                    failed = true;
                }
            }
        }
        if (ended) {
            if (MODE == 0) {
                lens[sampled<MODE>(R, pad, h)] = wk.k;
            } else if (MODE == 3) {
                lens[h] = wk.k;
                excess[h] = wk.k > pad ? wk.k - pad : 0;
            } else if (!failed && wk.k != wk.expect) {
                dev_fail(status, kDevTraceMismatch);
            }
            live = false;
            for (h += T; h < n_half; h += T)
                if ((live = begin_walk<MODE>(m, R, o_begin, h, lens, offs, base, cap, pad, resume, status, wk))) break;
        }
    }
    if (counters) {
        atomicAdd(counters + 2, (unsigned long long)n_steps);
        atomicAdd(counters + 3, (unsigned long long)n_exact);
    }
}

// Grid of the strided walk: ctas_per_sm CTAs of 128 threads per SM (7, the
// register cap's limit, when not positive), at most as many as can be resident at once (so the whole
// grid is one wave and every lane's share of half-rays runs concurrently),
// fewer when there are fewer half-rays.
template <int MODE>
unsigned trace_grid(int64_t n_half, int ctas_per_sm = 0) {
    int dev = 0, sms = 152, fit = 7;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, k_trace<MODE>, 128, 0) != cudaSuccess || fit < 1) fit = 1;
    int per = ctas_per_sm > 0 ? ctas_per_sm : 7;
    if (per > fit) per = fit;
    const int64_t want = (n_half + 127) / 128;
    const int64_t cap = int64_t(sms) * per;
    return unsigned(want < cap ? want : cap);
}

}  // namespace

void launch_trace_count(const DevMesh &m, const DevRays &R, int32_t o_begin, int32_t o_end,
                        int64_t *lens, int *status, unsigned long long *counters, cudaStream_t st,
                        int32_t o_stride) {
    if (o_stride < 1) o_stride = 1;
    const int64_t n_half = (int64_t(o_end - o_begin) + o_stride - 1) / o_stride * R.npairs * 2;
    if (n_half == 0) return;
    k_trace<0><<<trace_grid<0>(n_half), 128, 0, st>>>(m, R, o_begin, n_half, lens, nullptr, 0, 0, nullptr, nullptr,
                                                  nullptr, status, counters, o_stride, nullptr, nullptr);
}

void launch_trace_emit(const DevMesh &m, const DevRays &R, int32_t o_begin, int32_t o_end,
                       const int64_t *offs, int64_t base, int64_t cap, int32_t *idx, double *Z, double *delta,
                       int *status, cudaStream_t st) {
    const int64_t n_half = int64_t(o_end - o_begin) * R.npairs * 2;
    if (n_half == 0) return;
    if (Z) {
        k_trace<2><<<trace_grid<2>(n_half), 128, 0, st>>>(m, R, o_begin, n_half, nullptr, offs, base, cap, idx, Z,
                                                      delta, status, nullptr, 0, nullptr, nullptr);
    } else {
        k_trace<1><<<trace_grid<1>(n_half), 128, 0, st>>>(m, R, o_begin, n_half, nullptr, offs, base, cap, idx,
                                                      nullptr, nullptr, status, nullptr, 0, nullptr, nullptr);
    }
}

void launch_trace_pad(const DevMesh &m, const DevRays &R, int32_t o_begin, int32_t o_end, int32_t pad,
                      int64_t *lens, int64_t *excess, int4 *resume, int32_t *rows, int *status,
                      unsigned long long *counters, cudaStream_t st, int ctas_per_sm) {
    const int64_t n_half = int64_t(o_end - o_begin) * R.npairs * 2;
    if (n_half == 0) return;
    k_trace<3><<<trace_grid<3>(n_half, ctas_per_sm), 128, 0, st>>>(m, R, o_begin, n_half, lens, nullptr, 0, 0, rows, nullptr,
                                                  nullptr, status, counters, pad, excess, resume);
}

void launch_trace_tail(const DevMesh &m, const DevRays &R, int32_t o_begin, int32_t o_end, int32_t pad,
                       const int64_t *lens, const int4 *resume, const int64_t *offs, int64_t base, int64_t cap,
                       int32_t *tail, int *status, cudaStream_t st, int ctas_per_sm) {
    const int64_t n_half = int64_t(o_end - o_begin) * R.npairs * 2;
    if (n_half == 0) return;
    k_trace<4><<<trace_grid<4>(n_half, ctas_per_sm), 128, 0, st>>>(m, R, o_begin, n_half, const_cast<int64_t *>(lens), offs, base,
                                                  cap, tail, nullptr, nullptr, status, nullptr, pad, nullptr,
                                                  const_cast<int4 *>(resume));
}

}  // namespace mgx
