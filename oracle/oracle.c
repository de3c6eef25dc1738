/*
 * oracle.c -- plain, slow FP64 CPU implementation of the Magritte radiation-field
 * hot path (De Ceuster et al. 2020, "Magritte II: adaptive ray-tracing, mesh
 * construction and reduction").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the CUDA
 * path is checked against.  Only the test-suite, the package smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header, table
 * or constant generator with the CUDA library, and the CUDA library never calls it.
 *
 * Everything is double precision, evaluated in source order (compiled with
 * -ffp-contract=off so that no multiply-add is fused).  Each function names the
 * passage of the paper it follows.  Where the paper is silent (it defers the
 * discretisation details to Magritte I), the reading taken is stated in place.
 *
 * Parity status of each part (what pins it in the CPU test-suite):
 *   HEALPix pix2vec/vec2pix .......... pinned (ring closed forms, round trip,
 *                                       nested parenthood, pixel counts, uniformity)
 *   adaptive ray set ................. pinned (552 / 3072 ray counts, weights sum to 1,
 *                                       brute-force re-ranking of the counts)
 *   tracer ........................... pinned (exhaustive brute force on tiny meshes,
 *                                       straight grid lines)
 *   line mapping / sub-division ...... pinned (closed-form profile argument in
 *                                       50-digit arithmetic, trapezoid sums)
 *   Feautrier solve .................. pinned (dense linear solve, homogeneous closed
 *                                       form, second-order convergence, J -> S)
 *   velocity-sampling threshold, dtau_max and continuum-floor VALUES:
 *                                       parity unpinned (conventions, not in the paper)
 *   reduction criterion .............. pinned (hand-computed graphs, Gf in [0,1],
 *                                       thinning rate)
 *   Hermitian solve .................. pinned (uniform-grid Numerov system, exact
 *                                       quadratics, third-order convergence)
 *   per-ray u ........................ pinned (sum of 2 w u equals J)
 *   analytic size field .............. pinned (exponential closed form, Gaussian
 *                                       convergence, thinning rate)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_C_KMS 299792.458 /* speed of light in km/s */

/* ------------------------------------------------------------------------- */
/* HEALPix, nested ordering (Gorski et al. 2005), used by Section 2.1.3.      */
/* A level l has nside = 2^l and 12*4^l equal-area pixels.                    */
/* ------------------------------------------------------------------------- */

/* Ring row (in units of nside) of the southern corner of each base face, and
 * the longitude column of each base face (in units of pi/4).  These follow
 * from the geometry of the 12 base pixels in Gorski et al. (2005), Fig. 3. */
static const int64_t base_row[12] = {2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4};
static const int64_t base_col[12] = {1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7};

static int64_t bits_spread(int64_t v) /* bit k of v -> bit 2k of the result */
{
    int64_t r = 0;
    for (int k = 0; k < 31; ++k) r |= ((v >> k) & 1LL) << (2 * k);
    return r;
}

static int64_t bits_gather(int64_t v) /* bit 2k of v -> bit k of the result */
{
    int64_t r = 0;
    for (int k = 0; k < 31; ++k) r |= ((v >> (2 * k)) & 1LL) << k;
    return r;
}

int64_t orc_npix(int l) { return 12LL << (2 * l); }

/* Centre direction of nested pixel p at level l.  The pixel's ring number i
 * (1 .. 4 nside - 1, counted from the north pole) and its position j in the
 * ring give z and phi by the closed forms of Gorski et al. (2005):
 *   polar caps:   z = 1 - i^2 / (3 nside^2),  phi = pi/(2i) (j - 1/2)
 *   belt:         z = 4/3 - 2 i / (3 nside),  phi = pi/(2 nside) (j - s/2)
 * with s = 1 on rings i - nside even and 0 otherwise. */
void orc_pix2vec_nest(int l, int64_t p, double v[3])
{
    const int64_t ns = 1LL << l, npf = ns * ns;
    const int64_t f = p / npf, q = p % npf;
    const int64_t x = bits_gather(q), y = bits_gather(q >> 1);
    const int64_t i = base_row[f] * ns - x - y - 1;
    int64_t nr, shift;
    double z;
    if (i < ns) {
        nr = i;
        shift = 0;
        z = 1.0 - (double)(nr * nr) / (double)(3 * ns * ns);
    } else if (i > 3 * ns) {
        nr = 4 * ns - i;
        shift = 0;
        z = (double)(nr * nr) / (double)(3 * ns * ns) - 1.0;
    } else {
        nr = ns;
        shift = (i - ns) & 1;
        z = (double)(2 * (2 * ns - i)) / (double)(3 * ns);
    }
    int64_t j = (base_col[f] * nr + x - y + 1 + shift) / 2;
    if (j > 4 * nr) j -= 4 * nr;
    if (j < 1) j += 4 * nr;
    const double phi = (double)(2 * j - 1 - shift) * M_PI / (double)(4 * nr);
    const double st = sqrt((1.0 - z) * (1.0 + z));
    v[0] = st * cos(phi);
    v[1] = st * sin(phi);
    v[2] = z;
}

/* Nested pixel at level l that contains direction d (d need not be unit). */
int64_t orc_vec2pix_nest(int l, const double d[3])
{
    const int64_t ns = 1LL << l;
    const double len = sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
    const double z = d[2] / len;
    const double za = fabs(z);
    double t = atan2(d[1], d[0]) * M_2_PI; /* longitude in units of pi/2 */
    if (t < 0.0) t += 4.0;
    if (t >= 4.0) t -= 4.0;
    int64_t f, x, y;
    if (za <= 2.0 / 3.0) {
        /* equatorial zone: pixel edges are the lines t +- 3z/4 = const */
        const double c1 = (double)ns * (0.5 + t);
        const double c2 = (double)ns * (0.75 * z);
        const int64_t up = (int64_t)(c1 - c2);
        const int64_t dn = (int64_t)(c1 + c2);
        const int64_t fu = up >> l, fd = dn >> l;
        if (fu == fd) f = fu | 4;
        else if (fu < fd) f = fu;
        else f = fd + 8;
        x = dn & (ns - 1);
        y = ns - 1 - (up & (ns - 1));
    } else {
        /* polar caps: edges are lines of constant t*sqrt(3(1-|z|)) */
        int64_t k = (int64_t)t;
        if (k > 3) k = 3;
        const double tp = t - (double)k;
        const double w = (double)ns * sqrt(3.0 * (1.0 - za));
        int64_t a = (int64_t)(tp * w);
        int64_t b = (int64_t)((1.0 - tp) * w);
        if (a > ns - 1) a = ns - 1;
        if (b > ns - 1) b = ns - 1;
        if (z >= 0.0) {
            f = k;
            x = ns - 1 - b;
            y = ns - 1 - a;
        } else {
            f = k + 8;
            x = a;
            y = b;
        }
    }
    return f * ns * ns + bits_spread(x) + 2 * bits_spread(y);
}

/* The pixel containing the direction opposite to the centre of p. */
int64_t orc_antipode(int l, int64_t p)
{
    double v[3];
    orc_pix2vec_nest(l, p, v);
    v[0] = -v[0];
    v[1] = -v[1];
    v[2] = -v[2];
    return orc_vec2pix_nest(l, v);
}

/* ------------------------------------------------------------------------- */
/* Adaptive hierarchical ray set (Section 2.1.3, Eq. 4, Fig. 1).               */
/* Reading: refinement is counted in antipodal PAIRS -- at each level the top  */
/* half of the candidate pairs (ranked by the number of sample directions that */
/* fall in either member, ties to the smaller nested index) is refined, the    */
/* rest become rays of that level; at l_max every candidate is a ray.  With    */
/* l_min = 1, l_max = 4 this gives the paper's 552 rays.                        */
/* A ray set entry is packed as (level << 28) | nested pixel of the pair member */
/* with the smaller index; the other member points the opposite way.           */
/* ------------------------------------------------------------------------- */

int64_t orc_rayset_npairs(int l_min, int l_max)
{
    if (l_min == l_max) return orc_npix(l_min) / 2;
    int64_t cand = orc_npix(l_min) / 2, total = 0;
    for (int l = l_min; l < l_max; ++l) {
        total += cand / 2;
        cand = (cand / 2) * 4;
    }
    return total + cand;
}

typedef struct {
    int64_t score;
    int64_t pix;
} orc_cand;

static int cand_cmp(const void *a, const void *b)
{
    const orc_cand *x = (const orc_cand *)a, *y = (const orc_cand *)b;
    if (x->score != y->score) return x->score > y->score ? -1 : 1;
    return (x->pix < y->pix) ? -1 : (x->pix > y->pix);
}

static int u32_cmp(const void *a, const void *b)
{
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return (x < y) ? -1 : (x > y);
}

/* Ray set of origin i.  sample[0..n_sample) are the point indices of the
 * global sample of Section 2.1.3 (drawn by the caller); the origin itself and
 * points at the origin's position are skipped.  Writes orc_rayset_npairs()
 * entries, sorted ascending (level, then pixel).  Returns 0 or -1 on bad args. */
int orc_rayset_one(int64_t n, const double *pos, int64_t i, int64_t n_sample,
                   const int32_t *sample, int l_min, int l_max, uint32_t *out)
{
    if (l_min < 0 || l_max < l_min || l_max > 8) return -1;
    const int64_t np = orc_rayset_npairs(l_min, l_max);
    int64_t n_out = 0;
    if (l_min == l_max) {
        for (int64_t p = 0; p < orc_npix(l_min); ++p)
            if (p < orc_antipode(l_min, p)) out[n_out++] = ((uint32_t)l_min << 28) | (uint32_t)p;
        qsort(out, (size_t)n_out, sizeof(uint32_t), u32_cmp);
        return n_out == np ? 0 : -1;
    }
    /* direction counts at the finest level (Section 2.1.3: only the finest
     * level is histogrammed, coarser levels by nested downgrading) */
    const int64_t nfine = orc_npix(l_max);
    int64_t *cnt = (int64_t *)calloc((size_t)nfine, sizeof(int64_t));
    const double *xi = pos + 3 * i;
    for (int64_t s = 0; s < n_sample; ++s) {
        const int64_t j = sample[s];
        if (j == i || j < 0 || j >= n) continue;
        double d[3] = {pos[3 * j] - xi[0], pos[3 * j + 1] - xi[1], pos[3 * j + 2] - xi[2]};
        if (d[0] == 0.0 && d[1] == 0.0 && d[2] == 0.0) continue;
        cnt[orc_vec2pix_nest(l_max, d)] += 1;
    }
    int64_t ncand = 0;
    orc_cand *cand = (orc_cand *)malloc(sizeof(orc_cand) * (size_t)(orc_npix(l_max) / 2 + 8));
    for (int64_t p = 0; p < orc_npix(l_min); ++p)
        if (p < orc_antipode(l_min, p)) cand[ncand++].pix = p;
    for (int l = l_min; l < l_max; ++l) {
        const int sh = 2 * (l_max - l);
        for (int64_t c = 0; c < ncand; ++c) {
            const int64_t p = cand[c].pix, a = orc_antipode(l, p);
            int64_t s = 0;
            for (int64_t q = p << sh; q < (p + 1) << sh; ++q) s += cnt[q];
            for (int64_t q = a << sh; q < (a + 1) << sh; ++q) s += cnt[q];
            cand[c].score = s;
        }
        qsort(cand, (size_t)ncand, sizeof(orc_cand), cand_cmp);
        const int64_t nref = ncand / 2;
        for (int64_t c = nref; c < ncand; ++c)
            out[n_out++] = ((uint32_t)l << 28) | (uint32_t)cand[c].pix;
        int64_t nnew = 0;
        orc_cand *next = (orc_cand *)malloc(sizeof(orc_cand) * (size_t)(nref * 4 + 8));
        for (int64_t c = 0; c < nref; ++c)
            for (int64_t ch = 4 * cand[c].pix; ch < 4 * cand[c].pix + 4; ++ch) {
                const int64_t a = orc_antipode(l + 1, ch);
                next[nnew].pix = ch < a ? ch : a;
                next[nnew].score = 0;
                ++nnew;
            }
        free(cand);
        cand = next;
        ncand = nnew;
    }
    for (int64_t c = 0; c < ncand; ++c) out[n_out++] = ((uint32_t)l_max << 28) | (uint32_t)cand[c].pix;
    free(cand);
    free(cnt);
    qsort(out, (size_t)n_out, sizeof(uint32_t), u32_cmp);
    return n_out == np ? 0 : -1;
}

/* Ray sets of origins [0, n) -> out[n][npairs]; OpenMP over origins. */
int orc_rayset(int64_t n, const double *pos, int64_t n_sample, const int32_t *sample,
               int l_min, int l_max, uint32_t *out, int threads)
{
    const int64_t np = orc_rayset_npairs(l_min, l_max);
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) num_threads(threads) reduction(| : bad)
    for (int64_t i = 0; i < n; ++i)
        bad |= orc_rayset_one(n, pos, i, n_sample, sample, l_min, l_max, out + i * np) != 0;
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------------- */
/* Model description shared by the tracer and the solver.                     */
/* ------------------------------------------------------------------------- */
typedef struct {
    int64_t n;               /* points                                        */
    const double *pos;       /* [n][3]                                        */
    const double *vel;       /* [n][3] km/s                                   */
    const int64_t *nbr_off;  /* [n+1] CSR row offsets                         */
    const int32_t *nbr_idx;  /* [E]   neighbour indices                       */
    int32_t n_lines;         /* L                                             */
    const double *nu0;       /* [L] line-centre frequencies                   */
    const double *chi0;      /* [n][L] line-centre opacity                    */
    const double *eta0;      /* [n][L] line-centre emissivity                 */
    const double *dvw;       /* [n] Doppler width, km/s                       */
    const double *chi_c;     /* [n] continuum opacity                         */
    const double *eta_c;     /* [n] continuum emissivity                      */
    int32_t n_freq;          /* bins per line                                 */
    double x_span;           /* bins span [-x_span, x_span] Doppler widths    */
    int32_t l_min, l_max;    /* ray-set levels                                */
    const uint32_t *rays;    /* [n][npairs] packed ray set                    */
} orc_model;

typedef struct {
    double dtau_max; /* Eq. 2 */
    double dv_max;   /* velocity step limit, in units of the smaller Doppler width (<= 0: off) */
    double I_bdy;    /* boundary intensity entering both ends of every ray    */
    int32_t order;    /* 2: the second-order scheme with second-order boundary
                         conditions; 4: Auer's (1976) Hermitian fourth-order
                         scheme with third-order boundary conditions (Section 2.1) */
} orc_params;

/* ------------------------------------------------------------------------- */
/* Tracer (Section 2.1, Fig. 2).  From the current point c, the next point is  */
/* the neighbour of c that lies strictly further along the ray (Z_n > Z_c,     */
/* Z = (x_n - x_o).d) and closest to it (smallest |(x_n - x_o) - Z d|^2, ties   */
/* to the smaller index).  The half-ray ends when c has no such neighbour.     */
/* Writes up to cap entries; returns the half-ray length.                      */
/* ------------------------------------------------------------------------- */
int64_t orc_trace_half(const orc_model *m, int64_t o, const double d[3], int64_t cap,
                       int32_t *idx, double *Z)
{
    const double *xo = m->pos + 3 * o;
    int64_t c = o, k = 0;
    double zc = 0.0;
    for (;;) {
        int64_t best = -1;
        double qbest = 0.0, zbest = 0.0;
        for (int64_t e = m->nbr_off[c]; e < m->nbr_off[c + 1]; ++e) {
            const int64_t nb = m->nbr_idx[e];
            const double dx = m->pos[3 * nb] - xo[0];
            const double dy = m->pos[3 * nb + 1] - xo[1];
            const double dz = m->pos[3 * nb + 2] - xo[2];
            const double zn = (dx * d[0] + dy * d[1]) + dz * d[2];
            if (!(zn > zc)) continue;
            const double ex = dx - zn * d[0], ey = dy - zn * d[1], ez = dz - zn * d[2];
            const double q = (ex * ex + ey * ey) + ez * ez;
            if (best < 0 || q < qbest || (q == qbest && nb < best)) {
                best = nb;
                qbest = q;
                zbest = zn;
            }
        }
        if (best < 0) break;
        if (k < cap) {
            idx[k] = (int32_t)best;
            Z[k] = zbest;
        }
        ++k;
        c = best;
        zc = zbest;
        if (k > m->n) break; /* cannot happen: Z increases strictly */
    }
    return k;
}

/* ------------------------------------------------------------------------- */
/* Line data along one ray pair (Sections 2.1.1 and 2.1.2).                   */
/* ------------------------------------------------------------------------- */

/* Doppler-shifted profile argument of line lp at the frequency of bin k of
 * line l, for a point whose projected velocity relative to the origin is
 * delta (km/s) and whose Doppler width is dv.  Reading (Magritte I): bins are
 * uniform in x in [-x_span, x_span] origin Doppler widths around each line
 * centre, nu = nu_l (1 + x dv_o / c); a point moving with projected velocity
 * delta towards the origin sees nu (1 + delta / c); the Gaussian argument is
 * (nu (1 + delta/c) - nu_lp) / (nu_lp dv / c).  Written in velocity units: */
double orc_profile_arg(double nu_l, double nu_lp, double x, double dv_o, double delta, double dv)
{
    const double r = nu_l / nu_lp;
    const double ub = x * dv_o;
    return (ORC_C_KMS * (r - 1.0) + r * ub + r * (1.0 + ub / ORC_C_KMS) * delta) / dv;
}

double orc_bin_x(int32_t n_freq, double x_span, int32_t k)
{
    if (n_freq == 1) return 0.0;
    return -x_span + 2.0 * x_span * (double)k / (double)(n_freq - 1);
}

/* Frequency-independent samples along the pair line after adaptive velocity
 * sampling (Section 2.1.1).  At most ORC_MAX_LINES lines. */
#define ORC_MAX_LINES 16
typedef struct {
    double s, delta, dvw, chic, etac;
    double chi0[ORC_MAX_LINES], eta0[ORC_MAX_LINES];
} orc_sample;

typedef struct {
    int64_t cap, m; /* capacity and count   */
    int64_t io;     /* index of the origin  */
    orc_sample *p;
} orc_vline;

static void vline_free(orc_vline *v) { free(v->p); }

static void vline_push(orc_vline *v, const orc_sample *x)
{
    if (v->m == v->cap) {
        v->cap = v->cap * 2 + 16;
        v->p = (orc_sample *)realloc(v->p, sizeof(orc_sample) * (size_t)v->cap);
    }
    v->p[v->m++] = *x;
}

static void sample_of_point(const orc_model *m, int64_t id, double s, double delta, orc_sample *x)
{
    const int L = m->n_lines;
    x->s = s;
    x->delta = delta;
    x->dvw = m->dvw[id];
    x->chic = m->chi_c[id];
    x->etac = m->eta_c[id];
    for (int l = 0; l < L; ++l) {
        x->chi0[l] = m->chi0[id * L + l];
        x->eta0[l] = m->eta0[id * L + l];
    }
}

/* linear interpolation a + (b - a) t of every quantity (Section 2.1.1) */
static void sample_lerp(int L, const orc_sample *a, const orc_sample *b, double t, orc_sample *x)
{
    x->s = a->s + (b->s - a->s) * t;
    x->delta = a->delta + (b->delta - a->delta) * t;
    x->dvw = a->dvw + (b->dvw - a->dvw) * t;
    x->chic = a->chic + (b->chic - a->chic) * t;
    x->etac = a->etac + (b->etac - a->etac) * t;
    for (int l = 0; l < L; ++l) {
        x->chi0[l] = a->chi0[l] + (b->chi0[l] - a->chi0[l]) * t;
        x->eta0[l] = a->eta0[l] + (b->eta0[l] - a->eta0[l]) * t;
    }
}

/* Build the velocity-sampled pair line of origin o along +-r.  The base points
 * are the backward half-ray (traced along -r, listed from its far end), the
 * origin, and the forward half-ray (along +r), at signed distance s = -Z, 0,
 * +Z.  A point on the half along direction d (= -r or +r) gets the projected
 * velocity difference delta = (v_n - v_o).d; the origin gets 0.  Between
 * consecutive base points a and b with |delta_b - delta_a| larger than
 * dv_max * min(dv_a, dv_b), the interval is split into
 * ceil(|delta_b - delta_a| / (dv_max min(dv_a, dv_b))) equal parts with every
 * quantity interpolated linearly (reading of Section 2.1.1). */
static void build_vline(const orc_model *m, const orc_params *pr, int64_t o, const double r[3],
                        orc_vline *v)
{
    const int64_t n = m->n;
    const int L = m->n_lines;
    int32_t *bi = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    double *bz = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    int32_t *fi = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    double *fz = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    const double rm[3] = {-r[0], -r[1], -r[2]};
    const int64_t nb = orc_trace_half(m, o, rm, n + 1, bi, bz);
    const int64_t nf = orc_trace_half(m, o, r, n + 1, fi, fz);
    const double *vo = m->vel + 3 * o;
    v->cap = 0;
    v->m = 0;
    v->io = -1;
    v->p = NULL;
    orc_sample prev, cur, mid;
    memset(&prev, 0, sizeof prev);
    for (int64_t k = 0; k < nb + 1 + nf; ++k) {
        if (k < nb) { /* backward half, far end first */
            const int64_t id = bi[nb - 1 - k];
            const double *vn = m->vel + 3 * id;
            const double de = ((vn[0] - vo[0]) * rm[0] + (vn[1] - vo[1]) * rm[1]) + (vn[2] - vo[2]) * rm[2];
            sample_of_point(m, id, -bz[nb - 1 - k], de, &cur);
        } else if (k == nb) {
            sample_of_point(m, o, 0.0, 0.0, &cur);
        } else {
            const int64_t id = fi[k - nb - 1];
            const double *vn = m->vel + 3 * id;
            const double de = ((vn[0] - vo[0]) * r[0] + (vn[1] - vo[1]) * r[1]) + (vn[2] - vo[2]) * r[2];
            sample_of_point(m, id, fz[k - nb - 1], de, &cur);
        }
        if (k > 0 && pr->dv_max > 0.0) {
            int64_t parts = 1;
            const double jump = fabs(cur.delta - prev.delta);
            const double lim = pr->dv_max * fmin(prev.dvw, cur.dvw);
            if (jump > lim) parts = (int64_t)ceil(jump / lim);
            if (parts > 1) {
                for (int64_t j = 1; j < parts; ++j) {
                    sample_lerp(L, &prev, &cur, (double)j / (double)parts, &mid);
                    vline_push(v, &mid);
                }
            }
        }
        vline_push(v, &cur);
        if (k == nb) v->io = v->m - 1;
        prev = cur;
    }
    free(bi); free(bz); free(fi); free(fz);
}

/* Total opacity and emissivity at every velocity sample for bin k of line l. */
static void line_optics(const orc_model *m, const orc_vline *v, double dv_o, int32_t l, int32_t k,
                        double *chi, double *eta)
{
    const int L = m->n_lines;
    const double x = orc_bin_x(m->n_freq, m->x_span, k);
    for (int64_t i = 0; i < v->m; ++i) {
        const orc_sample *p = &v->p[i];
        double c = p->chic, e = p->etac;
        for (int lp = 0; lp < L; ++lp) {
            const double a = orc_profile_arg(m->nu0[l], m->nu0[lp], x, dv_o, p->delta, p->dvw);
            const double g = exp(-(a * a));
            c += p->chi0[lp] * g;
            e += p->eta0[lp] * g;
        }
        chi[i] = c;
        eta[i] = e;
    }
}

/* Adaptive optical-depth sub-division (Section 2.1.2, Eq. 2): between samples
 * i and i+1 at distance ds, n_inter = ceil(max(chi_i, chi_i+1) ds / dtau_max)
 * (at least 1) equal parts, with chi and eta linear on the sub-intervals and
 * the optical depth of each part by the trapezoid rule.  Outputs the optical
 * depth increments dtau[0..M) and the source function S[0..M] = eta/chi of the
 * sub-divided line, and the index of the origin.  Returns M, or -1 when the
 * line would exceed max_pts. */
int64_t orc_subdivide(int64_t mv, const double *s, const double *chi, const double *eta,
                      int64_t io, double dtau_max, int64_t max_pts, double *dtau, double *S,
                      int64_t *io_out)
{
    int64_t M = 0;
    S[0] = eta[0] / chi[0];
    if (io == 0) *io_out = 0;
    for (int64_t i = 0; i + 1 < mv; ++i) {
        const double ds = s[i + 1] - s[i];
        const double cmax = fmax(chi[i], chi[i + 1]);
        int64_t ni = (int64_t)ceil(cmax * ds / dtau_max); /* Eq. 2 */
        if (ni < 1) ni = 1;
        if (M + ni > max_pts) return -1;
        const double h = ds / (double)ni;
        double cprev = chi[i];
        for (int64_t j = 1; j <= ni; ++j) {
            double cj, ej;
            if (j == ni) {
                cj = chi[i + 1];
                ej = eta[i + 1];
            } else {
                const double t = (double)j / (double)ni;
                cj = chi[i] + (chi[i + 1] - chi[i]) * t;
                ej = eta[i] + (eta[i + 1] - eta[i]) * t;
            }
            dtau[M] = h * (cprev + cj) * 0.5;
            ++M;
            S[M] = ej / cj;
            cprev = cj;
        }
        if (i + 1 == io) *io_out = M;
    }
    return M;
}

static int64_t orc_subdivide_v(const orc_vline *v, const double *chi, const double *eta,
                               const orc_params *pr, int64_t max_pts, double *dtau, double *S, int64_t *io)
{
    double *s = (double *)malloc(sizeof(double) * (size_t)v->m);
    for (int64_t i = 0; i < v->m; ++i) s[i] = v->p[i].s;
    const int64_t M = orc_subdivide(v->m, s, chi, eta, v->io, pr->dtau_max, max_pts, dtau, S, io);
    free(s);
    return M;
}

/* ------------------------------------------------------------------------- */
/* Feautrier solve (Eq. 1, Section 2.1).                                       */
/* Reading (Magritte I / Auer 1967): rows 0..M of                               */
/*   -A_i u_{i-1} + (1 + A_i + C_i) u_i - C_i u_{i+1} = S_i,                    */
/*   A_i = 2 / (dtau_{i-1} (dtau_{i-1} + dtau_i)),                              */
/*   C_i = 2 / (dtau_i (dtau_{i-1} + dtau_i)),                                  */
/* closed at both ends by the second-order boundary condition for an incoming */
/* intensity I:                                                                 */
/*   (1 + 2/dt + 2/dt^2) u_end - (2/dt^2) u_next = S_end + 2 I / dt.            */
/* Solved by Gaussian elimination in the form of Rybicki & Hummer (1991):      */
/* F_i = (1 + A_i F_{i-1}/(1 + F_{i-1})) / C_i, z_i = (S_i + A_i z_{i-1}) /      */
/* (C_i (1 + F_i)), then back substitution u_i = u_{i+1}/(1+F_i) + z_i.          */
/* Returns u at row io; if u_all is not NULL it receives every row.             */
/* A line of a single point (M = 0) has no medium: u = I.                       */
/* ------------------------------------------------------------------------- */
double orc_feautrier(int64_t M, const double *dtau, const double *S, int64_t io, double I,
                     double *u_all)
{
    if (M == 0) {
        if (u_all) u_all[0] = I;
        return I;
    }
    double *F = (double *)malloc(sizeof(double) * (size_t)M);
    double *z = (double *)malloc(sizeof(double) * (size_t)M);
    double *u = u_all ? u_all : (double *)malloc(sizeof(double) * (size_t)(M + 1));
    const double t0 = dtau[0];
    F[0] = t0 + t0 * t0 * 0.5;
    z[0] = (S[0] + 2.0 * I / t0) / (1.0 + 2.0 / t0 + 2.0 / (t0 * t0));
    for (int64_t i = 1; i < M; ++i) {
        const double tm = dtau[i - 1], tp = dtau[i];
        const double A = 2.0 / (tm * (tm + tp));
        const double C = 2.0 / (tp * (tm + tp));
        F[i] = (1.0 + A * F[i - 1] / (1.0 + F[i - 1])) / C;
        z[i] = (S[i] + A * z[i - 1]) / (C * (1.0 + F[i]));
    }
    const double tl = dtau[M - 1];
    const double AM = 2.0 / (tl * tl);
    u[M] = (S[M] + 2.0 * I / tl + AM * z[M - 1]) /
           (1.0 + 2.0 / tl + AM * F[M - 1] / (1.0 + F[M - 1]));
    for (int64_t i = M - 1; i >= 0; --i) u[i] = u[i + 1] / (1.0 + F[i]) + z[i];
    const double uo = u[io];
    free(F);
    free(z);
    if (!u_all) free(u);
    return uo;
}

/* ------------------------------------------------------------------------- */
/* Hermitian (fourth-order) Feautrier solve, Auer (1976), named in Section 2.1 */
/* as the more accurate scheme Magritte provides, with the third-order          */
/* boundary condition of Auer (1967).                                           */
/* Interior row i (h- = dtau_{i-1}, h+ = dtau_i): the compact approximation     */
/*   2/(h- + h+) [(u_{i+1} - u_i)/h+ - (u_i - u_{i-1})/h-]                      */
/*     = a f_{i-1} + b f_i + g f_{i+1},   f = u - S  (Eq. 1: d2u/dtau2 = u - S), */
/* with the weights that make it exact for polynomials of degree four on a      */
/* non-uniform grid (Taylor expansion about tau_i):                             */
/*   a = (h-^2 + h- h+ - h+^2) / (6 h- (h- + h+)),                              */
/*   g = (h+^2 + h- h+ - h-^2) / (6 h+ (h- + h+)),   b = 1 - a - g,             */
/* (1/12, 10/12, 1/12 on a uniform grid), i.e.                                  */
/*   -(A_i - a) u_{i-1} + (1 + A_i - a + C_i - g) u_i - (C_i - g) u_{i+1}        */
/*       = a S_{i-1} + b S_i + g S_{i+1}.                                        */
/* Boundary row (h the increment to the neighbour, I the incoming intensity):   */
/* du/dtau = u - I at the surface, the derivative from the Taylor series to     */
/* third order, its third-derivative term from the difference of f over the     */
/* first increment:                                                             */
/*   (2/3 + 2/h + 2/h^2) u_end - (2/h^2 - 1/3) u_next = 2/3 S_end + 1/3 S_next   */
/*                                                      + 2 I / h.              */
/* Every row has diagonal excess (diagonal minus off-diagonals) 1 inside and    */
/* 1 + 2/h at the ends, so the elimination keeps the form of Rybicki & Hummer   */
/* with general off-diagonals a_i, c_i:                                         */
/*   F_i = (B_i + a_i F_{i-1}/(1 + F_{i-1})) / c_i,                              */
/*   z_i = (r_i + a_i z_{i-1}) / (c_i (1 + F_i)),  u_i = u_{i+1}/(1 + F_i) + z_i. */
/* The right-hand side is formed as S_i + a (S_{i-1} - S_i) + g (S_{i+1} - S_i). */
/* Reading: the weights a, g grow like the ratio of the two increments, so the  */
/* rounding of S would be amplified without bound next to a vanishing increment */
/* (traced points nearly level along the ray); a row whose increments differ by */
/* more than a factor HERM_RATIO uses the second-order weights (a = g = 0).     */
/* Returns u at row io (every row in u_all if not NULL); M = 0: u = I.          */
/* ------------------------------------------------------------------------- */
#define HERM_RATIO 64.0

double orc_feautrier4(int64_t M, const double *dtau, const double *S, int64_t io, double I, double *u_all)
{
    if (M == 0) {
        if (u_all) u_all[0] = I;
        return I;
    }
    double *F = (double *)malloc(sizeof(double) * (size_t)M);
    double *z = (double *)malloc(sizeof(double) * (size_t)M);
    double *u = u_all ? u_all : (double *)malloc(sizeof(double) * (size_t)(M + 1));
    {   /* boundary row 0 */
        const double h = dtau[0];
        const double c0 = 2.0 / (h * h) - 1.0 / 3.0;
        const double B0 = 1.0 + 2.0 / h;
        const double r0 = 2.0 / 3.0 * S[0] + 1.0 / 3.0 * S[1] + 2.0 * I / h;
        F[0] = B0 / c0;
        z[0] = r0 / (c0 * (1.0 + F[0]));
    }
    for (int64_t i = 1; i < M; ++i) {
        const double hm = dtau[i - 1], hp = dtau[i], hs = hm + hp;
        const double A = 2.0 / (hm * hs), C = 2.0 / (hp * hs);
        double wa = (hm * hm + hm * hp - hp * hp) / (6.0 * hm * hs);
        double wg = (hp * hp + hm * hp - hm * hm) / (6.0 * hp * hs);
        if (hp > HERM_RATIO * hm || hm > HERM_RATIO * hp) wa = wg = 0.0;  /* second-order row */
        const double a = A - wa, c = C - wg;
        /* a S_{i-1} + b S_i + g S_{i+1} with b = 1 - a - g, written on the
         * differences: next to a vanishing increment the weights grow like the
         * ratio of the increments and b = 1 - a - g would cancel */
        const double r = S[i] + wa * (S[i - 1] - S[i]) + wg * (S[i + 1] - S[i]);
        F[i] = (1.0 + a * F[i - 1] / (1.0 + F[i - 1])) / c;
        z[i] = (r + a * z[i - 1]) / (c * (1.0 + F[i]));
    }
    {   /* boundary row M */
        const double h = dtau[M - 1];
        const double aM = 2.0 / (h * h) - 1.0 / 3.0;
        const double BM = 1.0 + 2.0 / h;
        const double rM = 2.0 / 3.0 * S[M] + 1.0 / 3.0 * S[M - 1] + 2.0 * I / h;
        u[M] = (rM + aM * z[M - 1]) / (BM + aM * F[M - 1] / (1.0 + F[M - 1]));
    }
    for (int64_t i = M - 1; i >= 0; --i) u[i] = u[i + 1] / (1.0 + F[i]) + z[i];
    const double uo = u[io];
    free(F);
    free(z);
    if (!u_all) free(u);
    return uo;
}

/* ------------------------------------------------------------------------- */
/* One pair line for one bin, exposed for the tests: fills dtau[0..M), S[0..M]  */
/* and returns M (and the origin row in *io), or -1 on overflow of max_pts.      */
/* ------------------------------------------------------------------------- */
int64_t orc_pair_line(const orc_model *m, const orc_params *pr, int64_t o, uint32_t ray,
                      int32_t l, int32_t k, int64_t max_pts, double *dtau, double *S, int64_t *io)
{
    double r[3];
    orc_pix2vec_nest((int)(ray >> 28), (int64_t)(ray & 0x0FFFFFFFu), r);
    orc_vline v;
    build_vline(m, pr, o, r, &v);
    double *chi = (double *)malloc(sizeof(double) * (size_t)v.m);
    double *eta = (double *)malloc(sizeof(double) * (size_t)v.m);
    line_optics(m, &v, m->dvw[o], l, k, chi, eta);
    const int64_t M = orc_subdivide_v(&v, chi, eta, pr, max_pts, dtau, S, io);
    free(chi);
    free(eta);
    vline_free(&v);
    return M;
}

/* Sizes of the velocity-sampled line (number of samples and origin index). */
int64_t orc_vline_size(const orc_model *m, const orc_params *pr, int64_t o, uint32_t ray, int64_t *io)
{
    double r[3];
    orc_pix2vec_nest((int)(ray >> 28), (int64_t)(ray & 0x0FFFFFFFu), r);
    orc_vline v;
    build_vline(m, pr, o, r, &v);
    const int64_t mv = v.m;
    *io = v.io;
    vline_free(&v);
    return mv;
}

/* ------------------------------------------------------------------------- */
/* Mean intensity (Eq. 3 and Eq. 4): J_o(nu) = sum over rays w u = sum over     */
/* pairs 2 w_l u, w_l = 1/(12 4^l), accumulated in ascending pair order with     */
/* Neumaier's compensated summation.  J_out[no][L * n_freq], bin index l*F + k. */
/* Returns 0, or -1 if a sub-divided line exceeds max_pts.                      */
/* ------------------------------------------------------------------------- */
/* J of the given origins (J_out [n_orig][L*F], may be NULL) and, when u_out is */
/* not NULL, u at the origin of every pair line (u_out [n_orig][pairs][L*F]).   */
static int solve_origins(const orc_model *m, const orc_params *pr, int64_t n_orig, const int64_t *origins,
                         int64_t max_pts, double *J_out, double *u_out, int threads)
{
    const int64_t np = orc_rayset_npairs(m->l_min, m->l_max);
    const int L = m->n_lines, F = m->n_freq, nb = L * F;
    if (L < 1 || L > ORC_MAX_LINES || F < 1) return -1;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads) reduction(| : bad)
    for (int64_t q = 0; q < n_orig; ++q) {
        const int64_t o = origins[q];
        double *sum = (double *)calloc((size_t)nb, sizeof(double));
        double *comp = (double *)calloc((size_t)nb, sizeof(double));
        double *dtau = (double *)malloc(sizeof(double) * (size_t)max_pts);
        double *S = (double *)malloc(sizeof(double) * (size_t)(max_pts + 1));
        double *chi = NULL, *eta = NULL;
        for (int64_t p = 0; p < np && !bad; ++p) {
            const uint32_t ray = m->rays[o * np + p];
            const int lev = (int)(ray >> 28);
            double r[3];
            orc_pix2vec_nest(lev, (int64_t)(ray & 0x0FFFFFFFu), r);
            const double w2 = 2.0 / (double)orc_npix(lev);
            orc_vline v;
            build_vline(m, pr, o, r, &v);
            chi = (double *)realloc(chi, sizeof(double) * (size_t)v.m);
            eta = (double *)realloc(eta, sizeof(double) * (size_t)v.m);
            for (int l = 0; l < L; ++l)
                for (int k = 0; k < F; ++k) {
                    line_optics(m, &v, m->dvw[o], l, k, chi, eta);
                    int64_t io = 0;
                    const int64_t M = orc_subdivide_v(&v, chi, eta, pr, max_pts, dtau, S, &io);
                    if (M < 0) {
                        bad = 1;
                        break;
                    }
                    const double uo = pr->order == 4 ? orc_feautrier4(M, dtau, S, io, pr->I_bdy, NULL)
                                                     : orc_feautrier(M, dtau, S, io, pr->I_bdy, NULL);
                    const double x = w2 * uo;
                    const int b = l * F + k;
                    if (u_out) u_out[(q * np + p) * nb + b] = uo;
                    const double t = sum[b] + x;
                    if (fabs(sum[b]) >= fabs(x)) comp[b] += (sum[b] - t) + x;
                    else comp[b] += (x - t) + sum[b];
                    sum[b] = t;
                }
            vline_free(&v);
        }
        if (J_out)
            for (int b = 0; b < nb; ++b) J_out[q * nb + b] = sum[b] + comp[b];
        free(sum); free(comp); free(dtau); free(S); free(chi); free(eta);
    }
    return bad ? -1 : 0;
}

int orc_solve_J(const orc_model *m, const orc_params *pr, int64_t n_orig, const int64_t *origins,
                int64_t max_pts, double *J_out, int threads)
{
    return solve_origins(m, pr, n_orig, origins, max_pts, J_out, NULL, threads);
}

/* u at the origin of every pair line of the given origins, [n_orig][pairs][L*F]
 * (the per-ray mean intensity that J weights with Eq. 4). */
int orc_solve_u(const orc_model *m, const orc_params *pr, int64_t n_orig, const int64_t *origins,
                int64_t max_pts, double *u_out, int threads)
{
    return solve_origins(m, pr, n_orig, origins, max_pts, NULL, u_out, threads);
}

/* ------------------------------------------------------------------------- */
/* Mesh-reduction criterion (Section 2.2.2, Eqs. 6-8, Table 1).                */
/*   Gf_i = max_n |(f_i - f_n)/(f_i + f_n)|   (0 where f_i + f_n = 0)           */
/*   L_i  = mean_n |x_i - x_n|                                                  */
/*   ell_i = L_i f_small if Gf_i >= G_thres, else L_i f_large                    */
/* Reading (Gmsh is not available): the re-mesh is replaced by thinning; point */
/* i is kept when u_i < min(1, (L_i/ell_i)^3), u_i = splitmix64 uniform of      */
/* (seed, i) (Steele, Lea & Flood 2014); points without neighbours are kept.    */
/* ------------------------------------------------------------------------- */
double orc_uniform01(uint64_t seed, int64_t i)
{
    uint64_t z = seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z = z ^ (z >> 31);
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

void orc_reduce(int64_t n, const double *pos, const int64_t *nbr_off, const int32_t *nbr_idx,
                const double *f, double f_small, double f_large, double G_thres, uint64_t seed,
                double *Gf, double *L, double *ell, uint8_t *keep)
{
    for (int64_t i = 0; i < n; ++i) {
        double g = 0.0, sum = 0.0;
        const int64_t deg = nbr_off[i + 1] - nbr_off[i];
        for (int64_t e = nbr_off[i]; e < nbr_off[i + 1]; ++e) {
            const int64_t j = nbr_idx[e];
            const double den = f[i] + f[j];
            const double gi = den == 0.0 ? 0.0 : fabs((f[i] - f[j]) / den);
            if (gi > g) g = gi;
            const double dx = pos[3 * i] - pos[3 * j], dy = pos[3 * i + 1] - pos[3 * j + 1],
                         dz = pos[3 * i + 2] - pos[3 * j + 2];
            sum += sqrt((dx * dx + dy * dy) + dz * dz);
        }
        const double Li = deg > 0 ? sum / (double)deg : 0.0;
        const double fac = (g >= G_thres) ? f_small : f_large;
        Gf[i] = g;
        L[i] = Li;
        ell[i] = Li * fac;
        const double p = 1.0 / (fac * fac * fac);
        keep[i] = (deg == 0 || orc_uniform01(seed, i) < p) ? 1 : 0;
    }
}

/* ------------------------------------------------------------------------- */
/* Element-size field of an analytic model (Section 2.2.1, Eq. 5).           */
/* f > 0 is the tracer on a regular Cartesian background mesh of spacing h,  */
/* index (i ny + j) nz + k.  Gf = max_n n.grad f / f = ||grad f|| / f, the    */
/* gradient by central differences (first differences on the faces, 0 along */
/* an axis with one point); ell maps [max Gf, min Gf] linearly onto         */
/* [ell_min, ell_max] (all ell_max when Gf is constant).  Reading (Gmsh is   */
/* not available): the mesh is the background mesh (density h^-3) thinned to */
/* the density ell^-3, point i kept when u_i < (h / ell_i)^3, u_i the        */
/* SplitMix64 uniform of (seed, i) as in the reduction (h <= ell_min).       */
/* Returns the number kept.                                                   */
/* ------------------------------------------------------------------------- */
static double axis_diff(const double *f, int64_t idx, int64_t stride, int32_t pos, int32_t n, double h)
{
    if (n < 2) return 0.0;
    if (pos == 0) return (f[idx + stride] - f[idx]) / h;
    if (pos == n - 1) return (f[idx] - f[idx - stride]) / h;
    return (f[idx + stride] - f[idx - stride]) / (2.0 * h);
}

int64_t orc_analytic_mesh(int32_t nx, int32_t ny, int32_t nz, const double *f, double h, double ell_min,
                          double ell_max, uint64_t seed, double *Gf, double *ell, uint8_t *keep)
{
    const int64_t n = (int64_t)nx * ny * nz;
    double gmin = INFINITY, gmax = -INFINITY;
    for (int32_t i = 0; i < nx; ++i)
        for (int32_t j = 0; j < ny; ++j)
            for (int32_t k = 0; k < nz; ++k) {
                const int64_t q = ((int64_t)i * ny + j) * nz + k;
                const double gx = axis_diff(f, q, (int64_t)ny * nz, i, nx, h);
                const double gy = axis_diff(f, q, nz, j, ny, h);
                const double gz = axis_diff(f, q, 1, k, nz, h);
                Gf[q] = sqrt(gx * gx + gy * gy + gz * gz) / f[q];
                if (Gf[q] < gmin) gmin = Gf[q];
                if (Gf[q] > gmax) gmax = Gf[q];
            }
    int64_t kept = 0;
    for (int64_t q = 0; q < n; ++q) {
        ell[q] = gmax > gmin ? ell_max - (Gf[q] - gmin) * (ell_max - ell_min) / (gmax - gmin) : ell_max;
        const double r = h / ell[q];
        keep[q] = orc_uniform01(seed, q) < r * r * r ? 1 : 0;
        kept += keep[q];
    }
    return kept;
}
