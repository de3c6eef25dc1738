// hpx_host.cpp -- host-side HEALPix tables for the ray sets (Section 2.1.3).
//
// Pixel-centre directions are evaluated once per level on the host with the C
// library's sqrt/cos/sin, in double precision and without contraction
// (compiled with -ffp-contract=off), so the tracer walks exactly the directions
// the closed forms of Gorski et al. (2005) give:
//   ring i < nside (north cap):  z = 1 - i^2/(3 nside^2),   phi = (j - 1/2) pi/(2i)
//   nside <= i <= 3 nside (belt): z = 2 (2 nside - i)/(3 nside),
//                                phi = (j - (1 + s)/2) pi/(2 nside), s = (i - nside) mod 2
//   south cap by symmetry; the unit vector is (sin t cos phi, sin t sin phi, z)
//   with sin t = sqrt((1 - z)(1 + z)).
#include <cmath>
#include <cstdint>

#include "mgx_internal.cuh"

namespace mgx {

namespace {

// southern-corner ring of each base face in units of nside, and its longitude
// column in units of pi/4 (the 12 base pixels of the HEALPix sphere)
constexpr int64_t kFaceRing[12] = {2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4};
constexpr int64_t kFaceCol[12] = {1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7};

int64_t deinterleave(int64_t v) {
    int64_t out = 0;
    for (int b = 0; b < 31; ++b) out |= ((v >> (2 * b)) & 1) << b;
    return out;
}

int64_t interleave(int64_t v) {
    int64_t out = 0;
    for (int b = 0; b < 31; ++b) out |= ((v >> b) & 1) << (2 * b);
    return out;
}

}  // namespace

int64_t hpx_npix(int l) { return int64_t(12) << (2 * l); }

void hpx_pix2vec(int l, int64_t p, double v[3]) {
    const int64_t ns = int64_t(1) << l;
    const int64_t face = p >> (2 * l);
    const int64_t local = p & ((ns * ns) - 1);
    const int64_t x = deinterleave(local);
    const int64_t y = deinterleave(local >> 1);
    const int64_t ring = kFaceRing[face] * ns - x - y - 1;
    int64_t nr = ns, s = 0;
    double z;
    if (ring < ns) {
        nr = ring;
        z = 1.0 - double(nr * nr) / double(3 * ns * ns);
    } else if (ring > 3 * ns) {
        nr = 4 * ns - ring;
        z = double(nr * nr) / double(3 * ns * ns) - 1.0;
    } else {
        s = (ring - ns) & 1;
        z = double(2 * (2 * ns - ring)) / double(3 * ns);
    }
    int64_t j = (kFaceCol[face] * nr + x - y + 1 + s) / 2;
    if (j > 4 * nr) j -= 4 * nr;
    if (j < 1) j += 4 * nr;
    const double phi = double(2 * j - 1 - s) * M_PI / double(4 * nr);
    const double sint = std::sqrt((1.0 - z) * (1.0 + z));
    v[0] = sint * std::cos(phi);
    v[1] = sint * std::sin(phi);
    v[2] = z;
}

// Pixel of level l containing direction d; used on the host only to pair each
// pixel with its antipode (pixel centres lie well inside their pixels).
int64_t hpx_vec2pix(int l, const double d[3]) {
    const int64_t ns = int64_t(1) << l;
    const double len = std::sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
    const double z = d[2] / len;
    double t = std::atan2(d[1], d[0]) * M_2_PI;
    if (t < 0.0) t += 4.0;
    if (t >= 4.0) t -= 4.0;
    int64_t face, x, y;
    if (std::fabs(z) <= 2.0 / 3.0) {
        const double a = double(ns) * (0.5 + t);
        const double b = double(ns) * (0.75 * z);
        const int64_t asc = int64_t(a - b), dsc = int64_t(a + b);
        const int64_t fa = asc >> l, fd = dsc >> l;
        face = (fa == fd) ? (fa | 4) : (fa < fd ? fa : fd + 8);
        x = dsc & (ns - 1);
        y = ns - 1 - (asc & (ns - 1));
    } else {
        int64_t q = int64_t(t);
        if (q > 3) q = 3;
        const double tp = t - double(q);
        const double w = double(ns) * std::sqrt(3.0 * (1.0 - std::fabs(z)));
        int64_t a = int64_t(tp * w), b = int64_t((1.0 - tp) * w);
        if (a > ns - 1) a = ns - 1;
        if (b > ns - 1) b = ns - 1;
        if (z >= 0.0) {
            face = q;
            x = ns - 1 - b;
            y = ns - 1 - a;
        } else {
            face = q + 8;
            x = a;
            y = b;
        }
    }
    return (face << (2 * l)) + interleave(x) + 2 * interleave(y);
}

int64_t rayset_npairs(int lmin, int lmax) {
    if (lmin < 0 || lmax < lmin) return -1;
    if (lmin == lmax) return hpx_npix(lmin) / 2;
    int64_t cand = hpx_npix(lmin) / 2, rays = 0;
    for (int l = lmin; l < lmax; ++l) {
        rays += cand / 2;       // bottom half stays at level l
        cand = (cand / 2) * 4;  // each refined pair has four child pairs
    }
    return rays + cand;
}

}  // namespace mgx
