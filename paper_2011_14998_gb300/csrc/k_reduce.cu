// k_reduce.cu -- mesh-reduction criterion (Section 2.2.2, Eqs. 6-8, Table 1).
//
// One thread per point walks its neighbour list once:
//   Gf_i = max_n |(f_i - f_n)/(f_i + f_n)|  (0 where f_i + f_n = 0)     Eq. 6
//   L_i  = mean_n |x_i - x_n|                                           Eq. 8
//   ell_i = L_i * (f_small if Gf_i >= G_thres else f_large)             Eq. 7
// and thins the mesh in place of the paper's Gmsh re-meshing: keep i when
// u_i < min(1, (L_i/ell_i)^3), u_i the SplitMix64 uniform of (seed, i), or when
// i has no neighbours.  Operations are explicitly rounded, so the outputs are
// reproducible bit for bit.
#include "mgx_internal.cuh"

namespace mgx {

namespace {

__global__ void k_reduce(DevMesh m, const double *__restrict__ f, double f_small, double f_large,
                         double G_thres, uint64_t seed, double *Gf, double *L, double *ell,
                         uint8_t *keep) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= m.n) return;
    const double fi = f[i];
    const double xi = m.x[i], yi = m.y[i], zi = m.z[i];
    double g = 0.0, sum = 0.0;
    const int32_t e0 = m.off[i], e1 = m.off[i + 1];
    for (int32_t e = e0; e < e1; ++e) {
        const int32_t j = __ldg(m.nbr + e);
        const double fj = __ldg(f + j);
        const double den = __dadd_rn(fi, fj);
        const double gj = den == 0.0 ? 0.0 : fabs(__ddiv_rn(__dsub_rn(fi, fj), den));
        if (gj > g) g = gj;
        const double dx = __dsub_rn(xi, __ldg(m.x + j));
        const double dy = __dsub_rn(yi, __ldg(m.y + j));
        const double dz = __dsub_rn(zi, __ldg(m.z + j));
        sum = __dadd_rn(sum, __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                                                  __dmul_rn(dz, dz))));
    }
    const int32_t deg = e1 - e0;
    const double Li = deg > 0 ? __ddiv_rn(sum, double(deg)) : 0.0;
    const double fac = (g >= G_thres) ? f_small : f_large;
    const double p = __ddiv_rn(1.0, __dmul_rn(__dmul_rn(fac, fac), fac));
    if (Gf) Gf[i] = g;
    if (L) L[i] = Li;
    if (ell) ell[i] = __dmul_rn(Li, fac);
    keep[i] = (deg == 0 || splitmix_uniform(seed, i) < p) ? 1 : 0;
}

}  // namespace

void launch_reduce(const DevMesh &m, const double *f, double f_small, double f_large, double G_thres,
                   uint64_t seed, double *Gf, double *L, double *ell, uint8_t *keep, cudaStream_t st) {
    const int tb = 256;
    k_reduce<<<unsigned((m.n + tb - 1) / tb), tb, 0, st>>>(m, f, f_small, f_large, G_thres, seed, Gf, L,
                                                          ell, keep);
}

}  // namespace mgx
