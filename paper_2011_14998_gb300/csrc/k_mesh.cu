// k_mesh.cu -- ingest of the point cloud, neighbour graph and line data
// (Section 2.2: Magritte needs "a point cloud and nearest neighbour
// information").  The caller's array-of-structures input is split into
// structure-of-arrays device copies (double for tracing, float copies for the
// single-precision solve), and every value is range-checked on the device.
#include "mgx_internal.cuh"

namespace mgx {

__global__ void k_ingest_points(int32_t n, const double *__restrict__ pos,
                                const double *__restrict__ vel, const int64_t *__restrict__ off64,
                                int64_t E, double *x, double *y, double *z, double *vx, double *vy,
                                double *vz, float *vxf, float *vyf, float *vzf, int32_t *off32,
                                float4 *phi, unsigned int *xmax_bits, int *status) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i > n) return;
    const int64_t o = off64[i];
    if (o < 0 || o > E || (i < n && off64[i + 1] < o)) dev_fail(status, kDevBadCsr);
    off32[i] = int32_t(o);
    if (i == n) return;
    const double px = pos[3 * i], py = pos[3 * i + 1], pz = pos[3 * i + 2];
    const double ux = vel[3 * i], uy = vel[3 * i + 1], uz = vel[3 * i + 2];
    if (!isfinite(px) || !isfinite(py) || !isfinite(pz) || !isfinite(ux) || !isfinite(uy) ||
        !isfinite(uz) || fabs(px) > 1e30 || fabs(py) > 1e30 || fabs(pz) > 1e30)
        dev_fail(status, kDevNonFinite);
    x[i] = px;
    y[i] = py;
    z[i] = pz;
    vx[i] = ux;
    vy[i] = uy;
    vz[i] = uz;
    vxf[i] = float(ux);
    vyf[i] = float(uy);
    vzf[i] = float(uz);
    phi[i] = make_float4(__double2float_rn(px), __double2float_rn(py), __double2float_rn(pz), 0.0f);
    const float s = __double2float_ru(fabs(px) + fabs(py) + fabs(pz));
    if (isfinite(s)) atomicMax(xmax_bits, __float_as_uint(s));  // non-negative: bit order = value order
}

__global__ void k_check_nbr(int32_t n, const int32_t *__restrict__ off, const int32_t *__restrict__ nbr,
                            int *status) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    for (int32_t e = off[i]; e < off[i + 1]; ++e) {
        const int32_t j = nbr[e];
        if (j < 0 || j >= n || j == i) dev_fail(status, kDevBadCsr);
    }
}

void launch_ingest_mesh(int32_t n, const double *pos_aos, const double *vel_aos, const int64_t *off64,
                        int64_t E, double *x, double *y, double *z, double *vx, double *vy,
                        double *vz, float *vxf, float *vyf, float *vzf, int32_t *off32,
                        const int32_t *nbr, float4 *phi, unsigned int *xmax_bits, int *status,
                        cudaStream_t st) {
    const int tb = 256;
    k_ingest_points<<<unsigned((n + 1 + tb - 1) / tb), tb, 0, st>>>(
        n, pos_aos, vel_aos, off64, E, x, y, z, vx, vy, vz, vxf, vyf, vzf, off32, phi, xmax_bits, status);
    k_check_nbr<<<unsigned((n + tb - 1) / tb), tb, 0, st>>>(n, off32, nbr, status);
}

// neighbour records for the tracer's single-precision screen: the float
// position of nbr[e] minus the float position of its point, next to its id, in
// CSR order (the spare record after the last stays zero)
__global__ void k_pack_neighbours(int32_t n, const int32_t *__restrict__ off, const int32_t *__restrict__ nbr,
                                  float4 *__restrict__ phi, float4 *__restrict__ nrec) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    const float4 hi = phi[i];
    float smax = 0.0f;
    for (int32_t e = off[i]; e < off[i + 1]; ++e) {
        const int32_t j = nbr[e];
        const float4 h = phi[j];
        // x_j - x_i exactly as the tracer's screen forms it (differences of the float positions)
        const float dx = h.x - hi.x, dy = h.y - hi.y, dz = h.z - hi.z;
        nrec[e] = make_float4(dx, dy, dz, __int_as_float(j));
        smax = fmaxf(smax, fabsf(dx) + fabsf(dy) + fabsf(dz));
    }
    phi[i].w = smax;  // only w: the positions other threads read stay as they are
}

void launch_pack_neighbours(int32_t n, const int32_t *off, const int32_t *nbr, float4 *phi, float4 *nrec,
                            cudaStream_t st) {
    const int tb = 256;
    k_pack_neighbours<<<unsigned((n + tb - 1) / tb), tb, 0, st>>>(n, off, nbr, phi, nrec);
}

__global__ void k_ingest_lines(int32_t n, int32_t L, const double *__restrict__ chi0,
                               const double *__restrict__ eta0, const double *__restrict__ dvw,
                               const double *__restrict__ chic, const double *__restrict__ etac,
                               float *chi0f, float *eta0f, float *dvwf, float *chicf, float *etacf,
                               int *status) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    for (int l = 0; l < L; ++l) {
        const double c = chi0[i * L + l], e = eta0[i * L + l];
        if (!(c >= 0.0) || !(e >= 0.0) || !isfinite(c) || !isfinite(e)) dev_fail(status, kDevBadInput);
        chi0f[i * L + l] = float(c);
        eta0f[i * L + l] = float(e);
    }
    const double w = dvw[i], cc = chic[i], ec = etac[i];
    if (!(w > 0.0) || !(cc > 0.0) || !(ec >= 0.0) || !isfinite(w) || !isfinite(cc) || !isfinite(ec))
        dev_fail(status, kDevBadInput);
    dvwf[i] = float(w);
    chicf[i] = float(cc);
    etacf[i] = float(ec);
}

void launch_ingest_lines(int32_t n, int32_t L, const double *chi0, const double *eta0,
                         const double *dvw, const double *chic, const double *etac, float *chi0f,
                         float *eta0f, float *dvwf, float *chicf, float *etacf, int *status,
                         cudaStream_t st) {
    const int tb = 256;
    k_ingest_lines<<<unsigned((n + tb - 1) / tb), tb, 0, st>>>(n, L, chi0, eta0, dvw, chic, etac,
                                                               chi0f, eta0f, dvwf, chicf, etacf,
                                                               status);
}

}  // namespace mgx
