// Field loading on the device: E = -grad(phi) by central differences of the
// baked potentials (the paper derives E from the baked potentials; its
// spline derivative is read as second-order central differences, one-sided
// at the domain edges, E_r = 0 on the symmetry axis), then packing of the
// FP32 node records and the FP32 mask/distance field ("Gas field and
// electrode mask coupling").
#include "common.cuh"

namespace mucite {

__global__ void efield_kernel(const double *__restrict__ phi, int nr, int nz, double dr, double dz,
                              double *__restrict__ er, double *__restrict__ ez)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)nr * nz) return;
    const int i = (int)(idx % nr), j = (int)(idx / nr);
    const double *row = phi + (size_t)j * nr;
    double dpr;
    if (i == 0) dpr = 0.0;
    else if (i == nr - 1) dpr = (row[i] - row[i - 1]) / dr;
    else dpr = (row[i + 1] - row[i - 1]) / (2.0 * dr);
    double dpz;
    if (j == 0) dpz = (phi[idx + nr] - phi[idx]) / dz;
    else if (j == nz - 1) dpz = (phi[idx] - phi[idx - nr]) / dz;
    else dpz = (phi[idx + nr] - phi[idx - nr]) / (2.0 * dz);
    er[idx] = -dpr;
    ez[idx] = -dpz;
}

__global__ void pack_nodes_kernel(const double *er_dc, const double *ez_dc, const double *er_rf,
                                  const double *ez_rf, const double *p, const double *T,
                                  const double *ur, const double *uz, const uint8_t *mask,
                                  const double *dist, int n, NodeF *node, float *dmask)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    NodeF nd;
    nd.a = make_float4((float)er_dc[idx], (float)ez_dc[idx], (float)er_rf[idx], (float)ez_rf[idx]);
    nd.b = make_float4((float)p[idx], (float)T[idx], (float)ur[idx], (float)uz[idx]);
    node[idx] = nd;
    dmask[idx] = mask[idx] ? -1.0f : (float)dist[idx];
}

void launch_efield(const double *phi, int nr, int nz, double dr, double dz, double *er, double *ez,
                   cudaStream_t s)
{
    const int64_t n = (int64_t)nr * nz;
    efield_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(phi, nr, nz, dr, dz, er, ez);
}

void launch_pack_nodes(const double *er_dc, const double *ez_dc, const double *er_rf,
                       const double *ez_rf, const double *p, const double *T, const double *ur,
                       const double *uz, const uint8_t *mask, const double *dist, int n,
                       NodeF *node, float *dmask, cudaStream_t s)
{
    pack_nodes_kernel<<<(n + 255) / 256, 256, 0, s>>>(er_dc, ez_dc, er_rf, ez_rf, p, T, ur, uz, mask,
                                                      dist, n, node, dmask);
}

} // namespace mucite
