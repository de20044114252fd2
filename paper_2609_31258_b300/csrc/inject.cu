// Source sampling ("Continuous current Gaussian source"): packs placed on the
// source plane (or, for a prefill, uniformly in z), transverse position
// uniform over a disc or from a Gaussian truncated at the hard radius
// (inverse CDF of the truncated Rayleigh law), Maxwellian velocity at T_vel
// with v_z folded to >= 0 on request, E_int = E_int(T_init), and the
// Exp(1) optical depth to the first collision candidate. FP64 arithmetic;
// Philox counter (pack id, 0, block, 1).
#include "kernels.cuh"

namespace mucite {


__device__ __forceinline__ int32_t q32i(double v)
{
    const double r = rint(v);
    if (r < -2147483648.0) return INT32_MIN;
    if (r > 2147483647.0) return INT32_MAX;
    return (int32_t)r;
}

__global__ void inject_kernel(InjectArgs A)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= A.count) return;
    const int64_t p = A.p0 + t;
    const uint4 a = philox10(make_uint4((uint32_t)p, 0u, 0u, 1u), A.key0, A.key1);
    const uint4 b = philox10(make_uint4((uint32_t)p, 0u, 1u, 1u), A.key0, A.key1);
    const uint4 c = philox10(make_uint4((uint32_t)p, 0u, 2u, 1u), A.key0, A.key1);
    const double tau = -log(u01d(c.x));
    double r;
    if (A.profile == 0) {
        r = A.radius * sqrt(u01d(a.x));
    } else {
        const double tail = expm1(-A.radius * A.radius / (2.0 * A.sigma * A.sigma));
        r = A.sigma * sqrt(-2.0 * log1p(u01d(a.x) * tail));
    }
    double sn, cs;
    sincospi(2.0 * u01d(a.y), &sn, &cs);
    const double x = r * cs, y = r * sn;
    const double z = A.prefill ? A.pz0 + (A.pz1 - A.pz0) * u01d(a.z) : A.z_plane;
    const double r01 = sqrt(-2.0 * log(u01d(b.x))), r23 = sqrt(-2.0 * log(u01d(b.z)));
    double sn1, cs1;
    sincospi(2.0 * u01d(b.y), &sn1, &cs1);
    const double vx = A.sd * r01 * cs1, vy = A.sd * r01 * sn1;
    double vz = A.sd * r23 * cospi(2.0 * u01d(b.w));
    if (A.half_space) vz = fabs(vz);
    if (A.precision == MUCITE_FP32) {
        const double sx = kLat / A.R, sz = kLat / (A.gz1 - A.gz0);
        ((int32_t *)A.x)[p] = q32i(x * sx);
        ((int32_t *)A.y)[p] = q32i(y * sx);
        ((int32_t *)A.z)[p] = q32i((z - A.gz0) * sz);
        ((float *)A.vx)[p] = (float)vx;
        ((float *)A.vy)[p] = (float)vy;
        ((float *)A.vz)[p] = (float)vz;
        ((float *)A.eint)[p] = (float)A.e0;
        ((float *)A.lnsy)[p] = 0.0f;
        ((float *)A.tau)[p] = (float)tau;
    } else {
        ((double *)A.x)[p] = x;
        ((double *)A.y)[p] = y;
        ((double *)A.z)[p] = z;
        ((double *)A.vx)[p] = vx;
        ((double *)A.vy)[p] = vy;
        ((double *)A.vz)[p] = vz;
        ((double *)A.eint)[p] = A.e0;
        ((double *)A.lnsy)[p] = 0.0;
        ((double *)A.tau)[p] = tau;
    }
    A.status[p] = MUCITE_ACTIVE;
    A.t_term[p] = -1;
}

void launch_inject(const InjectArgs &A, cudaStream_t s)
{
    if (A.count <= 0) return;
    inject_kernel<<<(unsigned)((A.count + 255) / 256), 256, 0, s>>>(A);
}

} // namespace mucite
