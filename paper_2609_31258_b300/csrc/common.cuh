// Shared device-side definitions of the MuCITE B300 library: physical
// constants, the Philox4x32-10 counter-based generator, the fixed-point
// position lattice and the per-instance parameter blocks the kernels read.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mucite.h"

namespace mucite {

constexpr double kE = 1.602176634e-19;     // elementary charge [C]
constexpr double kKB = 1.380649e-23;       // Boltzmann constant [J/K]
constexpr double kDa = 1.66053906660e-27;  // dalton [kg]
constexpr double kEps0 = 8.8541878128e-12; // vacuum permittivity [F/m]
constexpr double kPi = 3.14159265358979323846;
constexpr double kPlanck = 6.62607015e-34;           // Planck constant [J s]
constexpr double kR = 1.380649e-23 * 6.02214076e23;  // molar gas constant k_B N_A [J/(mol K)]
constexpr int kCounters = 4;            // per-instance device counters (InstF32::counters)
constexpr int kEagerWeight = 6;         // candidate weight of the eager collision schedule
constexpr double kLat = 1073741824.0;      // 2^30 lattice units per R (r) or per (z1 - z0) (z)
constexpr int kKmax = 32;                  // collision candidates examined per pack per step

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds, each taking
// two 32x32 -> 64-bit products of counter words 0 and 2 with the round
// multipliers, the key advanced by the two Weyl increments between rounds.
// Counter = (pack id, step, draw block, purpose); key = (seed lo, seed hi).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox_round(uint4 &c, uint32_t k0, uint32_t k1)
{
    // each product as one 32 x 32 -> 64-bit multiply
    const uint64_t p0 = (uint64_t)c.x * 0xD2511F53u;
    const uint64_t p1 = (uint64_t)c.z * 0xCD9E8D57u;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
}

__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        philox_round(c, k0, k1);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// One block with precomputed round keys.
__device__ __forceinline__ uint4 philox10(uint4 c, const uint2 *rk)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint2 k = rk[round];
        philox_round(c, k.x, k.y);
    }
    return c;
}

// Two blocks with precomputed round keys, rounds interleaved.
__device__ __forceinline__ void philox10x2(uint4 &a, uint4 &b, const uint2 *rk)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint2 k = rk[round];
        philox_round(a, k.x, k.y);
        philox_round(b, k.x, k.y);
    }
}

// Two blocks under the same key, rounds interleaved (one key schedule).
__device__ __forceinline__ void philox10x2(uint4 &a, uint4 &b, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        philox_round(a, k0, k1);
        philox_round(b, k0, k1);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// 23-bit uniform in (0,1): ((x >> 9) + 1/2) * 2^-23, exact in FP32 and FP64.
__device__ __forceinline__ float u01f(uint32_t x)
{
    return ((float)(x >> 9) + 0.5f) * (1.0f / 8388608.0f);
}
__device__ __forceinline__ double u01d(uint32_t x)
{
    return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0);
}

// Packed static-field node of the FP32 path: a = (Er_dc, Ez_dc, Er_rf, Ez_rf),
// b = (p, T, u_r, u_z). One 32-byte sector per node.
struct __align__(32) NodeF {
    float4 a;
    float4 b;
};

// Static grid as the FP32 step kernel sees it.
struct GridF32 {
    const NodeF *node;
    const float *dmask; // -1 at metal nodes, else surface distance [m]
    int nr, nz;
    float sr;           // (nr - 1) * 2^-30: lattice r -> grid units
};

// Static grid of the plain FP64 path (structure of arrays, FP64).
struct GridF64 {
    const double *er_dc, *ez_dc, *er_rf, *ez_rf, *gas_p, *gas_T, *gas_ur, *gas_uz;
    const float *dmask;
    int nr, nz;
    double R, z0, z1;
};

// Heat-capacity profile Cv/k_B = 3N min(1, c0 + c1 T): E_int(T) = 3N (c0 T +
// c1 T^2 / 2) below Tcap = (1 - c0)/c1, linear above.
struct Profile {
    double n3, c0, c1, tcap, ecap; // ecap per 3N
};

// Per-instance parameters of the fused FP32 step (one entry per instance in
// a device array; copied to shared memory by every block).
struct InstF32 {
    int32_t *xq, *yq, *zq;
    float *vx, *vy, *vz, *eint, *lnsy;
    float *tau;                // optical depth left until the next collision candidate
    uint8_t *status;
    int32_t *t_term;
    int64_t n_slots;
    int64_t step0;
    double v_rf, dtf, phi_rf;  // RF scalar V cos(2 pi frac(phase0 + (n - seg0) dt f) + phi), FP64
    double rf_phase0;          // RF phase (cycles) at the start of the current dt segment
    int64_t seg_step0;         // step count at the start of the current dt segment
    float *rf;                 // RF scalars of the launch at half-step spacing: [2k] step k, [2k+1] k + 1/2
    int rk4;                   // RK4 pusher instead of the leapfrog
    float kick;                // q e dt / m
    float dc_scale;
    float cxs, czs;            // dt * 2^30 / R, dt * 2^30 / (z1 - z0): velocity -> lattice step
    float dt;
    float psig;                // p_scale * sigma / k_B  (n sigma = psig * p / T)
    float s_coef;              // 2 k_B / m_gas  (s^2 = s_coef * T)
    float fM, fm;              // M/(M+m), m/(M+m)
    float mu_2kb;              // mu / (2 k_B): relative KE in kelvin units
    float g_coef;              // 2 k_B / mu
    float n3, inv_n3, c0, c1, tcap, ecap;
    int tst;                   // dissociation (Eq. 7) on
    float tst_a_dt, tst_b;     // k dt = tst_a_dt * T * exp(-tst_b / T)
    int langevin;              // hybrid Langevin branch on
    int64_t lv_zq0, lv_zq1;    // window on the z lattice
    float lv_switch;           // lambda dt threshold
    float lv_c;                // gamma = lv_c * (n sigma) * sqrt(T)
    float lv_kM;               // k_B / M
    uint32_t key0, key1;
    uint2 rkey[10];            // Philox round keys (key0 + r W0, key1 + r W1), r = 0..9, formed on
                               // the host once: the kernels read them instead of advancing the key
                               // between rounds
    int64_t zexit_q;           // first lattice z counted as crossed
    uint64_t rdet2;            // (floor(r_det / R * 2^30))^2
    float hit;                 // electrode-hit distance [m]
    const float4 *esc4;        // space-charge field per PIC cell: [cell][0] = (E_r, E_z) at its lower
                               // nodes (i, j), (i+1, j), [cell][1] at (i, j+1), (i+1, j+1); or NULL
    int pnr, pnz;
    float psr;                 // (pnr - 1) * 2^-30
    unsigned long long *dep_q; // charge grid the launch deposits its active packs into at the end, or NULL
    int64_t dep_qw;            // charge number * weight of a pack (its CIC contributions: dep_qw w_r w_z)
    unsigned long long *counters; // [0] pack-steps, [1] collisions, [2] candidate-cap hits,
                                  // [3] bounded device waits that gave up (warps)
    int hold_tile;                // test hook of the streamed kernel: block-local tile whose staged copies
                                  // are withheld (its waits then run out), -1 = none
};

// Per-instance parameters of the plain FP64 step.
struct InstF64 {
    double *x, *y, *z, *vx, *vy, *vz, *eint, *lnsy, *tau;
    uint8_t *status;
    int32_t *t_term;
    int64_t n_slots;
    double qm, dc_scale, dt, p_scale, sigma, M, mg, T_unused;
    Profile prof;
    int tst;
    double tst_a, tst_b;       // k = tst_a * T * exp(-tst_b / T)
    int langevin;
    double lv_z0, lv_z1, lv_switch;
    double q_abs;              // |q| e
    int rk4;
    uint64_t seed;
    int64_t zexit_q, rdet_q;
    float hit;
    const double *er_sc, *ez_sc;  // space-charge field on the PIC grid (FP64) or NULL
    int pnr, pnz;
    unsigned long long *counters;
};

// Kernel launchers (defined in the .cu files, called from api.cu).
void launch_efield(const double *phi, int nr, int nz, double dr, double dz, double *er, double *ez,
                   cudaStream_t s);
void launch_pack_nodes(const double *er_dc, const double *ez_dc, const double *er_rf,
                       const double *ez_rf, const double *p, const double *T, const double *ur,
                       const double *uz, const uint8_t *mask, const double *dist, int n,
                       NodeF *node, float *dmask, cudaStream_t s);

} // namespace mucite
