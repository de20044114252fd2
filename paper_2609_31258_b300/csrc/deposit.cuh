// Charge deposit of one pack on the int32 position lattice (cloud in cell on
// the axisymmetric PIC grid, Methods "Axisymmetric PIC space charge update"),
// shared by the standalone deposit kernel and the step kernels' end-of-launch
// deposit. Integer arithmetic throughout, so every caller produces the same
// contributions bit for bit.
#pragma once
#include "common.cuh"

namespace mucite {

// floor(sqrt(v)) for v < 2^62, exact. An FP32 estimate (within ~2^-23
// relative, i.e. below 2^8 for v < 2^62) refined by one Newton correction
// from the exact integer residual v - r0^2 leaves r within 1 of the answer;
// the integer tests settle it. FP32 keeps the deposit off the slow FP64 pipe.
__device__ __forceinline__ uint64_t isqrt_floor(uint64_t v)
{
    if (v == 0) return 0;
    const uint64_t r0 = (uint64_t)__fsqrt_rn((float)v);
    const int64_t e = (int64_t)(v - r0 * r0); // |e| <= 2^9 r0 + 2^16, exact in 64 bits
    int64_t r = (int64_t)r0 + (int64_t)__float2ll_rn((float)e / (2.0f * (float)r0));
    if (r < 0) r = 0;
    uint64_t u = (uint64_t)r;
    while (u * u > v) --u;
    while ((u + 1) * (u + 1) <= v) ++u;
    return u;
}

// Cell (j * pnr + i of its lower-left node) and the four CIC contributions
// (i, j), (i+1, j), (i, j+1), (i+1, j+1) of a pack at lattice position
// (xq, yq, zq) with charge-weight product qw, in units of e * 2^-30: the
// lattice radius r = floor(sqrt(xq^2 + yq^2)) and z map onto the PIC nodes
// through integer products, 15-bit fractions. False when the pack is outside
// the PIC box.
__device__ __forceinline__ bool cic_lattice(int32_t xq, int32_t yq, int32_t zq, int pnr, int pnz, int64_t qw,
                                            uint32_t &cell, unsigned long long w[4])
{
    const uint64_t r2 = (uint64_t)((int64_t)xq * xq) + (uint64_t)((int64_t)yq * yq);
    const uint64_t r = isqrt_floor(r2);
    if (r >= (1ULL << 30) || zq < 0 || zq > (1 << 30)) return false;
    const uint64_t tr = r * (uint64_t)(pnr - 1);
    const uint64_t tz = (uint64_t)zq * (uint64_t)(pnz - 1);
    int64_t i = (int64_t)(tr >> 30), j = (int64_t)(tz >> 30);
    int64_t fr = (int64_t)((tr & ((1ULL << 30) - 1)) >> 15);
    int64_t fz = (int64_t)((tz & ((1ULL << 30) - 1)) >> 15);
    if (i > pnr - 2) { i = pnr - 2; fr = 1 << 15; }
    if (j > pnz - 2) { j = pnz - 2; fz = 1 << 15; }
    const int64_t wr0 = (1 << 15) - fr, wr1 = fr, wz0 = (1 << 15) - fz, wz1 = fz;
    cell = (uint32_t)(j * pnr + i);
    w[0] = (unsigned long long)(qw * wr0 * wz0);
    w[1] = (unsigned long long)(qw * wr1 * wz0);
    w[2] = (unsigned long long)(qw * wr0 * wz1);
    w[3] = (unsigned long long)(qw * wr1 * wz1);
    return true;
}

} // namespace mucite
