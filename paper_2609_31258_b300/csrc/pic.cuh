// Device-side descriptors of the space-charge solve (see pic.cu).
#pragma once

#include <algorithm>

#include "common.cuh"

namespace mucite {

// Fixed operator data of one PIC grid (shared by the instances using it).
struct PicGeom {
    int pnr, pnz, M, Nu;     // M = pnz - 2 axial unknowns, Nu = pnr - 1 radial unknowns
    double dr, dz;
    double bscale;           // -(e 2^-30) / (eps0 pi dz): node charge units -> right-hand side
    const float *S;          // [M][M] sin(pi j k / (M + 1)), j, k = 1..M
    const float *cp;         // [Nu][M] Thomas upper factors c_i / m_i(k)
    const float *invm;       // [Nu][M] 1 / m_i(k)
    const float *lo;         // [Nu] a_i (sub-diagonal)
    const double *a, *c, *A; // [Nu] FP64 operator coefficients
    const uint8_t *metal;    // [pnz][pnr] metal nodes (mask-aware solve) or NULL
};

// Per-instance buffers of the space-charge solve.
struct PicInst {
    unsigned long long *Q;   // [pnz][pnr] node charge, units e * 2^-30
    double *phi;             // [pnz][pnr] potential (zero on the Dirichlet boundary)
    float *r32;              // [M][Nu] residual in FP32
    float *hat;              // [Nu][M] transformed residual / correction
    float *d32;              // [M][Nu] correction
    float2 *esc;             // [pnz][pnr] (E_r, E_z)
    double *er64, *ez64;     // FP64 copies for the FP64 path (or NULL)
    double *red;             // [0] ||b||^2, [1] ||r||^2, [2] rel. residual, [3] iterations, [4..6] PCG scalars
    int *conv;               // converged flag
    double *r64, *z64, *q64; // [M][Nu] PCG vectors (mask-aware solve) or NULL
    double *p64;             // [pnz][pnr] PCG search direction or NULL
};

struct DepositArgs {
    int precision;
    const void *x, *y, *z;
    const uint8_t *status;
    int64_t n;
    double sx, sz, gz0;
    int pnr, pnz;
    int64_t qw;
    unsigned long long *Q;
};

struct DstGemm {
    const float *S;
    int a_is_S, a_sel, b_is_S, b_sel, c_sel; // sel: 0 = r32, 1 = hat, 2 = d32
    int Mo, No, K;
    int64_t a_sm, a_sk, b_sk, b_sn, c_sm, c_sn;
    float alpha;
};

// Batched over instances: tile t of 256 packs belongs to the instance i with
// tile_start[i] <= t < tile_start[i + 1].
void launch_deposit(const DepositArgs *d_args, const int32_t *d_tile_start, int n_inst, int total_tiles,
                    cudaStream_t s);
void launch_pic_prepare(const PicGeom &G, const PicInst *d_insts, int n_inst, cudaStream_t s);
// Returns the number of kernel launches issued.
int launch_pic_solve(const PicGeom &G, const PicInst *d_insts, int n_inst, int max_refine, double tol,
                     cudaStream_t s);
// Maskless fast solve A d = r: r32 -> (DST-I, Thomas per mode, inverse DST-I) -> d32.
int launch_fast_solve(const PicGeom &G, const PicInst *d_insts, int n_inst, cudaStream_t s);
// Mask-aware solve by PCG preconditioned with the fast solve (pic_masked.cu).
int launch_pic_solve_masked(const PicGeom &G, const PicInst *d_insts, int n_inst, int max_iter, double tol,
                            cudaStream_t s);
// E_SCE by central differences of Phi.
void launch_esc(const PicGeom &G, const PicInst *d_insts, int n_inst, cudaStream_t s);

} // namespace mucite
