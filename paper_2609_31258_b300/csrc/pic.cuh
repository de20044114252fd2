// Device-side descriptors of the space-charge solve (see pic.cu).
#pragma once
#include <algorithm>
#include <vector>

#include <cuda.h>

#include "common.cuh"

namespace mucite {

// Fixed operator data of one PIC grid (shared by the instances using it).
struct PicGeom {
    int pnr, pnz, M, Nu;     // M = pnz - 2 axial unknowns, Nu = pnr - 1 radial unknowns
    int hld;                 // leading dimension of hat (M rounded up to a multiple of 4: 16-byte rows)
    double dr, dz;
    double bscale;           // -(e 2^-30) / (eps0 pi dz): node charge units -> right-hand side
    const float *S;          // [M][M] sin(pi j k / (M + 1)), j, k = 1..M
    const float *cp;         // [Nu][M] Thomas upper factors c_i / m_i(k)
    const float *invm;       // [Nu][M] 1 / m_i(k)
    const float *lo;         // [Nu] a_i (sub-diagonal)
    const double *a, *c, *A; // [Nu] FP64 operator coefficients
    const uint8_t *metal;    // [pnz][pnr] metal nodes (mask-aware solve) or NULL
    int n_sm;                // SMs of the device (0: 148), sizes the split of small contractions
};

// Per-instance buffers of the space-charge solve.
struct PicInst {
    unsigned long long *Q;   // [pnz][pnr] node charge, units e * 2^-30
    unsigned long long *Qn;  // [pnz][pnr] charge deposited by the step kernels at the end of a macro
                             // step's launch, taken over by the next solve (FP32 graph replays) or NULL
    double *phi;             // [pnz][pnr] potential (zero on the Dirichlet boundary)
    double *phi_prev;        // [pnz][pnr] Phi of the update before, for the extrapolated start of a
                             // warm-started solve, or NULL (start from the last Phi)
    int *phi_hist;           // nonzero once phi_prev holds a solved Phi (set by esc_kernel)
    float *r32;              // [M][Nu] residual in FP32
    float *hat;              // [Nu][hld] transformed residual / correction
    float *hat_lo;           // [Nu][hld] with the tensor-core contractions: the tridiagonal solves write
                             // hat rounded to TF32 into hat and the rest here; else NULL
    float *rT, *rT_lo;       // [Nu][hld] with the tensor-core contractions: the residual written
                             // transposed (i-major, j contiguous) as a TF32 pair; else NULL
    float *d32;              // [M][Nu] correction
    float2 *esc;             // [pnz][pnr] (E_r, E_z)
    float4 *esc4;            // [pnz-1][pnr-1][2] the same per cell, the four nodes of a cell in one
                             // 32-byte sector for the step kernels' gather (FP32 instances) or NULL
    double *er64, *ez64;     // FP64 copies for the FP64 path (or NULL)
    double *red;             // [0] ||b||^2, [1] ||r||^2, [2] rel. residual, [3] iterations, [4..6] PCG scalars,
                             // [7] pass counter of a captured solve loop (first instance of a launch)
    int *conv;               // converged flag
    double *r64, *z64, *q64; // [M][Nu] PCG vectors (mask-aware solve) or NULL
    double *p64;             // [pnz][pnr] PCG search direction or NULL
    double *part;            // [2][kRedBlocks] per-block partial sums (block-ordered reductions)
    unsigned *ticket;        // arrival counter of those partial sums (zero between launches)
};

// Tensor-core DST-I contractions (dst_tc.cu): every operand is a pair of
// FP32 arrays, x_hi (x rounded to TF32) and x_lo = x - x_hi. Per instance
// the TMA descriptors of a solve are kTcMaps consecutive CUtensorMap in
// device memory: the forward contraction's A = rT (hi, lo) and B = S (hi,
// lo), then the inverse's A = S (hi, lo) and B = hat (hi, lo).
constexpr int kTcMaps = 8;
// Rows of the TMA box of an A operand (output tile rows) and of a B operand
// (output tile columns).
constexpr int kTcBoxA = 128, kTcBoxB = 128;

// Most blocks a solve kernel launches per instance (8 per SM on 148 SMs).
constexpr int kRedBlocks = 1184;

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

// Batched over instances: tile t of 256 packs belongs to the instance i with
// tile_start[i] <= t < tile_start[i + 1].
void launch_deposit(const DepositArgs *d_args, const int32_t *d_tile_start, int n_inst, int total_tiles,
                    cudaStream_t s);
void launch_pic_prepare(const PicGeom &G, const PicInst *d_insts, int n_inst, cudaStream_t s);
// As launch_pic_prepare, but the charge of the solve is taken from Qn
// (Q <- Qn, Qn <- 0) instead of being cleared for a deposit.
void launch_pic_take(const PicGeom &G, const PicInst *d_insts, int n_inst, cudaStream_t s);
// Clears Qn (before a standalone deposit into it).
void launch_pic_clear_next(const PicGeom &G, const PicInst *d_insts, int n_inst, cudaStream_t s);
// Returns the number of kernel launches issued. When `s` is being captured
// into a CUDA graph and `aux` is a stream of this device, the correction
// passes become the body of a device-controlled while loop (a conditional
// graph node, its body captured on `aux`), so a replay runs only the passes
// the solve needs instead of the fixed maximum; otherwise the passes are
// issued as a fixed sequence whose kernels return at once after convergence.
int launch_pic_solve(const PicGeom &G, const PicInst *d_insts, int n_inst, int max_refine, double tol,
                     cudaStream_t s, cudaStream_t aux = nullptr, const CUtensorMap *tc_maps = nullptr,
                     int *tc_err = nullptr);
// Maskless fast solve A d = r: r32 -> (DST-I, Thomas per mode, inverse DST-I) -> d32;
// with tc_maps (the instances' descriptors, kTcMaps each) the residual comes
// as rT and both contractions run on the tensor cores. With acc_phi the
// correction is added to Phi (Phi[j+1][i] += d[j][i]) instead of stored.
int launch_fast_solve(const PicGeom &G, const PicInst *d_insts, int n_inst, cudaStream_t s,
                      const CUtensorMap *tc_maps = nullptr, int *tc_err = nullptr, bool acc_phi = false);
// C[m][n] = alpha sum_k A[m][k] B[n][k] per instance z (A: Mg x K, B: Ng x K,
// K-major, each a TF32 pair of FP32 rows read by TMA through the descriptors
// maps[z * kTcMaps + first .. + 3] = A_hi, A_lo, B_hi, B_lo), formed on the
// tensor cores as A_hi B_hi + A_hi B_lo + A_lo B_hi; C is instance z's hat
// (forward, leading dimension hld) or d32 (inverse, leading dimension Nu).
// Returns false when the launch is not possible.
bool launch_dst_tc(const CUtensorMap *maps, int first, const PicInst *d_insts, int n_inst, bool forward,
                   const PicGeom &G, float alpha, int *err, cudaStream_t s);
// x rounded to TF32 (10 mantissa bits, to nearest, ties away from zero).
__device__ __forceinline__ float tf32_round(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
// Tensor map of a row-major FP32 matrix (rows x cols, leading dimension ld
// floats, ld * 4 a multiple of 16) for 32-column x box_rows boxes with the
// 128-byte swizzle; false when the encoder is unavailable or refuses.
bool make_tc_map(CUtensorMap *map, const float *base, int rows, int cols, int ld, int box_rows);
// Whether a grid's contractions fit the tensor-core kernel.
bool tc_shape_ok(const PicGeom &G);
// Once per device (current) before the first tensor-core launch: sets the
// kernel's shared-memory limit and checks that its clusters can be resident.
bool tc_prepare();
// Mask-aware solve by PCG preconditioned with the fast solve (pic_masked.cu).
int launch_pic_solve_masked(const PicGeom &G, const PicInst *d_insts, int n_inst, int max_iter, double tol,
                            cudaStream_t s, cudaStream_t aux = nullptr);

// Device-controlled loop for a stream under capture: adds a while node after
// the captured work of `s`, captures `body(aux)` as its body and lets the
// capture of `s` continue after the node. The body must end with
// launch_loop_ctl. The condition starts at 1 (the body runs at least once)
// after launch_loop_reset; with `done` >= 0 it starts at 0 and a kernel
// captured before the node (launch_loop_open) opens the loop only while a
// listed instance is unconverged and fewer than max_passes passes, counting
// the `done` passes issued before the node, have run. Returns false when `s`
// is not being captured, `aux` is null or a graph call fails (the capture is
// then unusable).
template <class Body>
bool capture_while(cudaStream_t s, cudaStream_t aux, const PicInst *d_insts, Body body, int n_inst = 0,
                   int done = -1, int max_passes = 0);
// Loop control of a captured while node: counts the passes (kept in the
// first instance's red[7], cleared by launch_loop_reset before the node) and
// continues while a listed instance is unconverged and fewer than max_passes
// passes have run.
void launch_loop_reset(const PicInst *d_insts, cudaStream_t s);
void launch_loop_open(const PicInst *d_insts, int n_inst, int done, int max_passes, cudaGraphConditionalHandle h,
                      cudaStream_t s);
void launch_loop_ctl(const PicInst *d_insts, int n_inst, int max_passes, cudaGraphConditionalHandle h,
                     cudaStream_t s);

inline bool stream_capturing(cudaStream_t s, cudaStream_t aux)
{
    if (aux == nullptr) return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive;
}

template <class Body>
bool capture_while(cudaStream_t s, cudaStream_t aux, const PicInst *d_insts, Body body, int n_inst, int done,
                   int max_passes)
{
    if (!stream_capturing(s, aux)) return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    if (cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr) != cudaSuccess ||
        cs != cudaStreamCaptureStatusActive)
        return false;
    cudaGraphConditionalHandle h;
    if (cudaGraphConditionalHandleCreate(&h, g, done >= 0 ? 0u : 1u, cudaGraphCondAssignDefault) != cudaSuccess)
        return false;
    if (done >= 0)
        launch_loop_open(d_insts, n_inst, done, max_passes, h, s);
    else
        launch_loop_reset(d_insts, s);
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    if (cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd) != cudaSuccess ||
        cs != cudaStreamCaptureStatusActive)
        return false;
    const std::vector<cudaGraphNode_t> dep(deps, deps + nd);
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    if (cudaGraphAddNode(&node, g, dep.data(), nullptr, dep.size(), &p) != cudaSuccess) return false;
    cudaGraph_t bg = p.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(aux, bg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess)
        return false;
    body(aux, h);
    cudaGraph_t fin = nullptr;
    if (cudaStreamEndCapture(aux, &fin) != cudaSuccess) return false;
    return cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies) ==
           cudaSuccess;
}

// E_SCE by central differences of Phi, at the nodes (esc) and, for the
// instances that have esc4, regrouped per cell.
void launch_esc(const PicGeom &G, const PicInst *d_insts, int n_inst, cudaStream_t s);

} // namespace mucite
