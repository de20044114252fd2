// Mask-aware space-charge solve (Methods, Axisymmetric PIC space charge
// update: the space-charge potential vanishes at both axial ends, at the
// outer radius and on the metal nodes of the electrode mask).
//
// A direct DST/tridiagonal solve cannot impose Phi = 0 at interior metal
// nodes, so the masked system A_m Phi = b_m (metal rows replaced by the
// identity, metal columns removed, b = 0 at metal) is solved by
// preconditioned conjugate gradients in FP64, with the maskless fast solver
// of pic.cu (FP32 DST-I + per-mode Thomas + inverse DST-I) as preconditioner,
// restricted to the fluid nodes: z = P A^-1 P r. A_m and A are both negative
// definite, so the usual PCG recurrences apply unchanged. Scalars (alpha,
// beta, convergence) live on the device; iterations stop at
// ||b - A_m Phi|| / ||b|| <= tol without a host round trip.
// blockIdx.z selects the instance.
#include "common.cuh"
#include "pic.cuh"

namespace mucite {

namespace {

// red slots of a masked solve
enum { kBB = 0, kRR = 1, kREL = 2, kIT = 3, kRZ = 4, kRZN = 5, kPQ = 6 };

__device__ __forceinline__ double block_sum_m(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    v = 0.0;
    if (w == 0) {
        v = l < (int)(blockDim.x >> 5) ? sh[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

// Order-independent grid sum of one instance: every block stores its partial
// sums, and the last block to arrive adds all of them in block order and
// writes the totals to red[s0] (and red[s1]), so the result, and with it
// every PCG scalar, does not depend on the order in which blocks finish.
// Called by all threads of a block with its partials v0 (and v1) in thread 0.
__device__ void grid_sum(const PicInst &I, double v0, double v1, bool two, int s0, int s1, double *sh)
{
    __shared__ bool last;
    if (threadIdx.x == 0) {
        I.part[blockIdx.x] = v0;
        if (two) I.part[kRedBlocks + blockIdx.x] = v1;
        __threadfence();
        last = atomicAdd(I.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double a = 0.0, b = 0.0;
    for (unsigned k = threadIdx.x; k < gridDim.x; k += blockDim.x) {
        a += __ldcg(I.part + k);
        if (two) b += __ldcg(I.part + kRedBlocks + k);
    }
    a = block_sum_m(a, sh);
    __syncthreads();
    if (two) b = block_sum_m(b, sh);
    if (threadIdx.x == 0) {
        I.red[s0] = a;
        if (two) I.red[s1] = b;
        *I.ticket = 0u;
    }
}

// (A x)_ij on an unknown node for a full-grid vector x (zero on the Dirichlet
// boundary and, for the vectors used here, on metal nodes).
__device__ __forceinline__ double apply_A(const PicGeom &G, const double *x, int i, int j)
{
    const double *ph = x + (size_t)j * G.pnr + i;
    const double c = ph[0];
    const double w = i > 0 ? ph[-1] : 0.0;
    return G.a[i] * w + G.c[i] * ph[1] - (G.a[i] + G.c[i]) * c + G.A[i] * (ph[G.pnr] - 2.0 * c + ph[-G.pnr]);
}

__device__ __forceinline__ bool is_metal(const PicGeom &G, int i, int j)
{
    return G.metal[(size_t)j * G.pnr + i] != 0;
}

} // namespace

// r = b_m - A_m Phi on the unknowns (FP64 and FP32 copies), ||b_m||^2.
__global__ void __launch_bounds__(256) pcg_init_kernel(PicGeom G, const PicInst *insts)
{
    __shared__ double sh[32];
    const PicInst &I = insts[blockIdx.z];
    const int64_t n = (int64_t)G.M * G.Nu;
    double bb = 0.0, rr = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / G.Nu) + 1, i = (int)(e % G.Nu);
        double r = 0.0;
        if (!is_metal(G, i, j)) {
            const double b = G.bscale * (double)(long long)I.Q[(size_t)j * G.pnr + i];
            r = b - apply_A(G, I.phi, i, j);
            bb += b * b;
        }
        I.r64[e] = r;
        I.r32[e] = (float)r;
        rr += r * r;
    }
    bb = block_sum_m(bb, sh);
    __syncthreads();
    rr = block_sum_m(rr, sh);
    grid_sum(I, bb, rr, true, kBB, kRR, sh);
}

// z = P A^-1 P r from the fast solve's output d32; rz = r . z.
__global__ void __launch_bounds__(256) pcg_z_kernel(PicGeom G, const PicInst *insts)
{
    __shared__ double sh[32];
    const PicInst &I = insts[blockIdx.z];
    if (*I.conv) return;
    const int64_t n = (int64_t)G.M * G.Nu;
    double rz = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / G.Nu) + 1, i = (int)(e % G.Nu);
        const double z = is_metal(G, i, j) ? 0.0 : (double)I.d32[e];
        I.z64[e] = z;
        rz += I.r64[e] * z;
    }
    rz = block_sum_m(rz, sh);
    grid_sum(I, rz, 0.0, false, kRZN, kRZN, sh);
}

// beta = rz_new / rz (0 on the first iteration), p = z + beta p (full grid).
__global__ void __launch_bounds__(256) pcg_p_kernel(PicGeom G, const PicInst *insts, int first)
{
    const PicInst &I = insts[blockIdx.z];
    if (*I.conv) return;
    __shared__ double sb;
    if (threadIdx.x == 0) sb = first ? 0.0 : I.red[kRZN] / I.red[kRZ]; // one FP64 division per block
    __syncthreads();
    const double beta = sb;
    const int64_t n = (int64_t)G.M * G.Nu;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / G.Nu) + 1, i = (int)(e % G.Nu);
        double *p = I.p64 + (size_t)j * G.pnr + i;
        *p = I.z64[e] + beta * *p;
    }
}

// q = A_m p, pq = p . q.
__global__ void __launch_bounds__(256) pcg_q_kernel(PicGeom G, const PicInst *insts)
{
    __shared__ double sh[32];
    const PicInst &I = insts[blockIdx.z];
    if (*I.conv) return;
    const int64_t n = (int64_t)G.M * G.Nu;
    double pq = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / G.Nu) + 1, i = (int)(e % G.Nu);
        const double q = is_metal(G, i, j) ? 0.0 : apply_A(G, I.p64, i, j);
        I.q64[e] = q;
        pq += I.p64[(size_t)j * G.pnr + i] * q;
    }
    pq = block_sum_m(pq, sh);
    grid_sum(I, pq, 0.0, false, kPQ, kPQ, sh);
}

// alpha = rz / pq; Phi += alpha p; r -= alpha q; ||r||^2.
__global__ void __launch_bounds__(256) pcg_xr_kernel(PicGeom G, const PicInst *insts)
{
    __shared__ double sh[32];
    const PicInst &I = insts[blockIdx.z];
    if (*I.conv) return;
    __shared__ double sa;
    if (threadIdx.x == 0) sa = I.red[kRZ] / I.red[kPQ]; // one FP64 division per block
    __syncthreads();
    const double alpha = sa;
    const int64_t n = (int64_t)G.M * G.Nu;
    double rr = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / G.Nu) + 1, i = (int)(e % G.Nu);
        const size_t f = (size_t)j * G.pnr + i;
        I.phi[f] += alpha * I.p64[f];
        const double r = I.r64[e] - alpha * I.q64[e];
        I.r64[e] = r;
        I.r32[e] = (float)r;
        rr += r * r;
    }
    rr = block_sum_m(rr, sh);
    grid_sum(I, rr, 0.0, false, kRR, kRR, sh);
}

// One thread per instance: rel = ||r|| / ||b|| after the initial residual
// (phase 0) or after an update (phase 2, also counts the iteration); the
// solve is converged when rel <= tol.
__global__ void pcg_scalar_kernel(const PicInst *insts, double tol, int phase)
{
    const PicInst &I = insts[blockIdx.x];
    if (threadIdx.x != 0 || *I.conv) return;
    double *red = I.red;
    const double rel = red[kBB] > 0.0 ? sqrt(red[kRR] / red[kBB]) : 0.0;
    red[kREL] = rel;
    red[kRR] = 0.0;
    if (phase == 2) red[kIT] += 1.0;
    if (rel <= tol) *I.conv = 1;
}

// After p = z + beta p: rz <- rz_new, clear the accumulators of the next round.
__global__ void pcg_rotate_kernel(const PicInst *insts)
{
    const PicInst &I = insts[blockIdx.x];
    if (threadIdx.x != 0 || *I.conv) return;
    I.red[kRZ] = I.red[kRZN];
    I.red[kRZN] = 0.0;
    I.red[kPQ] = 0.0;
}

int launch_pic_solve_masked(const PicGeom &G, const PicInst *d_insts, int n_inst, int max_iter, double tol,
                            cudaStream_t s, cudaStream_t aux)
{
    int launches = 0;
    const int64_t nu = (int64_t)G.M * G.Nu;
    const unsigned blocks = (unsigned)std::min<int64_t>((nu + 255) / 256, kRedBlocks);
    const dim3 gv(blocks, 1, n_inst);
    pcg_init_kernel<<<gv, 256, 0, s>>>(G, d_insts);
    pcg_scalar_kernel<<<n_inst, 32, 0, s>>>(d_insts, tol, 0);
    launches += 2;
    // z0 = P A^-1 P r0, p0 = z0
    launches += launch_fast_solve(G, d_insts, n_inst, s);
    pcg_z_kernel<<<gv, 256, 0, s>>>(G, d_insts);
    pcg_p_kernel<<<gv, 256, 0, s>>>(G, d_insts, 1);
    pcg_rotate_kernel<<<n_inst, 32, 0, s>>>(d_insts);
    launches += 3;
    // graph capture: the first (q, x/r, scalars) step, then at most
    // max_iter - 1 further iterations under device control
    if (max_iter > 1 && stream_capturing(s, aux)) {
        pcg_q_kernel<<<gv, 256, 0, s>>>(G, d_insts);
        pcg_xr_kernel<<<gv, 256, 0, s>>>(G, d_insts);
        pcg_scalar_kernel<<<n_inst, 32, 0, s>>>(d_insts, tol, 2);
        const bool looped = capture_while(s, aux, d_insts, [&](cudaStream_t b, cudaGraphConditionalHandle h) {
            launch_fast_solve(G, d_insts, n_inst, b);
            pcg_z_kernel<<<gv, 256, 0, b>>>(G, d_insts);
            pcg_p_kernel<<<gv, 256, 0, b>>>(G, d_insts, 0);
            pcg_rotate_kernel<<<n_inst, 32, 0, b>>>(d_insts);
            pcg_q_kernel<<<gv, 256, 0, b>>>(G, d_insts);
            pcg_xr_kernel<<<gv, 256, 0, b>>>(G, d_insts);
            pcg_scalar_kernel<<<n_inst, 32, 0, b>>>(d_insts, tol, 2);
            launch_loop_ctl(d_insts, n_inst, max_iter - 1, h, b);
        });
        return looped ? launches + 5 : -1;
    }
    for (int it = 0; it < max_iter; ++it) {
        pcg_q_kernel<<<gv, 256, 0, s>>>(G, d_insts);
        pcg_xr_kernel<<<gv, 256, 0, s>>>(G, d_insts);
        pcg_scalar_kernel<<<n_inst, 32, 0, s>>>(d_insts, tol, 2);
        launches += 3;
        if (it == max_iter - 1) break;
        launches += launch_fast_solve(G, d_insts, n_inst, s);
        pcg_z_kernel<<<gv, 256, 0, s>>>(G, d_insts);
        pcg_p_kernel<<<gv, 256, 0, s>>>(G, d_insts, 0);
        pcg_rotate_kernel<<<n_inst, 32, 0, s>>>(d_insts);
        launches += 3;
    }
    return launches;
}

} // namespace mucite
