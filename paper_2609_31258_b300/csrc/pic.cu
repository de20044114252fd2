// Space-charge macro step ("Axisymmetric PIC space charge update").
//
// 1. CIC deposit of q*W onto the (r, z) PIC nodes as int64 fixed point
//    (units e * 2^-30). The deposit is defined on the position lattice:
//    r = floor(sqrt(xq^2 + yq^2)) exactly, cell index and 15-bit fractions
//    from integer products, so the node charges are exact and independent of
//    the order of the atomic additions.
// 2. Finite-volume cylindrical Poisson operator over annular control volumes
//    (no flux through the axis, Phi = 0 at both axial ends and at r = R),
//    divided through by pi dz:
//      a_i Phi_{i-1} + c_i Phi_{i+1} - (a_i + c_i) Phi_i
//        + A_i (Phi_{j+1} - 2 Phi_j + Phi_{j-1}) = -Q_ij / (eps0 pi dz)
//    with a_i = 2(i - 1/2), c_i = 2(i + 1/2), A_i = 2 i dr^2/dz^2 for i >= 1
//    and a_0 = 0, c_0 = 1, A_0 = dr^2 / (4 dz^2).
// 3. Iterative refinement: residual r = b - A Phi in FP64; correction from
//    an FP32 fast solve -- DST-I in z as a dense contraction with the sine
//    matrix S_jk = sin(pi j k / (M + 1)), a tridiagonal (Thomas) solve in r
//    per axial mode with eigenvalue 4 sin^2(pi k / (2 (M + 1))), inverse
//    DST-I -- accumulated into FP64 Phi until ||r|| / ||b|| <= tol
//    (tol = 1e-6, the paper's Poisson tolerance). Convergence is decided on
//    the device, so the macro step needs no host round trip.
// 4. E_SCE = -grad(Phi) by central differences on the PIC grid (one-sided at
//    the edges, E_r = 0 on the axis).
// blockIdx.z selects the instance in batched launches.
#include <cooperative_groups.h>

#include "common.cuh"
#include "deposit.cuh"
#include "pic.cuh"

namespace mucite {

namespace {

__device__ __forceinline__ int32_t q32p(double v)
{
    const double r = rint(v);
    if (r < -2147483648.0) return INT32_MIN;
    if (r > 2147483647.0) return INT32_MAX;
    return (int32_t)r;
}

__device__ __forceinline__ double block_sum(double v, double *sh)
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

// Row-blocked loops of the grid kernels: a block of 256 threads covers
// 256 >> lw rows of width 2^lw (the smallest power of two >= the row length
// n, from 32 to 256; longer rows are walked in steps of 256), so a thread's
// node follows from shifts and masks instead of an index division.
__host__ __device__ __forceinline__ int row_shift(int n)
{
    int lw = 5;
    while ((1 << lw) < n && lw < 8) ++lw;
    return lw;
}

// Blocks of a row-blocked launch over `rows` rows of length n.
inline unsigned row_blocks(int rows, int n)
{
    const int per = 256 >> row_shift(n);
    return (unsigned)std::min((rows + per - 1) / per, kRedBlocks);
}

// End of a residual launch for one instance, called by all threads of each
// of its nblk blocks (this one is block blk) with the thread's partial sums
// of ||r||^2 and, on the first residual of a solve, ||b||^2: every block
// stores its partials, and the last block to arrive adds them up in block
// order and takes the convergence decision -- red[2] = ||r|| / ||b||, conv
// when <= tol, else one more correction pass counted in red[3]. The sums and
// the decision do not depend on the order in which the blocks finished.
template <bool kFirst>
__device__ void residual_close(const PicInst &I, double rr, double bb, double tol, unsigned blk, unsigned nblk,
                               double *sh)
{
    __shared__ bool last;
    rr = block_sum(rr, sh);
    if (kFirst) {
        __syncthreads();
        bb = block_sum(bb, sh);
    }
    if (threadIdx.x == 0) {
        I.part[blk] = rr;
        if (kFirst) I.part[kRedBlocks + blk] = bb;
        __threadfence();
        last = atomicAdd(I.ticket, 1u) == nblk - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double a = 0.0, b = 0.0;
    for (unsigned k = threadIdx.x; k < nblk; k += blockDim.x) {
        a += __ldcg(I.part + k);
        if (kFirst) b += __ldcg(I.part + kRedBlocks + k);
    }
    a = block_sum(a, sh);
    if (kFirst) {
        __syncthreads();
        b = block_sum(b, sh);
    }
    if (threadIdx.x != 0) return;
    I.red[1] = a;
    if (kFirst) I.red[0] = b;
    const double bn = kFirst ? b : I.red[0];
    const double rel = bn > 0.0 ? sqrt(a / bn) : 0.0;
    I.red[2] = rel;
    if (rel <= tol) *I.conv = 1;
    else I.red[3] += 1.0;
    *I.ticket = 0u;
}

// A solved hat value: as is, or, with the tensor-core contractions, as the
// TF32 pair (hat rounded to TF32, hat_lo the rest).
__device__ __forceinline__ void store_hat(const PicInst &I, size_t e, float v)
{
    if (I.hat_lo != nullptr) {
        const float hi = tf32_round(v);
        I.hat[e] = hi;
        I.hat_lo[e] = v - hi;
    } else {
        I.hat[e] = v;
    }
}

} // namespace

// Cell (j * pnr + i of its lower-left node) and the four CIC contributions
// of pack p, in units of e * 2^-30; false when the pack deposits nothing
// (inactive, or outside the PIC box).
__device__ __forceinline__ bool deposit_weights(const DepositArgs &A, int64_t p, uint32_t &cell,
                                                unsigned long long w[4])
{
    if (p >= A.n || A.status[p] != MUCITE_ACTIVE) return false;
    int32_t xq, yq, zq;
    if (A.precision == MUCITE_FP32) {
        xq = ((const int32_t *)A.x)[p];
        yq = ((const int32_t *)A.y)[p];
        zq = ((const int32_t *)A.z)[p];
    } else {
        xq = q32p(__dmul_rn(((const double *)A.x)[p], A.sx));
        yq = q32p(__dmul_rn(((const double *)A.y)[p], A.sx));
        zq = q32p(__dmul_rn(__dsub_rn(((const double *)A.z)[p], A.gz0), A.sz));
    }
    return cic_lattice(xq, yq, zq, A.pnr, A.pnz, A.qw, cell, w);
}

// Charge deposit of one 256-pack tile. Packs of a beam crowd into few
// cells, and atomics on one address serialise in L2; the block therefore
// first sums its packs' contributions per cell in a shared-memory table
// (open addressing on the cell index; the table has twice as many slots as
// the block has packs, so every insertion finds a slot), then adds each
// cell's four sums to the grid with one atomic per node. Integer addition
// is exact and order-independent, so the result is bit-exact.
constexpr int kDepBits = 9, kDepSlots = 1 << kDepBits;
constexpr uint32_t kDepEmpty = 0xFFFFFFFFu;

// Tile t of 256 packs belongs to instance i with tile_start[i] <= t < tile_start[i+1].
__global__ void __launch_bounds__(256) deposit_kernel(const DepositArgs *args, const int32_t *tile_start,
                                                      int n_inst)
{
    __shared__ int s_inst;
    __shared__ uint32_t s_key[kDepSlots];
    __shared__ unsigned long long s_acc[kDepSlots][4];
    for (int k = threadIdx.x; k < kDepSlots; k += blockDim.x) {
        s_key[k] = kDepEmpty;
        s_acc[k][0] = s_acc[k][1] = s_acc[k][2] = s_acc[k][3] = 0ull;
    }
    const int b = blockIdx.x;
    if (threadIdx.x == 0) {
        int lo = 0, hi = n_inst - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tile_start[mid] <= b) lo = mid;
            else hi = mid - 1;
        }
        s_inst = lo;
    }
    __syncthreads();
    const DepositArgs &A = args[s_inst];
    uint32_t cell;
    unsigned long long w[4];
    if (deposit_weights(A, (int64_t)(b - tile_start[s_inst]) * blockDim.x + threadIdx.x, cell, w)) {
        uint32_t h = (cell * 2654435761u) >> (32 - kDepBits);
        for (int probe = 0; probe < kDepSlots; ++probe) {
            const uint32_t prev = atomicCAS(&s_key[h], kDepEmpty, cell);
            if (prev == kDepEmpty || prev == cell) break;
            h = (h + 1) & (kDepSlots - 1);
        }
        atomicAdd(&s_acc[h][0], w[0]);
        atomicAdd(&s_acc[h][1], w[1]);
        atomicAdd(&s_acc[h][2], w[2]);
        atomicAdd(&s_acc[h][3], w[3]);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kDepSlots; k += blockDim.x) {
        const uint32_t c = s_key[k];
        if (c == kDepEmpty) continue;
        unsigned long long *Q = A.Q + c;
        if (s_acc[k][0]) atomicAdd(Q, s_acc[k][0]);
        if (s_acc[k][1]) atomicAdd(Q + 1, s_acc[k][1]);
        if (s_acc[k][2]) atomicAdd(Q + A.pnr, s_acc[k][2]);
        if (s_acc[k][3]) atomicAdd(Q + A.pnr + 1, s_acc[k][3]);
    }
}

// Start of a warm-started solve: with phi_prev, Phi_n = 2 Phi_{n-1} - Phi_{n-2}
// (the last two solutions extrapolated linearly in time; from the second
// solve on) and phi_prev <- Phi_{n-1}. Any start converges to the same
// tolerance; this one leaves the first correction a smaller residual, the
// charge moving steadily between updates.
__device__ __forceinline__ void start_phi(const PicInst &I, int64_t e, bool ext)
{
    if (I.phi_prev == nullptr) return;
    const double p = I.phi[e];
    if (ext) I.phi[e] = 2.0 * p - I.phi_prev[e];
    I.phi_prev[e] = p;
}

// Clears the node charges and the convergence bookkeeping of every instance
// before a macro step (blockIdx.y = instance); the start of the solve.
__global__ void __launch_bounds__(256) pic_prepare_kernel(PicGeom G, const PicInst *insts)
{
    const PicInst &I = insts[blockIdx.y];
    const int64_t n = (int64_t)G.pnr * G.pnz;
    const bool ext = I.phi_prev != nullptr && *I.phi_hist != 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        I.Q[e] = 0ull;
        start_phi(I, e, ext);
    }
    if (blockIdx.x == 0 && threadIdx.x < 8) I.red[threadIdx.x] = 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) *I.conv = 0;
}

__global__ void __launch_bounds__(256) pic_take_kernel(PicGeom G, const PicInst *insts)
{
    const PicInst &I = insts[blockIdx.y];
    const int64_t n = (int64_t)G.pnr * G.pnz;
    const bool ext = I.phi_prev != nullptr && *I.phi_hist != 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        I.Q[e] = I.Qn[e];
        I.Qn[e] = 0ull;
        start_phi(I, e, ext);
    }
    if (blockIdx.x == 0 && threadIdx.x < 8) I.red[threadIdx.x] = 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) *I.conv = 0;
}

__global__ void __launch_bounds__(256) pic_clear_next_kernel(PicGeom G, const PicInst *insts)
{
    const PicInst &I = insts[blockIdx.y];
    const int64_t n = (int64_t)G.pnr * G.pnz;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x)
        I.Qn[e] = 0ull;
}

// r = b - A Phi (FP64) on the unknowns, r32 = (float) r; ||r||^2 (and, on
// the first residual of a solve, ||b||^2) and the convergence decision by
// residual_close. Rows q = j - 1 of the unknowns, row-blocked.
template <bool kFirst>
__global__ void __launch_bounds__(256) residual_kernel(PicGeom G, const PicInst *insts, double tol)
{
    __shared__ double sh[32];
    const PicInst &I = insts[blockIdx.z];
    if (*I.conv) return;
    const int lw = row_shift(G.Nu), per = 256 >> lw;
    const int sub = threadIdx.x >> lw, t = threadIdx.x & ((1 << lw) - 1);
    double rr = 0.0, bb = 0.0;
    for (int q = blockIdx.x * per + sub; q < G.M; q += gridDim.x * per) {
        const int j = q + 1;
        for (int i = t; i < G.Nu; i += 1 << lw) {
            const double *ph = I.phi + (size_t)j * G.pnr + i;
            const double c = ph[0];
            const double w = i > 0 ? ph[-1] : 0.0;
            const double east = ph[1]; // i + 1 <= pnr - 1, Phi = 0 there
            const double ax = G.a[i] * w + G.c[i] * east - (G.a[i] + G.c[i]) * c +
                              G.A[i] * (ph[G.pnr] - 2.0 * c + ph[-G.pnr]);
            const double b = G.bscale * (double)(long long)I.Q[(size_t)j * G.pnr + i];
            const double r = b - ax;
            I.r32[(size_t)q * G.Nu + i] = (float)r;
            rr += r * r;
            if (kFirst) bb += b * b;
        }
    }
    residual_close<kFirst>(I, rr, bb, tol, blockIdx.x, gridDim.x, sh);
}

// The residual of residual_kernel written transposed for the tensor-core
// contractions as a TF32 pair: rT[i][j - 1] (rounded to TF32) and rT_lo (the
// rest), i-major with leading dimension hld. A block takes a 32 x 32 tile of
// (j, i), reads Phi and Q along i (coalesced), and writes rT along j through
// a shared-memory transpose; the norms and the decision as residual_kernel.
template <bool kFirst>
__global__ void __launch_bounds__(256) residual_t_kernel(PicGeom G, const PicInst *insts, double tol)
{
    __shared__ float tile[32][33];
    __shared__ double sh[32];
    const PicInst &I = insts[blockIdx.z];
    if (*I.conv) return;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int i0 = blockIdx.x * 32, q0 = blockIdx.y * 32; // q = j - 1
    double rr = 0.0, bb = 0.0;
    for (int r = ty; r < 32; r += 8) {
        const int q = q0 + r, i = i0 + tx;
        float v = 0.0f;
        if (q < G.M && i < G.Nu) {
            const int j = q + 1;
            const double *ph = I.phi + (size_t)j * G.pnr + i;
            const double c = ph[0];
            const double w = i > 0 ? ph[-1] : 0.0;
            const double east = ph[1];
            const double ax = G.a[i] * w + G.c[i] * east - (G.a[i] + G.c[i]) * c +
                              G.A[i] * (ph[G.pnr] - 2.0 * c + ph[-G.pnr]);
            const double b = G.bscale * (double)(long long)I.Q[(size_t)j * G.pnr + i];
            const double res = b - ax;
            v = (float)res;
            rr += res * res;
            if (kFirst) bb += b * b;
        }
        tile[r][tx] = v;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int i = i0 + r, q = q0 + tx;
        if (i < G.Nu && q < G.M) {
            const float v = tile[tx][r], hi = tf32_round(v);
            I.rT[(size_t)i * G.hld + q] = hi;
            I.rT_lo[(size_t)i * G.hld + q] = v - hi;
        }
    }
    residual_close<kFirst>(I, rr, bb, tol, blockIdx.y * gridDim.x + blockIdx.x, gridDim.x * gridDim.y, sh);
}

// DST-I contractions of the fast solve with the sine matrix's symmetry:
// with S[j][k] = sin(pi (j+1)(k+1) / (M+1)) (0-based), row M-1-j equals row j
// in the even columns k = 2c and its negative in the odd ones k = 2c+1
// (S[M-1-j][k] = (-1)^k S[j][k]), and S is symmetric. So each transform is
// two contractions over H = ceil(M/2) terms instead of one over M, half the
// arithmetic:
//   forward (kInv = false), hat[i][k] = alpha sum_j r[j][i] S[j][k]:
//     hat[i][2c]   = alpha sum_{j<H} (r[j][i] + r[M-1-j][i]) S[j][2c]
//     hat[i][2c+1] = alpha sum_{j<H} (r[j][i] - r[M-1-j][i]) S[j][2c+1]
//   inverse (kInv = true), d[j][i] = sum_k S[j][k] hat[i][k], for j < H:
//     O = sum_{c<H} S[2c][j] hat[i][2c], E = sum_{c<H} S[2c+1][j] hat[i][2c+1],
//     d[j][i] = O + E, d[M-1-j][i] = O - E,
// where for odd M the middle row j = H-1 pairs with itself (r enters once;
// S[H-1][2c+1] = 0). A CTA computes a 64 x 64 tile of both sums, 4 x 4
// outputs of each per thread, over 16-deep k slices double-buffered in
// shared memory. Small problems split the k range over the CTAs of a
// thread-block cluster (`splits` CTAs along x, cluster rank = split): each
// CTA leaves its partial tiles in its shared memory and, after a cluster
// barrier, CTA r adds the partials of its share of the rows through
// distributed shared memory in rank order. Every output's sum has a fixed
// order, so results are deterministic. With kAcc (inverse only) the
// correction is not stored but added to Phi at once, Phi[j+1][i] +=
// (double) d[j][i], the refinement's update fused into the epilogue.
template <bool kInv, bool kAcc = false>
__global__ void __launch_bounds__(256, 2) dst_sym_kernel(PicGeom G, const PicInst *insts, int splits, float alpha)
{
    constexpr int KS = 16, BM = 64, BN = 64, PAD = 4;
    constexpr int L = BM * KS / 256; // elements of each operand tile loaded per thread per slice (BM == BN)
    const PicInst &I = insts[blockIdx.z];
    if (*I.conv) return; // uniform over a cluster: its CTAs share blockIdx.z
    const int M = G.M, Nu = G.Nu, H = (M + 1) / 2;
    const float *S = G.S;
    const float *R = kInv ? I.hat : I.r32;
    // operand tiles [buffer][set][k][m or n]; set 0: the even-column sum, 1: the odd-column sum
    __shared__ __align__(16) float smem[2 * 2 * KS * (BM + PAD) * 2];
    float(*As)[2][KS][BM + PAD] = reinterpret_cast<float(*)[2][KS][BM + PAD]>(smem);
    float(*Bs)[2][KS][BN + PAD] = reinterpret_cast<float(*)[2][KS][BN + PAD]>(smem + 2 * 2 * KS * (BM + PAD));
    const int tid = threadIdx.x;
    const int split = (int)(blockIdx.x % (unsigned)splits);
    const int m0 = blockIdx.y * BM, n0 = (int)(blockIdx.x / (unsigned)splits) * BN;
    const int Mo = kInv ? H : Nu, No = kInv ? Nu : H;
    const int tx = tid & 15, ty = tid >> 4;
    const int nsl = (H + KS - 1) / KS, per = (nsl + splits - 1) / splits;
    const int kb = split * per * KS, ke = min(H, (split + 1) * per * KS);
    float a0[L], a1[L], b0[L], b1[L];
    auto load = [&](int k0) {
#pragma unroll
        for (int q = 0; q < L; ++q) {
            const int e = tid + 256 * q;
            const int mm = e & (BM - 1), kk = e / BM; // A: consecutive threads along m
            const int gm = m0 + mm, gk = k0 + kk;
            float x0 = 0.0f, x1 = 0.0f;
            if (gm < Mo && gk < ke) {
                if (kInv) {
                    // A(j, c) = S[2c][j], S[2c+1][j]
                    x0 = S[(size_t)(2 * gk) * M + gm];
                    x1 = 2 * gk + 1 < M ? S[(size_t)(2 * gk + 1) * M + gm] : 0.0f;
                } else {
                    // A(i, j) = r[j][i] +- r[M-1-j][i]
                    const float u = R[(size_t)gk * Nu + gm];
                    const int jm = M - 1 - gk;
                    const float v = jm != gk ? R[(size_t)jm * Nu + gm] : 0.0f;
                    x0 = u + v;
                    x1 = u - v;
                }
            }
            a0[q] = x0;
            a1[q] = x1;
        }
#pragma unroll
        for (int q = 0; q < L; ++q) {
            const int e = tid + 256 * q;
            int nn, kk;
            if (kInv) { kk = e % KS; nn = e / KS; } // B = hat: consecutive threads along k
            else { nn = e & (BN - 1); kk = e / BN; } // B = S rows: along n
            const int gn = n0 + nn, gk = k0 + kk;
            float y0 = 0.0f, y1 = 0.0f;
            if (gn < No && gk < ke) {
                if (kInv) {
                    // B(c, i) = hat[i][2c], hat[i][2c+1]
                    y0 = R[(size_t)gn * G.hld + 2 * gk];
                    y1 = 2 * gk + 1 < M ? R[(size_t)gn * G.hld + 2 * gk + 1] : 0.0f;
                } else {
                    // B(j, c) = S[j][2c], S[j][2c+1]
                    y0 = S[(size_t)gk * M + 2 * gn];
                    y1 = 2 * gn + 1 < M ? S[(size_t)gk * M + 2 * gn + 1] : 0.0f;
                }
            }
            b0[q] = y0;
            b1[q] = y1;
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int q = 0; q < L; ++q) {
            const int e = tid + 256 * q;
            const int mm = e & (BM - 1), kk = e / BM;
            As[buf][0][kk][mm] = a0[q];
            As[buf][1][kk][mm] = a1[q];
        }
#pragma unroll
        for (int q = 0; q < L; ++q) {
            const int e = tid + 256 * q;
            int nn, kk;
            if (kInv) { kk = e % KS; nn = e / KS; }
            else { nn = e & (BN - 1); kk = e / BN; }
            Bs[buf][0][kk][nn] = b0[q];
            Bs[buf][1][kk][nn] = b1[q];
        }
    };
    float acc0[4][4] = {}, acc1[4][4] = {};
    if (kb < ke) {
        load(kb);
        store(0);
        __syncthreads();
        int buf = 0;
        for (int k0 = kb; k0 < ke; k0 += KS) {
            const bool more = k0 + KS < ke;
            if (more) load(k0 + KS);
#pragma unroll
            for (int kk = 0; kk < KS; ++kk) {
                const float4 p0 = *reinterpret_cast<const float4 *>(&As[buf][0][kk][ty * 4]);
                const float4 p1 = *reinterpret_cast<const float4 *>(&As[buf][1][kk][ty * 4]);
                const float4 q0 = *reinterpret_cast<const float4 *>(&Bs[buf][0][kk][tx * 4]);
                const float4 q1 = *reinterpret_cast<const float4 *>(&Bs[buf][1][kk][tx * 4]);
                const float ua[4] = {p0.x, p0.y, p0.z, p0.w}, ub[4] = {p1.x, p1.y, p1.z, p1.w};
                const float va[4] = {q0.x, q0.y, q0.z, q0.w}, vb[4] = {q1.x, q1.y, q1.z, q1.w};
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        acc0[u][v] = fmaf(ua[u], va[v], acc0[u][v]);
                        acc1[u][v] = fmaf(ub[u], vb[v], acc1[u][v]);
                    }
            }
            if (more) store(buf ^ 1);
            __syncthreads();
            buf ^= 1;
        }
    }
    // epilogue for output (row m, column n) of the tile with sums x0 (even
    // columns / O) and x1 (odd columns / E)
    auto put = [&](int mm, int nn, float x0, float x1) {
        const int gm = m0 + mm, gn = n0 + nn;
        if (gm >= Mo || gn >= No) return;
        if (kInv && kAcc) {
            I.phi[(size_t)(gm + 1) * G.pnr + gn] += (double)(x0 + x1);
            const int jm = M - 1 - gm;
            if (jm != gm) I.phi[(size_t)(jm + 1) * G.pnr + gn] += (double)(x0 - x1);
        } else if (kInv) {
            float *D = I.d32;
            D[(size_t)gm * Nu + gn] = x0 + x1;
            const int jm = M - 1 - gm;
            if (jm != gm) D[(size_t)jm * Nu + gn] = x0 - x1;
        } else {
            float *D = I.hat + (size_t)gm * G.hld;
            D[2 * gn] = alpha * x0;
            if (2 * gn + 1 < M) D[2 * gn + 1] = alpha * x1;
        }
    };
    if (splits == 1) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) put(ty * 4 + u, tx * 4 + v, acc0[u][v], acc1[u][v]);
        return;
    }
    // split-K: partial tiles to shared memory (the slice buffers are free
    // after the loop's last barrier), rank-ordered sums over the cluster
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    float(*Ps)[BM][BN + PAD] = reinterpret_cast<float(*)[BM][BN + PAD]>(smem);
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            Ps[0][ty * 4 + u][tx * 4 + v] = acc0[u][v];
            Ps[1][ty * 4 + u][tx * 4 + v] = acc1[u][v];
        }
    cluster.sync();
    const int rows = BM / splits, r0 = split * rows;
    for (int e = tid; e < rows * BN; e += 256) {
        const int rr = r0 + e / BN, cc = e % BN;
        // all remote reads in flight together, then added in rank order
        float y0[8], y1[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (q < splits) {
                const float *rp = cluster.map_shared_rank(&Ps[0][0][0], (unsigned)q);
                y0[q] = rp[rr * (BN + PAD) + cc];
                y1[q] = rp[BM * (BN + PAD) + rr * (BN + PAD) + cc];
            }
        }
        float x0 = 0.0f, x1 = 0.0f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (q < splits) {
                x0 += y0[q];
                x1 += y1[q];
            }
        }
        put(rr, cc, x0, x1);
    }
    cluster.sync(); // partials stay readable until every CTA of the cluster is done
}

// Tridiagonal solve per axial mode k, staged in shared memory: a block takes
// kThModes consecutive modes, loads their right-hand sides and elimination
// factors for all Nu <= kThRows radial rows with the whole block (coalesced
// along k), runs the sequential forward and backward sweeps of one mode per
// thread on shared memory, and writes the solution back. The sweeps are a
// dependent chain of Nu steps; the operands of the next 8 rows are fetched
// into registers while the current 8 are eliminated, so a step costs the
// chain's arithmetic rather than a shared-memory round trip. Grids with more
// radial unknowns use thomas_kernel below.
constexpr int kThModes = 8, kThRows = 256;

__global__ void __launch_bounds__(256) thomas_smem_kernel(PicGeom G, const PicInst *insts)
{
    constexpr int U = 8;
    __shared__ float sh[kThRows][kThModes], sm[kThRows][kThModes], sc[kThRows][kThModes], sl[kThRows];
    const PicInst &I = insts[blockIdx.z];
    if (*I.conv) return;
    const int k0 = blockIdx.x * kThModes;
    const int Nu = G.Nu;
    const int n = Nu * kThModes;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int i = e / kThModes, kk = e % kThModes, k = k0 + kk;
        if (k < G.M) {
            const size_t o = (size_t)i * G.M + k;
            sh[i][kk] = I.hat[(size_t)i * G.hld + k];
            sm[i][kk] = G.invm[o];
            sc[i][kk] = G.cp[o];
        }
    }
    for (int i = threadIdx.x; i < Nu; i += blockDim.x) sl[i] = G.lo[i];
    __syncthreads();
    const int t = threadIdx.x;
    if (t < kThModes && k0 + t < G.M) {
        // forward: y_0 = h_0 / m_0, y_i = (h_i - a_i y_{i-1}) / m_i
        float ch[U], cm[U], cl[U], nh[U], nm[U], nl[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool ok = u < Nu;
            ch[u] = ok ? sh[u][t] : 0.0f;
            cm[u] = ok ? sm[u][t] : 0.0f;
            cl[u] = ok && u > 0 ? sl[u] : 0.0f; // row 0 has no sub-diagonal term
        }
        float y = 0.0f;
        for (int i0 = 0; i0 < Nu; i0 += U) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = i0 + U + u;
                const bool ok = i < Nu;
                nh[u] = ok ? sh[i][t] : 0.0f;
                nm[u] = ok ? sm[i][t] : 0.0f;
                nl[u] = ok ? sl[i] : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = i0 + u;
                if (i < Nu) {
                    y = (ch[u] - cl[u] * y) * cm[u];
                    sh[i][t] = y;
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                ch[u] = nh[u];
                cm[u] = nm[u];
                cl[u] = nl[u];
            }
        }
        // backward: x_{Nu-1} = y_{Nu-1}, x_i = y_i - (c_i / m_i) x_{i+1}
        float x = y;
        float cy[U], cc[U], ny[U], nc[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = Nu - 2 - u;
            const bool ok = i >= 0;
            cy[u] = ok ? sh[i][t] : 0.0f;
            cc[u] = ok ? sc[i][t] : 0.0f;
        }
        for (int i1 = Nu - 2; i1 >= 0; i1 -= U) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = i1 - U - u;
                const bool ok = i >= 0;
                ny[u] = ok ? sh[i][t] : 0.0f;
                nc[u] = ok ? sc[i][t] : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = i1 - u;
                if (i >= 0) {
                    x = cy[u] - cc[u] * x;
                    sh[i][t] = x;
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                cy[u] = ny[u];
                cc[u] = nc[u];
            }
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int i = e / kThModes, kk = e % kThModes, k = k0 + kk;
        if (k < G.M) store_hat(I, (size_t)i * G.hld + k, sh[i][kk]);
    }
}

// Tridiagonal solve per axial mode k, in place on hat[i][k] (i = 0..Nu-1),
// with the elimination factors of the fixed operator precomputed.
__global__ void __launch_bounds__(256) thomas_kernel(PicGeom G, const PicInst *insts)
{
    const PicInst &I = insts[blockIdx.z];
    if (*I.conv) return;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= G.M) return;
    float *h = I.hat + k;
    float y = h[0] * G.invm[k];
    h[0] = y;
    for (int i = 1; i < G.Nu; ++i) {
        y = (h[(size_t)i * G.hld] - G.lo[i] * y) * G.invm[(size_t)i * G.M + k];
        h[(size_t)i * G.hld] = y;
    }
    float x = y;
    if (I.hat_lo != nullptr) store_hat(I, (size_t)(G.Nu - 1) * G.hld + k, x);
    for (int i = G.Nu - 2; i >= 0; --i) {
        x = h[(size_t)i * G.hld] - G.cp[(size_t)i * G.M + k] * x;
        if (I.hat_lo != nullptr)
            store_hat(I, (size_t)i * G.hld + k, x);
        else
            h[(size_t)i * G.hld] = x;
    }
}

// Phi += (double) d32 on the unknowns (row-blocked like residual_kernel).
__global__ void __launch_bounds__(256) update_kernel(PicGeom G, const PicInst *insts)
{
    const PicInst &I = insts[blockIdx.z];
    if (*I.conv) return;
    const int lw = row_shift(G.Nu), per = 256 >> lw;
    const int sub = threadIdx.x >> lw, t = threadIdx.x & ((1 << lw) - 1);
    for (int q = blockIdx.x * per + sub; q < G.M; q += gridDim.x * per)
        for (int i = t; i < G.Nu; i += 1 << lw)
            I.phi[(size_t)(q + 1) * G.pnr + i] += (double)I.d32[(size_t)q * G.Nu + i];
}

// E_SCE at the nodes (esc, and er64 / ez64 for FP64 instances) and, for
// the instances that have esc4, regrouped per cell in the same pass: node
// (i, j) is corner 00 of cell (i, j), 10 of cell (i-1, j), 01 of cell
// (i, j-1) and 11 of cell (i-1, j-1), the float2 slots 0..3 of a cell's
// 32 bytes. Rows j of the grid, row-blocked.
__global__ void __launch_bounds__(256) esc_kernel(PicGeom G, const PicInst *insts)
{
    // FP64 division is slow on this part: the four step reciprocals are
    // formed once per block and the differences multiplied by them
    __shared__ double rcp[4];
    if (threadIdx.x == 0) {
        rcp[0] = 1.0 / G.dr;
        rcp[1] = 1.0 / (2.0 * G.dr);
        rcp[2] = 1.0 / G.dz;
        rcp[3] = 1.0 / (2.0 * G.dz);
    }
    __syncthreads();
    const double idr = rcp[0], i2dr = rcp[1], idz = rcp[2], i2dz = rcp[3];
    const PicInst &I = insts[blockIdx.z];
    if (I.phi_hist != nullptr && blockIdx.x == 0 && threadIdx.x == 0) *I.phi_hist = 1; // Phi is solved
    const int lw = row_shift(G.pnr), per = 256 >> lw;
    const int sub = threadIdx.x >> lw, t = threadIdx.x & ((1 << lw) - 1);
    const int cr = G.pnr - 1, cz = G.pnz - 1;
    float2 *c4 = reinterpret_cast<float2 *>(I.esc4);
    for (int j = blockIdx.x * per + sub; j < G.pnz; j += gridDim.x * per)
        for (int i = t; i < G.pnr; i += 1 << lw) {
            const size_t e = (size_t)j * G.pnr + i;
            const double *ph = I.phi + e;
            double dpr, dpz;
            if (i == 0) dpr = 0.0;
            else if (i == G.pnr - 1) dpr = (ph[0] - ph[-1]) * idr;
            else dpr = (ph[1] - ph[-1]) * i2dr;
            if (j == 0) dpz = (ph[G.pnr] - ph[0]) * idz;
            else if (j == G.pnz - 1) dpz = (ph[0] - ph[-G.pnr]) * idz;
            else dpz = (ph[G.pnr] - ph[-G.pnr]) * i2dz;
            const float2 v = make_float2((float)-dpr, (float)-dpz);
            I.esc[e] = v;
            if (I.er64) {
                I.er64[e] = -dpr;
                I.ez64[e] = -dpz;
            }
            if (c4 != nullptr) {
                if (j < cz) {
                    if (i < cr) c4[4 * ((size_t)j * cr + i)] = v;
                    if (i > 0) c4[4 * ((size_t)j * cr + i - 1) + 1] = v;
                }
                if (j > 0) {
                    if (i < cr) c4[4 * ((size_t)(j - 1) * cr + i) + 2] = v;
                    if (i > 0) c4[4 * ((size_t)(j - 1) * cr + i - 1) + 3] = v;
                }
            }
        }
}

void launch_pic_prepare(const PicGeom &G, const PicInst *d_insts, int n_inst, cudaStream_t s)
{
    const int64_t nn = (int64_t)G.pnr * G.pnz;
    const unsigned bx = (unsigned)std::min<int64_t>((nn + 255) / 256, 512);
    pic_prepare_kernel<<<dim3(bx, n_inst), 256, 0, s>>>(G, d_insts);
}

void launch_pic_take(const PicGeom &G, const PicInst *d_insts, int n_inst, cudaStream_t s)
{
    const int64_t nn = (int64_t)G.pnr * G.pnz;
    const unsigned bx = (unsigned)std::min<int64_t>((nn + 255) / 256, 512);
    pic_take_kernel<<<dim3(bx, n_inst), 256, 0, s>>>(G, d_insts);
}

void launch_pic_clear_next(const PicGeom &G, const PicInst *d_insts, int n_inst, cudaStream_t s)
{
    const int64_t nn = (int64_t)G.pnr * G.pnz;
    const unsigned bx = (unsigned)std::min<int64_t>((nn + 255) / 256, 512);
    pic_clear_next_kernel<<<dim3(bx, n_inst), 256, 0, s>>>(G, d_insts);
}

void launch_deposit(const DepositArgs *d_args, const int32_t *d_tile_start, int n_inst, int total_tiles,
                    cudaStream_t s)
{
    if (total_tiles <= 0) return;
    deposit_kernel<<<total_tiles, 256, 0, s>>>(d_args, d_tile_start, n_inst);
}

// Launch of a contraction with `splits` CTAs per cluster along x.
void launch_sym(void (*kern)(PicGeom, const PicInst *, int, float), dim3 grid, int splits, const PicGeom &G,
                const PicInst *d_insts, float alpha, cudaStream_t s)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)splits;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, G, d_insts, splits, alpha);
}

// Radial tridiagonal solves of every axial mode: the 8-mode blocks on
// shared memory up to kThRows radial unknowns, the global-memory sweep
// above. Both run the Thomas recurrences with the elimination factors formed
// in FP64 (stored in FP32): in FP32 they leave the correction accurate
// enough that a warm-started solve on 256 x 1024 meets 1e-6 after one pass
// (residual about 2e-7), where parallel cyclic reduction, faster per call
// but with its eliminations rounded in FP32 at every level, left 1e-5 and
// needed a second pass.
void launch_thomas(const PicGeom &G, const PicInst *d_insts, int n_inst, cudaStream_t s)
{
    if (G.Nu <= kThRows)
        thomas_smem_kernel<<<dim3((G.M + kThModes - 1) / kThModes, 1, n_inst), 256, 0, s>>>(G, d_insts);
    else
        thomas_kernel<<<dim3((G.M + 255) / 256, 1, n_inst), 256, 0, s>>>(G, d_insts);
}

int launch_fast_solve(const PicGeom &G, const PicInst *d_insts, int n_inst, cudaStream_t s,
                      const CUtensorMap *tc_maps, int *tc_err, bool acc_phi)
{
    if (tc_maps != nullptr) {
        // hat[i][k] = 2/(M+1) sum_j rT[i][j] S[k][j]  (S symmetric)
        launch_dst_tc(tc_maps, 0, d_insts, n_inst, true, G, (float)(2.0 / (G.M + 1)), tc_err, s);
        launch_thomas(G, d_insts, n_inst, s);
        // d32[j][i] = sum_k S[j][k] hat[i][k]
        launch_dst_tc(tc_maps, 4, d_insts, n_inst, false, G, 1.0f, tc_err, s);
        if (!acc_phi) return 3;
        update_kernel<<<dim3(row_blocks(G.M, G.Nu), 1, n_inst), 256, 0, s>>>(G, d_insts);
        return 4;
    }
    // split the k range over a cluster of 2 to 8 CTAs while the 64 x 64
    // tiles would leave the SMs without a second resident CTA
    const int sms = G.n_sm > 0 ? G.n_sm : 148;
    const int H = (G.M + 1) / 2;
    const int64_t tiles = (int64_t)((H + 63) / 64) * ((G.Nu + 63) / 64) * n_inst;
    int splits = 1;
    while (splits < 8 && tiles * splits < 2 * sms && (H + 15) / 16 >= 4 * splits) splits *= 2;
    const dim3 gf((unsigned)(((H + 63) / 64) * splits), (G.Nu + 63) / 64, n_inst);
    const dim3 gi((unsigned)(((G.Nu + 63) / 64) * splits), (H + 63) / 64, n_inst);
    // hat[i][k] = 2/(M+1) sum_j r32[j][i] S[j][k]
    launch_sym(dst_sym_kernel<false>, gf, splits, G, d_insts, (float)(2.0 / (G.M + 1)), s);
    launch_thomas(G, d_insts, n_inst, s);
    // d32[j][i] = sum_k S[j][k] hat[i][k], or Phi[j+1][i] += that
    launch_sym(acc_phi ? dst_sym_kernel<true, true> : dst_sym_kernel<true, false>, gi, splits, G, d_insts, 1.0f,
               s);
    return 3;
}

void launch_esc(const PicGeom &G, const PicInst *d_insts, int n_inst, cudaStream_t s)
{
    esc_kernel<<<dim3(row_blocks(G.pnz, G.pnr), 1, n_inst), 256, 0, s>>>(G, d_insts);
}

__global__ void loop_reset_kernel(const PicInst *insts)
{
    if (threadIdx.x == 0) insts[0].red[7] = 0.0;
}

__global__ void loop_ctl_kernel(const PicInst *insts, int n_inst, int max_passes, cudaGraphConditionalHandle h)
{
    if (threadIdx.x != 0) return;
    const double c = insts[0].red[7] + 1.0;
    insts[0].red[7] = c;
    bool open = false;
    for (int i = 0; i < n_inst; ++i) open = open || *insts[i].conv == 0;
    cudaGraphSetConditional(h, (open && c < (double)max_passes) ? 1u : 0u);
}

__global__ void loop_open_kernel(const PicInst *insts, int n_inst, int done, int max_passes,
                                 cudaGraphConditionalHandle h)
{
    if (threadIdx.x != 0) return;
    insts[0].red[7] = (double)done;
    bool open = false;
    for (int i = 0; i < n_inst; ++i) open = open || *insts[i].conv == 0;
    cudaGraphSetConditional(h, (open && done < max_passes) ? 1u : 0u);
}

void launch_loop_open(const PicInst *d_insts, int n_inst, int done, int max_passes, cudaGraphConditionalHandle h,
                      cudaStream_t s)
{
    loop_open_kernel<<<1, 32, 0, s>>>(d_insts, n_inst, done, max_passes, h);
}

void launch_loop_reset(const PicInst *d_insts, cudaStream_t s)
{
    loop_reset_kernel<<<1, 32, 0, s>>>(d_insts);
}

void launch_loop_ctl(const PicInst *d_insts, int n_inst, int max_passes, cudaGraphConditionalHandle h,
                     cudaStream_t s)
{
    loop_ctl_kernel<<<1, 32, 0, s>>>(d_insts, n_inst, max_passes, h);
}

int launch_pic_solve(const PicGeom &G, const PicInst *d_insts, int n_inst, int max_refine, double tol,
                     cudaStream_t s, cudaStream_t aux, const CUtensorMap *tc_maps, int *tc_err)
{
    int launches = 0;
    // with the tensor-core contractions the residual is written transposed
    // by 32 x 32 tiles (at most kRedBlocks, tc_shape_ok)
    const dim3 gt((unsigned)((G.Nu + 31) / 32), (unsigned)((G.M + 31) / 32), (unsigned)n_inst);
    const dim3 gr(row_blocks(G.M, G.Nu), 1, (unsigned)n_inst);
    // each residual also takes the convergence decision (residual_close);
    // the first of a solve also forms ||b||^2
    auto residual = [&](cudaStream_t st, bool first) {
        if (tc_maps != nullptr) {
            if (first) residual_t_kernel<true><<<gt, 256, 0, st>>>(G, d_insts, tol);
            else residual_t_kernel<false><<<gt, 256, 0, st>>>(G, d_insts, tol);
        } else {
            if (first) residual_kernel<true><<<gr, 256, 0, st>>>(G, d_insts, tol);
            else residual_kernel<false><<<gr, 256, 0, st>>>(G, d_insts, tol);
        }
    };
    // graph capture: initial residual, the first kFixedPasses passes of (fast
    // solve with the update fused, residual) as plain nodes (their kernels
    // return at once after convergence), then the rest of the at most
    // max_refine passes under device control. A warm-started solve mostly
    // converges within the plain pass, and a loop that its opening kernel
    // leaves closed costs less than loop iterations do.
    if (max_refine > 0 && stream_capturing(s, aux)) {
        constexpr int kFixedPasses = 1;
        const int fixed = std::min(max_refine, kFixedPasses);
        residual(s, true);
        for (int k = 0; k < fixed; ++k) {
            launch_fast_solve(G, d_insts, n_inst, s, tc_maps, tc_err, true);
            residual(s, false);
        }
        if (max_refine > fixed) {
            const bool looped = capture_while(
                s, aux, d_insts,
                [&](cudaStream_t b, cudaGraphConditionalHandle h) {
                    launch_fast_solve(G, d_insts, n_inst, b, tc_maps, tc_err, true);
                    residual(b, false);
                    launch_loop_ctl(d_insts, n_inst, max_refine, h, b);
                },
                n_inst, fixed, max_refine);
            if (!looped) return -1;
        }
        launch_esc(G, d_insts, n_inst, s);
        return 3 + 4 * fixed;
    }
    for (int it = 0; it <= max_refine; ++it) {
        residual(s, it == 0);
        launches += 1;
        if (it == max_refine) break;
        launches += launch_fast_solve(G, d_insts, n_inst, s, tc_maps, tc_err, true);
    }
    launch_esc(G, d_insts, n_inst, s);
    return launches + 1;
}

} // namespace mucite
