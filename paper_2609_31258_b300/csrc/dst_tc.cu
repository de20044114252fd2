// DST-I contractions of the space-charge fast solve on the tensor cores
// ("Axisymmetric PIC space charge update": each refinement pass corrects Phi
// by a DST-I in z, a tridiagonal solve per axial mode in r and the inverse
// DST-I; both transforms are dense contractions with the sine matrix
// S[j][k] = sin(pi (j+1)(k+1) / (M+1)), which is symmetric).
//
//   C[m][n] = alpha sum_k A[m][k] B[n][k],   A and B stored K-major, C row-major:
//   forward: hat[i][k] = 2/(M+1) sum_j rT[i][j] S[k][j]   (A = rT,  B = S)
//   inverse: d[j][i]   = sum_k S[j][k] hat[i][k]           (A = S,   B = hat)
//
// Precision: every operand comes as a pair x = x_hi + x_lo with x_hi the
// value rounded to TF32 (10 mantissa bits) and x_lo the rest, and each
// product is formed as A_hi B_hi + A_hi B_lo + A_lo B_hi (three TF32 MMAs):
// about 2^-21 relative error, the accuracy of the FP32 contraction. A single
// TF32 product (2^-11) is not enough here: the error of the inverse transform
// is white in z, the next residual applies the operator to it, and the
// operator amplifies its high modes by its condition number, so the FP64
// refinement around the solve (pic.cu) would need several more passes.
//
// One CTA (4 warps) computes a 128 x 128 output tile over a share of the K
// range: TMA brings 32-column chunks of the four operand tiles (A_hi, A_lo,
// B_hi, B_lo; 128-byte swizzle) into a ring of three 64 KB slots of shared
// memory (one "full" mbarrier per slot); one thread issues tcgen05.mma
// (kind::tf32, M = N = 128, K = 8 per instruction) into a 128 x 128 FP32
// accumulator in tensor memory and, after each chunk, tcgen05.commit to the
// slot's "empty" mbarrier, which frees the slot for the chunk three ahead.
// The four warps read their 32 lanes of the accumulator back with
// tcgen05.ld. The K range is split over the CTAs of a thread-block cluster
// (up to 8): every CTA leaves its partial tile in shared memory and, after a
// cluster barrier, CTA r adds the partials of its share of the rows through
// distributed shared memory in rank order, so every output is a sum in a
// fixed order (deterministic).
//
// Every wait is bounded: a wait that gives up raises *err, waits (again
// bounded) for the copies and products still in flight, frees the tensor
// memory and still joins both cluster barriers, so no CTA of the cluster is
// left waiting.
#include <cooperative_groups.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "pic.cuh"

namespace mucite {

namespace {

constexpr int kTile = 128;     // output tile rows and columns (UMMA M = N = 128)
constexpr int kChunk = 32;     // K elements per staged chunk: one 128-byte swizzled row
constexpr int kSlots = 3;      // ring of staged chunks per CTA
constexpr int kMaxChunks = 16; // chunks of one CTA's K share
constexpr int kPadN = kTile + 4; // row stride (floats) of the partial tile in shared memory
constexpr uint32_t kSpins = 1u << 26;          // backstop on the polls of one wait
constexpr uint64_t kWaitNs = 250ull * 1000 * 1000; // wall-clock bound of one wait (0.25 s)
constexpr uint32_t kSlice = (uint32_t)kTile * kChunk * 4u; // bytes of one operand's chunk (16 KB)
constexpr uint32_t kChunkBytes = 4u * kSlice;              // A_hi, A_lo, B_hi, B_lo slices of one chunk

// Instruction descriptor of tcgen05.mma kind::tf32: D in FP32 (bits 4-5 = 1),
// A and B in TF32 (bits 7-9 and 10-12 = 2), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTile >> 3) << 17) |
                            ((uint32_t)(kTile >> 4) << 24);

__device__ __forceinline__ uint32_t su32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// true once the phase of the given parity has completed; false when it has
// not after kWaitNs of wall-clock time (%globaltimer) or kSpins polls
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity)
{
    uint64_t t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (uint32_t it = 0; it < kSpins; ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(bar), "r"(parity)
                     : "memory");
        if (done) return true;
        if ((it & 63u) == 63u) {
            uint64_t t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            if (t - t0 > kWaitNs) return false;
        }
    }
    return false;
}

// Shared-memory matrix descriptor of a K-major operand with the 128-byte
// swizzle: start address >> 4 (bits 0-13), leading byte offset 16 (unused
// for this layout), stride byte offset 1024 between 8-row groups (bits
// 32-45), descriptor version 1 (bits 46-47), swizzle mode 2 = 128 bytes
// (bits 61-63). The chunk's base is 1024-byte aligned; the K step within the
// 128-byte row advances the start address by 32 bytes.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int c0, int c1, uint64_t *bar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3}], [%4];" ::"r"(su32(dst)),
                 "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(su32(bar))
                 : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "setp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                 "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
                 : "memory");
}

// 16 consecutive accumulator columns of this thread's lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v)
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                 "%12, %13, %14, %15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                   "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

} // namespace

// grid (n tiles x splits, m tiles), cluster (splits, 1, 1), 128 threads;
// dynamic shared memory: the ring of slots (or the partial tile, if larger)
// + 1 KB for alignment.
__global__ void __launch_bounds__(128, 1)
    dst_tc_kernel(const CUtensorMap *maps, int first, const PicInst *insts, int forward, int ldc, int Mg, int Ng,
                  int n_chunks, int per_split, float alpha, int *err)
{
    namespace cg = cooperative_groups;
    extern __shared__ unsigned char dyn[];
    __shared__ __align__(8) uint64_t full_bar[kSlots];
    __shared__ __align__(8) uint64_t empty_bar[kSlots];
    __shared__ __align__(8) uint64_t mma_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int fail;
    const PicInst &I = insts[blockIdx.z];
    if (*I.conv) return; // this instance has converged: every CTA of its clusters returns
    float *C = forward ? I.hat : I.d32;
    const CUtensorMap *ta_hi = maps + (size_t)blockIdx.z * kTcMaps + first, *ta_lo = ta_hi + 1,
                      *tb_hi = ta_hi + 2, *tb_lo = ta_hi + 3;
    cg::cluster_group cluster = cg::this_cluster();
    const unsigned splits = cluster.num_blocks();
    const unsigned rank = cluster.block_rank();
    unsigned char *sm = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(dyn) + 1023) &
                                                          ~static_cast<uintptr_t>(1023));
    const int tid = threadIdx.x, warp = tid >> 5;
    const int m0 = blockIdx.y * kTile, n0 = (int)(blockIdx.x / splits) * kTile;
    const int cb = (int)rank * per_split;
    const int nc = max(0, min(per_split, n_chunks - cb));
    if (tid == 0) {
        for (int k = 0; k < kSlots; ++k) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&full_bar[k])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&empty_bar[k])) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&mma_bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fail = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_slot)),
                     "r"(kTile)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    int issued = 0;   // chunks whose copies were issued (thread 0)
    int consumed = 0; // chunks whose products were issued (thread 0)
    bool committed = false;
    if (tid == 0 && nc > 0) {
        // the descriptors were copied into device memory before the launch:
        // make them visible to the tensor-map proxy before the first copy
        for (int q = 0; q < 4; ++q)
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(ta_hi + q) : "memory");
        auto load = [&](int c) {
            const int sl = c % kSlots;
            unsigned char *a = sm + (size_t)sl * kChunkBytes;
            const int k0 = (cb + c) * kChunk;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(&full_bar[sl])),
                         "r"(kChunkBytes)
                         : "memory");
            tma_load_2d(a, ta_hi, k0, m0, &full_bar[sl]);
            tma_load_2d(a + kSlice, ta_lo, k0, m0, &full_bar[sl]);
            tma_load_2d(a + 2 * kSlice, tb_hi, k0, n0, &full_bar[sl]);
            tma_load_2d(a + 3 * kSlice, tb_lo, k0, n0, &full_bar[sl]);
            ++issued;
        };
        for (int c = 0; c < nc && c < kSlots; ++c) load(c);
        bool ok = true;
        for (int c = 0; c < nc; ++c) {
            const int sl = c % kSlots;
            if (!(ok = bar_wait(su32(&full_bar[sl]), (uint32_t)(c / kSlots) & 1u))) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ahi = su32(sm + (size_t)sl * kChunkBytes), alo = ahi + kSlice, bhi = ahi + 2 * kSlice,
                           blo = ahi + 3 * kSlice;
#pragma unroll
            for (int kk = 0; kk < kChunk / 8; ++kk) {
                const uint32_t o = 32u * kk;
                mma_tf32(tmem, sw128_desc(ahi + o), sw128_desc(bhi + o), (c > 0 || kk > 0) ? 1u : 0u);
                mma_tf32(tmem, sw128_desc(ahi + o), sw128_desc(blo + o), 1u);
                mma_tf32(tmem, sw128_desc(alo + o), sw128_desc(bhi + o), 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             su32(&empty_bar[sl]))
                         : "memory");
            ++consumed;
            // refill the slot of the previous chunk once its products are done
            // (one chunk of products stays queued behind the wait)
            if (c >= 1 && c - 1 + kSlots < nc) {
                const int p = c - 1;
                if (!(ok = bar_wait(su32(&empty_bar[p % kSlots]), (uint32_t)(p / kSlots) & 1u))) break;
                load(p + kSlots);
            }
        }
        // every product issued so far completes on mma_bar (also on failure,
        // so that the tensor memory is not released under running products)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         su32(&mma_bar))
                     : "memory");
        committed = true;
        if (!ok) fail = 1;
    }
    __syncthreads();
    bool ok = fail == 0;
    if (ok && nc > 0) ok = bar_wait(su32(&mma_bar), 0);
    const bool bad = __syncthreads_or(!ok) != 0;
    if (bad && tid == 0) {
        // copies still in flight land and the products finish before the
        // shared and tensor memory they use are released (each wait bounded)
        for (int c = consumed; c < issued; ++c) (void)bar_wait(su32(&full_bar[c % kSlots]), (uint32_t)(c / kSlots) & 1u);
        if (committed) (void)bar_wait(su32(&mma_bar), 0);
        atomicExch(err, 1);
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // the partial tile over the slots (their products are complete)
    float *P = reinterpret_cast<float *>(sm);
    if (!bad && nc > 0) {
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c0 = 0; c0 < kTile; c0 += 16) {
            float v[16];
            tmem_ld16(lane_base + (uint32_t)c0, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) P[tid * kPadN + c0 + q] = v[q];
        }
    } else {
        for (int q = 0; q < kTile; ++q) P[tid * kPadN + q] = 0.0f;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTile) : "memory");
    // rows [r0, r0 + rows) of the tile: the cluster's partials in rank order
    cluster.sync();
    const int rows = kTile / (int)splits, r0 = (int)rank * rows;
    for (int e = tid; e < rows * kTile; e += blockDim.x) {
        const int rr = r0 + e / kTile, cc = e % kTile;
        float acc = 0.0f;
        for (unsigned q = 0; q < splits; ++q) acc += cluster.map_shared_rank(P, q)[rr * kPadN + cc];
        const int gm = m0 + rr, gn = n0 + cc;
        if (gm < Mg && gn < Ng) C[(size_t)gm * ldc + gn] = alpha * acc;
    }
    cluster.sync(); // the partials stay readable until every CTA of the cluster is done
}

namespace {

size_t tc_smem_bytes()
{
    return std::max<size_t>((size_t)kSlots * kChunkBytes, (size_t)kTile * kPadN * 4) + 1024;
}

void tc_split(int K, int &n_chunks, int &splits, int &per)
{
    n_chunks = (K + kChunk - 1) / kChunk;
    splits = 1;
    while (splits < 8 && splits * 2 <= n_chunks) splits *= 2;
    per = (n_chunks + splits - 1) / splits;
}

} // namespace

bool tc_shape_ok(const PicGeom &G)
{
    int n_chunks, splits, per;
    tc_split(G.M, n_chunks, splits, per);
    const int64_t tiles = (int64_t)((G.Nu + 31) / 32) * ((G.M + 31) / 32); // transposed-residual blocks
    return per <= kMaxChunks && G.hld % 4 == 0 && G.Nu >= 1 && G.M >= 1 && tiles <= kRedBlocks;
}

bool launch_dst_tc(const CUtensorMap *maps, int first, const PicInst *d_insts, int n_inst, bool forward,
                   const PicGeom &G, float alpha, int *err, cudaStream_t s)
{
    // forward: hat[i][k] (Mg = Nu, Ng = M); inverse: d[j][i] (Mg = M, Ng = Nu); K = M
    const int Mg = forward ? G.Nu : G.M, Ng = forward ? G.M : G.Nu, ldc = forward ? G.hld : G.Nu;
    int n_chunks, splits, per;
    tc_split(G.M, n_chunks, splits, per);
    if (per > kMaxChunks) return false;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(((Ng + kTile - 1) / kTile) * splits), (unsigned)((Mg + kTile - 1) / kTile),
                       (unsigned)n_inst);
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = tc_smem_bytes();
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)splits;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, dst_tc_kernel, maps, first, d_insts, forward ? 1 : 0, ldc, Mg, Ng, n_chunks,
                              per, alpha, err) == cudaSuccess;
}

bool tc_prepare()
{
    // the largest dynamic shared memory a launch asks for, set once (not a
    // stream operation, so never inside a capture); then whether a cluster of
    // 8 such CTAs can be resident at all
    const size_t smem = tc_smem_bytes();
    if (cudaFuncSetAttribute(dst_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return false;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(8, 1, 1);
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 8;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, dst_tc_kernel, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return clusters >= 1;
}

bool make_tc_map(CUtensorMap *map, const float *base, int rows, int cols, int ld, int box_rows)
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    std::call_once(once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    if (encode == nullptr || ((uintptr_t)base & 15u) != 0 || ((size_t)ld * 4) % 16 != 0 || box_rows < 1 ||
        box_rows > 256)
        return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    const cuuint32_t box[2] = {(cuuint32_t)kChunk, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

} // namespace mucite
