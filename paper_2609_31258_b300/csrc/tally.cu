// Observables of one instance from its pack pool ("Terminal events,
// snapshots, and reported observables"; Eq. 8; conservation of represented
// weight, "Continuous current Gaussian source"): counts and represented
// weight per status, exit-time histogram of transmitted weight (Eq. 8 up to
// the factor qe/dt), exit-radius, KE and T_eff histograms of the transmitted
// weight (percentiles and the 95% beam radius are read from them), and the
// electrode loss map. Quantities that decide a bin are formed in FP64 (KE,
// T_eff) or FP32 (lattice radius) with explicit round-to-nearest operations
// in a fixed order, so the bins are exact functions of the state.
#include "kernels.cuh"

namespace mucite {


namespace {

__device__ __forceinline__ int32_t q32t(double v)
{
    const double r = rint(v);
    if (r < -2147483648.0) return INT32_MIN;
    if (r > 2147483647.0) return INT32_MAX;
    return (int32_t)r;
}

__device__ __forceinline__ int64_t bin_d(double v, int n)
{
    if (!(v < (double)n)) return n - 1;
    const int64_t b = __double2ll_rz(v);
    return b < 0 ? 0 : b;
}

__device__ __forceinline__ int64_t bin_f(float v, int n)
{
    if (!(v < (float)n)) return n - 1;
    const int64_t b = __float2ll_rz(v);
    return b < 0 ? 0 : b;
}

__device__ __forceinline__ double teff_exact(const Profile &pf, double eint)
{
    const double e = __ddiv_rn(eint, pf.n3);
    if (e <= pf.ecap) {
        const double disc = __dadd_rn(__dmul_rn(pf.c0, pf.c0), __dmul_rn(__dmul_rn(2.0, pf.c1), e));
        return __ddiv_rn(__dmul_rn(2.0, e), __dadd_rn(pf.c0, __dsqrt_rn(disc)));
    }
    return __dadd_rn(pf.tcap, __dsub_rn(e, pf.ecap));
}

} // namespace

__global__ void __launch_bounds__(256) tally_kernel(TallyArgs A)
{
    __shared__ unsigned long long s_cnt[8];
    __shared__ double s_ke[8], s_te[8], s_sy[8];
    if (threadIdx.x < 8) {
        s_cnt[threadIdx.x] = 0;
        s_ke[threadIdx.x] = 0.0;
        s_te[threadIdx.x] = 0.0;
        s_sy[threadIdx.x] = 0.0;
    }
    __syncthreads();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int st = 8;
    double wke = 0.0, wte = 0.0, wsy = 0.0; // the pack's weighted KE, T_eff and SY
    if (p < A.n) {
        st = A.status[p];
        if (st < 8) {
            int32_t xq, yq, zq;
            double vx, vy, vz, ei, ls;
            if (A.precision == MUCITE_FP32) {
                xq = ((const int32_t *)A.x)[p];
                yq = ((const int32_t *)A.y)[p];
                zq = ((const int32_t *)A.z)[p];
                vx = ((const float *)A.vx)[p];
                vy = ((const float *)A.vy)[p];
                vz = ((const float *)A.vz)[p];
                ei = ((const float *)A.eint)[p];
                ls = ((const float *)A.lnsy)[p];
            } else {
                xq = q32t(__dmul_rn(((const double *)A.x)[p], A.sx));
                yq = q32t(__dmul_rn(((const double *)A.y)[p], A.sx));
                zq = q32t(__dmul_rn(__dsub_rn(((const double *)A.z)[p], A.gz0), A.sz));
                vx = ((const double *)A.vx)[p];
                vy = ((const double *)A.vy)[p];
                vz = ((const double *)A.vz)[p];
                ei = ((const double *)A.eint)[p];
                ls = ((const double *)A.lnsy)[p];
            }
            double v2 = __dmul_rn(vx, vx);
            v2 = __dadd_rn(v2, __dmul_rn(vy, vy));
            v2 = __dadd_rn(v2, __dmul_rn(vz, vz));
            const double ke = __dmul_rn(v2, A.c_ke);
            const double te = teff_exact(A.prof, ei);
            const double W = (double)A.weight;
            wke = W * ke;
            wte = W * te;
            wsy = W * exp(ls);
            const float fx = (float)xq, fy = (float)yq;
            const float rr = __fsqrt_rn(__fadd_rn(__fmul_rn(fx, fx), __fmul_rn(fy, fy)));
            const unsigned long long Wu = (unsigned long long)A.weight;
            if (st == MUCITE_TRANSMITTED) {
                int64_t b = (int64_t)A.t_term[p] / A.exit_bin_steps;
                b = b < 0 ? 0 : (b > A.n_exit_bins - 1 ? A.n_exit_bins - 1 : b);
                atomicAdd(&A.exit_hist[b], Wu);
                atomicAdd(&A.r_hist[bin_f(__fmul_rn(rr, A.r_scale), A.n_r_bins)], Wu);
                atomicAdd(&A.ke_hist[bin_d(__dmul_rn(ke, A.ke_scale), A.n_ke_bins)], Wu);
                atomicAdd(&A.teff_hist[bin_d(__dmul_rn(te, A.t_scale), A.n_teff_bins)], Wu);
            } else if (st == MUCITE_ELECTRODE) {
                const int64_t br = bin_f(__fmul_rn(rr, A.lr_scale), A.n_loss_r);
                int64_t bz = ((int64_t)zq * A.n_loss_z) >> 30;
                bz = bz < 0 ? 0 : (bz > A.n_loss_z - 1 ? A.n_loss_z - 1 : bz);
                atomicAdd(&A.loss_map[bz * A.n_loss_r + br], Wu);
            }
        }
    }
    // per status, the warp's packs summed first (lanes of one status at a
    // time, a butterfly over the warp), then one shared-memory atomic per
    // status present instead of one per pack
    constexpr unsigned kAll = 0xffffffffu;
    const bool valid = st < 8;
    unsigned todo = __ballot_sync(kAll, valid);
    while (todo != 0u) {
        const int src = __ffs(todo) - 1;
        const int s = __shfl_sync(kAll, st, src);
        const bool mine = valid && st == s;
        const unsigned m = __ballot_sync(kAll, mine);
        double a = mine ? wke : 0.0, b = mine ? wte : 0.0, c = mine ? wsy : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(kAll, a, o);
            b += __shfl_xor_sync(kAll, b, o);
            c += __shfl_xor_sync(kAll, c, o);
        }
        if ((int)(threadIdx.x & 31u) == src) {
            atomicAdd(&s_cnt[s], (unsigned long long)__popc(m));
            atomicAdd(&s_ke[s], a);
            atomicAdd(&s_te[s], b);
            atomicAdd(&s_sy[s], c);
        }
        todo &= ~m;
    }
    __syncthreads();
    if (threadIdx.x < 8 && s_cnt[threadIdx.x]) {
        const int st = threadIdx.x;
        atomicAdd(&A.count[st], s_cnt[st]);
        atomicAdd(&A.wsum[st], s_cnt[st] * (unsigned long long)A.weight);
        atomicAdd(&A.sum_ke[st], s_ke[st]);
        atomicAdd(&A.sum_teff[st], s_te[st]);
        atomicAdd(&A.sum_sy[st], s_sy[st]);
    }
}

void launch_tally(const TallyArgs &A, cudaStream_t s)
{
    if (A.n <= 0) return;
    tally_kernel<<<(unsigned)((A.n + 255) / 256), 256, 0, s>>>(A);
}

} // namespace mucite
