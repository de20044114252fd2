// Space-charge Poisson solve without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs after start-up under a
// fixed device-memory budget (a serving process whose memory is fully
// reserved up front, or a host framework whose own pool owns the device
// memory and forbids allocations outside it), and real-time loops that must
// not block on the allocator. For them, mucite_poisson_solve_noalloc keeps
// all of its scratch -- the sine matrix, the tridiagonal factors, the residual
// and transform buffers and the convergence bookkeeping -- in one file-scope
// device array of fixed size, MUCITE_NOALLOC_SCRATCH_BYTES, that every device
// which loads the library holds until the process exits. The caller passes
// the node charges and the output buffers; nothing is allocated on any call.
// The sine matrix and the tridiagonal factors depend on the grid only: they
// are rebuilt when a call's grid differs from the one they were last built
// for on that device.
#include <mutex>

#include "pic.cuh"

namespace mucite {

namespace {

constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[MUCITE_NOALLOC_SCRATCH_BYTES];

std::mutex g_setup_mutex;
unsigned char *g_scratch_addr[kMaxDevices] = {};
int g_n_sm[kMaxDevices] = {};

// Grid whose tables the scratch of a device holds (guarded by g_setup_mutex).
struct TableKey {
    int nr = 0, nz = 0;
    double R = 0.0, z0 = 0.0, z1 = 0.0;
    bool operator==(const TableKey &o) const
    {
        return nr == o.nr && nz == o.nz && R == o.R && z0 == o.z0 && z1 == o.z1;
    }
};
TableKey g_tables[kMaxDevices];

// Byte layout of the scratch for an M x Nu problem (256-byte aligned pieces).
struct ScratchLayout {
    size_t inst, red, conv, part, ticket, S, cp, invm, lo, a, c, A, r32, hat, d32, total;
};

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

ScratchLayout scratch_layout(int M, int Nu)
{
    ScratchLayout L{};
    size_t off = 0;
    auto put = [&](size_t &o, size_t bytes) {
        o = off;
        off += up256(bytes);
    };
    put(L.inst, sizeof(PicInst));
    put(L.red, 4 * sizeof(double));
    put(L.conv, sizeof(int));
    put(L.part, 2 * (size_t)kRedBlocks * sizeof(double));
    put(L.ticket, sizeof(unsigned));
    put(L.S, (size_t)M * M * sizeof(float));
    put(L.cp, (size_t)Nu * M * sizeof(float));
    put(L.invm, (size_t)Nu * M * sizeof(float));
    put(L.lo, (size_t)Nu * sizeof(float));
    put(L.a, (size_t)Nu * sizeof(double));
    put(L.c, (size_t)Nu * sizeof(double));
    put(L.A, (size_t)Nu * sizeof(double));
    put(L.r32, (size_t)M * Nu * sizeof(float));
    put(L.hat, (size_t)((M + 3) / 4 * 4) * Nu * sizeof(float));
    put(L.d32, (size_t)M * Nu * sizeof(float));
    L.total = off;
    return L;
}

// Operator coefficients and the sine matrix of the DST-I (same definitions as
// the context path): a_i, c_i, A_i per radial row; S_jk = sin(pi j k/(M+1)).
__global__ void na_tables_kernel(int M, int Nu, double rz, float *S, float *lo, double *a, double *c,
                                 double *A)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < (int64_t)M * M) {
        const int j = (int)(e / M) + 1, k = (int)(e % M) + 1;
        const int64_t jk = ((int64_t)j * k) % (2LL * (M + 1));
        S[e] = (float)sinpi((double)jk / (double)(M + 1));
    }
    if (e < Nu) {
        const int i = (int)e;
        const double ai = i == 0 ? 0.0 : 2.0 * (i - 0.5);
        const double ci = i == 0 ? 1.0 : 2.0 * (i + 0.5);
        const double Ai = i == 0 ? rz / 4.0 : 2.0 * i * rz;
        a[i] = ai;
        c[i] = ci;
        A[i] = Ai;
        lo[i] = (float)ai;
    }
}

// Elimination factors of the tridiagonal system of axial mode k (one thread
// per mode, sequential in r).
__global__ void na_thomas_factors_kernel(int M, int Nu, const double *a, const double *c,
                                         const double *A, float *cp, float *invm)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M) return;
    const double s = sinpi((double)(k + 1) / (2.0 * (M + 1)));
    const double lam = 4.0 * s * s;
    double cprev = 0.0;
    for (int i = 0; i < Nu; ++i) {
        const double d = -(a[i] + c[i] + A[i] * lam);
        const double m = i == 0 ? d : d - a[i] * cprev;
        const double cpi = c[i] / m;
        cp[(size_t)i * M + k] = (float)cpi;
        invm[(size_t)i * M + k] = (float)(1.0 / m);
        cprev = cpi;
    }
}

__global__ void na_set_inst_kernel(PicInst *dst, PicInst v)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *dst = v;
}

__global__ void na_copy_rel_kernel(const double *red, double *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *out = red[2];
}

} // namespace

} // namespace mucite

using namespace mucite;

extern "C" mucite_status mucite_poisson_solve_noalloc(int device, void *cuda_stream,
                                                      const mucite_grid *pic, const int64_t *d_Q,
                                                      double *d_phi, float *d_esc,
                                                      double *d_rel_residual)
{
    if (!pic || !d_Q || !d_phi || !d_esc) return MUCITE_E_ARG;
    if (device < 0 || device >= kMaxDevices) return MUCITE_E_ARG;
    if (pic->nr < 3 || pic->nz < 3 || !(pic->R > 0.0) || !(pic->z1 > pic->z0)) return MUCITE_E_ARG;
    const int M = pic->nz - 2, Nu = pic->nr - 1;
    const ScratchLayout L = scratch_layout(M, Nu);
    if (L.total > (size_t)MUCITE_NOALLOC_SCRATCH_BYTES) return MUCITE_E_ARG; // grid beyond the fixed scratch
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return MUCITE_E_CUDA;
    if (prev != device && cudaSetDevice(device) != cudaSuccess) return MUCITE_E_CUDA;
    mucite_status st = MUCITE_OK;
    do {
        // an error left by unrelated earlier work is not this call's
        (void)cudaGetLastError();
        // One-time set-up on this device, with the device current: the host
        // name of the array is only a stand-in, so take its device address.
        // Under lazy module loading this lookup is also what loads the module
        // and reserves the array on the device.
        unsigned char *base = nullptr;
        int n_sm = 0;
        bool rebuild = false;
        const TableKey key{pic->nr, pic->nz, pic->R, pic->z0, pic->z1};
        {
            std::lock_guard<std::mutex> lock(g_setup_mutex);
            if (!g_scratch_addr[device]) {
                void *p = nullptr;
                int sms = 0;
                if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess ||
                    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
                    st = MUCITE_E_CUDA;
                    break;
                }
                g_scratch_addr[device] = (unsigned char *)p;
                g_n_sm[device] = sms;
            }
            base = g_scratch_addr[device];
            n_sm = g_n_sm[device];
            rebuild = !(g_tables[device] == key);
            g_tables[device] = key; // the tables below are enqueued before any later call's work
        }
        cudaStream_t s = (cudaStream_t)cuda_stream;
        PicGeom G{};
        G.pnr = pic->nr;
        G.pnz = pic->nz;
        G.M = M;
        G.Nu = Nu;
        G.hld = (M + 3) / 4 * 4;
        G.dr = pic->R / (pic->nr - 1);
        G.dz = (pic->z1 - pic->z0) / (pic->nz - 1);
        G.bscale = -(kE / kLat) / (kEps0 * kPi * G.dz);
        G.S = (float *)(base + L.S);
        G.cp = (float *)(base + L.cp);
        G.invm = (float *)(base + L.invm);
        G.lo = (float *)(base + L.lo);
        G.a = (double *)(base + L.a);
        G.c = (double *)(base + L.c);
        G.A = (double *)(base + L.A);
        G.n_sm = n_sm;
        if (rebuild) {
            const double rz = (G.dr * G.dr) / (G.dz * G.dz);
            const int64_t nt = std::max<int64_t>((int64_t)M * M, Nu);
            na_tables_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(M, Nu, rz, (float *)G.S,
                                                                         (float *)G.lo, (double *)G.a,
                                                                         (double *)G.c, (double *)G.A);
            na_thomas_factors_kernel<<<(M + 127) / 128, 128, 0, s>>>(M, Nu, G.a, G.c, G.A, (float *)G.cp,
                                                                   (float *)G.invm);
        }
        PicInst I{};
        I.Q = (unsigned long long *)d_Q;
        I.phi = d_phi;
        I.r32 = (float *)(base + L.r32);
        I.hat = (float *)(base + L.hat);
        I.d32 = (float *)(base + L.d32);
        I.esc = (float2 *)d_esc;
        I.er64 = nullptr;
        I.ez64 = nullptr;
        I.red = (double *)(base + L.red);
        I.conv = (int *)(base + L.conv);
        // per-block partial sums added up in block order: the norms, the
        // convergence decision and the reported residual are reproducible
        I.part = (double *)(base + L.part);
        I.ticket = (unsigned *)(base + L.ticket);
        PicInst *d_inst = (PicInst *)(base + L.inst);
        na_set_inst_kernel<<<1, 32, 0, s>>>(d_inst, I);
        // the solve starts from Phi = 0; bookkeeping left by the previous call is cleared
        if (cudaMemsetAsync(d_phi, 0, (size_t)pic->nr * pic->nz * sizeof(double), s) != cudaSuccess ||
            cudaMemsetAsync(I.red, 0, 4 * sizeof(double), s) != cudaSuccess ||
            cudaMemsetAsync(I.conv, 0, sizeof(int), s) != cudaSuccess ||
            cudaMemsetAsync(I.ticket, 0, sizeof(unsigned), s) != cudaSuccess) {
            st = MUCITE_E_CUDA;
            break;
        }
        launch_pic_solve(G, d_inst, 1, 8, 1e-6, s);
        if (d_rel_residual) na_copy_rel_kernel<<<1, 32, 0, s>>>(I.red, d_rel_residual);
        if (cudaGetLastError() != cudaSuccess) st = MUCITE_E_CUDA;
    } while (0);
    if (st != MUCITE_OK) {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        g_tables[device] = TableKey{}; // the tables may not have been built
    }
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    return st;
}
