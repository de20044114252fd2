// Host side of the C ABI declared in include/mucite.h: context, field
// loading, instances (pack pools owned by the caller), stepping with the
// space-charge macro step interleaved, tallies. All device work is enqueued
// on the context stream; calls return a status and never throw.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "pic.cuh"

using namespace mucite;

namespace {

struct Instance {
    bool used = false;
    mucite_ion_template ion{};
    mucite_source src{};
    mucite_run run{};
    void *pool = nullptr;
    int64_t capacity = 0;
    mucite_layout lay{};
    int64_t n_slots = 0;
    int64_t step = 0;
    double rf_phase0 = 0.0;  // RF phase at the start of the current dt segment
    int64_t seg_step0 = 0;   // step at the start of the current dt segment
    double src_acc = 0.0;
    unsigned long long *d_counters = nullptr; // [kCounters]
    // tally buffers: [0..7] count, [8..15] wsum, then hist arrays; sums in d_tsum
    unsigned long long *d_tally = nullptr;
    double *d_tsum = nullptr; // [24]: sum_ke[8], sum_teff[8], sum_sy[8]
    int64_t tally_len = 0;
    bool has_pic = false;
    bool pic_masked = false;
    PicInst pic{};
    InstF32 f32{};
    InstF64 f64{};
    // tensor-core contractions of a maskless solve: transposed residual and
    // the TMA descriptors of its operands (tc_on when all could be made)
    bool tc_on = false;
    float *tc_rT = nullptr, *tc_rT_lo = nullptr, *tc_hat_lo = nullptr;
    CUtensorMap tc_maps[kTcMaps]{}; // rT, rT_lo, S, S_lo (forward), S, S_lo, hat, hat_lo (inverse)
};

} // namespace

static_assert(MUCITE_SCHEDULE_EAGER == kEagerWeight, "the eager schedule is the eager kernel instantiation");

struct mucite_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t aux = nullptr; // captures the bodies of device-controlled solve loops
    // streams the per-instance collision launches of a batch run side by side
    // on (forked from and joined back into the context stream by events)
    static constexpr int kStepStreams = 16;
    cudaStream_t step_streams[kStepStreams] = {};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[kStepStreams] = {};
    bool device_loops = true;   // cleared if a driver cannot build them: fixed pass sequences instead
    std::string err;
    bool fields = false;
    mucite_grid g{};
    NodeF *d_node = nullptr;
    float *d_dmask = nullptr;
    double *d_f64[8] = {};
    bool has_pic_grid = false;
    mucite_grid pg_grid{};
    PicGeom pg{};
    float *d_S = nullptr, *d_cp = nullptr, *d_invm = nullptr, *d_lo = nullptr;
    // tensor-core DST-I (single-instance maskless solves): the sine matrix as
    // a TF32 pair with rows of hld floats, its TMA descriptors, and an error
    // word raised when a bounded wait of the contraction gives up
    float *d_Spad = nullptr, *d_Spad_lo = nullptr;
    CUtensorMap map_S{}, map_S_lo{}, map_SA{}, map_SA_lo{}; // S as a B operand, as an A operand
    bool tc_ok = false;              // device and PIC grid allow the tensor-core contractions
    bool use_tc = false;             // the caller chose them (mucite_set_pic_solver)
    int *d_tc_err = nullptr;
    CUtensorMap *d_tc_maps = nullptr; // [MUCITE_MAX_INSTANCES][kTcMaps] descriptors of a PIC upload's plain group
    bool tc_group = false;            // the plain solves of the last PIC upload take the tensor cores
    double *d_a = nullptr, *d_c = nullptr, *d_A = nullptr;
    uint8_t *d_pic_metal = nullptr; // metal flags of the PIC nodes
    unsigned *d_limits = nullptr;   // Eq. 1 reduction scratch [3]
    bool pic_has_metal = false;
    Instance inst[MUCITE_MAX_INSTANCES];
    InstF32 *d_insts = nullptr;
    int32_t *d_tiles = nullptr;
    unsigned *d_ticket = nullptr;   // arrival ticket of the streamed single-step kernel (zero between launches)
    bool last_stream = false;       // the last step launch was the streamed single-step kernel
    int hold_tile = -1;             // test hook: withhold the staged copies of this tile of the next streamed launch
    PicInst *d_picinst = nullptr;
    DepositArgs *d_dep = nullptr;
    int32_t *d_dep_tiles = nullptr;
    float *d_rf = nullptr;       // per-instance RF scalars of the current launch
    size_t rf_cap = 0;
    int sm_count = 0;
    bool gas_free = false;       // no gas anywhere on the static grid
    int steps_per_launch = 256;
    int threads = 256;
    int persistent = 0;          // blocks per SM of a persistent launch, 0 = one block per tile
    int schedule = MUCITE_SCHEDULE_BALANCED; // candidate weight of the collision loop (kEagerWeight: eager)
    int use_graphs = 1;
    int64_t launches = 0;
    int64_t graph_replays = 0, graph_captures = 0;
    InstF32 inst0{};             // host copy of the first descriptor of the last step upload
    std::vector<InstF32> h_insts;   // host copies of the descriptors of the last step upload
    std::vector<int32_t> h_tiles;   // and of its tile starts
    // captured macro step of the last group (replayed while the group is unchanged)
    cudaGraphExec_t graph = nullptr;
    std::vector<const void *> graph_key;
    int64_t graph_launches = 0;
};

namespace {

std::string g_create_err;

mucite_status fail(mucite_ctx *ctx, mucite_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    else g_create_err = buf;
    return st;
}

struct DevGuard {
    int prev = -1, want;
    explicit DevGuard(int d) : want(d)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != d) cudaSetDevice(d);
    }
    ~DevGuard()
    {
        if (prev >= 0 && prev != want) cudaSetDevice(prev);
    }
};

#define CK(call)                                                                                 \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? MUCITE_E_OOM : MUCITE_E_CUDA,     \
                        "%s failed: %s", #call, cudaGetErrorString(e_));                         \
    } while (0)

#define CKL()                                                                                    \
    do {                                                                                         \
        cudaError_t e_ = cudaGetLastError();                                                     \
        if (e_ != cudaSuccess)                                                                   \
            return fail(ctx, MUCITE_E_CUDA, "kernel launch failed: %s", cudaGetErrorString(e_)); \
    } while (0)

template <typename T> void dfree(T *&p)
{
    if (p) cudaFree((void *)p);
    p = nullptr;
}

int64_t align256(int64_t v) { return (v + 255) / 256 * 256; }

constexpr int kPicRefine = 4; // FP32 correction passes of a plain space-charge solve
// PCG iterations of a mask-aware solve: 13-59 were needed on the ring stack
// (PIC 65 x 257 and 256 x 1024, cold and warm starts); iterations after
// convergence still cost their launches, so the cap stays near that
constexpr int kPcgIter = 100;

void layout_of(int precision, int64_t cap, mucite_layout *L)
{
    const int pb = precision == MUCITE_FP64 ? 8 : 4, vb = pb;
    int64_t off = 0;
    auto put = [&](int64_t &o, int64_t bytes) {
        o = off;
        off += align256(bytes);
    };
    put(L->off_x, cap * pb);
    put(L->off_y, cap * pb);
    put(L->off_z, cap * pb);
    put(L->off_vx, cap * vb);
    put(L->off_vy, cap * vb);
    put(L->off_vz, cap * vb);
    put(L->off_eint, cap * vb);
    put(L->off_status, cap);
    put(L->off_t_term, cap * 4);
    put(L->off_lnsy, cap * vb);
    put(L->off_tau, cap * vb);
    L->total_bytes = off;
    L->pos_bytes = pb;
    L->vel_bytes = vb;
}

Profile profile_of(const mucite_ion_template &ion)
{
    Profile p;
    p.n3 = 3.0 * ion.n_atoms;
    p.c0 = ion.cv_c0;
    p.c1 = ion.cv_c1;
    if (ion.cv_c1 > 0.0) {
        p.tcap = (1.0 - ion.cv_c0) / ion.cv_c1;
        p.ecap = ion.cv_c0 * p.tcap + 0.5 * ion.cv_c1 * p.tcap * p.tcap;
    } else {
        p.tcap = INFINITY;
        p.ecap = INFINITY;
    }
    return p;
}

double eint_of_T(const Profile &p, double T)
{
    if (T <= p.tcap) return p.n3 * (p.c0 * T + 0.5 * p.c1 * T * T);
    return p.n3 * (p.ecap + (T - p.tcap));
}

void free_instance(Instance &I)
{
    dfree(I.d_counters);
    dfree(I.d_tally);
    dfree(I.d_tsum);
    dfree(I.pic.Q);
    dfree(I.pic.phi);
    dfree(I.pic.phi_prev);
    dfree(I.pic.phi_hist);
    dfree(I.pic.r32);
    dfree(I.pic.hat);
    dfree(I.tc_rT);
    dfree(I.tc_rT_lo);
    dfree(I.tc_hat_lo);
    I.tc_on = false;
    dfree(I.pic.d32);
    dfree(I.pic.esc);
    dfree(I.pic.er64);
    dfree(I.pic.ez64);
    dfree(I.pic.red);
    dfree(I.pic.conv);
    dfree(I.pic.r64);
    dfree(I.pic.z64);
    dfree(I.pic.q64);
    dfree(I.pic.p64);
    dfree(I.pic.part);
    dfree(I.pic.ticket);
    dfree(I.pic.Qn);
    dfree(I.pic.esc4);
    I = Instance();
}

void free_fields(mucite_ctx *ctx)
{
    dfree(ctx->d_node);
    dfree(ctx->d_dmask);
    for (auto &p : ctx->d_f64) dfree(p);
    dfree(ctx->d_S);
    dfree(ctx->d_Spad);
    dfree(ctx->d_Spad_lo);
    ctx->tc_ok = false;
    dfree(ctx->d_cp);
    dfree(ctx->d_invm);
    dfree(ctx->d_lo);
    dfree(ctx->d_a);
    dfree(ctx->d_c);
    dfree(ctx->d_A);
    dfree(ctx->d_pic_metal);
    ctx->pic_has_metal = false;
    ctx->fields = false;
    ctx->has_pic_grid = false;
}

template <typename T> T *at(void *pool, int64_t off) { return (T *)((char *)pool + off); }

void bind_params(mucite_ctx *ctx, Instance &I)
{
    const mucite_run &r = I.run;
    const mucite_ion_template &ion = I.ion;
    const mucite_grid &g = ctx->g;
    const double M = ion.mass_da * kDa, mg = r.m_gas_da * kDa;
    const double mu = M * mg / (M + mg);
    const Profile pf = profile_of(ion);
    const int64_t zexit_q = (int64_t)ceil((r.z_exit - g.z0) / (g.z1 - g.z0) * kLat);
    const int64_t rdet_q = (int64_t)floor(r.r_det / g.R * kLat);
    {
        InstF32 &P = I.f32;
        P = InstF32{};
        if (I.lay.pos_bytes == 4) {
        P.xq = at<int32_t>(I.pool, I.lay.off_x);
        P.yq = at<int32_t>(I.pool, I.lay.off_y);
        P.zq = at<int32_t>(I.pool, I.lay.off_z);
        P.vx = at<float>(I.pool, I.lay.off_vx);
        P.vy = at<float>(I.pool, I.lay.off_vy);
        P.vz = at<float>(I.pool, I.lay.off_vz);
        P.eint = at<float>(I.pool, I.lay.off_eint);
        P.status = at<uint8_t>(I.pool, I.lay.off_status);
        P.t_term = at<int32_t>(I.pool, I.lay.off_t_term);
        P.lnsy = at<float>(I.pool, I.lay.off_lnsy);
        P.tau = at<float>(I.pool, I.lay.off_tau);
        }
        P.rk4 = r.integrator == 1 ? 1 : 0;
        P.rf_phase0 = I.rf_phase0;
        P.seg_step0 = I.seg_step0;
        P.tst = ion.dH_kJmol > 0.0 ? 1 : 0;
        P.tst_a_dt = (float)(kKB / kPlanck * exp(ion.dS_JmolK / kR) * r.dt);
        P.tst_b = (float)(ion.dH_kJmol * 1000.0 / kR);
        P.langevin = r.langevin ? 1 : 0;
        P.lv_zq0 = (int64_t)ceil((r.lv_z0 - g.z0) / (g.z1 - g.z0) * kLat);
        P.lv_zq1 = (int64_t)floor((r.lv_z1 - g.z0) / (g.z1 - g.z0) * kLat);
        P.lv_switch = (float)r.lv_switch;
        P.lv_c = (float)(16.0 / 3.0 * sqrt(mu * kKB / (2.0 * kPi)) / M);
        P.lv_kM = (float)(kKB / M);
        P.v_rf = r.v_rf;
        P.dtf = r.dt * r.f_rf;
        P.phi_rf = r.phi_rf;
        P.kick = (float)(ion.charge * kE * r.dt / M);
        P.dc_scale = (float)r.dc_scale;
        P.cxs = (float)(r.dt * kLat / g.R);
        P.czs = (float)(r.dt * kLat / (g.z1 - g.z0));
        P.dt = (float)r.dt;
        P.psig = (float)(r.p_scale * ion.ccs_m2 / kKB);
        P.s_coef = (float)(2.0 * kKB / mg);
        P.fM = (float)(M / (M + mg));
        P.fm = (float)(mg / (M + mg));
        P.mu_2kb = (float)(mu / (2.0 * kKB));
        P.g_coef = (float)(2.0 * kKB / mu);
        P.n3 = (float)pf.n3;
        P.inv_n3 = (float)(1.0 / pf.n3);
        P.c0 = (float)pf.c0;
        P.c1 = (float)pf.c1;
        P.tcap = std::isinf(pf.tcap) ? 3.0e38f : (float)pf.tcap;
        P.ecap = std::isinf(pf.ecap) ? 3.0e38f : (float)pf.ecap;
        P.key0 = (uint32_t)r.seed;
        P.key1 = (uint32_t)(r.seed >> 32);
        for (int k = 0; k < 10; ++k)
            P.rkey[k] = make_uint2(P.key0 + (uint32_t)k * 0x9E3779B9u, P.key1 + (uint32_t)k * 0xBB67AE85u);
        P.zexit_q = zexit_q;
        P.rdet2 = (uint64_t)(rdet_q * rdet_q);
        P.hit = (float)r.hit_dist;
        if (I.has_pic) {
            P.esc4 = I.pic.esc4;
            P.pnr = ctx->pg.pnr;
            P.pnz = ctx->pg.pnz;
            P.psr = (float)(ctx->pg.pnr - 1) * (1.0f / 1073741824.0f);
        }
        P.counters = I.d_counters;
        P.hold_tile = -1;
    }
    if (I.lay.pos_bytes == 8) {
        InstF64 &P = I.f64;
        P = InstF64{};
        P.x = at<double>(I.pool, I.lay.off_x);
        P.y = at<double>(I.pool, I.lay.off_y);
        P.z = at<double>(I.pool, I.lay.off_z);
        P.vx = at<double>(I.pool, I.lay.off_vx);
        P.vy = at<double>(I.pool, I.lay.off_vy);
        P.vz = at<double>(I.pool, I.lay.off_vz);
        P.eint = at<double>(I.pool, I.lay.off_eint);
        P.status = at<uint8_t>(I.pool, I.lay.off_status);
        P.t_term = at<int32_t>(I.pool, I.lay.off_t_term);
        P.lnsy = at<double>(I.pool, I.lay.off_lnsy);
        P.tau = at<double>(I.pool, I.lay.off_tau);
        P.tst = ion.dH_kJmol > 0.0 ? 1 : 0;
        P.tst_a = kKB / kPlanck * exp(ion.dS_JmolK / kR);
        P.tst_b = ion.dH_kJmol * 1000.0 / kR;
        P.langevin = r.langevin ? 1 : 0;
        P.lv_z0 = r.lv_z0;
        P.lv_z1 = r.lv_z1;
        P.lv_switch = r.lv_switch;
        P.q_abs = fabs((double)ion.charge) * kE;
        P.rk4 = r.integrator == 1 ? 1 : 0;
        P.qm = ion.charge * kE / (ion.mass_da * kDa);
        P.dc_scale = r.dc_scale;
        P.dt = r.dt;
        P.p_scale = r.p_scale;
        P.sigma = ion.ccs_m2;
        P.M = M;
        P.mg = mg;
        P.prof = pf;
        P.seed = r.seed;
        P.zexit_q = zexit_q;
        P.rdet_q = rdet_q;
        P.hit = (float)r.hit_dist;
        if (I.has_pic) {
            P.er_sc = I.pic.er64;
            P.ez_sc = I.pic.ez64;
            P.pnr = ctx->pg.pnr;
            P.pnz = ctx->pg.pnz;
        }
        P.counters = I.d_counters;
    }
}

GridF32 grid_f32(const mucite_ctx *ctx)
{
    GridF32 G;
    G.node = ctx->d_node;
    G.dmask = ctx->d_dmask;
    G.nr = ctx->g.nr;
    G.nz = ctx->g.nz;
    G.sr = (float)(ctx->g.nr - 1) * (1.0f / 1073741824.0f);
    return G;
}

GridF64 grid_f64(const mucite_ctx *ctx)
{
    GridF64 G;
    G.er_dc = ctx->d_f64[0];
    G.ez_dc = ctx->d_f64[1];
    G.er_rf = ctx->d_f64[2];
    G.ez_rf = ctx->d_f64[3];
    G.gas_p = ctx->d_f64[4];
    G.gas_T = ctx->d_f64[5];
    G.gas_ur = ctx->d_f64[6];
    G.gas_uz = ctx->d_f64[7];
    G.dmask = ctx->d_dmask;
    G.nr = ctx->g.nr;
    G.nz = ctx->g.nz;
    G.R = ctx->g.R;
    G.z0 = ctx->g.z0;
    G.z1 = ctx->g.z1;
    return G;
}

// RF scalar of Eq. 4 at step n (plus `half` of a step) of the instance's
// current dt segment: V cos(2 pi frac(phase0 + (n - seg0) dt f) + phi).
double rf_scalar(const Instance &I, int64_t n, double half = 0.0)
{
    const mucite_run &r = I.run;
    if (r.v_rf == 0.0 || r.f_rf == 0.0) return 0.0;
    const double x = I.rf_phase0 + ((double)(n - I.seg_step0) + half) * (r.dt * r.f_rf);
    const double frac = x - floor(x);
    return r.v_rf * cos(2.0 * kPi * frac + r.phi_rf);
}

mucite_status inject_packs(mucite_ctx *ctx, Instance &I, int64_t p0, int64_t count, bool prefill)
{
    if (count <= 0) return MUCITE_OK;
    InjectArgs A{};
    A.p0 = p0;
    A.count = count;
    A.profile = I.src.profile;
    A.half_space = I.src.half_space;
    A.prefill = prefill && I.src.prefill_z1 > I.src.prefill_z0;
    A.z_plane = I.src.z_plane;
    A.radius = I.src.radius;
    A.sigma = I.src.sigma;
    A.sd = sqrt(kKB * I.src.T_vel / (I.ion.mass_da * kDa));
    A.pz0 = I.src.prefill_z0;
    A.pz1 = I.src.prefill_z1;
    A.e0 = eint_of_T(profile_of(I.ion), I.ion.T_init);
    A.key0 = (uint32_t)I.run.seed;
    A.key1 = (uint32_t)(I.run.seed >> 32);
    A.precision = I.run.precision;
    A.x = (char *)I.pool + I.lay.off_x;
    A.y = (char *)I.pool + I.lay.off_y;
    A.z = (char *)I.pool + I.lay.off_z;
    A.vx = (char *)I.pool + I.lay.off_vx;
    A.vy = (char *)I.pool + I.lay.off_vy;
    A.vz = (char *)I.pool + I.lay.off_vz;
    A.eint = (char *)I.pool + I.lay.off_eint;
    A.lnsy = (char *)I.pool + I.lay.off_lnsy;
    A.tau = (char *)I.pool + I.lay.off_tau;
    A.status = at<uint8_t>(I.pool, I.lay.off_status);
    A.t_term = at<int32_t>(I.pool, I.lay.off_t_term);
    A.R = ctx->g.R;
    A.gz0 = ctx->g.z0;
    A.gz1 = ctx->g.z1;
    launch_inject(A, ctx->stream);
    ctx->launches++;
    CKL();
    return MUCITE_OK;
}

// Packs released by the continuous source over nsteps (Eq. 5): the
// accumulator gains I dt / (z e) real ions per step and releases one pack
// per W accumulated.
int64_t source_emit(Instance &I, int64_t nsteps)
{
    if (!(I.src.current_A > 0.0) || I.src.weight <= 0) return 0;
    const double per_step = I.src.current_A * I.run.dt / ((double)I.ion.charge * kE);
    int64_t emitted = 0;
    for (int64_t k = 0; k < nsteps; ++k) {
        I.src_acc += per_step;
        while (I.src_acc >= (double)I.src.weight) {
            I.src_acc -= (double)I.src.weight;
            ++emitted;
        }
    }
    return emitted;
}

DepositArgs deposit_args(const mucite_ctx *ctx, const Instance &I)
{
    DepositArgs D{};
    D.precision = I.run.precision;
    D.x = (char *)I.pool + I.lay.off_x;
    D.y = (char *)I.pool + I.lay.off_y;
    D.z = (char *)I.pool + I.lay.off_z;
    D.status = at<uint8_t>(I.pool, I.lay.off_status);
    D.n = I.n_slots;
    D.sx = kLat / ctx->g.R;
    D.sz = kLat / (ctx->g.z1 - ctx->g.z0);
    D.gz0 = ctx->g.z0;
    D.pnr = ctx->pg.pnr;
    D.pnz = ctx->pg.pnz;
    D.qw = (int64_t)I.ion.charge * I.src.weight;
    D.Q = I.pic.Q;
    return D;
}

// Upload the descriptors of a space-charge group (outside any capture).
mucite_status pic_upload(mucite_ctx *ctx, const std::vector<Instance *> &grp_in, int &total_tiles,
                         int &n_masked, bool into_next = false)
{
    // maskless instances first, mask-aware ones after: two batched solves
    std::vector<Instance *> grp;
    for (Instance *I : grp_in)
        if (!I->pic_masked) grp.push_back(I);
    for (Instance *I : grp_in)
        if (I->pic_masked) grp.push_back(I);
    n_masked = (int)std::count_if(grp_in.begin(), grp_in.end(), [](Instance *I) { return I->pic_masked; });
    const size_t n = grp.size();
    // the plain solves take the tensor cores when the grid's rule says so
    // (every plain instance then has its operands)
    const size_t n_plain = n - (size_t)n_masked;
    bool tc = ctx->tc_ok && ctx->use_tc && n_plain > 0;
    for (size_t k = 0; k < n_plain; ++k) tc = tc && grp[k]->tc_on;
    ctx->tc_group = tc;
    if (tc) {
        std::vector<CUtensorMap> maps(n_plain * kTcMaps);
        for (size_t k = 0; k < n_plain; ++k)
            for (int q = 0; q < kTcMaps; ++q) maps[k * kTcMaps + q] = grp[k]->tc_maps[q];
        CK(cudaMemcpyAsync(ctx->d_tc_maps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice,
                           ctx->stream));
    }
    std::vector<DepositArgs> dep(n);
    std::vector<PicInst> pi(n);
    std::vector<int32_t> tiles(n + 1);
    int64_t total = 0;
    for (size_t k = 0; k < n; ++k) {
        dep[k] = deposit_args(ctx, *grp[k]);
        if (into_next) dep[k].Q = grp[k]->pic.Qn;
        pi[k] = grp[k]->pic;
        // the transposed residual and the TF32 pairs only for solves whose
        // contractions run on the tensor cores
        const bool tk = tc && k < n_plain;
        pi[k].rT = tk ? grp[k]->tc_rT : nullptr;
        pi[k].rT_lo = tk ? grp[k]->tc_rT_lo : nullptr;
        pi[k].hat_lo = tk ? grp[k]->tc_hat_lo : nullptr;
        tiles[k] = (int32_t)total;
        total += (grp[k]->n_slots + 255) / 256;
    }
    tiles[n] = (int32_t)total;
    total_tiles = (int)total;
    CK(cudaMemcpyAsync(ctx->d_dep, dep.data(), n * sizeof(DepositArgs), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_dep_tiles, tiles.data(), (n + 1) * sizeof(int32_t), cudaMemcpyHostToDevice,
                       ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_picinst, pi.data(), n * sizeof(PicInst), cudaMemcpyHostToDevice, ctx->stream));
    return MUCITE_OK;
}

// Space-charge macro step of a group: clear, deposit, solve, E_SCE -- a fixed
// number of launches for any number of instances. Issued directly, passes
// after convergence still launch (and return at once), so the caps are kept
// near what the warm-started solves need; under graph capture the solve loops
// become device-controlled while nodes that stop at convergence. With take,
// the charge is not deposited here but taken over from Qn, where the previous
// step launch deposited it. Returns the launches issued, or -1 when a
// captured loop could not be built.
int64_t pic_launch(mucite_ctx *ctx, int n_inst, int total_tiles, int n_masked, bool take = false)
{
    int64_t l = 1;
    if (take) {
        // the charge was deposited by the previous step launch (into Qn)
        launch_pic_take(ctx->pg, ctx->d_picinst, n_inst, ctx->stream);
    } else {
        launch_pic_prepare(ctx->pg, ctx->d_picinst, n_inst, ctx->stream);
        launch_deposit(ctx->d_dep, ctx->d_dep_tiles, n_inst, total_tiles, ctx->stream);
        ++l;
    }
    const int n_plain = n_inst - n_masked;
    if (n_plain > 0) {
        const int k = launch_pic_solve(ctx->pg, ctx->d_picinst, n_plain, kPicRefine, 1e-6, ctx->stream,
                                       ctx->device_loops ? ctx->aux : nullptr,
                                       ctx->tc_group ? ctx->d_tc_maps : nullptr, ctx->d_tc_err);
        if (k < 0) return -1;
        l += k;
    }
    if (n_masked > 0) {
        PicGeom Gm = ctx->pg;
        Gm.metal = ctx->d_pic_metal;
        const int k =
            launch_pic_solve_masked(Gm, ctx->d_picinst + n_plain, n_masked, kPcgIter, 1e-6, ctx->stream,
                                    ctx->device_loops ? ctx->aux : nullptr);
        if (k < 0) return -1;
        launch_esc(Gm, ctx->d_picinst + n_plain, n_masked, ctx->stream);
        l += k + 1;
    }
    return l;
}

mucite_status pic_update_group(mucite_ctx *ctx, const std::vector<Instance *> &grp)
{
    if (grp.empty()) return MUCITE_OK;
    int total = 0, nm = 0;
    const mucite_status st = pic_upload(ctx, grp, total, nm);
    if (st != MUCITE_OK) return st;
    const int64_t l = pic_launch(ctx, (int)grp.size(), total, nm);
    if (l < 0) return fail(ctx, MUCITE_E_CUDA, "capture of the solve loop failed");
    ctx->launches += l;
    CKL();
    return MUCITE_OK;
}

mucite_status check_instance(mucite_ctx *ctx, int instance)
{
    if (!ctx) return MUCITE_E_ARG;
    if (instance < 0 || instance >= MUCITE_MAX_INSTANCES)
        return fail(ctx, MUCITE_E_ARG, "instance %d out of range", instance);
    if (!ctx->inst[instance].used) return fail(ctx, MUCITE_E_STATE, "instance %d not injected", instance);
    return MUCITE_OK;
}

void drop_graph(mucite_ctx *ctx)
{
    if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    ctx->graph = nullptr;
    ctx->graph_key.clear();
}

mucite_status ensure_rf(mucite_ctx *ctx, size_t floats)
{
    if (floats <= ctx->rf_cap) return MUCITE_OK;
    CK(cudaStreamSynchronize(ctx->stream));
    drop_graph(ctx);
    dfree(ctx->d_rf);
    CK(cudaMalloc(&ctx->d_rf, floats * sizeof(float)));
    ctx->rf_cap = floats;
    return MUCITE_OK;
}

// Upload the step descriptors of a group (clocks, slot counts, tiles).
mucite_status step_upload(mucite_ctx *ctx, const std::vector<Instance *> &grp, int chunk, int &total_tiles,
                          bool deposit_next = false)
{
    const size_t n = grp.size();
    std::vector<InstF32> host(n);
    std::vector<int32_t> tiles(n + 1);
    int64_t total = 0;
    for (size_t k = 0; k < n; ++k) {
        Instance *I = grp[k];
        host[k] = I->f32;
        host[k].n_slots = I->n_slots;
        host[k].step0 = I->step;
        host[k].rf = ctx->d_rf + k * (size_t)(2 * chunk + 1);
        host[k].dep_q = deposit_next ? I->pic.Qn : nullptr;
        host[k].dep_qw = (int64_t)I->ion.charge * I->src.weight;
        tiles[k] = (int32_t)total;
        total += (I->n_slots + ctx->threads - 1) / ctx->threads;
    }
    tiles[n] = (int32_t)total;
    if (total > INT32_MAX) return fail(ctx, MUCITE_E_ARG, "too many tiles in one launch");
    total_tiles = (int)total;
    CK(cudaMemcpyAsync(ctx->d_insts, host.data(), sizeof(InstF32) * n, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_tiles, tiles.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice,
                       ctx->stream));
    ctx->inst0 = host[0]; // the descriptor a single-instance launch takes as a kernel parameter
    ctx->inst0.hold_tile = -1;
    ctx->h_insts = host;  // the descriptors collision launches take as kernel parameters
    ctx->h_tiles = tiles;
    return MUCITE_OK;
}

// Collisions can happen only with gas on the grid, a non-zero pressure scale
// and a non-zero cross section (otherwise the collision-free kernel runs).
bool can_collide(const mucite_ctx *ctx, const Instance &I)
{
    return !ctx->gas_free && I.run.p_scale > 0.0 && I.ion.ccs_m2 > 0.0;
}

int64_t step_launch(mucite_ctx *ctx, const std::vector<Instance *> &grp, int total_tiles, int chunk)
{
    ctx->last_stream = false;
    if (total_tiles <= 0) return 0;
    bool collide = false, extras = false, pic = false;
    for (const Instance *I : grp) {
        collide = collide || can_collide(ctx, *I);
        extras = extras || I->f32.tst || I->f32.langevin || I->f32.rk4;
        pic = pic || I->has_pic;
    }
    int grid = total_tiles;
    // one collision-free micro step of one instance: the staged streaming
    // kernel (pool arrays 16-byte aligned for its bulk copies)
    if (chunk == 1 && !collide && !extras && grp.size() == 1 && ctx->threads == 256) {
        InstF32 &P = ctx->inst0;
        P.hold_tile = ctx->hold_tile;
        ctx->hold_tile = -1; // one launch only
        const void *arr[] = {P.xq, P.yq, P.zq, P.vx, P.vy, P.vz, P.status};
        bool aligned = true;
        for (const void *a : arr) aligned = aligned && ((uintptr_t)a & 15u) == 0;
        if (aligned) {
            const int per_sm = std::max(1, step_f32_stream_blocks_per_sm());
            grid = std::min(total_tiles, per_sm * ctx->sm_count);
            launch_step_f32_stream(grid_f32(ctx), P, ctx->d_insts, total_tiles, grid, ctx->d_ticket, ctx->stream);
            ctx->last_stream = true;
            return 1;
        }
    }
    // Launches of a few micro steps (streamed) default to an occupancy-sized
    // grid striding over the tiles, which spares every tile the block start
    // (descriptor copy, barriers); long fused launches and launches with
    // collisions default to one block per tile, so blocks whose packs finish
    // early free their SM slot (with collisions a block's warps finish at
    // different times: 4.5 % less time per step in 10-step launches).
    const int pers = ctx->persistent > 0 ? ctx->persistent : (chunk <= 16 && !collide ? 32 : 0);
    if (pers > 0) {
        const int per_sm = std::min(pers, std::max(1, step_f32_blocks_per_sm(grid_f32(ctx), ctx->threads, chunk, collide, extras, pic)));
        grid = std::min(total_tiles, per_sm * ctx->sm_count);
    }
    const GridF32 G = grid_f32(ctx);
    if (collide && !step_f32_large_grid(G)) {
        // one launch per instance, each with its descriptor as the kernel
        // parameter; a batch's launches forked onto the step streams
        const int n = (int)grp.size();
        launch_rf_table(ctx->d_insts, n, chunk, ctx->stream);
        auto one = [&](int k, cudaStream_t st) {
            const int tiles = ctx->h_tiles[k + 1] - ctx->h_tiles[k];
            const int g = grid >= total_tiles ? tiles : std::min(grid, tiles);
            launch_step_f32_one(G, ctx->h_insts[k], ctx->d_insts + k, tiles, ctx->threads, chunk, g, extras, pic,
                                ctx->schedule, st);
        };
        if (n == 1) {
            one(0, ctx->stream);
            return 2;
        }
        const int ns = std::min(n, mucite_ctx::kStepStreams);
        cudaEventRecord(ctx->ev_fork, ctx->stream);
        for (int i = 0; i < ns; ++i) cudaStreamWaitEvent(ctx->step_streams[i], ctx->ev_fork, 0);
        for (int k = 0; k < n; ++k) one(k, ctx->step_streams[k % ns]);
        for (int i = 0; i < ns; ++i) {
            cudaEventRecord(ctx->ev_join[i], ctx->step_streams[i]);
            cudaStreamWaitEvent(ctx->stream, ctx->ev_join[i], 0);
        }
        return 1 + n;
    }
    launch_step_f32(G, ctx->d_insts, ctx->d_tiles, (int)grp.size(), total_tiles, ctx->threads, chunk, grid,
                    collide, extras, pic, ctx->stream);
    return 2;
}

// Advance a group of FP32 instances together by nsteps: per chunk, the
// space-charge macro step of the instances that are due, then one fused
// launch over the packs of all instances. When every instance shares the
// PIC schedule, a whole macro step is captured once as a CUDA graph (PIC,
// RF table, step, clock advance on the device) and replayed.
mucite_status step_f32_group(mucite_ctx *ctx, std::vector<Instance *> &grp, int64_t nsteps)
{
    const size_t n = grp.size();
    const int P0 = grp[0]->has_pic ? grp[0]->run.pic_interval : 0;
    bool uniform = true;
    for (Instance *I : grp) {
        const int P = I->has_pic ? I->run.pic_interval : 0;
        uniform = uniform && P == P0 && (P == 0 || I->step % P == 0);
    }
    int64_t done = 0;
    // the legacy default stream cannot be captured
    const bool capturable = ctx->stream != nullptr && ctx->stream != cudaStreamLegacy;
    if (ctx->use_graphs && uniform && capturable) {
        const int chunk = P0 > 0 ? P0 : ctx->steps_per_launch;
        // single micro steps without space charge: several per captured graph
        // (consecutive kernels of one graph start sooner than consecutive graphs)
        const int unroll = (P0 == 0 && chunk == 1) ? 8 : 1;
        const int64_t reps = (nsteps - done) / ((int64_t)chunk * unroll);
        if (reps >= 2) {
            mucite_status st = ensure_rf(ctx, n * (size_t)(2 * chunk + 1));
            if (st != MUCITE_OK) return st;
            std::vector<const void *> key;
            key.push_back((const void *)(intptr_t)chunk);
            key.push_back((const void *)(intptr_t)unroll);
            key.push_back((const void *)(intptr_t)ctx->threads);
            key.push_back((const void *)(intptr_t)ctx->persistent);
            key.push_back((const void *)(intptr_t)ctx->schedule);
            for (Instance *I : grp) {
                key.push_back(I);
                key.push_back((const void *)(intptr_t)I->n_slots);
            }
            // each replay's step launch deposits the charge its successor's
            // solve needs (into Qn) while the positions are in registers;
            // the first replay takes the charge deposited here
            bool fused = P0 > 0;
            for (Instance *I : grp) fused = fused && I->pic.Qn != nullptr;
            key.push_back((const void *)(intptr_t)fused);
            int tiles = 0, ptiles = 0, pmasked = 0;
            st = step_upload(ctx, grp, chunk, tiles, fused);
            if (st != MUCITE_OK) return st;
            {
                // the kernels take descriptors by value: any change of them
                // other than the clock needs a new capture
                uint64_t h = 1469598103934665603ull; // FNV-1a
                std::vector<InstF32> all = ctx->h_insts;
                all.push_back(ctx->inst0);
                for (InstF32 d : all) {
                    d.step0 = 0;
                    const unsigned char *b = reinterpret_cast<const unsigned char *>(&d);
                    for (size_t k = 0; k < sizeof d; ++k) h = (h ^ b[k]) * 1099511628211ull;
                }
                key.push_back((const void *)(uintptr_t)h);
            }
            if (P0 > 0) {
                st = pic_upload(ctx, grp, ptiles, pmasked, fused);
                if (st != MUCITE_OK) return st;
            }
            if (fused) {
                launch_pic_clear_next(ctx->pg, ctx->d_picinst, (int)n, ctx->stream);
                launch_deposit(ctx->d_dep, ctx->d_dep_tiles, (int)n, ptiles, ctx->stream);
                ctx->launches += 2;
                CKL();
            }
            if (!ctx->graph || key != ctx->graph_key) {
                drop_graph(ctx);
                cudaGraph_t g = nullptr;
                int64_t l = 0;
                // with device-controlled solve loops first; if they cannot be
                // built, once more with the fixed pass sequences
                for (int attempt = 0;; ++attempt) {
                    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
                    const int64_t lp = P0 > 0 ? pic_launch(ctx, (int)n, ptiles, pmasked, fused) : 0;
                    l = lp;
                    for (int u = 0; u < unroll; ++u) {
                        l += step_launch(ctx, grp, tiles, chunk);
                        // the streamed single-step kernel advances the clock itself
                        if (!ctx->last_stream) {
                            launch_advance_clock(ctx->d_insts, (int)n, chunk, ctx->stream);
                            l += 1;
                        }
                    }
                    const cudaError_t ce = cudaStreamEndCapture(ctx->stream, &g);
                    if (lp >= 0) {
                        if (ce != cudaSuccess)
                            return fail(ctx, MUCITE_E_CUDA, "graph capture failed: %s", cudaGetErrorString(ce));
                        break;
                    }
                    if (ce == cudaSuccess) cudaGraphDestroy(g);
                    g = nullptr;
                    cudaGetLastError();
                    if (attempt > 0 || !ctx->device_loops)
                        return fail(ctx, MUCITE_E_CUDA, "graph capture of the solve loop failed");
                    ctx->device_loops = false;
                }
                const cudaError_t ie = cudaGraphInstantiate(&ctx->graph, g, 0);
                cudaGraphDestroy(g);
                if (ie != cudaSuccess) {
                    ctx->graph = nullptr;
                    return fail(ctx, MUCITE_E_CUDA, "graph instantiate failed: %s", cudaGetErrorString(ie));
                }
                ctx->graph_key = key;
                ctx->graph_launches = l;
                ctx->graph_captures += 1;
            }
            for (int64_t r = 0; r < reps; ++r) {
                CK(cudaGraphLaunch(ctx->graph, ctx->stream));
                ctx->launches += ctx->graph_launches;
                ctx->graph_replays += 1;
            }
            for (Instance *I : grp) I->step += reps * chunk * unroll;
            done += reps * chunk * unroll;
        }
    }
    while (done < nsteps) {
        int64_t chunk = std::min<int64_t>(nsteps - done, ctx->steps_per_launch);
        std::vector<Instance *> due;
        for (Instance *I : grp) {
            const int P = I->has_pic ? I->run.pic_interval : 0;
            if (P > 0) {
                if (I->step % P == 0) due.push_back(I);
                chunk = std::min<int64_t>(chunk, P - I->step % P);
            }
        }
        mucite_status st = pic_update_group(ctx, due);
        if (st != MUCITE_OK) return st;
        st = ensure_rf(ctx, n * (size_t)(2 * chunk + 1));
        if (st != MUCITE_OK) return st;
        int tiles = 0;
        st = step_upload(ctx, grp, (int)chunk, tiles);
        if (st != MUCITE_OK) return st;
        ctx->launches += step_launch(ctx, grp, tiles, (int)chunk);
        CKL();
        for (Instance *I : grp) I->step += chunk;
        done += chunk;
    }
    return MUCITE_OK;
}

mucite_status step_f64_one(mucite_ctx *ctx, Instance &I, int64_t nsteps)
{
    const GridF64 G = grid_f64(ctx);
    for (int64_t k = 0; k < nsteps; ++k) {
        const int P = I.has_pic ? I.run.pic_interval : 0;
        if (P > 0 && I.step % P == 0) {
            std::vector<Instance *> one{&I};
            const mucite_status st = pic_update_group(ctx, one);
            if (st != MUCITE_OK) return st;
        }
        InstF64 p = I.f64;
        p.n_slots = I.n_slots;
        launch_step_f64(G, p, I.step, rf_scalar(I, I.step), rf_scalar(I, I.step, 0.5), rf_scalar(I, I.step + 1),
                        ctx->stream);
        ctx->launches++;
        CKL();
        I.step += 1;
    }
    return MUCITE_OK;
}

} // namespace

extern "C" {

static void destroy_step_streams(mucite_ctx *ctx)
{
    for (int i = 0; i < mucite_ctx::kStepStreams; ++i) {
        if (ctx->step_streams[i]) cudaStreamDestroy(ctx->step_streams[i]);
        if (ctx->ev_join[i]) cudaEventDestroy(ctx->ev_join[i]);
    }
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
}

mucite_status mucite_create(mucite_ctx **out, int device, void *cuda_stream)
{
    if (!out) return fail(nullptr, MUCITE_E_ARG, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return fail(nullptr, MUCITE_E_ARG, "no CUDA device %d", device);
    mucite_ctx *ctx = new (std::nothrow) mucite_ctx();
    if (!ctx) return fail(nullptr, MUCITE_E_OOM, "host allocation failed");
    ctx->device = device;
    ctx->stream = (cudaStream_t)cuda_stream;
    DevGuard dg(device);
    cudaError_t e = cudaMalloc(&ctx->d_insts, sizeof(InstF32) * MUCITE_MAX_INSTANCES);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_tiles, sizeof(int32_t) * (MUCITE_MAX_INSTANCES + 1));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_picinst, sizeof(PicInst) * MUCITE_MAX_INSTANCES);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_dep, sizeof(DepositArgs) * MUCITE_MAX_INSTANCES);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_dep_tiles, sizeof(int32_t) * (MUCITE_MAX_INSTANCES + 1));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_limits, 4 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_ticket, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_ticket, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_tc_err, sizeof(int));
    if (e == cudaSuccess)
        e = cudaMalloc(&ctx->d_tc_maps, sizeof(CUtensorMap) * kTcMaps * MUCITE_MAX_INSTANCES);
    if (e == cudaSuccess) e = cudaMemset(ctx->d_tc_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking);
    for (int i = 0; i < mucite_ctx::kStepStreams && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&ctx->step_streams[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_join[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        fail(nullptr, MUCITE_E_OOM, "cudaMalloc failed: %s", cudaGetErrorString(e));
        dfree(ctx->d_insts);
        dfree(ctx->d_tiles);
        dfree(ctx->d_picinst);
        dfree(ctx->d_dep);
        dfree(ctx->d_dep_tiles);
        dfree(ctx->d_limits);
        dfree(ctx->d_ticket);
        dfree(ctx->d_tc_err);
        dfree(ctx->d_tc_maps);
        if (ctx->aux) cudaStreamDestroy(ctx->aux);
        destroy_step_streams(ctx);
        delete ctx;
        return MUCITE_E_OOM;
    }
    *out = ctx;
    return MUCITE_OK;
}

void mucite_destroy(mucite_ctx *ctx)
{
    if (!ctx) return;
    DevGuard dg(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto &I : ctx->inst)
        if (I.used) free_instance(I);
    free_fields(ctx);
    dfree(ctx->d_insts);
    dfree(ctx->d_tiles);
    dfree(ctx->d_picinst);
    dfree(ctx->d_dep);
    dfree(ctx->d_dep_tiles);
    dfree(ctx->d_ticket);
    dfree(ctx->d_tc_err);
    dfree(ctx->d_tc_maps);
    dfree(ctx->d_rf);
    dfree(ctx->d_limits);
    drop_graph(ctx);
    if (ctx->aux) cudaStreamDestroy(ctx->aux);
    destroy_step_streams(ctx);
    delete ctx;
}

const char *mucite_last_error(const mucite_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : g_create_err.c_str();
}

mucite_status mucite_state_layout(int precision, int64_t capacity, mucite_layout *out)
{
    if (!out || capacity < 0 || (precision != MUCITE_FP32 && precision != MUCITE_FP64))
        return MUCITE_E_ARG;
    layout_of(precision, capacity, out);
    return MUCITE_OK;
}

mucite_status mucite_load_fields(mucite_ctx *ctx, const mucite_grid *g, const double *phi_dc,
                                 const double *phi_rf_basis, const double *gas_p,
                                 const double *gas_T, const double *gas_ur, const double *gas_uz,
                                 const uint8_t *metal_mask, const double *surf_dist,
                                 const mucite_grid *pic)
{
    if (!ctx) return MUCITE_E_ARG;
    if (!g || !phi_dc || !phi_rf_basis || !gas_p || !gas_T || !gas_ur || !gas_uz || !metal_mask ||
        !surf_dist)
        return fail(ctx, MUCITE_E_ARG, "NULL field array");
    if (g->nr < 2 || g->nz < 2 || g->nr > (1 << 20) || g->nz > (1 << 20) || !(g->R > 0.0) || !(g->z1 > g->z0))
        return fail(ctx, MUCITE_E_ARG, "bad grid (nr=%d nz=%d R=%g z0=%g z1=%g)", g->nr, g->nz, g->R,
                    g->z0, g->z1);
    if (pic && (pic->nr < 3 || pic->nz < 3 || pic->nr > (1 << 20) || pic->nz > (1 << 20) || pic->R != g->R ||
                pic->z0 != g->z0 || pic->z1 != g->z1))
        return fail(ctx, MUCITE_E_ARG, "PIC grid must have >= 3 nodes per axis and span the static box");
    for (auto &I : ctx->inst)
        if (I.used) return fail(ctx, MUCITE_E_STATE, "release all instances before reloading fields");
    DevGuard dg(ctx->device);
    free_fields(ctx);
    const int64_t n = (int64_t)g->nr * g->nz;
    if (n > (1LL << 31) / 2) return fail(ctx, MUCITE_E_ARG, "grid too large");
    ctx->g = *g;
    for (auto &p : ctx->d_f64) CK(cudaMalloc(&p, n * sizeof(double)));
    CK(cudaMalloc(&ctx->d_node, n * sizeof(NodeF)));
    CK(cudaMalloc(&ctx->d_dmask, n * sizeof(float)));
    double *d_phi = nullptr, *d_dist = nullptr;
    uint8_t *d_mask = nullptr;
    CK(cudaMalloc(&d_phi, 2 * n * sizeof(double)));
    CK(cudaMalloc(&d_dist, n * sizeof(double)));
    CK(cudaMalloc(&d_mask, n));
    const size_t nb = n * sizeof(double);
    CK(cudaMemcpyAsync(d_phi, phi_dc, nb, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(d_phi + n, phi_rf_basis, nb, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_f64[4], gas_p, nb, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_f64[5], gas_T, nb, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_f64[6], gas_ur, nb, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_f64[7], gas_uz, nb, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(d_dist, surf_dist, nb, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(d_mask, metal_mask, n, cudaMemcpyHostToDevice, ctx->stream));
    ctx->gas_free = true;
    for (int64_t k = 0; k < n && ctx->gas_free; ++k) ctx->gas_free = !(gas_p[k] > 0.0);
    const double dr = g->R / (g->nr - 1), dz = (g->z1 - g->z0) / (g->nz - 1);
    launch_efield(d_phi, g->nr, g->nz, dr, dz, ctx->d_f64[0], ctx->d_f64[1], ctx->stream);
    launch_efield(d_phi + n, g->nr, g->nz, dr, dz, ctx->d_f64[2], ctx->d_f64[3], ctx->stream);
    launch_pack_nodes(ctx->d_f64[0], ctx->d_f64[1], ctx->d_f64[2], ctx->d_f64[3], ctx->d_f64[4],
                      ctx->d_f64[5], ctx->d_f64[6], ctx->d_f64[7], d_mask, d_dist, (int)n, ctx->d_node,
                      ctx->d_dmask, ctx->stream);
    ctx->launches += 3;
    CKL();
    CK(cudaStreamSynchronize(ctx->stream));
    cudaFree(d_phi);
    cudaFree(d_dist);
    cudaFree(d_mask);
    if (pic) {
        PicGeom &G = ctx->pg;
        G = PicGeom{};
        G.n_sm = ctx->sm_count;
        G.pnr = pic->nr;
        G.pnz = pic->nz;
        G.M = pic->nz - 2;
        G.Nu = pic->nr - 1;
        G.dr = pic->R / (pic->nr - 1);
        G.dz = (pic->z1 - pic->z0) / (pic->nz - 1);
        G.bscale = -(kE / kLat) / (kEps0 * kPi * G.dz);
        G.hld = (G.M + 3) / 4 * 4;
        const int M = G.M, Nu = G.Nu;
        std::vector<float> S((size_t)M * M), cp((size_t)Nu * M), invm((size_t)Nu * M), lo(Nu);
        std::vector<double> a(Nu), c(Nu), A(Nu);
        const double rz = (G.dr * G.dr) / (G.dz * G.dz);
        for (int i = 0; i < Nu; ++i) {
            if (i == 0) {
                a[i] = 0.0;
                c[i] = 1.0;
                A[i] = rz / 4.0;
            } else {
                a[i] = 2.0 * (i - 0.5);
                c[i] = 2.0 * (i + 0.5);
                A[i] = 2.0 * i * rz;
            }
            lo[i] = (float)a[i];
        }
        const int64_t period = 2LL * (M + 1);
        for (int j = 1; j <= M; ++j)
            for (int k = 1; k <= M; ++k) {
                const int64_t jk = ((int64_t)j * k) % period;
                S[(size_t)(j - 1) * M + (k - 1)] = (float)sin(kPi * (double)jk / (double)(M + 1));
            }
        for (int k = 1; k <= M; ++k) {
            const double s = sin(kPi * k / (2.0 * (M + 1)));
            const double lam = 4.0 * s * s;
            double cprev = 0.0;
            for (int i = 0; i < Nu; ++i) {
                const double d = -(a[i] + c[i] + A[i] * lam);
                const double m = i == 0 ? d : d - a[i] * cprev;
                const double cpi = c[i] / m;
                cp[(size_t)i * M + (k - 1)] = (float)cpi;
                invm[(size_t)i * M + (k - 1)] = (float)(1.0 / m);
                cprev = cpi;
            }
        }
        CK(cudaMalloc(&ctx->d_S, S.size() * sizeof(float)));
        CK(cudaMalloc(&ctx->d_cp, cp.size() * sizeof(float)));
        CK(cudaMalloc(&ctx->d_invm, invm.size() * sizeof(float)));
        CK(cudaMalloc(&ctx->d_lo, lo.size() * sizeof(float)));
        CK(cudaMalloc(&ctx->d_a, Nu * sizeof(double)));
        CK(cudaMalloc(&ctx->d_c, Nu * sizeof(double)));
        CK(cudaMalloc(&ctx->d_A, Nu * sizeof(double)));
        CK(cudaMemcpy(ctx->d_S, S.data(), S.size() * sizeof(float), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ctx->d_cp, cp.data(), cp.size() * sizeof(float), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ctx->d_invm, invm.data(), invm.size() * sizeof(float), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ctx->d_lo, lo.data(), lo.size() * sizeof(float), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ctx->d_a, a.data(), Nu * sizeof(double), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ctx->d_c, c.data(), Nu * sizeof(double), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ctx->d_A, A.data(), Nu * sizeof(double), cudaMemcpyHostToDevice));
        // the tensor-core contractions read S through TMA: rows padded to hld
        // floats (16-byte rows)
        ctx->tc_ok = false;
        if (tc_shape_ok(G) && tc_prepare()) {
            // S = S_hi + S_lo, S_hi rounded to TF32 (10 mantissa bits, to
            // nearest with ties away from zero: add half a unit of the 13
            // dropped bits to the magnitude, then clear them)
            std::vector<float> hi((size_t)M * G.hld, 0.0f), lo((size_t)M * G.hld, 0.0f);
            for (int j = 0; j < M; ++j)
                for (int k = 0; k < M; ++k) {
                    const float v = S[(size_t)j * M + k];
                    uint32_t b;
                    std::memcpy(&b, &v, 4);
                    b = (b + 0x1000u) & 0xFFFFE000u;
                    float h;
                    std::memcpy(&h, &b, 4);
                    hi[(size_t)j * G.hld + k] = h;
                    lo[(size_t)j * G.hld + k] = v - h;
                }
            CK(cudaMalloc(&ctx->d_Spad, hi.size() * sizeof(float)));
            CK(cudaMalloc(&ctx->d_Spad_lo, lo.size() * sizeof(float)));
            CK(cudaMemcpy(ctx->d_Spad, hi.data(), hi.size() * sizeof(float), cudaMemcpyHostToDevice));
            CK(cudaMemcpy(ctx->d_Spad_lo, lo.data(), lo.size() * sizeof(float), cudaMemcpyHostToDevice));
            // S is the B operand of the forward contraction and the A operand
            // of the inverse one
            ctx->tc_ok = make_tc_map(&ctx->map_S, ctx->d_Spad, M, M, G.hld, kTcBoxB) &&
                         make_tc_map(&ctx->map_S_lo, ctx->d_Spad_lo, M, M, G.hld, kTcBoxB) &&
                         make_tc_map(&ctx->map_SA, ctx->d_Spad, M, M, G.hld, kTcBoxA) &&
                         make_tc_map(&ctx->map_SA_lo, ctx->d_Spad_lo, M, M, G.hld, kTcBoxA);
        }
        cudaGetLastError(); // a refused check leaves no error behind: the fast solve then stays on SIMT
        // metal flag of each PIC node: the electrode mask at the nearest static node
        std::vector<uint8_t> pm((size_t)pic->nr * pic->nz);
        const double sdr = g->R / (g->nr - 1), sdz = (g->z1 - g->z0) / (g->nz - 1);
        for (int j = 0; j < pic->nz; ++j)
            for (int i = 0; i < pic->nr; ++i) {
                int si = (int)std::lrint(i * G.dr / sdr), sj = (int)std::lrint(j * G.dz / sdz);
                si = std::min(std::max(si, 0), g->nr - 1);
                sj = std::min(std::max(sj, 0), g->nz - 1);
                pm[(size_t)j * pic->nr + i] = metal_mask[(size_t)sj * g->nr + si] ? 1 : 0;
                ctx->pic_has_metal = ctx->pic_has_metal || pm[(size_t)j * pic->nr + i];
            }
        CK(cudaMalloc(&ctx->d_pic_metal, pm.size()));
        CK(cudaMemcpy(ctx->d_pic_metal, pm.data(), pm.size(), cudaMemcpyHostToDevice));
        G.S = ctx->d_S;
        G.cp = ctx->d_cp;
        G.invm = ctx->d_invm;
        G.lo = ctx->d_lo;
        G.a = ctx->d_a;
        G.c = ctx->d_c;
        G.A = ctx->d_A;
        ctx->has_pic_grid = true;
        ctx->pg_grid = *pic;
    }
    ctx->fields = true;
    return MUCITE_OK;
}

mucite_status mucite_inject(mucite_ctx *ctx, int instance, const mucite_ion_template *ion,
                            const mucite_source *src, const mucite_run *run, void *d_state,
                            int64_t capacity)
{
    if (!ctx) return MUCITE_E_ARG;
    if (instance < 0 || instance >= MUCITE_MAX_INSTANCES)
        return fail(ctx, MUCITE_E_ARG, "instance %d out of range", instance);
    if (!ctx->fields) return fail(ctx, MUCITE_E_STATE, "mucite_load_fields has not been called");
    if (!ion || !src || !run || !d_state) return fail(ctx, MUCITE_E_ARG, "NULL argument");
    if (((uintptr_t)d_state & 255) != 0) return fail(ctx, MUCITE_E_ARG, "pack pool not 256-byte aligned");
    if (capacity < 0 || capacity > (1LL << 31) - 1024)
        return fail(ctx, MUCITE_E_ARG, "capacity %lld out of range", (long long)capacity);
    if (src->n_initial < 0 || src->n_initial > capacity)
        return fail(ctx, MUCITE_E_ARG, "n_initial %lld exceeds capacity %lld", (long long)src->n_initial,
                    (long long)capacity);
    if (run->precision != MUCITE_FP32 && run->precision != MUCITE_FP64)
        return fail(ctx, MUCITE_E_ARG, "bad precision");
    if (!(run->dt > 0.0) || !(ion->mass_da > 0.0) || ion->charge == 0 || !(ion->n_atoms > 0.0) ||
        src->weight <= 0 || run->m_gas_da <= 0.0)
        return fail(ctx, MUCITE_E_ARG, "bad physical parameter (dt, mass, charge, atoms, weight)");
    if (run->exit_bin_steps <= 0 || run->n_exit_bins <= 0 || run->n_r_bins <= 0 || run->n_ke_bins <= 0 ||
        run->n_teff_bins <= 0 || run->n_loss_r <= 0 || run->n_loss_z <= 0 || !(run->ke_max_ev > 0.0) ||
        !(run->teff_max > 0.0) || !(run->r_det > 0.0))
        return fail(ctx, MUCITE_E_ARG, "bad tally layout");
    if (src->profile == 1 && !(src->sigma > 0.0)) return fail(ctx, MUCITE_E_ARG, "Gaussian source needs sigma > 0");
    const bool pic_on = ctx->has_pic_grid && run->pic_interval > 0;
    if (run->pic_interval > 0 && !ctx->has_pic_grid)
        return fail(ctx, MUCITE_E_STATE, "pic_interval > 0 but no PIC grid was loaded");
    if (pic_on) {
        const double bound = (double)capacity * std::fabs((double)ion->charge) * (double)src->weight;
        if (bound >= 8589934592.0)
            return fail(ctx, MUCITE_E_OVERFLOW, "capacity*|q|*W = %.3g >= 2^33 (fixed-point charge bound)",
                        bound);
    }
    DevGuard dg(ctx->device);
    drop_graph(ctx);
    Instance &I = ctx->inst[instance];
    if (I.used) {
        cudaStreamSynchronize(ctx->stream);
        free_instance(I);
    }
    I.ion = *ion;
    I.src = *src;
    I.run = *run;
    I.pool = d_state;
    I.capacity = capacity;
    layout_of(run->precision, capacity, &I.lay);
    I.used = true;
    CK(cudaMalloc(&I.d_counters, kCounters * sizeof(unsigned long long)));
    CK(cudaMemsetAsync(I.d_counters, 0, kCounters * sizeof(unsigned long long), ctx->stream));
    I.tally_len = 16 + run->n_exit_bins + run->n_r_bins + run->n_ke_bins + run->n_teff_bins +
                  (int64_t)run->n_loss_r * run->n_loss_z;
    CK(cudaMalloc(&I.d_tally, I.tally_len * sizeof(unsigned long long)));
    CK(cudaMalloc(&I.d_tsum, 24 * sizeof(double)));
    I.has_pic = pic_on;
    if (pic_on) {
        const PicGeom &G = ctx->pg;
        const size_t nn = (size_t)G.pnr * G.pnz, nu = (size_t)G.M * G.Nu;
        CK(cudaMalloc(&I.pic.Q, nn * sizeof(unsigned long long)));
        CK(cudaMalloc(&I.pic.phi, nn * sizeof(double)));
        CK(cudaMalloc(&I.pic.phi_prev, nn * sizeof(double)));
        CK(cudaMalloc(&I.pic.phi_hist, sizeof(int)));
        CK(cudaMemsetAsync(I.pic.phi_prev, 0, nn * sizeof(double), ctx->stream));
        CK(cudaMemsetAsync(I.pic.phi_hist, 0, sizeof(int), ctx->stream));
        CK(cudaMalloc(&I.pic.r32, nu * sizeof(float)));
        CK(cudaMalloc(&I.pic.hat, (size_t)G.Nu * G.hld * sizeof(float)));
        CK(cudaMalloc(&I.pic.d32, nu * sizeof(float)));
        CK(cudaMalloc(&I.pic.esc, nn * sizeof(float2)));
        CK(cudaMalloc(&I.pic.red, 8 * sizeof(double)));
        CK(cudaMalloc(&I.pic.conv, sizeof(int)));
        CK(cudaMemsetAsync(I.pic.phi, 0, nn * sizeof(double), ctx->stream));
        CK(cudaMemsetAsync(I.pic.esc, 0, nn * sizeof(float2), ctx->stream));
        CK(cudaMemsetAsync(I.pic.Q, 0, nn * sizeof(unsigned long long), ctx->stream));
        CK(cudaMemsetAsync(I.pic.red, 0, 8 * sizeof(double), ctx->stream));
        I.pic_masked = run->pic_masked != 0 && ctx->pic_has_metal;
        if (ctx->tc_ok && ctx->use_tc && !I.pic_masked) {
            const size_t nt = (size_t)G.Nu * G.hld;
            CK(cudaMalloc(&I.tc_rT, nt * sizeof(float)));
            CK(cudaMalloc(&I.tc_rT_lo, nt * sizeof(float)));
            CK(cudaMalloc(&I.tc_hat_lo, nt * sizeof(float)));
            CUtensorMap *m = I.tc_maps;
            I.tc_on = make_tc_map(&m[0], I.tc_rT, G.Nu, G.M, G.hld, kTcBoxA) &&
                      make_tc_map(&m[1], I.tc_rT_lo, G.Nu, G.M, G.hld, kTcBoxA) &&
                      make_tc_map(&m[6], I.pic.hat, G.Nu, G.M, G.hld, kTcBoxB) &&
                      make_tc_map(&m[7], I.tc_hat_lo, G.Nu, G.M, G.hld, kTcBoxB);
            m[2] = ctx->map_S;
            m[3] = ctx->map_S_lo;
            m[4] = ctx->map_SA;
            m[5] = ctx->map_SA_lo;
        }
        if (I.pic_masked) {
            CK(cudaMalloc(&I.pic.r64, nu * sizeof(double)));
            CK(cudaMalloc(&I.pic.z64, nu * sizeof(double)));
            CK(cudaMalloc(&I.pic.q64, nu * sizeof(double)));
            CK(cudaMalloc(&I.pic.p64, nn * sizeof(double)));
            CK(cudaMemsetAsync(I.pic.p64, 0, nn * sizeof(double), ctx->stream));
        }
        CK(cudaMalloc(&I.pic.part, 2 * kRedBlocks * sizeof(double)));
        CK(cudaMalloc(&I.pic.ticket, sizeof(unsigned)));
        CK(cudaMemsetAsync(I.pic.ticket, 0, sizeof(unsigned), ctx->stream));
        if (run->precision == MUCITE_FP32) {
            const size_t nc = (size_t)(ctx->pg.pnr - 1) * (ctx->pg.pnz - 1);
            CK(cudaMalloc(&I.pic.Qn, nn * sizeof(unsigned long long)));
            CK(cudaMalloc(&I.pic.esc4, nc * 2 * sizeof(float4)));
            CK(cudaMemsetAsync(I.pic.esc4, 0, nc * 2 * sizeof(float4), ctx->stream));
        }
        if (run->precision == MUCITE_FP64) {
            CK(cudaMalloc(&I.pic.er64, nn * sizeof(double)));
            CK(cudaMalloc(&I.pic.ez64, nn * sizeof(double)));
            CK(cudaMemsetAsync(I.pic.er64, 0, nn * sizeof(double), ctx->stream));
            CK(cudaMemsetAsync(I.pic.ez64, 0, nn * sizeof(double), ctx->stream));
        }
    }
    // every slot starts empty (status 255, t_term -1)
    CK(cudaMemsetAsync((char *)d_state + I.lay.off_status, 0xFF, (size_t)capacity, ctx->stream));
    CK(cudaMemsetAsync((char *)d_state + I.lay.off_t_term, 0xFF, (size_t)capacity * 4, ctx->stream));
    bind_params(ctx, I);
    I.n_slots = src->n_initial;
    I.step = 0;
    I.src_acc = 0.0;
    return inject_packs(ctx, I, 0, src->n_initial, true);
}

mucite_status mucite_release(mucite_ctx *ctx, int instance)
{
    const mucite_status st = check_instance(ctx, instance);
    if (st != MUCITE_OK) return st;
    DevGuard dg(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    drop_graph(ctx);
    free_instance(ctx->inst[instance]);
    return MUCITE_OK;
}

mucite_status mucite_resume(mucite_ctx *ctx, int instance, int64_t n_slots, int64_t step)
{
    const mucite_status st = check_instance(ctx, instance);
    if (st != MUCITE_OK) return st;
    Instance &I = ctx->inst[instance];
    if (n_slots < 0 || n_slots > I.capacity || step < 0)
        return fail(ctx, MUCITE_E_ARG, "n_slots %lld / step %lld out of range", (long long)n_slots,
                    (long long)step);
    DevGuard dg(ctx->device);
    drop_graph(ctx);
    I.n_slots = n_slots;
    I.step = step;
    CK(cudaMemsetAsync(I.d_counters, 0, kCounters * sizeof(unsigned long long), ctx->stream));
    return MUCITE_OK;
}

namespace {

// Advance the selected instances together (see mucite_step).
mucite_status step_selected(mucite_ctx *ctx, const std::vector<Instance *> &sel, int n_steps)
{
    DevGuard dg(ctx->device);
    // continuous source: release the packs accumulated over this call's steps
    for (Instance *I : sel) {
        const int64_t k = source_emit(*I, n_steps);
        if (k > 0) {
            if (I->n_slots + k > I->capacity)
                return fail(ctx, MUCITE_E_ARG, "pack pool full (capacity %lld)", (long long)I->capacity);
            const mucite_status st = inject_packs(ctx, *I, I->n_slots, k, false);
            if (st != MUCITE_OK) return st;
            I->n_slots += k;
        }
    }
    std::vector<Instance *> f32;
    for (Instance *I : sel) {
        if (I->run.precision == MUCITE_FP32) {
            f32.push_back(I);
        } else {
            const mucite_status st = step_f64_one(ctx, *I, n_steps);
            if (st != MUCITE_OK) return st;
        }
    }
    if (!f32.empty()) {
        // instances advance together only while their PIC schedules agree
        bool same = true;
        for (Instance *I : f32)
            same = same && I->run.pic_interval == f32[0]->run.pic_interval &&
                   (!I->has_pic || I->step % I->run.pic_interval == f32[0]->step % I->run.pic_interval);
        if (same) return step_f32_group(ctx, f32, n_steps);
        for (Instance *I : f32) {
            std::vector<Instance *> one{I};
            const mucite_status st = step_f32_group(ctx, one, n_steps);
            if (st != MUCITE_OK) return st;
        }
    }
    return MUCITE_OK;
}

} // namespace

mucite_status mucite_step(mucite_ctx *ctx, int instance, int n_steps)
{
    if (!ctx) return MUCITE_E_ARG;
    if (n_steps < 0) return fail(ctx, MUCITE_E_ARG, "n_steps < 0");
    std::vector<Instance *> sel;
    if (instance == -1) {
        for (auto &I : ctx->inst)
            if (I.used) sel.push_back(&I);
    } else {
        const mucite_status st = check_instance(ctx, instance);
        if (st != MUCITE_OK) return st;
        sel.push_back(&ctx->inst[instance]);
    }
    return step_selected(ctx, sel, n_steps);
}

mucite_status mucite_step_set(mucite_ctx *ctx, const int *instances, int count, int n_steps)
{
    if (!ctx) return MUCITE_E_ARG;
    if (n_steps < 0) return fail(ctx, MUCITE_E_ARG, "n_steps < 0");
    if (count < 0 || (count > 0 && !instances)) return fail(ctx, MUCITE_E_ARG, "bad instance list");
    std::vector<Instance *> sel;
    std::vector<bool> seen(MUCITE_MAX_INSTANCES, false);
    for (int k = 0; k < count; ++k) {
        const mucite_status st = check_instance(ctx, instances[k]);
        if (st != MUCITE_OK) return st;
        if (seen[instances[k]]) return fail(ctx, MUCITE_E_ARG, "instance %d listed twice", instances[k]);
        seen[instances[k]] = true;
        sel.push_back(&ctx->inst[instances[k]]);
    }
    return step_selected(ctx, sel, n_steps);
}

namespace {

// Device and host state of a set of instances that stepping changes: pack
// pools, clocks, slot counts, source accumulators, counters and the
// space-charge charge, potential (the solver's warm start) and field.
struct Snapshot {
    std::vector<Instance *> sel;
    std::vector<size_t> off;
    std::vector<int64_t> step, n_slots;
    std::vector<double> src_acc;
    std::vector<unsigned long long> counters;
    char *d = nullptr;
    size_t bytes = 0;
};

size_t pic_state_bytes(const mucite_ctx *ctx)
{
    const size_t nn = (size_t)ctx->pg.pnr * ctx->pg.pnz;
    const size_t nc = (size_t)(ctx->pg.pnr - 1) * (ctx->pg.pnz - 1);
    return nn * (sizeof(unsigned long long) + 2 * sizeof(double) + sizeof(float2)) + nc * 2 * sizeof(float4) +
           256;
}

mucite_status snapshot_take(mucite_ctx *ctx, Snapshot &S)
{
    size_t b = 0;
    for (Instance *I : S.sel) {
        S.off.push_back(b);
        b += align256(I->lay.total_bytes);
        if (I->has_pic) b += align256((int64_t)pic_state_bytes(ctx));
        S.step.push_back(I->step);
        S.n_slots.push_back(I->n_slots);
        S.src_acc.push_back(I->src_acc);
    }
    S.bytes = b;
    if (cudaMalloc(&S.d, b) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, MUCITE_E_OOM, "no device memory for the tuning snapshot (%zu bytes)", b);
    }
    S.counters.resize(kCounters * S.sel.size());
    const size_t nn = (size_t)ctx->pg.pnr * ctx->pg.pnz;
    const size_t nc = (size_t)(ctx->pg.pnr - 1) * (ctx->pg.pnz - 1);
    for (size_t k = 0; k < S.sel.size(); ++k) {
        Instance *I = S.sel[k];
        char *dst = S.d + S.off[k];
        CK(cudaMemcpyAsync(dst, I->pool, I->lay.total_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
        if (I->has_pic) {
            char *q = dst + align256(I->lay.total_bytes);
            CK(cudaMemcpyAsync(q, I->pic.Q, nn * 8, cudaMemcpyDeviceToDevice, ctx->stream));
            CK(cudaMemcpyAsync(q + nn * 8, I->pic.phi, nn * 8, cudaMemcpyDeviceToDevice, ctx->stream));
            CK(cudaMemcpyAsync(q + nn * 16, I->pic.esc, nn * 8, cudaMemcpyDeviceToDevice, ctx->stream));
            if (I->pic.esc4)
                CK(cudaMemcpyAsync(q + nn * 24, I->pic.esc4, nc * 32, cudaMemcpyDeviceToDevice, ctx->stream));
            char *h = q + nn * 24 + nc * 32;
            CK(cudaMemcpyAsync(h, I->pic.phi_prev, nn * 8, cudaMemcpyDeviceToDevice, ctx->stream));
            CK(cudaMemcpyAsync(h + nn * 8, I->pic.phi_hist, sizeof(int), cudaMemcpyDeviceToDevice, ctx->stream));
        }
        CK(cudaMemcpyAsync(&S.counters[kCounters * k], I->d_counters, kCounters * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return MUCITE_OK;
}

mucite_status snapshot_restore(mucite_ctx *ctx, const Snapshot &S)
{
    const size_t nn = (size_t)ctx->pg.pnr * ctx->pg.pnz;
    const size_t nc = (size_t)(ctx->pg.pnr - 1) * (ctx->pg.pnz - 1);
    for (size_t k = 0; k < S.sel.size(); ++k) {
        Instance *I = S.sel[k];
        const char *src = S.d + S.off[k];
        CK(cudaMemcpyAsync(I->pool, src, I->lay.total_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
        if (I->has_pic) {
            const char *q = src + align256(I->lay.total_bytes);
            CK(cudaMemcpyAsync(I->pic.Q, q, nn * 8, cudaMemcpyDeviceToDevice, ctx->stream));
            CK(cudaMemcpyAsync(I->pic.phi, q + nn * 8, nn * 8, cudaMemcpyDeviceToDevice, ctx->stream));
            CK(cudaMemcpyAsync(I->pic.esc, q + nn * 16, nn * 8, cudaMemcpyDeviceToDevice, ctx->stream));
            if (I->pic.esc4)
                CK(cudaMemcpyAsync(I->pic.esc4, q + nn * 24, nc * 32, cudaMemcpyDeviceToDevice, ctx->stream));
            const char *h = q + nn * 24 + nc * 32;
            CK(cudaMemcpyAsync(I->pic.phi_prev, h, nn * 8, cudaMemcpyDeviceToDevice, ctx->stream));
            CK(cudaMemcpyAsync(I->pic.phi_hist, h + nn * 8, sizeof(int), cudaMemcpyDeviceToDevice, ctx->stream));
        }
        CK(cudaMemcpyAsync(I->d_counters, &S.counters[kCounters * k], kCounters * sizeof(unsigned long long),
                           cudaMemcpyHostToDevice, ctx->stream));
        I->step = S.step[k];
        I->n_slots = S.n_slots[k];
        I->src_acc = S.src_acc[k];
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return MUCITE_OK;
}

} // namespace

mucite_status mucite_autotune(mucite_ctx *ctx, const int *instances, int count, int trial_steps,
                              mucite_tuning *out)
{
    if (!ctx) return MUCITE_E_ARG;
    if (!out || count <= 0 || !instances) return fail(ctx, MUCITE_E_ARG, "bad instance list or output");
    if (trial_steps < 1 || trial_steps > 100000)
        return fail(ctx, MUCITE_E_ARG, "trial_steps must be in [1, 100000]");
    Snapshot S;
    std::vector<bool> seen(MUCITE_MAX_INSTANCES, false);
    bool pic = false;
    for (int k = 0; k < count; ++k) {
        const mucite_status st = check_instance(ctx, instances[k]);
        if (st != MUCITE_OK) return st;
        if (seen[instances[k]]) return fail(ctx, MUCITE_E_ARG, "instance %d listed twice", instances[k]);
        seen[instances[k]] = true;
        Instance *I = &ctx->inst[instances[k]];
        if (I->run.precision != MUCITE_FP32)
            return fail(ctx, MUCITE_E_ARG, "instance %d is FP64: its plain step has no launch shape", instances[k]);
        pic = pic || I->has_pic;
        S.sel.push_back(I);
    }
    DevGuard dg(ctx->device);
    mucite_status st = snapshot_take(ctx, S);
    if (st != MUCITE_OK) return st;
    // candidate shapes; with space charge the PIC interval sets the steps per launch
    std::vector<int> spls;
    if (pic) {
        spls.push_back(ctx->steps_per_launch);
    } else {
        for (int v : {250, 500, 1000, 2000})
            if (v <= std::max(1, trial_steps / 2)) spls.push_back(v);
        if (spls.empty()) spls.push_back(std::max(1, trial_steps / 2));
    }
    const int threads_c[] = {64, 128, 256};
    const int pers_c[] = {0, 1, 2, 3};
    // launches as short as the PIC interval: both collision-loop schedules
    std::vector<int> scheds{MUCITE_SCHEDULE_BALANCED};
    if (pic) scheds.push_back(MUCITE_SCHEDULE_EAGER);
    const int save_spl = ctx->steps_per_launch, save_thr = ctx->threads, save_pers = ctx->persistent;
    const int save_sched = ctx->schedule;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double best = -1.0;
    int bspl = save_spl, bthr = save_thr, bpers = save_pers, bsched = save_sched, tried = 0;
    for (int spl : spls)
        for (int sched : scheds)
        for (int thr : threads_c)
            for (int pers : pers_c) {
                ctx->steps_per_launch = spl;
                ctx->threads = thr;
                ctx->persistent = pers;
                ctx->schedule = sched;
                drop_graph(ctx);
                // untimed pass of the same shape (graph capture, caches), then the timed one
                for (int pass = 0; pass < 2 && st == MUCITE_OK; ++pass) {
                    st = snapshot_restore(ctx, S);
                    if (st != MUCITE_OK) break;
                    if (pass == 1) cudaEventRecord(e0, ctx->stream);
                    st = step_selected(ctx, S.sel, trial_steps);
                    if (pass == 1) cudaEventRecord(e1, ctx->stream);
                }
                if (st != MUCITE_OK) break;
                CK(cudaEventSynchronize(e1));
                float ms = 0.0f;
                CK(cudaEventElapsedTime(&ms, e0, e1));
                ++tried;
                if (best < 0.0 || ms < best) {
                    best = ms;
                    bspl = spl;
                    bthr = thr;
                    bpers = pers;
                    bsched = sched;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const mucite_status rs = snapshot_restore(ctx, S);
    cudaFree(S.d);
    drop_graph(ctx);
    if (st != MUCITE_OK || rs != MUCITE_OK) {
        ctx->steps_per_launch = save_spl;
        ctx->threads = save_thr;
        ctx->persistent = save_pers;
        ctx->schedule = save_sched;
        return st != MUCITE_OK ? st : rs;
    }
    ctx->steps_per_launch = bspl;
    ctx->threads = bthr;
    ctx->persistent = bpers;
    ctx->schedule = bsched;
    out->steps_per_launch = bspl;
    out->threads_per_block = bthr;
    out->persistent_blocks_per_sm = bpers;
    out->schedule = bsched;
    out->n_tried = tried;
    out->best_ms_per_step = best / trial_steps;
    return MUCITE_OK;
}

mucite_status mucite_pic_update(mucite_ctx *ctx, int instance)
{
    const mucite_status st = check_instance(ctx, instance);
    if (st != MUCITE_OK) return st;
    Instance &I = ctx->inst[instance];
    if (!I.has_pic) return fail(ctx, MUCITE_E_STATE, "instance %d has no space charge", instance);
    DevGuard dg(ctx->device);
    std::vector<Instance *> one{&I};
    return pic_update_group(ctx, one);
}

mucite_status mucite_tally(mucite_ctx *ctx, int instance, mucite_tally_out *out)
{
    mucite_status st = check_instance(ctx, instance);
    if (st != MUCITE_OK) return st;
    if (!out) return fail(ctx, MUCITE_E_ARG, "out is NULL");
    Instance &I = ctx->inst[instance];
    const mucite_run &r = I.run;
    DevGuard dg(ctx->device);
    CK(cudaMemsetAsync(I.d_tally, 0, I.tally_len * sizeof(unsigned long long), ctx->stream));
    CK(cudaMemsetAsync(I.d_tsum, 0, 24 * sizeof(double), ctx->stream));
    TallyArgs A{};
    A.precision = r.precision;
    A.x = (char *)I.pool + I.lay.off_x;
    A.y = (char *)I.pool + I.lay.off_y;
    A.z = (char *)I.pool + I.lay.off_z;
    A.vx = (char *)I.pool + I.lay.off_vx;
    A.vy = (char *)I.pool + I.lay.off_vy;
    A.vz = (char *)I.pool + I.lay.off_vz;
    A.eint = (char *)I.pool + I.lay.off_eint;
    A.lnsy = (char *)I.pool + I.lay.off_lnsy;
    A.status = at<uint8_t>(I.pool, I.lay.off_status);
    A.t_term = at<int32_t>(I.pool, I.lay.off_t_term);
    A.n = I.n_slots;
    A.sx = kLat / ctx->g.R;
    A.sz = kLat / (ctx->g.z1 - ctx->g.z0);
    A.gz0 = ctx->g.z0;
    A.prof = profile_of(I.ion);
    const double M = I.ion.mass_da * kDa;
    A.c_ke = 0.5 * M / kE;
    A.ke_scale = (double)r.n_ke_bins / r.ke_max_ev;
    A.t_scale = (double)r.n_teff_bins / r.teff_max;
    A.r_scale = (float)((double)r.n_r_bins / (r.r_det / ctx->g.R) / kLat);
    A.lr_scale = (float)((double)r.n_loss_r / kLat);
    A.exit_bin_steps = r.exit_bin_steps;
    A.n_exit_bins = r.n_exit_bins;
    A.n_r_bins = r.n_r_bins;
    A.n_ke_bins = r.n_ke_bins;
    A.n_teff_bins = r.n_teff_bins;
    A.n_loss_r = r.n_loss_r;
    A.n_loss_z = r.n_loss_z;
    A.weight = I.src.weight;
    A.count = I.d_tally;
    A.wsum = I.d_tally + 8;
    A.sum_ke = I.d_tsum;
    A.sum_teff = I.d_tsum + 8;
    A.sum_sy = I.d_tsum + 16;
    A.exit_hist = I.d_tally + 16;
    A.r_hist = A.exit_hist + r.n_exit_bins;
    A.ke_hist = A.r_hist + r.n_r_bins;
    A.teff_hist = A.ke_hist + r.n_ke_bins;
    A.loss_map = A.teff_hist + r.n_teff_bins;
    launch_tally(A, ctx->stream);
    ctx->launches++;
    CKL();
    std::vector<unsigned long long> h(I.tally_len);
    double sums[24];
    unsigned long long cnt[kCounters];
    CK(cudaMemcpyAsync(h.data(), I.d_tally, I.tally_len * sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(sums, I.d_tsum, sizeof sums, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(cnt, I.d_counters, sizeof cnt, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < 8; ++k) {
        out->count[k] = (int64_t)h[k];
        out->weight[k] = (int64_t)h[8 + k];
        out->sum_w_ke[k] = sums[k];
        out->sum_w_teff[k] = sums[8 + k];
        out->sum_w_sy[k] = sums[16 + k];
    }
    out->emitted_count = I.n_slots;
    out->emitted_weight = I.n_slots * I.src.weight;
    out->pack_steps = (int64_t)cnt[0];
    out->collisions = (int64_t)cnt[1];
    out->candidate_overflow = (int64_t)cnt[2];
    out->step = I.step;
    int tc_err = 0;
    CK(cudaMemcpy(&tc_err, ctx->d_tc_err, sizeof tc_err, cudaMemcpyDeviceToHost));
    if (tc_err != 0 && I.has_pic)
        return fail(ctx, MUCITE_E_TIMEOUT, "a bounded wait of the tensor-core DST-I gave up: the space-charge "
                    "solution is not reliable");
    if (cnt[3] != 0)
        return fail(ctx, MUCITE_E_TIMEOUT, "instance %d: %llu bounded device waits gave up (staged state copies "
                    "that did not land); its state is not reliable", instance, cnt[3]);
    int64_t off = 16;
    auto copy_out = [&](int64_t *dst, int64_t len) {
        if (dst)
            for (int64_t k = 0; k < len; ++k) dst[k] = (int64_t)h[off + k];
        off += len;
    };
    copy_out(out->exit_hist, r.n_exit_bins);
    copy_out(out->r_hist, r.n_r_bins);
    copy_out(out->ke_hist, r.n_ke_bins);
    copy_out(out->teff_hist, r.n_teff_bins);
    copy_out(out->loss_map, (int64_t)r.n_loss_r * r.n_loss_z);
    return MUCITE_OK;
}

mucite_status mucite_pic_read(mucite_ctx *ctx, int instance, int64_t *Q, double *phi, float *er,
                              float *ez, double *rel_residual, int32_t *iterations)
{
    const mucite_status st = check_instance(ctx, instance);
    if (st != MUCITE_OK) return st;
    Instance &I = ctx->inst[instance];
    if (!I.has_pic) return fail(ctx, MUCITE_E_STATE, "instance %d has no space charge", instance);
    DevGuard dg(ctx->device);
    const size_t nn = (size_t)ctx->pg.pnr * ctx->pg.pnz;
    if (Q) CK(cudaMemcpyAsync(Q, I.pic.Q, nn * 8, cudaMemcpyDeviceToHost, ctx->stream));
    if (phi) CK(cudaMemcpyAsync(phi, I.pic.phi, nn * 8, cudaMemcpyDeviceToHost, ctx->stream));
    std::vector<float2> e;
    if (er || ez) {
        e.resize(nn);
        CK(cudaMemcpyAsync(e.data(), I.pic.esc, nn * sizeof(float2), cudaMemcpyDeviceToHost, ctx->stream));
    }
    double red[4] = {0, 0, 0, 0};
    int tc_err = 0;
    CK(cudaMemcpyAsync(red, I.pic.red, sizeof red, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(&tc_err, ctx->d_tc_err, sizeof tc_err, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (tc_err != 0)
        return fail(ctx, MUCITE_E_TIMEOUT, "a bounded wait of the tensor-core DST-I gave up: the space-charge "
                    "solution is not reliable");
    for (size_t k = 0; k < e.size(); ++k) {
        if (er) er[k] = e[k].x;
        if (ez) ez[k] = e[k].y;
    }
    if (rel_residual) *rel_residual = red[2];
    if (iterations) *iterations = (int32_t)red[3];
    return MUCITE_OK;
}

mucite_status mucite_set_tuning(mucite_ctx *ctx, int steps_per_launch, int threads_per_block)
{
    if (!ctx) return MUCITE_E_ARG;
    if (steps_per_launch < 0 || steps_per_launch > 6000)
        return fail(ctx, MUCITE_E_ARG, "steps_per_launch must be in [1, 6000]");
    if (threads_per_block < 0 || threads_per_block % 64 != 0 || threads_per_block > 256)
        return fail(ctx, MUCITE_E_ARG, "threads_per_block must be a multiple of 64 in [64, 256]");
    drop_graph(ctx);
    if (steps_per_launch) ctx->steps_per_launch = steps_per_launch;
    if (threads_per_block) ctx->threads = threads_per_block;
    return MUCITE_OK;
}

mucite_status mucite_set_dt(mucite_ctx *ctx, int instance, double dt)
{
    const mucite_status st = check_instance(ctx, instance);
    if (st != MUCITE_OK) return st;
    if (!(dt > 0.0)) return fail(ctx, MUCITE_E_ARG, "dt must be > 0");
    Instance &I = ctx->inst[instance];
    DevGuard dg(ctx->device);
    drop_graph(ctx);
    if (I.run.f_rf != 0.0) {
        const double x = I.rf_phase0 + (double)(I.step - I.seg_step0) * (I.run.dt * I.run.f_rf);
        I.rf_phase0 = x - floor(x);
    }
    I.seg_step0 = I.step;
    I.run.dt = dt;
    bind_params(ctx, I);
    return MUCITE_OK;
}

mucite_status mucite_dt_limits(mucite_ctx *ctx, int instance, double out[6])
{
    const mucite_status st = check_instance(ctx, instance);
    if (st != MUCITE_OK) return st;
    if (!out) return fail(ctx, MUCITE_E_ARG, "out is NULL");
    Instance &I = ctx->inst[instance];
    DevGuard dg(ctx->device);
    unsigned *d_out = ctx->d_limits;
    const unsigned init[3] = {0u, 0u, 0x7f800000u};
    CK(cudaMemcpyAsync(d_out, init, sizeof init, cudaMemcpyHostToDevice, ctx->stream));
    LimitArgs A{};
    A.precision = I.run.precision;
    A.x = (char *)I.pool + I.lay.off_x;
    A.y = (char *)I.pool + I.lay.off_y;
    A.z = (char *)I.pool + I.lay.off_z;
    A.vx = (char *)I.pool + I.lay.off_vx;
    A.vy = (char *)I.pool + I.lay.off_vy;
    A.vz = (char *)I.pool + I.lay.off_vz;
    A.status = at<uint8_t>(I.pool, I.lay.off_status);
    A.n = I.n_slots;
    A.sx_inv = kLat / ctx->g.R;
    A.sz_inv = kLat / (ctx->g.z1 - ctx->g.z0);
    A.gz0 = ctx->g.z0;
    A.srf = rf_scalar(I, I.step);
    const double M = I.ion.mass_da * kDa;
    A.kick_m = (float)(I.ion.charge * kE / M);
    A.kT_over_M_coef = (float)(kKB / M);
    A.out = d_out;
    launch_dt_limits(grid_f32(ctx), I.f32, A, ctx->stream);
    ctx->launches++;
    CKL();
    unsigned h[3];
    CK(cudaMemcpyAsync(h, d_out, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    float lam, vmax, acc;
    memcpy(&lam, &h[0], 4);
    memcpy(&vmax, &h[1], 4);
    memcpy(&acc, &h[2], 4);
    const double dr = ctx->g.R / (ctx->g.nr - 1), dz = (ctx->g.z1 - ctx->g.z0) / (ctx->g.nz - 1);
    out[0] = (I.run.f_rf > 0.0 && I.run.v_rf != 0.0) ? 0.05 / I.run.f_rf : INFINITY;
    out[1] = lam > 0.0f ? 0.1 / lam : INFINITY;
    out[2] = acc;
    out[3] = vmax > 0.0f ? 0.5 * std::min(dr, dz) / vmax : INFINITY;
    out[4] = I.run.langevin ? 2e-9 : INFINITY;
    out[5] = out[0];
    for (int k = 1; k < 5; ++k) out[5] = std::min(out[5], out[k]);
    return MUCITE_OK;
}

mucite_status mucite_set_launch_mode(mucite_ctx *ctx, int persistent_blocks_per_sm, int use_graphs)
{
    if (!ctx) return MUCITE_E_ARG;
    if (persistent_blocks_per_sm < 0 || persistent_blocks_per_sm > 32)
        return fail(ctx, MUCITE_E_ARG, "persistent_blocks_per_sm must be in [0, 32]");
    DevGuard dg(ctx->device);
    drop_graph(ctx);
    ctx->persistent = persistent_blocks_per_sm;
    ctx->use_graphs = use_graphs ? 1 : 0;
    return MUCITE_OK;
}

mucite_status mucite_set_schedule(mucite_ctx *ctx, int schedule)
{
    if (!ctx) return MUCITE_E_ARG;
    if (schedule != MUCITE_SCHEDULE_BALANCED && schedule != MUCITE_SCHEDULE_EAGER)
        return fail(ctx, MUCITE_E_ARG, "unknown collision-loop schedule %d", schedule);
    DevGuard dg(ctx->device);
    if (schedule != ctx->schedule) drop_graph(ctx);
    ctx->schedule = schedule;
    return MUCITE_OK;
}

int64_t mucite_launch_count(const mucite_ctx *ctx) { return ctx ? ctx->launches : 0; }

mucite_status mucite_test_hook(mucite_ctx *ctx, int hook, int value)
{
    if (!ctx) return MUCITE_E_ARG;
    if (hook != MUCITE_HOOK_HOLD_STAGED_COPY || value < -1)
        return fail(ctx, MUCITE_E_ARG, "unknown test hook %d or value %d", hook, value);
    ctx->hold_tile = value;
    return MUCITE_OK;
}

mucite_status mucite_set_pic_solver(mucite_ctx *ctx, int contraction)
{
    if (!ctx) return MUCITE_E_ARG;
    if (contraction != MUCITE_DST_SIMT && contraction != MUCITE_DST_TENSOR_CORES)
        return fail(ctx, MUCITE_E_ARG, "contraction must be MUCITE_DST_SIMT or MUCITE_DST_TENSOR_CORES");
    if (!ctx->has_pic_grid) return fail(ctx, MUCITE_E_STATE, "load fields with a PIC grid first");
    for (auto &I : ctx->inst)
        if (I.used && I.has_pic) return fail(ctx, MUCITE_E_STATE, "choose the solver before injecting instances");
    if (contraction == MUCITE_DST_TENSOR_CORES && !ctx->tc_ok)
        return fail(ctx, MUCITE_E_STATE, "the tensor-core contractions are not available for this device or grid");
    drop_graph(ctx);
    ctx->use_tc = contraction == MUCITE_DST_TENSOR_CORES;
    return MUCITE_OK;
}

mucite_status mucite_graph_stats(const mucite_ctx *ctx, int64_t *replays, int64_t *captures)
{
    if (!ctx) return MUCITE_E_ARG;
    if (replays) *replays = ctx->graph_replays;
    if (captures) *captures = ctx->graph_captures;
    return MUCITE_OK;
}

mucite_status mucite_sync(mucite_ctx *ctx)
{
    if (!ctx) return MUCITE_E_ARG;
    DevGuard dg(ctx->device);
    CK(cudaStreamSynchronize(ctx->stream));
    return MUCITE_OK;
}

} // extern "C"
