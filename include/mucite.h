/*
 * mucite.h -- C ABI of the B300 (sm_103a) ion-pack step library.
 *
 * The library advances weighted ion packs through baked axisymmetric (r,z)
 * fields, in the operator order of the paper's runtime (Methods, "Simulation
 * scope and modular architecture"): per micro step, gather gas and fields at
 * the ion -> ion-gas collisions (Eq. 6, IICT paragraph) -> leapfrog kick and
 * drift under E_DC + E_RF(t) + E_SCE (Eq. 3, Eq. 4) -> terminal
 * classification ("Terminal events"); per macro step, CIC deposit ->
 * cylindrical Poisson -> E_SCE ("Axisymmetric PIC space charge update").
 *
 * Conventions (all calls):
 *  - Every call returns a mucite_status (0 = MUCITE_OK, < 0 = error) and
 *    never throws or aborts; mucite_last_error() describes the last failure.
 *  - Host pointers passed in are read during the call and copied; the caller
 *    keeps ownership. Device pointers (the pack pool) stay owned by the
 *    caller and must outlive their instance.
 *  - Work is enqueued on the context's CUDA stream; only mucite_tally,
 *    mucite_pic_read and mucite_sync wait for it.
 *  - Node arrays are row-major [Nz][Nr]; node counts include both ends
 *    (Supporting Information Table S2: 2001 nodes for 20 mm at 0.01 mm).
 *  - SI units. Internal energy is stored as E_int / k_B (kelvin units).
 *  - Positions of the FP32 path live on a fixed-point lattice:
 *    x = xq * R * 2^-30, y = yq * R * 2^-30, z = z0 + zq * (z1 - z0) * 2^-30
 *    (int32). Every discrete decision (mask lookup, classification, deposit,
 *    tally bins) is taken on this lattice; the FP64 path quantises its FP64
 *    positions as rint(x * 2^30 / R), rint((z - z0) * 2^30 / (z1 - z0)).
 */
#ifndef MUCITE_H
#define MUCITE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mucite_ctx mucite_ctx;
typedef int mucite_status;

enum {
    MUCITE_OK = 0,
    MUCITE_E_ARG = -1,      /* invalid argument or size */
    MUCITE_E_OOM = -2,      /* device allocation failed */
    MUCITE_E_CUDA = -3,     /* a CUDA call or kernel launch failed */
    MUCITE_E_OVERFLOW = -4, /* fixed-point charge bound exceeded (sum |q W| >= 2^33) */
    MUCITE_E_STATE = -5,    /* call out of order (no fields, no instance, ...) */
    MUCITE_E_TIMEOUT = -6   /* a bounded device wait gave up */
};

enum { MUCITE_FP32 = 0, MUCITE_FP64 = 1 };

/* Pack status byte: terminal classes of "Terminal events, snapshots, and
 * reported observables". A terminal pack is never re-activated. */
enum {
    MUCITE_ACTIVE = 0,
    MUCITE_TRANSMITTED = 1,
    MUCITE_ELECTRODE = 2,
    MUCITE_RADIAL = 3,
    MUCITE_AXIAL = 4,
    MUCITE_EMPTY = 255
};

#define MUCITE_MAX_INSTANCES 256

/* Axisymmetric grid: nr x nz nodes over r in [0, R], z in [z0, z1]. */
typedef struct {
    int32_t nr, nz;
    double R, z0, z1;
} mucite_grid;

/* Ion template (Methods, "Simulation scope": the species is described by its
 * mass, its charge, its cross section for collisions with the gas, the number
 * of its atoms and how its heat capacity varies with T). Heat capacity
 * Cv / k_B = 3 n_atoms * min(1, cv_c0 + cv_c1 * T); classical: (1, 0). */
typedef struct {
    double mass_da;
    int32_t charge;
    double ccs_m2;
    double n_atoms;
    double cv_c0, cv_c1;
    double T_init; /* initial T_eff */
    /* Transition-state parameters of the dissociation model (Eq. 7, a loss
     * rate that depends on T_eff): activation
     * enthalpy [kJ/mol] and entropy [J/(mol K)]; dH_kJmol <= 0 disables it.
     * Every micro step, after the collisions, ln SY -= k(T_eff) dt with the
     * Eyring rate k = (k_B T/h) exp(dS/R) exp(-dH/(R T)). */
    double dH_kJmol, dS_JmolK;
} mucite_ion_template;

/* Source definition ("Continuous current Gaussian source", Eq. 5).
 * profile 0: uniform over the disc r <= radius; 1: Gaussian of width sigma
 * truncated at radius. n_initial packs are placed at once (on z_plane, or
 * uniformly in [prefill_z0, prefill_z1) when that range is non-empty); a
 * non-zero current_A then releases packs of weight W through the Eq. 5
 * accumulator at the start of every mucite_step call. */
typedef struct {
    int32_t profile;
    double z_plane, radius, sigma, T_vel;
    int32_t half_space; /* fold v_z to >= 0 */
    int64_t n_initial;
    double prefill_z0, prefill_z1;
    double current_A;
    int64_t weight;
} mucite_source;

/* Operating conditions and run settings of one instance. v_rf is the peak
 * voltage applied to the RF basis (V_ref = 1 V, Eq. 4); dc_scale multiplies
 * the DC basis; p_scale multiplies the gas pressure. Histogram layout of the
 * tallies is fixed here. */
typedef struct {
    double dt, v_rf, f_rf, phi_rf, dc_scale, p_scale;
    double hit_dist, z_exit, r_det, m_gas_da;
    uint64_t seed;
    int32_t precision;    /* MUCITE_FP32 (fused) or MUCITE_FP64 (plain) */
    int32_t pic_interval; /* steps between space-charge updates, 0 = none */
    int32_t exit_bin_steps, n_exit_bins, n_r_bins, n_ke_bins, n_teff_bins, n_loss_r, n_loss_z;
    double ke_max_ev, teff_max;
    /* Hybrid Langevin branch (Methods, Particle transport, collisions, and
     * effective internal temperature: the optional lumped-relaxation mode;
     * Table S2: switch at lambda dt >= 0.05): with langevin != 0, a pack in
     * z in [lv_z0, lv_z1] whose expected collision rate satisfies
     * lambda dt >= lv_switch gets an exact Ornstein-Uhlenbeck update of its
     * velocity relative to the gas flow (friction q/(M K), Mason-Schamp
     * mobility K) instead of explicit collisions; T_eff and the survival yield
     * are not updated in that step. */
    int32_t langevin;
    double lv_z0, lv_z1, lv_switch;
    /* pic_masked != 0: the space-charge solve also imposes Phi = 0 on metal
     * nodes of the PIC grid (the electrode mask at the nearest static node),
     * by conjugate gradients preconditioned with the maskless fast solve
     * (at most 100 iterations, same 1e-6 tolerance; mucite_pic_read reports
     * the iterations taken and the residual reached). */
    int32_t pic_masked;
    /* integrator 0: leapfrog (kick-drift, one field evaluation per step);
     * 1: fourth-order Runge-Kutta under the instantaneous total field (the
     * paper's pusher, "Particle transport, collisions, and effective internal
     * temperature"): field evaluations at t, t + dt/2 (twice) and t + dt. */
    int32_t integrator;
} mucite_run;

/* Byte offsets of the structure-of-arrays pack pool (each array 256-byte
 * aligned). FP32: xq, yq, zq int32; vx, vy, vz, eint, lnsy, tau float. FP64:
 * x, y, z, vx, vy, vz, eint, lnsy, tau double. Both: status uint8, t_term
 * int32 (step count at which the pack became terminal, -1 while active). lnsy
 * is the log of the precursor survival yield of Eq. 7 (0 when dissociation
 * is off); tau is the optical depth (an Exp(1) variate, dimensionless) left
 * until the pack's next collision candidate, drawn at injection and consumed
 * at the local candidate rate n sigma (|v - u| + 2 s / sqrt(pi)). */
typedef struct {
    int64_t off_x, off_y, off_z, off_vx, off_vy, off_vz, off_eint, off_status, off_t_term, off_lnsy,
        off_tau;
    int64_t total_bytes;
    int32_t pos_bytes, vel_bytes;
} mucite_layout;

/* Observables of one instance (Eq. 8; "reported observables"; conservation
 * of represented weight). Arrays are caller-owned host buffers sized by the
 * instance's run settings; a NULL array is skipped. */
typedef struct {
    int64_t count[8], weight[8];      /* by status code (index 0..4) */
    double sum_w_ke[8], sum_w_teff[8];/* sum of W * KE [eV] and W * T_eff [K] by status */
    double sum_w_sy[8];               /* sum of W * SY (surviving precursor weight, Eq. 7) by status */
    int64_t emitted_count, emitted_weight;
    int64_t pack_steps;               /* active pack-steps advanced so far */
    int64_t collisions;               /* accepted collision events so far */
    int64_t candidate_overflow;       /* steps that hit the per-step candidate cap */
    int64_t step;                     /* instance clock (steps taken) */
    int64_t *exit_hist;               /* [n_exit_bins] transmitted W by t_term / exit_bin_steps */
    int64_t *r_hist;                  /* [n_r_bins] transmitted W by exit radius over [0, r_det] */
    int64_t *ke_hist;                 /* [n_ke_bins] transmitted W by KE over [0, ke_max_ev] */
    int64_t *teff_hist;               /* [n_teff_bins] transmitted W by T_eff over [0, teff_max] */
    int64_t *loss_map;                /* [n_loss_z][n_loss_r] electrode-hit W over the domain */
} mucite_tally_out;

/* Context on one device; `cuda_stream` is a cudaStream_t (NULL = legacy
 * default stream), e.g. torch.cuda.current_stream().cuda_stream. */
mucite_status mucite_create(mucite_ctx **out, int device, void *cuda_stream);
void mucite_destroy(mucite_ctx *ctx);
/* Text of the last error on this context (or of a failed create when ctx is
 * NULL); valid until the next call on the context. */
const char *mucite_last_error(const mucite_ctx *ctx);

/* Load the baked static fields (Methods, "Coordinate system, static fields,
 * and RF convention"; "Gas field and electrode mask coupling").
 * phi_dc, phi_rf_basis: FP64 potentials [Nz][Nr] (RF basis: adjacent RF
 * electrodes at +1/-1 V); E = -grad(phi) is formed on the device by central
 * differences (one-sided at the domain edges, E_r = 0 on the axis).
 * gas_p [Pa], gas_T [K], gas_ur, gas_uz [m/s]: FP64 [Nz][Nr].
 * metal_mask: uint8 [Nz][Nr], 1 = metal node; surf_dist: FP64 [Nz][Nr]
 * distance to the metal surface [m].
 * pic: PIC grid for the space-charge field, or NULL for none; it must span
 * the same (r, z) box as `g`.
 * Errors: MUCITE_E_ARG (NULL arrays, nr or nz outside [2, 2^20] (PIC grid:
 * [3, 2^20]), more than 2^30 nodes, bad box), MUCITE_E_STATE (instances
 * already injected), MUCITE_E_OOM, MUCITE_E_CUDA. */
mucite_status mucite_load_fields(mucite_ctx *ctx, const mucite_grid *g, const double *phi_dc,
                                 const double *phi_rf_basis, const double *gas_p,
                                 const double *gas_T, const double *gas_ur, const double *gas_uz,
                                 const uint8_t *metal_mask, const double *surf_dist,
                                 const mucite_grid *pic);

/* Layout of a pack pool of `capacity` packs in the given precision. */
mucite_status mucite_state_layout(int precision, int64_t capacity, mucite_layout *out);

/* Create (or replace) instance `instance` in [0, MUCITE_MAX_INSTANCES):
 * binds the caller's device pool `d_state` (layout from
 * mucite_state_layout, 256-byte aligned, owned by the caller), marks all
 * slots empty, and places src->n_initial packs (source sampling of
 * "Continuous current Gaussian source"; Maxwellian velocities at T_vel;
 * E_int = E_int(T_init)). Random draws: Philox4x32-10 keyed by run->seed,
 * counter (pack id, 0, block, 1).
 * Errors: MUCITE_E_ARG (sizes, NULL pool, misaligned pool, n_initial >
 * capacity, bad histogram sizes), MUCITE_E_OVERFLOW (capacity * |q| * W >=
 * 2^33 with space charge on), MUCITE_E_STATE (no fields loaded), MUCITE_E_OOM. */
mucite_status mucite_inject(mucite_ctx *ctx, int instance, const mucite_ion_template *ion,
                            const mucite_source *src, const mucite_run *run, void *d_state,
                            int64_t capacity);

/* Free the instance's device buffers (the caller's pool is not touched). */
mucite_status mucite_release(mucite_ctx *ctx, int instance);

/* Declare that the caller has written `n_slots` packs into the instance's
 * pool (checkpoint import, or a state prepared by a test) and set the
 * instance clock to `step`; counters restart at zero.
 * Errors: MUCITE_E_ARG (n_slots > capacity, step < 0), MUCITE_E_STATE. */
mucite_status mucite_resume(mucite_ctx *ctx, int instance, int64_t n_slots, int64_t step);

/* Advance `n_steps` micro steps of instance `instance`, or of every FP32
 * instance in one batched launch per chunk plus every FP64 instance when
 * instance = -1. With space charge on, a PIC update runs whenever the
 * instance clock is a multiple of pic_interval before the next micro step.
 * Per micro step and active pack: gather -> collisions -> kick -> drift ->
 * classify. Random draws: candidate k of a step uses Philox blocks
 * (pack id, step, 2k, 0) and (pack id, step, 2k + 1, 0); the optical depth
 * to the next candidate is carried per pack (layout array tau).
 * Errors: MUCITE_E_ARG (n_steps < 0), MUCITE_E_STATE, MUCITE_E_CUDA. */
mucite_status mucite_step(mucite_ctx *ctx, int instance, int n_steps);

/* Advance the `count` instances listed in `instances` (host array, each
 * injected and listed once) by `n_steps` micro steps together: the FP32 ones
 * in one batched launch per chunk, as mucite_step(-1) does for all. No
 * counterpart in the paper (which runs cases as separate processes): it lets
 * a serving loop choose which admitted requests share the next launch.
 * Errors: MUCITE_E_ARG (n_steps < 0, count < 0, NULL list, an instance
 * listed twice), MUCITE_E_STATE (an instance not injected), MUCITE_E_CUDA. */
mucite_status mucite_step_set(mucite_ctx *ctx, const int *instances, int count, int n_steps);

/* Launch shape chosen by mucite_autotune. */
typedef struct {
    int32_t steps_per_launch;         /* micro steps fused per launch (PIC runs: unchanged) */
    int32_t threads_per_block;        /* packs per tile, as in mucite_set_tuning */
    int32_t persistent_blocks_per_sm; /* as in mucite_set_launch_mode (0 = automatic) */
    int32_t schedule;                 /* collision-loop schedule, as in mucite_set_schedule */
    int32_t n_tried;                  /* shapes timed */
    double best_ms_per_step;          /* device time of one micro step of the set, chosen shape */
} mucite_tuning;

/* Autotuner of the batched FP32 launch (no counterpart in the paper): times
 * `trial_steps` micro steps of the listed instances (host array, each an
 * injected FP32 instance, listed once) for every candidate shape -- packs
 * per tile {64, 128, 256} x persistent blocks per SM {0, 1, 2, 3} x steps
 * per launch {250, 500, 1000, 2000} up to trial_steps / 2 (with space
 * charge on, the PIC interval fixes the steps per launch, and both
 * schedules of mucite_set_schedule are tried as well) -- each from the
 * same saved state after an untimed pass of the same shape, then restores
 * that state (pools, clocks, slot counts, source accumulators, counters,
 * PIC charge, potential and field) and applies the fastest shape to the
 * context. Takes a device copy of the listed pools (and PIC state) for the
 * duration of the call. Synchronises the stream.
 * Errors: MUCITE_E_ARG (bad list, FP64 instance, trial_steps outside
 * [1, 100000]), MUCITE_E_STATE, MUCITE_E_OOM (no room for the copy),
 * MUCITE_E_CUDA. */
mucite_status mucite_autotune(mucite_ctx *ctx, const int *instances, int count, int trial_steps,
                              mucite_tuning *out);

/* Space-charge macro step of one instance: int64 CIC deposit of q*W in units
 * of e * 2^-30 -> finite-volume cylindrical Poisson (dPhi/dr = 0 on the
 * axis, Phi = 0 at both axial ends and at r = R) solved by an FP32 DST-I in z
 * with a tridiagonal solve per mode, refined in FP64 until
 * ||b - A Phi|| / ||b|| <= 1e-6 (at most 4 correction passes, started from
 * the last two solutions extrapolated linearly in time, 2 Phi_{n-1} -
 * Phi_{n-2}; one pass suffices in steady state on the config workloads, and
 * mucite_pic_read reports the residual reached and the passes taken) -> E_SCE
 * by central differences on the PIC grid.
 * Errors: MUCITE_E_STATE (no PIC grid or instance), MUCITE_E_CUDA. */
mucite_status mucite_pic_update(mucite_ctx *ctx, int instance);

/* Observables of the instance computed from its pack pool (synchronises the
 * stream). Integer counts and histograms are exact; FP64 sums are
 * accumulated with atomics (order-dependent in the last bits). */
mucite_status mucite_tally(mucite_ctx *ctx, int instance, mucite_tally_out *out);

/* Copy the instance's last space-charge solution to host buffers (any may be
 * NULL): Q int64 [pNz][pNr] (units e * 2^-30), phi FP64 [pNz][pNr],
 * E_r and E_z float [pNz][pNr], the final relative residual, and the number
 * of correction passes (fast FP32 solves, or PCG iterations for the
 * mask-aware solve) the last update took. Synchronises the stream. */
mucite_status mucite_pic_read(mucite_ctx *ctx, int instance, int64_t *Q, double *phi, float *er,
                              float *ez, double *rel_residual, int32_t *iterations);

/* Launch shape of the fused FP32 step: at most `steps_per_launch` micro
 * steps (1..6000) are fused per launch (state stays in registers between
 * them); a block advances a tile of `threads_per_block` packs (a multiple of
 * 64 in [64, 256]): one pack per thread with collisions, two per thread in
 * the collision-free kernel. 0 keeps the current value; other values return
 * MUCITE_E_ARG. */
mucite_status mucite_set_tuning(mucite_ctx *ctx, int steps_per_launch, int threads_per_block);

/* Start a new dt segment of instance `instance` at its current step (the
 * global micro step of Eq. 1 is chosen per macro step): the RF phase carries
 * over continuously, the step count (and with it the random-number counters)
 * continues. Errors: MUCITE_E_ARG (dt <= 0), MUCITE_E_STATE. */
mucite_status mucite_set_dt(mucite_ctx *ctx, int instance, double dt);

/* Limits of the global micro step of Eq. 1 on the instance's current state
 * (synchronises the stream): out[0] = 0.05 t_RF, out[1] = 0.1 tau_coll
 * (1 / largest expected collision rate of an active pack), out[2] = dt_acc =
 * 0.1 min over packs of max(|v|, sqrt(kT/M)) / |q E_tot / M|, out[3] =
 * dt_CFL = 0.5 min(dr, dz) / max |v|, out[4] = dt_L = 2 ns with the hybrid
 * Langevin branch on (Table S2), out[5] = the smallest; +inf where a limit
 * does not apply. dt_rem (time to the next scheduled boundary) is the
 * caller's to add. Limits are evaluated in FP32 for both precisions. */
mucite_status mucite_dt_limits(mucite_ctx *ctx, int instance, double out[6]);

/* Launch mode of the batched FP32 step (the paper runs independent cases as
 * separate processes, Supporting Information S6; here many instances are
 * stepped together: collision-free steps in one launch over all instances,
 * steps with collisions on grids up to 64 MB in one launch per instance, the
 * launches of a batch side by side on the context's step streams, larger
 * grids in one launch). persistent_blocks_per_sm > 0: persistent launches of
 * that many blocks per SM (capped by occupancy) whose blocks stride over the
 * tiles of their instances (block b takes tiles b, b + grid, ...); 0: automatic, the
 * occupancy-sized persistent grid for collision-free launches of at most 16
 * micro steps, one block per tile otherwise.
 * use_graphs != 0: when all stepped instances share the space-charge
 * schedule and the context stream is not the legacy default stream, one macro
 * step (PIC update, RF table, fused step, clock advance) is captured once as
 * a CUDA graph and replayed. In the replayed macro step the solve loops stop
 * on the device at convergence, and the step launch deposits the charge of
 * the next PIC update at its end (results identical to use_graphs == 0).
 * Errors: MUCITE_E_ARG (persistent_blocks_per_sm outside [0, 32]). */
mucite_status mucite_set_launch_mode(mucite_ctx *ctx, int persistent_blocks_per_sm, int use_graphs);

/* Contraction of the space-charge fast solve (the DST-I in z and its
 * inverse around the per-mode tridiagonal solve; Methods, "Axisymmetric PIC
 * space charge update"): MUCITE_DST_SIMT (default) runs both transforms as
 * FP32 SIMT contractions that use the sine matrix's row symmetry;
 * MUCITE_DST_TENSOR_CORES runs them on the tensor cores (tcgen05, TMA,
 * thread-block clusters) with every operand split into a TF32 pair
 * (x = x_hi + x_lo, products x_hi y_hi + x_hi y_lo + x_lo y_hi), which keeps
 * the accuracy of the FP32 contraction; the FP64 refinement to 1e-6 and all
 * other steps are the same. The choice applies to the maskless solves of the
 * context, batched or not, so batched and single-instance runs stay
 * bit-identical. Make it after mucite_load_fields (with a PIC grid) and
 * before injecting instances with space charge.
 * Errors: MUCITE_E_ARG (unknown contraction), MUCITE_E_STATE (no PIC grid
 * loaded, instances with space charge already injected, or the tensor-core
 * path unavailable for this device or grid). */
#define MUCITE_DST_SIMT 0
#define MUCITE_DST_TENSOR_CORES 1
mucite_status mucite_set_pic_solver(mucite_ctx *ctx, int contraction);

/* Schedule of the collision loop in the per-instance collision launches (no
 * counterpart in the paper; results do not depend on it). A lane of a warp
 * owns a pack, and each iteration of the warp either tries one pending
 * collision candidate of every lane that has one or finishes the micro step
 * of every lane that has none. MUCITE_SCHEDULE_BALANCED (default) takes
 * whichever serves more lanes, the better choice where candidates are common
 * and launches are long; MUCITE_SCHEDULE_EAGER takes the candidates as soon
 * as their lanes number at least a sixth of those ready to step, so that in
 * launches of a few micro steps (the steps between space-charge updates)
 * with rare candidates no lane falls steps behind and finishes the launch
 * nearly alone. mucite_autotune tries both when space charge fixes the
 * steps per launch. Errors: MUCITE_E_ARG (unknown schedule). */
#define MUCITE_SCHEDULE_BALANCED 1
#define MUCITE_SCHEDULE_EAGER 6
mucite_status mucite_set_schedule(mucite_ctx *ctx, int schedule);

/* Test hook (no counterpart in the paper; for tests of the failure path,
 * never for production runs). MUCITE_HOOK_HOLD_STAGED_COPY with value v >= 0:
 * the next streamed single-step launch (one collision-free micro step of one
 * instance) withholds the staged state copies of the v-th tile of every
 * block, so the bounded waits for them run out (about 0.25 s each); the
 * kernel then ends without faulting, counts the waits that gave up, and
 * mucite_tally of the instance returns MUCITE_E_TIMEOUT until mucite_resume
 * resets its counters (the pack state of that step is not reliable). v = -1
 * clears the hook. Errors: MUCITE_E_ARG (unknown hook or v < -1). */
#define MUCITE_HOOK_HOLD_STAGED_COPY 1
mucite_status mucite_test_hook(mucite_ctx *ctx, int hook, int value);

/* Number of kernels this context has launched since creation. */
int64_t mucite_launch_count(const mucite_ctx *ctx);

/* CUDA-graph use of this context since creation (no counterpart in the
 * paper; evidence of how the batched launches were issued): `replays` (out,
 * may be NULL) the macro-step graphs launched, `captures` (out, may be NULL)
 * the macro-step graphs captured and instantiated (a new one each time the
 * stepped set of instances, their slot counts or the launch shape changes).
 * Errors: MUCITE_E_ARG (ctx NULL). */
mucite_status mucite_graph_stats(const mucite_ctx *ctx, int64_t *replays, int64_t *captures);

/* Wait for all work enqueued on the context's stream. */
mucite_status mucite_sync(mucite_ctx *ctx);

/* Size of the fixed device scratch used by mucite_poisson_solve_noalloc. */
#define MUCITE_NOALLOC_SCRATCH_BYTES (10u * 1024u * 1024u)

/* Space-charge Poisson solve that allocates nothing (the paper has no
 * counterpart; it is a deployment variant of the maskless solve inside
 * mucite_pic_update).
 * Some callers cannot call cudaMalloc: processes whose device memory is fully
 * reserved up front (a serving process, or a host framework whose own pool
 * owns the device and forbids allocations outside it) and real-time loops
 * that must not block on the allocator. This entry point keeps all of its
 * scratch (sine matrix, tridiagonal factors, residual and transform buffers,
 * block partial sums, convergence flags) in one file-scope device array of
 * MUCITE_NOALLOC_SCRATCH_BYTES, which every GPU that loads the library holds
 * until the process exits; it calls no allocator on any call.
 * Arguments: `device` is the CUDA device to run on (made current for the
 * call); `cuda_stream` a cudaStream_t on that device (NULL = legacy default);
 * `pic` the PIC grid (nr x nz nodes over [0, R] x [z0, z1]); `d_Q` device int64
 * [nz][nr] node charges in units of e * 2^-30 (input, as deposited by the
 * library); `d_phi` device FP64 [nz][nr] (output; the solve starts from
 * Phi = 0 on every call, boundary nodes are 0); `d_esc` device float
 * [nz][nr][2] (output E_r, E_z); `d_rel_residual` device double (output, may be
 * NULL): the final ||b - A Phi|| / ||b||. The operator is the maskless one of
 * mucite_pic_update (Phi = 0 at both axial ends and at r = R only; metal
 * nodes inside the grid are not imposed, unlike a run with pic_masked set):
 * FP32 DST-I + tridiagonal correction, FP64 refinement to 1e-6 (at most 8
 * refinements, norms added up in block order, so the result is reproducible)
 * and E differencing. All work is enqueued on the stream.
 * Set-up: the first call on a device looks up the device address of the
 * scratch array and the device's SM count. Under CUDA's default lazy module
 * loading that first call is also what loads the module and reserves the
 * array's MUCITE_NOALLOC_SCRATCH_BYTES on the device, so it can fail with
 * MUCITE_E_CUDA once the device memory is fully reserved: make the first call
 * at start-up, before the memory budget is taken and before any stream
 * capture. The sine matrix and the tridiagonal factors are rebuilt only when
 * the grid differs from the previous call's on that device.
 * Every call shares the one scratch array, which keeps the last call's
 * contents (this call clears what it needs cleared): calls on the same device
 * that overlap on the GPU (different streams, or other host threads) race and
 * must be serialised by the caller.
 * Errors: MUCITE_E_ARG (NULL pointers, device out of [0, 64), fewer than 3
 * nodes per axis, or a grid whose scratch exceeds MUCITE_NOALLOC_SCRATCH_BYTES:
 * about 4 (nz - 2)^2 + 20 (nr - 1)(nz - 2) bytes, e.g. up to 256 x 1026 nodes);
 * MUCITE_E_CUDA (a CUDA call or launch failed). */
mucite_status mucite_poisson_solve_noalloc(int device, void *cuda_stream, const mucite_grid *pic,
                                           const int64_t *d_Q, double *d_phi, float *d_esc,
                                           double *d_rel_residual);

#ifdef __cplusplus
}
#endif

#endif /* MUCITE_H */
