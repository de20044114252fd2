// Argument blocks and launchers of the pack kernels (see the .cu files).
#pragma once

#include "common.cuh"

namespace mucite {

struct InjectArgs {
    int64_t p0, count;
    int profile, half_space, prefill;
    double z_plane, radius, sigma, sd, pz0, pz1, e0;
    uint32_t key0, key1;
    int precision;
    void *x, *y, *z, *vx, *vy, *vz, *eint, *lnsy, *tau;
    uint8_t *status;
    int32_t *t_term;
    double R, gz0, gz1;
};

struct TallyArgs {
    int precision;
    const void *x, *y, *z, *vx, *vy, *vz, *eint, *lnsy;
    const uint8_t *status;
    const int32_t *t_term;
    int64_t n;
    double sx, sz, gz0;  // FP64-path quantisation to the lattice
    Profile prof;
    double c_ke, ke_scale, t_scale;
    float r_scale, lr_scale;
    int exit_bin_steps, n_exit_bins, n_r_bins, n_ke_bins, n_teff_bins, n_loss_r, n_loss_z;
    int64_t weight;
    unsigned long long *count, *wsum;  // [8]
    double *sum_ke, *sum_teff, *sum_sy; // [8] each
    unsigned long long *exit_hist, *r_hist, *ke_hist, *teff_hist, *loss_map;
};

void launch_inject(const InjectArgs &A, cudaStream_t s);
void launch_tally(const TallyArgs &A, cudaStream_t s);
// grid == total_tiles: one tile per block; a smaller grid strides over the tiles.
// esc_cache: the collision tiles keep each lane's last PIC cell in shared
// memory (for groups with space charge).
void launch_step_f32(const GridF32 &G, InstF32 *d_insts, const int32_t *d_tile_start, int n_inst,
                     int total_tiles, int threads, int nsteps, int grid, bool collide, bool extras,
                     bool esc_cache, cudaStream_t s);
void launch_advance_clock(InstF32 *d_insts, int n_inst, int nsteps, cudaStream_t s);
// Grids above 64 MB of node records (their collision launches keep the
// batched kernel with its scalar arithmetic).
bool step_f32_large_grid(const GridF32 &G);
// RF scalars of the next nsteps micro steps of every instance (P.rf).
void launch_rf_table(InstF32 *d_insts, int n_inst, int nsteps, cudaStream_t s);
// Collision launch of one instance on a grid of at most 64 MB: h_inst (the
// host copy of the descriptor uploaded to d_inst) is the kernel parameter;
// tiles of threads packs; grid < total_tiles strides over them. The RF
// scalars come from launch_rf_table. cand_weight: the candidate weight of the
// collision loop's schedule, 1 or kEagerWeight (results do not depend on it).
void launch_step_f32_one(const GridF32 &G, const InstF32 &h_inst, const InstF32 *d_inst, int total_tiles,
                         int threads, int nsteps, int grid, bool extras, bool esc_cache, int cand_weight,
                         cudaStream_t s);
int step_f32_blocks_per_sm(const GridF32 &G, int threads, int nsteps, bool collide, bool extras,
                           bool esc_cache);
// One collision-free micro step of one instance (no Eq. 7, Langevin or RK4)
// with the pack state staged in shared memory by TMA bulk copies; the pool
// arrays must be 16-byte aligned. Tiles of 256 packs.
// `P` is the instance's descriptor as uploaded to d_insts[0]; the kernel
// reads the step clock from d_insts, forms the step's RF scalar itself and
// advances the clock by one at its end (the last block to arrive on
// `ticket`, a device word that is zero between launches).
void launch_step_f32_stream(const GridF32 &G, const InstF32 &P, InstF32 *d_insts, int total_tiles, int grid,
                            unsigned *ticket, cudaStream_t s);
int step_f32_stream_blocks_per_sm();
void launch_step_f64(const GridF64 &G, const InstF64 &P, int64_t step, double srf, double srf_half,
                     double srf_next, cudaStream_t s);
// Eq. 1 limits of one instance: out (device) [0] max rate, [1] max |v|,
// [2] min max(|v|, v_th)/|a|, as float bit patterns reduced with integer atomics.
struct LimitArgs {
    int precision;
    const void *x, *y, *z, *vx, *vy, *vz;
    const uint8_t *status;
    int64_t n;
    double sx_inv, sz_inv, gz0;   // lattice -> metres for the FP32 pool
    double srf;
    float kick_m;                 // q/M (acceleration per V/m)
    float kT_over_M_coef;         // k_B / M
    unsigned *out;
};
void launch_dt_limits(const GridF32 &G, const InstF32 &P, const LimitArgs &A, cudaStream_t s);

} // namespace mucite
