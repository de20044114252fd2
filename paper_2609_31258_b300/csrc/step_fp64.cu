// Plain FP64 ion-pack step: one thread per pack, one micro step per launch,
// FP64 positions, velocities, internal energy and fields, no staging and no
// fusion. It is the straightforward GPU form of the method and the reference
// the fused FP32 path is measured against.
//
// Same micro-step order and physics as the FP32 kernel (gather -> collisions
// -> kick -> drift -> classify, Methods "Simulation scope and modular
// architecture"; Eq. 3, Eq. 4, Eq. 6, IICT paragraph, "Terminal events"); the
// classification quantises the FP64 position to the int32 lattice
// (rint(x 2^30 / R)) and applies the lattice rules.
#include "kernels.cuh"

namespace mucite {

namespace {

__device__ __forceinline__ void cell_d(double g, int n, int &i0, double &f)
{
    const double fl = floor(g);
    const int i = (int)fl;
    if (i < 0) {
        i0 = 0;
        f = 0.0;
    } else if (i > n - 2) {
        i0 = n - 2;
        f = 1.0;
    } else {
        i0 = i;
        f = g - fl;
    }
}

__device__ __forceinline__ double bil(const double *a, int nr, int i0, int j0, double fr, double fz)
{
    const double *p = a + (size_t)j0 * nr + i0;
    return (1.0 - fr) * (1.0 - fz) * p[0] + fr * (1.0 - fz) * p[1] + (1.0 - fr) * fz * p[nr] +
           fr * fz * p[nr + 1];
}

struct LocalD {
    double ed[3], er[3], es[3], u[3];
    double n, T;
};

__device__ void gather_d(const GridF64 &G, const InstF64 &P, double x, double y, double z, LocalD &L)
{
    const double r = sqrt(x * x + y * y);
    const double dr = G.R / (G.nr - 1), dz = (G.z1 - G.z0) / (G.nz - 1);
    int i0, j0;
    double fr, fz;
    cell_d(r / dr, G.nr, i0, fr);
    cell_d((z - G.z0) / dz, G.nz, j0, fz);
    const double cx = r > 0.0 ? x / r : 0.0, cy = r > 0.0 ? y / r : 0.0;
    double er = bil(G.er_dc, G.nr, i0, j0, fr, fz), ez = bil(G.ez_dc, G.nr, i0, j0, fr, fz);
    L.ed[0] = er * cx; L.ed[1] = er * cy; L.ed[2] = ez;
    er = bil(G.er_rf, G.nr, i0, j0, fr, fz);
    ez = bil(G.ez_rf, G.nr, i0, j0, fr, fz);
    L.er[0] = er * cx; L.er[1] = er * cy; L.er[2] = ez;
    const double p = bil(G.gas_p, G.nr, i0, j0, fr, fz) * P.p_scale;
    const double T = bil(G.gas_T, G.nr, i0, j0, fr, fz);
    const double ur = bil(G.gas_ur, G.nr, i0, j0, fr, fz), uz = bil(G.gas_uz, G.nr, i0, j0, fr, fz);
    L.T = T;
    L.n = T > 0.0 ? p / (kKB * T) : 0.0;
    L.u[0] = ur * cx; L.u[1] = ur * cy; L.u[2] = uz;
    L.es[0] = L.es[1] = L.es[2] = 0.0;
    if (P.er_sc != nullptr) {
        const double pdr = G.R / (P.pnr - 1), pdz = (G.z1 - G.z0) / (P.pnz - 1);
        cell_d(r / pdr, P.pnr, i0, fr);
        cell_d((z - G.z0) / pdz, P.pnz, j0, fz);
        er = bil(P.er_sc, P.pnr, i0, j0, fr, fz);
        ez = bil(P.ez_sc, P.pnr, i0, j0, fr, fz);
        L.es[0] = er * cx; L.es[1] = er * cy; L.es[2] = ez;
    }
}

__device__ __forceinline__ void draw(const InstF64 &P, uint32_t pack, uint32_t step, uint32_t block,
                                     double u[4])
{
    const uint4 o = philox10(make_uint4(pack, step, block, 0u), (uint32_t)P.seed,
                             (uint32_t)(P.seed >> 32));
    u[0] = u01d(o.x); u[1] = u01d(o.y); u[2] = u01d(o.z); u[3] = u01d(o.w);
}

// 12 uniforms of candidate k of a step from Philox blocks 2k and 2k+1:
// fields 0..7 the top 21 bits of the eight words, fields 8..11 the low 11
// bits of word pairs (0,1), (2,3), (4,5), (6,7) joined into 22 bits.
__device__ __forceinline__ void draw_candidate(const InstF64 &P, uint32_t pack, uint32_t step, uint32_t k,
                                               double f[12])
{
    const uint32_t k0 = (uint32_t)P.seed, k1 = (uint32_t)(P.seed >> 32);
    const uint4 a = philox10(make_uint4(pack, step, 2u * k, 0u), k0, k1);
    const uint4 b = philox10(make_uint4(pack, step, 2u * k + 1u, 0u), k0, k1);
    const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    for (int j = 0; j < 8; ++j) f[j] = ((double)(w[j] >> 11) + 0.5) * 0x1p-21;
    for (int m = 0; m < 4; ++m)
        f[8 + m] = ((double)(((w[2 * m] & 0x7FFu) << 11) | (w[2 * m + 1] & 0x7FFu)) + 0.5) * 0x1p-22;
}

__device__ __forceinline__ double teff_d(const Profile &pf, double eint)
{
    const double e = eint / pf.n3;
    if (e <= pf.ecap) return 2.0 * e / (pf.c0 + sqrt(pf.c0 * pf.c0 + 2.0 * pf.c1 * e));
    return pf.tcap + (e - pf.ecap);
}

// Collisions of one pack during one step: candidates of a Poisson process of
// rate n sigma (|v - u| + cbar) at the carried optical depth tau.
__device__ int collide_d(const InstF64 &P, const LocalD &L, uint32_t pack, uint32_t step, double v[3],
                         double &eint, double &tau, int &ovf)
{
    ovf = 0;
    if (!(L.n > 0.0) || !(P.sigma > 0.0) || !(L.T > 0.0)) return 0;
    const double M = P.M, mg = P.mg, mu = M * mg / (M + mg);
    const double s = sqrt(2.0 * kKB * L.T / mg);
    const double cbar = 2.0 * s / sqrt(kPi);
    double t = 0.0;
    int acc = 0;
    for (int k = 0; k < kKmax; ++k) {
        const double w3[3] = {v[0] - L.u[0], v[1] - L.u[1], v[2] - L.u[2]};
        const double w = sqrt(w3[0] * w3[0] + w3[1] * w3[1] + w3[2] * w3[2]);
        const double nu = L.n * P.sigma * (w + cbar);
        const double room = nu * (P.dt - t);
        if (tau >= room) {
            tau -= room;
            return acc;
        }
        t += tau / nu;
        double f[12];
        draw_candidate(P, pack, step, (uint32_t)k, f);
        tau = -log(f[11]);
        // |c'|^2 / s^2 ~ Gamma(3/2) (Maxwellian) or Gamma(2) (speed-weighted)
        double fk = 1.0;
        if (f[0] * (w + cbar) < w) {
            const double cw = cospi(2.0 * f[2]);
            fk = cw * cw;
        }
        const double y = -log(f[3]) - log(f[4]) * fk;
        const double cmag = s * sqrt(y);
        double cp[3];
        {
            const double ct = 2.0 * f[5] - 1.0, st = sqrt(fmax(0.0, 1.0 - ct * ct));
            double sn, cs;
            sincospi(2.0 * f[6], &sn, &cs);
            cp[0] = cmag * st * cs;
            cp[1] = cmag * st * sn;
            cp[2] = cmag * ct;
        }
        const double g3[3] = {w3[0] - cp[0], w3[1] - cp[1], w3[2] - cp[2]};
        const double g = sqrt(g3[0] * g3[0] + g3[1] * g3[1] + g3[2] * g3[2]);
        if (!(f[1] * (w + cmag) < g)) continue;
        ++acc;
        double Vcm[3];
        for (int d = 0; d < 3; ++d) Vcm[d] = (M * v[d] + mg * (L.u[d] + cp[d])) / (M + mg);
        const double etr = 0.5 * mu * g * g / kKB;
        const double ec = etr + eint;
        const double Te = teff_d(P.prof, eint);
        const double fc = P.prof.c0 + P.prof.c1 * Te;
        const double acv = P.prof.n3 * (fc < 1.0 ? fc : 1.0);
        const double omb = -expm1(log(f[9]) / acv + log(f[10]) / (acv + 1.0));
        const double etr_new = ec * omb;
        eint = eint + (etr - etr_new);
        const double gnew = sqrt(2.0 * etr_new * kKB / mu);
        const double ct = 2.0 * f[7] - 1.0, st = sqrt(fmax(0.0, 1.0 - ct * ct));
        double sn, cs;
        sincospi(2.0 * f[8], &sn, &cs);
        const double nh[3] = {st * cs, st * sn, ct};
        for (int d = 0; d < 3; ++d) v[d] = Vcm[d] + (mg / (M + mg)) * gnew * nh[d];
    }
    ovf = 1;
    return acc;
}

__device__ double collision_rate_d(const InstF64 &P, const LocalD &L, const double v[3])
{
    if (!(L.n > 0.0) || !(P.sigma > 0.0) || !(L.T > 0.0)) return 0.0;
    const double s = sqrt(2.0 * kKB * L.T / P.mg);
    const double w = sqrt((v[0] - L.u[0]) * (v[0] - L.u[0]) + (v[1] - L.u[1]) * (v[1] - L.u[1]) +
                          (v[2] - L.u[2]) * (v[2] - L.u[2]));
    const double x = w / s;
    const double g = x > 1e-6 ? s * ((x + 0.5 / x) * erf(x) + exp(-x * x) / sqrt(kPi)) : 2.0 * s / sqrt(kPi);
    return L.n * P.sigma * g;
}

__device__ void langevin_d(const InstF64 &P, const LocalD &L, uint32_t pack, uint32_t step, double v[3])
{
    const double mu = P.M * P.mg / (P.M + P.mg);
    const double K = 3.0 * P.q_abs / (16.0 * L.n) * sqrt(2.0 * kPi / (mu * kKB * L.T)) / P.sigma;
    const double gamma = P.q_abs / (P.M * K);
    const double decay = exp(-gamma * P.dt);
    const double sd = sqrt(kKB * L.T / P.M * -expm1(-2.0 * gamma * P.dt));
    double u[4];
    draw(P, pack, step, 128u, u);
    const double r01 = sqrt(-2.0 * log(u[0])), r23 = sqrt(-2.0 * log(u[2]));
    double sn, cs;
    sincospi(2.0 * u[1], &sn, &cs);
    const double xi[3] = {r01 * cs, r01 * sn, r23 * cospi(2.0 * u[3])};
    for (int d = 0; d < 3; ++d) v[d] = L.u[d] + (v[d] - L.u[d]) * decay + sd * xi[d];
}

__device__ __forceinline__ int32_t q32(double v)
{
    const double r = rint(v);
    if (r < -2147483648.0) return INT32_MIN;
    if (r > 2147483647.0) return INT32_MAX;
    return (int32_t)r;
}

__device__ int classify_d(const GridF64 &G, const InstF64 &P, double x, double y, double z)
{
    const double sx = kLat / G.R, sz = kLat / (G.z1 - G.z0);
    const int32_t xq = q32(__dmul_rn(x, sx)), yq = q32(__dmul_rn(y, sx));
    const int32_t zq = q32(__dmul_rn(__dsub_rn(z, G.z0), sz));
    const float fx = (float)xq, fy = (float)yq;
    const float rr = __fsqrt_rn(__fadd_rn(__fmul_rn(fx, fx), __fmul_rn(fy, fy)));
    const float sr = (float)(G.nr - 1) * (1.0f / 1073741824.0f);
    int ir = __float2int_rz(__fadd_rn(__fmul_rn(rr, sr), 0.5f));
    ir = min(ir, G.nr - 1);
    int64_t iz = ((int64_t)zq * (int64_t)(G.nz - 1) + (1LL << 29)) >> 30;
    iz = iz < 0 ? 0 : (iz > G.nz - 1 ? G.nz - 1 : iz);
    if (G.dmask[(size_t)iz * G.nr + ir] <= P.hit) return MUCITE_ELECTRODE;
    const uint64_t r2 = (uint64_t)((int64_t)xq * xq) + (uint64_t)((int64_t)yq * yq);
    if (r2 >= (1ULL << 60)) return MUCITE_RADIAL;
    if ((int64_t)zq >= P.zexit_q)
        return r2 <= (uint64_t)(P.rdet_q * P.rdet_q) ? MUCITE_TRANSMITTED : MUCITE_AXIAL;
    if (zq < 0) return MUCITE_AXIAL;
    return MUCITE_ACTIVE;
}

} // namespace

// (q/m) E_tot at a position for a given RF scalar (Eq. 3, Eq. 4).
__device__ void accel_d(const GridF64 &G, const InstF64 &P, double x, double y, double z, double srf,
                        double a[3])
{
    LocalD L;
    gather_d(G, P, x, y, z, L);
    for (int d = 0; d < 3; ++d) a[d] = P.qm * (P.dc_scale * L.ed[d] + srf * L.er[d] + L.es[d]);
}

__global__ void __launch_bounds__(256) step_f64_kernel(GridF64 G, InstF64 P, int64_t step,
                                                       double srf, double srf_half, double srf_next)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned done = 0, coll = 0, ovf_n = 0;
    if (p < P.n_slots && P.status[p] == MUCITE_ACTIVE) {
        double x = P.x[p], y = P.y[p], z = P.z[p];
        double v[3] = {P.vx[p], P.vy[p], P.vz[p]};
        double eint = P.eint[p];
        double lnsy = P.tst ? P.lnsy[p] : 0.0;
        double tau = P.tau[p];
        LocalD L;
        gather_d(G, P, x, y, z, L);
        int ovf = 0;
        const bool lv = P.langevin && z >= P.lv_z0 && z <= P.lv_z1 &&
                        collision_rate_d(P, L, v) * P.dt >= P.lv_switch;
        if (lv) langevin_d(P, L, (uint32_t)p, (uint32_t)step, v);
        else coll = (unsigned)collide_d(P, L, (uint32_t)p, (uint32_t)step, v, eint, tau, ovf);
        ovf_n = (unsigned)ovf;
        if (P.tst && !lv) {
            // Eq. 7: ln SY decays at the Eyring rate of the current T_eff
            const double Te = teff_d(P.prof, eint);
            lnsy -= P.tst_a * Te * exp(-P.tst_b / Te) * P.dt;
        }
        if (P.rk4) {
            // RK4 under the instantaneous field: t, t + dt/2 (twice), t + dt
            const double h = P.dt;
            double a1[3], a2[3], a3[3], a4[3], v2[3], v3[3], v4[3];
            for (int d = 0; d < 3; ++d) a1[d] = P.qm * (P.dc_scale * L.ed[d] + srf * L.er[d] + L.es[d]);
            for (int d = 0; d < 3; ++d) v2[d] = v[d] + 0.5 * h * a1[d];
            accel_d(G, P, x + 0.5 * h * v[0], y + 0.5 * h * v[1], z + 0.5 * h * v[2], srf_half, a2);
            for (int d = 0; d < 3; ++d) v3[d] = v[d] + 0.5 * h * a2[d];
            accel_d(G, P, x + 0.5 * h * v2[0], y + 0.5 * h * v2[1], z + 0.5 * h * v2[2], srf_half, a3);
            for (int d = 0; d < 3; ++d) v4[d] = v[d] + h * a3[d];
            accel_d(G, P, x + h * v3[0], y + h * v3[1], z + h * v3[2], srf_next, a4);
            x += h / 6.0 * (v[0] + 2.0 * v2[0] + 2.0 * v3[0] + v4[0]);
            y += h / 6.0 * (v[1] + 2.0 * v2[1] + 2.0 * v3[1] + v4[1]);
            z += h / 6.0 * (v[2] + 2.0 * v2[2] + 2.0 * v3[2] + v4[2]);
            for (int d = 0; d < 3; ++d) v[d] += h / 6.0 * (a1[d] + 2.0 * a2[d] + 2.0 * a3[d] + a4[d]);
        } else {
            for (int d = 0; d < 3; ++d)
                v[d] += P.qm * (P.dc_scale * L.ed[d] + srf * L.er[d] + L.es[d]) * P.dt;
            x += v[0] * P.dt;
            y += v[1] * P.dt;
            z += v[2] * P.dt;
        }
        const int st = classify_d(G, P, x, y, z);
        P.x[p] = x; P.y[p] = y; P.z[p] = z;
        P.vx[p] = v[0]; P.vy[p] = v[1]; P.vz[p] = v[2];
        P.eint[p] = eint;
        if (P.tst) P.lnsy[p] = lnsy;
        P.tau[p] = tau;
        if (st != MUCITE_ACTIVE) {
            P.status[p] = (uint8_t)st;
            P.t_term[p] = (int32_t)(step + 1);
        }
        done = 1;
    }
    done = __reduce_add_sync(0xffffffffu, done);
    coll = __reduce_add_sync(0xffffffffu, coll);
    ovf_n = __reduce_add_sync(0xffffffffu, ovf_n);
    if ((threadIdx.x & 31) == 0) {
        if (done) atomicAdd(&P.counters[0], (unsigned long long)done);
        if (coll) atomicAdd(&P.counters[1], (unsigned long long)coll);
        if (ovf_n) atomicAdd(&P.counters[2], (unsigned long long)ovf_n);
    }
}

void launch_step_f64(const GridF64 &G, const InstF64 &P, int64_t step, double srf, double srf_half,
                     double srf_next, cudaStream_t s)
{
    if (P.n_slots <= 0) return;
    const int threads = 256;
    const int64_t blocks = (P.n_slots + threads - 1) / threads;
    step_f64_kernel<<<(unsigned)blocks, threads, 0, s>>>(G, P, step, srf, srf_half, srf_next);
}

} // namespace mucite
