// Fused FP32 ion-pack step: one thread per pack, up to K micro steps per
// launch with the pack state held in registers.
//
// Per micro step n and active pack (operator order of the paper's runtime,
// Methods "Simulation scope and modular architecture"):
//   1. gather at x_n: bilinear E_DC, E_RF basis, gas (p, T, u_r, u_z) from the
//      static grid, E_SCE from the PIC grid; E_r and u_r projected onto x, y
//      (Eq. 3, zero on the axis);
//   2. collisions (Eq. 6 and the IICT paragraph): null-collision sub-cycling
//      with the Maxwellian gas partner, hard-sphere isotropic scattering and
//      Borgnakke-Larsen internal exchange;
//   3. kick v += (q/m)(s_dc E_DC + s_rf(n) E_RF + E_SCE) dt, s_rf from Eq. 4
//      with the phase taken in FP64 once per (instance, step);
//   4. drift on the int32 lattice: xq += floor(v dt 2^30 / R + d), d a
//      uniform dither;
//   5. classification at x_{n+1} on the lattice ("Terminal events").
// Rounding: the per-step lattice displacement and the FP32 velocity update
// are rounded stochastically (a uniform dither from a hash of pack and step):
// in ballistic motion the same increment is rounded every step, and
// round-to-nearest would then add the same error every step; dithered
// rounding is unbiased and needs no state beyond the pack's own, so results
// do not depend on how the steps are split into launches.
// Positions, the mask lookup and the classification are integer or IEEE
// round-to-nearest FP32 operations without contraction, so they decide the
// same classes as any other implementation of the same lattice rules.
#include "deposit.cuh"
#include "kernels.cuh"

namespace mucite {

namespace {

// MurmurHash3 32-bit finalizer (Appleby): avalanche mix for the dither bits.
__device__ __forceinline__ uint32_t fmix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

// Dither words of pack-step (pack, n): h1 = fmix32(pack ^ key ^ n phi) with
// phi = 2^32 / golden ratio (odd: n phi is a bijection of n, so the words of
// one pack's steps are all distinct), h2 a bijective remix of h1 (xor-shift,
// odd multiplier); every 10-bit field of either word is uniform. `hp` is
// pack ^ key, formed once per pack.
__device__ __forceinline__ uint32_t dither_word(uint32_t hp, uint32_t n)
{
    return fmix32(hp ^ (n * 0x9E3779B9u));
}

__device__ __forceinline__ uint32_t remix32(uint32_t h)
{
    return (h ^ (h >> 16)) * 0x7FEB352Du;
}

__device__ __forceinline__ uint32_t pack_key(uint32_t pack, const InstF32 &P)
{
    return pack ^ (P.key0 * 0x9E3779B9u) ^ P.key1;
}

// Dither (b + 1/2) / 1024 in (0,1) from the 10 bits b of h starting at bit
// `sh`: b becomes the top of a mantissa in [1, 2), so no integer-to-float
// conversion is needed; dither_c is the same value minus 1/2.
__device__ __forceinline__ float dither(uint32_t h, int sh)
{
    return __int_as_float(0x3F801000u | (((h >> sh) & 0x3FFu) << 13)) - 1.0f;
}

__device__ __forceinline__ float dither_c(uint32_t h, int sh)
{
    return __int_as_float(0x3F801000u | (((h >> sh) & 0x3FFu) << 13)) - 1.5f;
}

// v + d with stochastic rounding: the sum is dithered by a uniform offset
// uc (centred, in (-1/2, 1/2)) of one unit in the last place of the result
// before rounding to nearest.
__device__ __forceinline__ float add_sr(float v, float d, float uc)
{
    const float t = v + d;
    const float ulp = __int_as_float(__float_as_int(t) & 0x7f800000) * 1.1920928955078125e-7f;
    return v + fmaf(uc, ulp, d);
}

// sqrt where the value decides nothing discrete (approximate reciprocal root).
__device__ __forceinline__ float sqrt_fast(float x)
{
    return x > 0.0f ? x * rsqrtf(x) : 0.0f;
}

// cos and sin of 2 pi u for u in (0,1), through the centred argument
// 2 pi (u - 1/2) in (-pi, pi) where the hardware approximation is accurate.
__device__ __forceinline__ void sincos_2pi(float u, float &sn, float &cs)
{
    __sincosf(6.283185307179586f * (u - 0.5f), &sn, &cs);
    sn = -sn;
    cs = -cs;
}

// Fields gathered at one position: radial and axial components of E_DC, of
// the RF basis field and of E_SCE, the transverse projection (cx, cy) =
// (x, y) / r (zero on the axis, Eq. 3), and the gas.
struct Local {
    float edr, edz, err, erz, esr, esz, cx, cy;
    float nsig, T, ux, uy, uz;
};

// Velocity increment (a m/s per unit field) from the gathered fields: the
// total field (Eq. 3-4) formed in (r, z) and projected once.
// kPack (here and in the functions below): pairs of components -- (r, z),
// (x, y) -- side by side in packed FP32x2 instructions, two results per
// issue slot; otherwise the scalar form. The instantiation for very large
// grids (80 registers, latency-bound on its L2 gathers) takes the scalar
// form, which runs faster there.
template <bool kPack = true>
__device__ __forceinline__ void field_kick(const Local &L, float a, float dc, float srf, float &kx, float &ky,
                                           float &kz)
{
    if constexpr (kPack) {
        // (r, z) side by side in packed FP32x2 instructions:
        // k_rz = a ((dc E_DC + srf E_RF) + E_SCE), then (kx, ky) = k_r (cx, cy)
        float2 t = __fmul2_rn(make_float2(dc, dc), make_float2(L.edr, L.edz));
        t = __ffma2_rn(make_float2(srf, srf), make_float2(L.err, L.erz), t);
        t = __fadd2_rn(t, make_float2(L.esr, L.esz));
        t = __fmul2_rn(make_float2(a, a), t);
        const float2 kxy = __fmul2_rn(make_float2(t.x, t.x), make_float2(L.cx, L.cy));
        kx = kxy.x;
        ky = kxy.y;
        kz = t.y;
    } else {
        const float kr = a * (dc * L.edr + srf * L.err + L.esr);
        kx = kr * L.cx;
        ky = kr * L.cy;
        kz = a * (dc * L.edz + srf * L.erz + L.esz);
    }
}

// Cell index and fraction along one axis; clamped to the last cell.
__device__ __forceinline__ void cell_r(float g, int n, int &i0, float &f)
{
    const int i = __float2int_rd(g);
    const bool last = i > n - 2;
    i0 = last ? n - 2 : i;
    f = last ? 1.0f : g - (float)i;
}

__device__ __forceinline__ void cell_z(int32_t zq, int n, int &j0, float &f)
{
    const int64_t t = (int64_t)zq * (int64_t)(n - 1);
    const int j = (int)(t >> 30); // |zq| < 2^31 and n < 2^20: fits
    const float fr = (float)(int)((uint32_t)t & 0x3FFFFFFFu) * (1.0f / 1073741824.0f);
    j0 = j < 0 ? 0 : (j > n - 2 ? n - 2 : j);
    f = j < 0 ? 0.0f : (j > n - 2 ? 1.0f : fr);
}

// Bilinear combination of four node records, each component summed in the
// order w00 a + w10 b + w01 c + w11 d (a product, then three fused
// multiply-adds); kPack: two components per packed FP32x2 instruction.
template <bool kPack = true>
__device__ __forceinline__ float4 lerp4(float4 a, float4 b, float4 c, float4 d, float w00, float w10,
                                        float w01, float w11)
{
    if constexpr (kPack) {
        const float2 p00 = make_float2(w00, w00), p10 = make_float2(w10, w10);
        const float2 p01 = make_float2(w01, w01), p11 = make_float2(w11, w11);
        float2 lo = __fmul2_rn(p00, make_float2(a.x, a.y));
        float2 hi = __fmul2_rn(p00, make_float2(a.z, a.w));
        lo = __ffma2_rn(p10, make_float2(b.x, b.y), lo);
        hi = __ffma2_rn(p10, make_float2(b.z, b.w), hi);
        lo = __ffma2_rn(p01, make_float2(c.x, c.y), lo);
        hi = __ffma2_rn(p01, make_float2(c.z, c.w), hi);
        lo = __ffma2_rn(p11, make_float2(d.x, d.y), lo);
        hi = __ffma2_rn(p11, make_float2(d.z, d.w), hi);
        return make_float4(lo.x, lo.y, hi.x, hi.y);
    } else {
        return make_float4(w00 * a.x + w10 * b.x + w01 * c.x + w11 * d.x,
                           w00 * a.y + w10 * b.y + w01 * c.y + w11 * d.y,
                           w00 * a.z + w10 * b.z + w01 * c.z + w11 * d.z,
                           w00 * a.w + w10 * b.w + w01 * c.w + w11 * d.w);
    }
}

// Per-lane cache of the last PIC cell read: its index and the E_SCE of its
// four nodes (32 bytes, in two shared-memory slots of the lane). The field
// is fixed for the length of a launch (the solve runs between launches) and
// a pack crosses a PIC cell boundary only every few tens of micro steps, so
// most steps read the cell from shared memory instead of L2. The values are
// the same either way. cell = -1: empty; lo = nullptr: no cache.
struct EscCache {
    int cell;
    float4 *lo, *hi;
};

template <bool kPack = true>
__device__ __forceinline__ void gather(const GridF32 &G, const InstF32 &P, float fx, float fy,
                                       float rr, int32_t zq, Local &L, EscCache *C = nullptr)
{
    int i0, j0;
    float ar, az;
    cell_r(rr * G.sr, G.nr, i0, ar);
    cell_z(zq, G.nz, j0, az);
    const NodeF *nd = G.node + (size_t)j0 * G.nr + i0;
    const float4 a00 = __ldg(&nd[0].a), a10 = __ldg(&nd[1].a);
    const float4 a01 = __ldg(&nd[G.nr].a), a11 = __ldg(&nd[G.nr + 1].a);
    const float4 b00 = __ldg(&nd[0].b), b10 = __ldg(&nd[1].b);
    const float4 b01 = __ldg(&nd[G.nr].b), b11 = __ldg(&nd[G.nr + 1].b);
    float w00, w10, w01, w11;
    if constexpr (kPack) {
        // (w00, w10) and (w01, w11): (1 - ar, ar) times 1 - az and az
        const float2 wr = make_float2(1.0f - ar, ar);
        const float2 wl = __fmul2_rn(wr, make_float2(1.0f - az, 1.0f - az));
        const float2 wh = __fmul2_rn(wr, make_float2(az, az));
        w00 = wl.x; w10 = wl.y;
        w01 = wh.x; w11 = wh.y;
    } else {
        w00 = (1.0f - ar) * (1.0f - az); w10 = ar * (1.0f - az);
        w01 = (1.0f - ar) * az; w11 = ar * az;
    }
    const float4 fa = lerp4<kPack>(a00, a10, a01, a11, w00, w10, w01, w11);
    const float4 fb = lerp4<kPack>(b00, b10, b01, b11, w00, w10, w01, w11);
    const float inv = rr > 0.0f ? __fdividef(1.0f, rr) : 0.0f;
    // Eq. 3: zero transverse projection on the axis
    float cx, cy;
    if constexpr (kPack) {
        const float2 cxy = __fmul2_rn(make_float2(fx, fy), make_float2(inv, inv));
        cx = cxy.x; cy = cxy.y;
    } else {
        cx = fx * inv; cy = fy * inv;
    }
    L.cx = cx;
    L.cy = cy;
    L.edr = fa.x; L.edz = fa.y;
    L.err = fa.z; L.erz = fa.w;
    L.T = fb.y;
    L.nsig = fb.y > 0.0f ? __fdividef(P.psig * fb.x, fb.y) : 0.0f;
    if constexpr (kPack) {
        const float2 uxy = __fmul2_rn(make_float2(fb.z, fb.z), make_float2(cx, cy));
        L.ux = uxy.x; L.uy = uxy.y;
    } else {
        L.ux = fb.z * cx; L.uy = fb.z * cy;
    }
    L.uz = fb.w;
    L.esr = L.esz = 0.0f;
    if (P.esc4 != nullptr) {
        int pi0, pj0;
        float pr, pz;
        cell_r(rr * P.psr, P.pnr, pi0, pr);
        cell_z(zq, P.pnz, pj0, pz);
        // the cell's four nodes in one 32-byte sector
        const int c = pj0 * (P.pnr - 1) + pi0;
        float4 lo, hi;
        if (C != nullptr && C->lo != nullptr && c == C->cell) {
            lo = *C->lo;
            hi = *C->hi;
        } else {
            const float4 *e = P.esc4 + 2 * (size_t)c;
            lo = __ldg(&e[0]);
            hi = __ldg(&e[1]);
            if (C != nullptr && C->lo != nullptr) {
                *C->lo = lo;
                *C->hi = hi;
                C->cell = c;
            }
        }
        if constexpr (kPack) {
            // (E_r, E_z) of the four nodes side by side: weights as above,
            // then a product and three fused multiply-adds per component
            const float2 vr = make_float2(1.0f - pr, pr);
            const float2 vl = __fmul2_rn(vr, make_float2(1.0f - pz, 1.0f - pz));
            const float2 vh = __fmul2_rn(vr, make_float2(pz, pz));
            float2 es = __fmul2_rn(make_float2(vl.x, vl.x), make_float2(lo.x, lo.y));
            es = __ffma2_rn(make_float2(vl.y, vl.y), make_float2(lo.z, lo.w), es);
            es = __ffma2_rn(make_float2(vh.x, vh.x), make_float2(hi.x, hi.y), es);
            es = __ffma2_rn(make_float2(vh.y, vh.y), make_float2(hi.z, hi.w), es);
            L.esr = es.x;
            L.esz = es.y;
        } else {
            const float v00 = (1.0f - pr) * (1.0f - pz), v10 = pr * (1.0f - pz), v01 = (1.0f - pr) * pz,
                        v11 = pr * pz;
            L.esr = v00 * lo.x + v10 * lo.z + v01 * hi.x + v11 * hi.z;
            L.esz = v00 * lo.y + v10 * lo.w + v01 * hi.y + v11 * hi.w;
        }
    }
}

// e^x - 1 for x <= 0 without cancellation: near 0 the Taylor series to x^5
// (truncation below 1.4e-9 relative for |x| < 1/16), else expf(x) - 1,
// whose rounding error is then small against |e^x - 1| >= 0.06.
__device__ __forceinline__ float expm1_neg(float x)
{
    if (x > -0.0625f)
        return x * (1.0f + x * (0.5f + x * (1.0f / 6.0f + x * (1.0f / 24.0f + x * (1.0f / 120.0f)))));
    return expf(x) - 1.0f;
}

// T_eff from E_int (kelvin units) through the heat-capacity profile.
__device__ __forceinline__ float teff_of(const InstF32 &P, float eint)
{
    const float e = eint * P.inv_n3;
    if (e <= P.ecap) return __fdividef(2.0f * e, P.c0 + sqrt_fast(P.c0 * P.c0 + 2.0f * P.c1 * e));
    return P.tcap + (e - P.ecap);
}

// Uniforms of a candidate from the eight words of its two Philox blocks:
// the top 21 bits of one word, or the low 11 bits of two words joined into
// 22 bits; both land mid-interval and are exact in FP32.
__device__ __forceinline__ float u21(uint32_t w)
{
    return ((float)(w >> 11) + 0.5f) * 4.76837158203125e-07f; // 2^-21
}

__device__ __forceinline__ float u22(uint32_t hi, uint32_t lo)
{
    const uint32_t v = ((hi & 0x7FFu) << 11) | (lo & 0x7FFu);
    return ((float)v + 0.5f) * 2.384185791015625e-07f; // 2^-22
}

// Gas and force of one step, gathered at the step's start position and held
// while the step's collision candidates are processed.
struct StepGas {
    float kx, ky, kz;          // velocity kick (q/m)(s_dc E_DC + s_rf(n) E_RF + E_SCE) dt
    float nsig, T, ux, uy, uz; // n sigma, gas temperature and flow
    float s;                   // thermal speed sqrt(2 k_B T / m_gas)
};

// Collisions (Eq. 6): candidates form a Poisson process of rate
// nu = n sigma (|v - u| + 2 s / sqrt(pi)); the pack carries the optical depth
// tau left until its next candidate, so a step without one costs a rate
// evaluation and draws nothing. One pass at time t of the step: the rest of
// the step holds nu (dt - t) of optical depth; returns true when tau runs out
// inside it (a candidate at t + tau / nu), else consumes that depth.
// The relative speed w = |v - u| of the pass is returned for the candidate.
template <bool kPack = true>
__device__ __forceinline__ bool next_candidate(const InstF32 &P, const StepGas &S, float vx, float vy,
                                               float vz, float &tau, float &t, float &w)
{
    const float cbar = 1.1283791670955126f * S.s; // 2 s / sqrt(pi)
    if constexpr (kPack) {
        const float2 wxy = __fadd2_rn(make_float2(vx, vy), make_float2(-S.ux, -S.uy));
        const float wz = vz - S.uz;
        const float2 sq = __fmul2_rn(wxy, wxy);
        w = sqrt_fast(fmaf(wz, wz, sq.x + sq.y));
    } else {
        const float wx = vx - S.ux, wy = vy - S.uy, wz = vz - S.uz;
        w = sqrt_fast(wx * wx + wy * wy + wz * wz);
    }
    const float nu = S.nsig * (w + cbar);
    const float room = nu * (P.dt - t);
    if (tau >= room) {
        tau -= room;
        return false;
    }
    t += __fdividef(tau, nu);
    return true;
}

// Candidate kc of a step (Philox blocks 2kc and 2kc+1, words A and B):
// fields A.x branch, A.y accept, A.z Maxwellian extra, A.w and B.x partner
// magnitude, B.y and B.z partner direction, B.w and (A.x, A.y low bits)
// scattering direction, (A.z, A.w) and (B.x, B.y) low bits the Beta uniforms,
// (B.z, B.w) low bits the next optical depth. Returns 1 when accepted.
// w: |v - u| from the pass of next_candidate that found the candidate.
template <bool kPack = true>
__device__ __forceinline__ int candidate(const InstF32 &P, const StepGas &S, uint32_t pack, uint32_t step,
                                         uint32_t kc, float w, float &vx, float &vy, float &vz, float &eint,
                                         float &tau)
{
    // kPack: the x and y components of the vector arithmetic side by side in
    // packed FP32x2 instructions (the same operations per component)
    const float s = S.s;
    const float cbar = 1.1283791670955126f * s;
    float wx, wy;
    if constexpr (kPack) {
        const float2 wxy = __fadd2_rn(make_float2(vx, vy), make_float2(-S.ux, -S.uy));
        wx = wxy.x; wy = wxy.y;
    } else {
        wx = vx - S.ux; wy = vy - S.uy;
    }
    const float wz = vz - S.uz;
    uint4 A = make_uint4(pack, step, 2u * kc, 0u), B = make_uint4(pack, step, 2u * kc + 1u, 0u);
    philox10x2(A, B, P.rkey);
    tau = -__logf(u22(B.z, B.w));
    // Partner |c'|^2 / s^2 ~ Gamma(k, 1), isotropic: k = 3/2 (Maxwellian)
    // or 2 (speed-weighted); Gamma(3/2) = Exp(1) + N^2/2 with
    // N^2/2 = -ln(u) cos^2(2 pi u'). One branch-free path for both laws.
    float f = 1.0f;
    if (u21(A.x) * (w + cbar) < w) {
        float sn0, cs0;
        sincos_2pi(u21(A.z), sn0, cs0);
        f = cs0 * cs0;
    }
    const float y = -__logf(u21(A.w)) - __logf(u21(B.x)) * f;
    const float cmag = s * sqrt_fast(y);
    float cx, cy, cz;
    {
        const float ct = 2.0f * u21(B.y) - 1.0f;
        const float st = sqrt_fast(fmaxf(0.0f, 1.0f - ct * ct));
        float sn, cs;
        sincos_2pi(u21(B.z), sn, cs);
        if constexpr (kPack) {
            const float cst = cmag * st;
            const float2 cxy = __fmul2_rn(make_float2(cst, cst), make_float2(cs, sn));
            cx = cxy.x; cy = cxy.y;
        } else {
            cx = cmag * st * cs;
            cy = cmag * st * sn;
        }
        cz = cmag * ct;
    }
    float g2;
    if constexpr (kPack) {
        const float2 gxy = __fadd2_rn(make_float2(wx, wy), make_float2(-cx, -cy));
        const float gz = wz - cz;
        const float2 gg = __fmul2_rn(gxy, gxy);
        g2 = fmaf(gz, gz, gg.x + gg.y);
    } else {
        const float gx = wx - cx, gy = wy - cy, gz = wz - cz;
        g2 = gx * gx + gy * gy + gz * gz;
    }
    const float g = sqrt_fast(g2);
    if (!(u21(A.y) * (w + cmag) < g)) return 0;
    float Vx, Vy;
    if constexpr (kPack) {
        const float2 Vxy = __ffma2_rn(make_float2(P.fM, P.fM), make_float2(vx, vy),
                                      __fmul2_rn(make_float2(P.fm, P.fm),
                                                 __fadd2_rn(make_float2(S.ux, S.uy), make_float2(cx, cy))));
        Vx = Vxy.x; Vy = Vxy.y;
    } else {
        Vx = P.fM * vx + P.fm * (S.ux + cx);
        Vy = P.fM * vy + P.fm * (S.uy + cy);
    }
    const float Vz = P.fM * vz + P.fm * (S.uz + cz);
    const float etr = P.mu_2kb * g2;
    const float ec = etr + eint;
    const float Te = teff_of(P, eint);
    const float a = P.n3 * fminf(1.0f, P.c0 + P.c1 * Te);
    // 1 - B for B ~ Beta(a, 2); expm1 keeps the precision of small exchanges
    const float omb = -expm1_neg(__fdividef(__logf(u22(A.z, A.w)), a) +
                                 __fdividef(__logf(u22(B.x, B.y)), a + 1.0f));
    const float etr_new = ec * omb;
    eint = eint + (etr - etr_new);
    const float gn = sqrt_fast(etr_new * P.g_coef) * P.fm;
    const float ct = 2.0f * u21(B.w) - 1.0f;
    const float st = sqrt_fast(fmaxf(0.0f, 1.0f - ct * ct));
    float sn, cs;
    sincos_2pi(u22(A.x, A.y), sn, cs);
    if constexpr (kPack) {
        const float gst = gn * st;
        const float2 nv = __ffma2_rn(make_float2(gst, gst), make_float2(cs, sn), make_float2(Vx, Vy));
        vx = nv.x; vy = nv.y;
    } else {
        vx = Vx + gn * st * cs;
        vy = Vy + gn * st * sn;
    }
    vz = Vz + gn * ct;
    return 1;
}

// Expected collision rate n sigma <|v - c|> (Eq. 6, Maxwellian partner):
// n sigma s [(x + 1/(2x)) erf(x) + exp(-x^2)/sqrt(pi)], x = |v - u| / s.
template <class Gas>
__device__ __forceinline__ float collision_rate(const InstF32 &P, const Gas &L, float vx, float vy, float vz)
{
    const float s = sqrt_fast(P.s_coef * L.T);
    const float wx = vx - L.ux, wy = vy - L.uy, wz = vz - L.uz;
    const float w = sqrt_fast(wx * wx + wy * wy + wz * wz);
    const float x = __fdividef(w, s);
    const float g = x > 1e-3f ? s * ((x + __fdividef(0.5f, x)) * erff(x) + __expf(-x * x) * 0.5641895835f)
                              : 1.1283791671f * s * (1.0f + x * x * (1.0f / 3.0f));
    return L.nsig * g;
}

// Hybrid Langevin step: exact Ornstein-Uhlenbeck update of v - u over dt with
// friction gamma = q / (M K) (Mason-Schamp K) and the gas temperature's
// equilibrium spread; normals from draw block 128 of the step.
__device__ __forceinline__ void langevin_step(const InstF32 &P, const StepGas &L, uint32_t pack,
                                              uint32_t step, float &vx, float &vy, float &vz)
{
    const float sqT = sqrt_fast(L.T);
    const float gdt = P.lv_c * L.nsig * sqT * P.dt;
    const float decay = __expf(-gdt);
    const float sd = sqT * sqrt_fast(P.lv_kM * -expm1f(-2.0f * gdt));
    const uint4 U = philox10(make_uint4(pack, step, 128u, 0u), P.rkey);
    const float r01 = sd * sqrt_fast(-2.0f * __logf(u01f(U.x)));
    const float r23 = sd * sqrt_fast(-2.0f * __logf(u01f(U.z)));
    float sn, cs, sn2, cs2;
    sincos_2pi(u01f(U.y), sn, cs);
    sincos_2pi(u01f(U.w), sn2, cs2);
    vx = L.ux + (vx - L.ux) * decay + r01 * cs;
    vy = L.uy + (vy - L.uy) * decay + r01 * sn;
    vz = L.uz + (vz - L.uz) * decay + r23 * cs2;
}

// Lattice displacement of one step, floor(d + u) with a uniform dither u,
// clamped to keep the int32 lattice from wrapping.
__device__ __forceinline__ int32_t lattice_step(float d, float u)
{
    d = fminf(fmaxf(d, -1.0e9f), 1.0e9f);
    return __float2int_rd(d + u);
}

// Lattice radius in FP32, IEEE round-to-nearest, no contraction.
__device__ __forceinline__ float lattice_r(float fx, float fy)
{
    return __fsqrt_rn(__fadd_rn(__fmul_rn(fx, fx), __fmul_rn(fy, fy)));
}

__device__ __forceinline__ int classify(const GridF32 &G, const InstF32 &P, int32_t xq, int32_t yq,
                                        int32_t zq, float rr)
{
    int ir = __float2int_rz(__fadd_rn(__fmul_rn(rr, G.sr), 0.5f));
    ir = min(ir, G.nr - 1);
    // nearest z node; |zq| < 2^31 and nz < 2^20, so the shifted value fits
    int iz = (int)(((int64_t)zq * (int64_t)(G.nz - 1) + (1LL << 29)) >> 30);
    iz = min(max(iz, 0), G.nz - 1);
    const float d = __ldg(&G.dmask[iz * G.nr + ir]);
    const uint64_t r2 = (uint64_t)((int64_t)xq * xq) + (uint64_t)((int64_t)yq * yq);
    // precedence: electrode, radial wall, exit plane (detector or not), z < 0;
    // selected without branches, the lowest precedence first
    int st = zq < 0 ? MUCITE_AXIAL : MUCITE_ACTIVE;
    st = zq >= P.zexit_q ? (r2 <= P.rdet2 ? MUCITE_TRANSMITTED : MUCITE_AXIAL) : st;
    st = r2 >= (1ULL << 60) ? MUCITE_RADIAL : st;
    return d <= P.hit ? MUCITE_ELECTRODE : st;
}

__device__ __forceinline__ unsigned warp_sum(unsigned v)
{
    return __reduce_add_sync(0xffffffffu, v);
}

// Velocity increment kick * E_tot over one step at the RK4 stage position
// x + h v (h v given in m/s times the step, i.e. the stage's fraction of
// the step times the stage velocity), with RF scalar srf.
template <bool kPack = true>
__device__ __forceinline__ void stage_kick(const GridF32 &G, const InstF32 &P, int32_t xq, int32_t yq,
                                           int32_t zq, float hvx, float hvy, float hvz, float srf, float &kx,
                                           float &ky, float &kz)
{
    const int32_t sx = xq + __float2int_rn(fminf(fmaxf(hvx * P.cxs, -1.0e9f), 1.0e9f));
    const int32_t sy = yq + __float2int_rn(fminf(fmaxf(hvy * P.cxs, -1.0e9f), 1.0e9f));
    const int32_t sz = zq + __float2int_rn(fminf(fmaxf(hvz * P.czs, -1.0e9f), 1.0e9f));
    const float fx = (float)sx, fy = (float)sy;
    Local L;
    gather<kPack>(G, P, fx, fy, lattice_r(fx, fy), sz, L);
    field_kick<kPack>(L, P.kick, P.dc_scale, srf, kx, ky, kz);
}

// Counters of a warp added to the instance's totals.
__device__ __forceinline__ void add_counters(const InstF32 &P, unsigned n_steps_done, unsigned n_coll,
                                             unsigned n_ovf)
{
    n_steps_done = warp_sum(n_steps_done);
    n_coll = warp_sum(n_coll);
    n_ovf = warp_sum(n_ovf);
    if ((threadIdx.x & 31) == 0) {
        if (n_steps_done) atomicAdd(&P.counters[0], (unsigned long long)n_steps_done);
        if (n_coll) atomicAdd(&P.counters[1], (unsigned long long)n_coll);
        if (n_ovf) atomicAdd(&P.counters[2], (unsigned long long)n_ovf);
    }
}

// End-of-launch charge deposit of a pack that is still active (the charge
// the next space-charge solve needs, deposited while the positions are in
// registers): the same integer CIC contributions as the standalone deposit.
__device__ __forceinline__ void deposit_at_end(const InstF32 &P, int32_t xq, int32_t yq, int32_t zq)
{
    uint32_t cell;
    unsigned long long w[4];
    if (!cic_lattice(xq, yq, zq, P.pnr, P.pnz, P.dep_qw, cell, w)) return;
    unsigned long long *Q = P.dep_q + cell;
    if (w[0]) atomicAdd(Q, w[0]);
    if (w[1]) atomicAdd(Q + 1, w[1]);
    if (w[2]) atomicAdd(Q + P.pnr, w[2]);
    if (w[3]) atomicAdd(Q + P.pnr + 1, w[3]);
}

// Kick and drift of step n with kick (kx, ky, kz) evaluated at x_n (RK4:
// the first stage), then the lattice radius and class at x_{n+1}.
template <bool kExtras, bool kPack = true>
__device__ __forceinline__ int push(const GridF32 &G, const InstF32 &P, const float *s_rf, int k,
                                    uint32_t h1, uint32_t h2, float kx, float ky, float kz, int32_t &xq,
                                    int32_t &yq, int32_t &zq, float &vx, float &vy, float &vz, float &fx,
                                    float &fy, float &rr)
{
    if (kExtras && P.rk4) {
        // RK4 under the instantaneous field: stages at t, t + dt/2 (x2)
        // and t + dt; stage positions rounded to the lattice
        const float sh = s_rf[2 * k + 1], s1 = s_rf[2 * k + 2];
        float k2x, k2y, k2z, k3x, k3y, k3z, k4x, k4y, k4z;
        stage_kick<kPack>(G, P, xq, yq, zq, 0.5f * vx, 0.5f * vy, 0.5f * vz, sh, k2x, k2y, k2z);
        const float v2x = vx + 0.5f * kx, v2y = vy + 0.5f * ky, v2z = vz + 0.5f * kz;
        stage_kick<kPack>(G, P, xq, yq, zq, 0.5f * v2x, 0.5f * v2y, 0.5f * v2z, sh, k3x, k3y, k3z);
        const float v3x = vx + 0.5f * k2x, v3y = vy + 0.5f * k2y, v3z = vz + 0.5f * k2z;
        stage_kick<kPack>(G, P, xq, yq, zq, v3x, v3y, v3z, s1, k4x, k4y, k4z);
        const float v4x = vx + k3x, v4y = vy + k3y, v4z = vz + k3z;
        const float c6 = 1.0f / 6.0f;
        const float ux = (vx + 2.0f * v2x + 2.0f * v3x + v4x) * c6;
        const float uy = (vy + 2.0f * v2y + 2.0f * v3y + v4y) * c6;
        const float uz = (vz + 2.0f * v2z + 2.0f * v3z + v4z) * c6;
        vx = add_sr(vx, (kx + 2.0f * k2x + 2.0f * k3x + k4x) * c6, dither_c(h1, 0));
        vy = add_sr(vy, (ky + 2.0f * k2y + 2.0f * k3y + k4y) * c6, dither_c(h1, 11));
        vz = add_sr(vz, (kz + 2.0f * k2z + 2.0f * k3z + k4z) * c6, dither_c(h1, 22));
        xq += lattice_step(ux * P.cxs, dither(h2, 0));
        yq += lattice_step(uy * P.cxs, dither(h2, 11));
        zq += lattice_step(uz * P.czs, dither(h2, 22));
    } else if (kPack) {
        // x and y side by side in packed FP32x2 instructions (the same
        // operations per component as add_sr and lattice_step)
        const float2 v = make_float2(vx, vy), d = make_float2(kx, ky);
        const float2 t = __fadd2_rn(v, d);
        const float2 ulp = __fmul2_rn(make_float2(__int_as_float(__float_as_int(t.x) & 0x7f800000),
                                                  __int_as_float(__float_as_int(t.y) & 0x7f800000)),
                                      make_float2(1.1920928955078125e-7f, 1.1920928955078125e-7f));
        const float2 nv = __fadd2_rn(v, __ffma2_rn(make_float2(dither_c(h1, 0), dither_c(h1, 11)), ulp, d));
        vx = nv.x;
        vy = nv.y;
        vz = add_sr(vz, kz, dither_c(h1, 22));
        const float2 sxy = __fmul2_rn(nv, make_float2(P.cxs, P.cxs));
        xq += lattice_step(sxy.x, dither(h2, 0));
        yq += lattice_step(sxy.y, dither(h2, 11));
        zq += lattice_step(vz * P.czs, dither(h2, 22));
    } else {
        vx = add_sr(vx, kx, dither_c(h1, 0));
        vy = add_sr(vy, ky, dither_c(h1, 11));
        vz = add_sr(vz, kz, dither_c(h1, 22));
        xq += lattice_step(vx * P.cxs, dither(h2, 0));
        yq += lattice_step(vy * P.cxs, dither(h2, 11));
        zq += lattice_step(vz * P.czs, dither(h2, 22));
    }
    fx = (float)xq;
    fy = (float)yq;
    rr = lattice_r(fx, fy);
    return classify(G, P, xq, yq, zq, rr);
}

// Kick of step k at the gathered fields.
template <bool kPack = true>
__device__ __forceinline__ void kick_of(const InstF32 &P, const Local &L, float srf, float &kx, float &ky,
                                        float &kz)
{
    field_kick<kPack>(L, P.kick, P.dc_scale, srf, kx, ky, kz);
}

// Collision-free tile: the U x blockDim.x packs of instance P starting at
// pack `off` advance `nsteps` micro steps (gather, kick, drift, classify).
// Each thread carries U packs whose steps are computed side by side (no
// branch between them, so their load and arithmetic chains overlap); a pack
// that has become terminal keeps its state and only its tentative step is
// discarded. The state of all U packs is loaded up front, not behind the
// status load, so the loads of a thread are in flight together.
template <bool kExtras, int U>
__device__ __forceinline__ void run_tile_free(const GridF32 &G, const InstF32 &P, const float *s_rf,
                                              int64_t off, int nsteps)
{
    int32_t xq[U], yq[U], zq[U], kd[U], st[U];
    float vx[U], vy[U], vz[U], eint[U], lnsy[U], fx[U], fy[U], rr[U];
    uint32_t hb[U];
    bool own[U], mv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int64_t p = off + threadIdx.x + (int64_t)u * blockDim.x;
        const int64_t q = p < P.n_slots ? p : 0; // an owned slot for the unconditional loads
        own[u] = p < P.n_slots && P.status[q] == MUCITE_ACTIVE;
        mv[u] = own[u];
        xq[u] = P.xq[q]; yq[u] = P.yq[q]; zq[u] = P.zq[q];
        vx[u] = P.vx[q]; vy[u] = P.vy[q]; vz[u] = P.vz[q];
        eint[u] = (kExtras && P.tst) ? P.eint[q] : 0.0f;
        lnsy[u] = (kExtras && P.tst) ? P.lnsy[q] : 0.0f;
        hb[u] = pack_key((uint32_t)p, P);
        fx[u] = (float)xq[u];
        fy[u] = (float)yq[u];
        rr[u] = lattice_r(fx[u], fy[u]);
        kd[u] = 0;
        st[u] = MUCITE_ACTIVE;
    }
    for (int k = 0; k < nsteps; ++k) {
        const uint32_t n = (uint32_t)(P.step0 + k);
        bool any = false;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            Local L;
            gather(G, P, fx[u], fy[u], rr[u], zq[u], L);
            float kx, ky, kz;
            kick_of(P, L, s_rf[2 * k], kx, ky, kz);
            const uint32_t h1 = dither_word(hb[u], n), h2 = remix32(h1);
            float ls = lnsy[u];
            if (kExtras && P.tst) {
                // Eq. 7: d ln SY / dt = -k(T_eff), Eyring rate at the current T_eff
                const float Te = teff_of(P, eint[u]);
                const float kdt = P.tst_a_dt * Te * __expf(-P.tst_b * __frcp_rn(Te));
                ls = add_sr(ls, -kdt, dither_c(fmix32(h1 ^ 0x68E31DA4u), 0));
            }
            int32_t x2 = xq[u], y2 = yq[u], z2 = zq[u];
            float wx = vx[u], wy = vy[u], wz = vz[u], gx, gy, gr;
            const int s2 = push<kExtras>(G, P, s_rf, k, h1, h2, kx, ky, kz, x2, y2, z2, wx, wy, wz, gx, gy, gr);
            if (mv[u]) {
                xq[u] = x2; yq[u] = y2; zq[u] = z2;
                vx[u] = wx; vy[u] = wy; vz[u] = wz;
                fx[u] = gx; fy[u] = gy; rr[u] = gr;
                lnsy[u] = ls;
                st[u] = s2;
                kd[u] = k + 1;
                mv[u] = s2 == MUCITE_ACTIVE;
            }
            any = any || mv[u];
        }
        if (!any) break;
    }
    unsigned n_steps_done = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if (!own[u]) continue;
        const int64_t p = off + threadIdx.x + (int64_t)u * blockDim.x;
        n_steps_done += (unsigned)kd[u];
        P.xq[p] = xq[u]; P.yq[p] = yq[u]; P.zq[p] = zq[u];
        P.vx[p] = vx[u]; P.vy[p] = vy[u]; P.vz[p] = vz[u];
        if (kExtras && P.tst) P.lnsy[p] = lnsy[u];
        if (st[u] != MUCITE_ACTIVE) {
            P.status[p] = (uint8_t)st[u];
            P.t_term[p] = (int32_t)(P.step0 + kd[u]);
        } else if (P.dep_q != nullptr) {
            deposit_at_end(P, xq[u], yq[u], zq[u]);
        }
    }
    add_counters(P, n_steps_done, 0u, 0u);
}

// Start of step k of one pack: gather at x_k, the step's kick, the Langevin
// switch, and the first pass of the candidate loop. Returns whether a
// collision candidate is pending.
template <bool kExtras, bool kPack = true>
__device__ __forceinline__ bool begin_step(const GridF32 &G, const InstF32 &P, const float *s_rf, int k,
                                           uint32_t pack, float fx, float fy, float rr, int32_t zq,
                                           float &vx, float &vy, float &vz, float &tau, float &t,
                                           float &w, bool &lv, StepGas &S, EscCache &C, int64_t step0)
{
    Local L;
    gather<kPack>(G, P, fx, fy, rr, zq, L, &C);
    kick_of<kPack>(P, L, s_rf[2 * k], S.kx, S.ky, S.kz);
    S.nsig = L.nsig; S.T = L.T;
    S.ux = L.ux; S.uy = L.uy; S.uz = L.uz;
    t = 0.0f;
    lv = false;
    if (!(S.nsig > 0.0f) || !(S.T > 0.0f)) return false;
    S.s = sqrt_fast(P.s_coef * S.T);
    if (kExtras && P.langevin && zq >= P.lv_zq0 && zq <= P.lv_zq1)
        lv = collision_rate(P, S, vx, vy, vz) * P.dt >= P.lv_switch;
    if (lv) {
        langevin_step(P, S, pack, (uint32_t)(step0 + k), vx, vy, vz);
        return false;
    }
    return next_candidate<kPack>(P, S, vx, vy, vz, tau, t, w);
}

// Tile with collisions. Each lane owns a pack and walks through its steps;
// a step may hold several collision candidates (a Poisson number). Rather
// than stepping all lanes together, which makes the warp run the candidate
// code as often as its busiest lane needs it, every iteration the warp
// either processes one candidate of each lane that has one pending or
// finishes the step (kick, drift, classify, next gather) of each lane that
// has none, whichever serves more lanes. Lanes drift apart in step index;
// every pack still takes exactly its own sequence of operations, so results
// do not depend on the schedule. kW > 1 serves the pending candidates as
// soon as their lanes are at least 1 / kW of those ready to push: in
// launches of a few micro steps, where candidates are rare, lanes that wait
// for enough others to have a candidate fall steps behind, and the launch
// ends with them running nearly alone.
template <bool kExtras, bool kPack, int kW = 1>
__device__ __forceinline__ void run_tile_coll(const GridF32 &G, const InstF32 &P, const float *s_rf,
                                              int64_t off, int nsteps, float4 *s_esc, int64_t step0)
{
    const int64_t p = off + threadIdx.x;
    const bool owned = p < P.n_slots && P.status[p] == MUCITE_ACTIVE;
    int32_t xq = 0, yq = 0, zq = 0;
    float vx = 0.0f, vy = 0.0f, vz = 0.0f, eint = 0.0f, tau = 0.0f, lnsy = 0.0f;
    if (owned) {
        xq = P.xq[p]; yq = P.yq[p]; zq = P.zq[p];
        vx = P.vx[p]; vy = P.vy[p]; vz = P.vz[p];
        eint = P.eint[p];
        tau = P.tau[p];
        if (kExtras && P.tst) lnsy = P.lnsy[p];
    }
    const uint32_t pack = (uint32_t)p;
    const uint32_t hbase = pack_key(pack, P);
    float fx = (float)xq, fy = (float)yq;
    float rr = lattice_r(fx, fy);
    unsigned n_coll = 0, n_ovf = 0;
    int k = 0, kc = 0, st = MUCITE_ACTIVE;
    float t = 0.0f, w = 0.0f;
    bool lv = false, live = owned && nsteps > 0, pend = false;
    StepGas S;
    EscCache C{-1, nullptr, nullptr};
    if (s_esc != nullptr && P.esc4 != nullptr) {
        C.lo = s_esc + threadIdx.x;
        C.hi = s_esc + blockDim.x + threadIdx.x;
    }
    if (live)
        pend = begin_step<kExtras, kPack>(G, P, s_rf, 0, pack, fx, fy, rr, zq, vx, vy, vz, tau, t, w, lv, S, C, step0);
    for (;;) {
        const bool can_push = live && !pend;
        const unsigned mc = __ballot_sync(0xffffffffu, pend);
        const unsigned mp = __ballot_sync(0xffffffffu, can_push);
        if ((mc | mp) == 0u) break;
        if (mc != 0u && kW * __popc(mc) >= __popc(mp)) {
            if (pend) {
                n_coll += (unsigned)candidate<kPack>(P, S, pack, (uint32_t)(step0 + k), (uint32_t)kc, w, vx, vy,
                                              vz, eint, tau);
                if (++kc == kKmax) {
                    ++n_ovf; // candidate cap: the rest of the step holds no further candidate
                    pend = false;
                } else {
                    pend = next_candidate<kPack>(P, S, vx, vy, vz, tau, t, w);
                }
            }
        } else if (can_push) {
            const uint32_t n = (uint32_t)(step0 + k);
            const uint32_t h1 = dither_word(hbase, n), h2 = remix32(h1);
            if (kExtras && P.tst && !lv) {
                // Eq. 7: d ln SY / dt = -k(T_eff), Eyring rate at the current T_eff
                const float Te = teff_of(P, eint);
                const float kdt = P.tst_a_dt * Te * __expf(-P.tst_b * __frcp_rn(Te));
                lnsy = add_sr(lnsy, -kdt, dither_c(fmix32(h1 ^ 0x68E31DA4u), 0));
            }
            st = push<kExtras, kPack>(G, P, s_rf, k, h1, h2, S.kx, S.ky, S.kz, xq, yq, zq, vx, vy, vz, fx, fy,
                                      rr);
            ++k;
            kc = 0;
            if (st != MUCITE_ACTIVE || k == nsteps)
                live = false;
            else
                pend = begin_step<kExtras, kPack>(G, P, s_rf, k, pack, fx, fy, rr, zq, vx, vy, vz, tau, t, w, lv,
                                                  S, C, step0);
        }
    }
    if (owned) {
        P.xq[p] = xq; P.yq[p] = yq; P.zq[p] = zq;
        P.vx[p] = vx; P.vy[p] = vy; P.vz[p] = vz;
        P.eint[p] = eint;
        P.tau[p] = tau;
        if (kExtras && P.tst) P.lnsy[p] = lnsy;
        if (st != MUCITE_ACTIVE) {
            P.status[p] = (uint8_t)st;
            P.t_term[p] = (int32_t)(step0 + k);
        } else if (P.dep_q != nullptr) {
            deposit_at_end(P, xq, yq, zq);
        }
    }
    add_counters(P, owned ? (unsigned)k : 0u, n_coll, n_ovf);
}

// RF scalar of Eq. 4 at time step0 + j/2 of an instance: the phase
// frac(phase0 + (n - seg0) dt f) taken in FP64 from the integer step count.
__device__ __forceinline__ float rf_scalar_at(const InstF32 &P, int64_t step0, int j)
{
    float v = 0.0f;
    if (P.v_rf != 0.0 && P.dtf != 0.0) {
        const double x = P.rf_phase0 + ((double)(step0 - P.seg_step0) + 0.5 * j) * P.dtf;
        v = (float)(P.v_rf * cos(2.0 * kPi * (x - floor(x)) + P.phi_rf));
    }
    return v;
}

// ---------------------------------------------------------------------------
// Streamed single step (one micro step per launch, collision-free, no Eq. 7,
// Langevin or RK4; one instance). The kernel is bound by the HBM stream of
// the pack state, 49 bytes per pack-step, and a block that loads its tile's
// state only when it starts the tile leaves the memory system idle while it
// computes. Here the state of the next tiles a block will take is copied to
// shared memory by TMA bulk copies (cp.async.bulk, completion counted on an
// mbarrier per stage) kStreamStages - 1 tiles ahead, so the HBM stream keeps
// flowing while the block computes. The per-pack arithmetic is that of the
// collision-free tile (same device functions), so results are identical.
// ---------------------------------------------------------------------------
constexpr int kStreamStages = 4;
constexpr int kStreamTile = 256; // packs per tile: two per thread, 128 threads
constexpr uint32_t kWaitSpins = 1u << 26;          // backstop on the polls of one wait
constexpr uint64_t kWaitNs = 250ull * 1000 * 1000; // wall-clock bound of one wait (0.25 s)

struct StreamStage {
    int32_t xq[kStreamTile], yq[kStreamTile], zq[kStreamTile];
    float vx[kStreamTile], vy[kStreamTile], vz[kStreamTile];
    uint8_t status[kStreamTile];
};
constexpr uint32_t kStageBytes = 6 * 4 * kStreamTile + kStreamTile;

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// true once the phase of the given parity has completed; false when it has
// not after kWaitNs of wall-clock time (%globaltimer) or kWaitSpins polls: a
// copy that never lands is reported, not waited for
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    const uint32_t a = smem_u32(bar);
    uint64_t t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (uint32_t it = 0; it < kWaitSpins; ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(a), "r"(parity)
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

// bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned)
// from global to shared memory, completion counted on `bar`
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// stage the state of full tile t (kStreamTile packs from pack t * kStreamTile)
__device__ __forceinline__ void stream_prefetch(const InstF32 &P, int64_t t, StreamStage &S, uint64_t *bar)
{
    const int64_t o = t * kStreamTile;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar, kStageBytes);
    bulk_g2s(S.xq, P.xq + o, 4 * kStreamTile, bar);
    bulk_g2s(S.yq, P.yq + o, 4 * kStreamTile, bar);
    bulk_g2s(S.zq, P.zq + o, 4 * kStreamTile, bar);
    bulk_g2s(S.vx, P.vx + o, 4 * kStreamTile, bar);
    bulk_g2s(S.vy, P.vy + o, 4 * kStreamTile, bar);
    bulk_g2s(S.vz, P.vz + o, 4 * kStreamTile, bar);
    bulk_g2s(S.status, P.status + o, kStreamTile, bar);
}

} // namespace

// Work list: tile t of the launch belongs to the instance i with
// tile_start[i] <= t < tile_start[i + 1] (tile = blockDim.x packs). Block b
// takes tiles b, b + gridDim.x, ... (one tile per block when the grid covers
// the list; a persistent grid strides over it). Every thread finds its tile's
// instance itself; the block copies the instance descriptor and its RF
// scalars (rf_table_kernel) into shared memory only when the instance changes.
// Packs per thread of the collision-free kernel (launched with
// threads / kFreeU threads per block over the same tiles).
constexpr int kFreeU = 2;

template <bool kCollide, bool kExtras, int kMinBlocks>
__global__ void __launch_bounds__(kCollide ? 256 : 128, kMinBlocks)
    step_f32_kernel(GridF32 G, const InstF32 *insts,
                                                       const int32_t *tile_start, int n_inst,
                                                       int total_tiles, int nsteps, int esc_cache)
{
    // dynamic shared memory: the RF scalars of the launch, then (esc_cache)
    // the per-lane PIC cell caches of the collision tiles
    extern __shared__ __align__(16) float s_rf[];
    float4 *s_esc = esc_cache ? reinterpret_cast<float4 *>(s_rf + ((2 * nsteps + 1 + 3) & ~3)) : nullptr;
    __shared__ __align__(16) unsigned char p_raw[sizeof(InstF32)];
    const InstF32 &P = *reinterpret_cast<const InstF32 *>(p_raw);
    int cur = -1;
    for (int t = blockIdx.x; t < total_tiles; t += gridDim.x) {
        int lo = 0, hi = n_inst - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(&tile_start[mid]) <= t) lo = mid;
            else hi = mid - 1;
        }
        if (lo != cur) {
            __syncthreads(); // the previous tile's readers are done with P and s_rf
            const uint32_t *src = reinterpret_cast<const uint32_t *>(insts + lo);
            for (int w = threadIdx.x; w < (int)(sizeof(InstF32) / 4); w += blockDim.x)
                reinterpret_cast<uint32_t *>(p_raw)[w] = src[w];
            __syncthreads();
            for (int k = threadIdx.x; k <= 2 * nsteps; k += blockDim.x) s_rf[k] = P.rf[k];
            __syncthreads();
            cur = lo;
        }
        constexpr int kU = kCollide ? 1 : kFreeU;
        const int64_t off = (int64_t)(t - __ldg(&tile_start[lo])) * (kU * blockDim.x);
        if (kCollide)
            run_tile_coll<kExtras, kMinBlocks != 3>(G, P, s_rf, off, nsteps, s_esc, P.step0);
        else
            run_tile_free<kExtras, kU>(G, P, s_rf, off, nsteps);
    }
}

// Collision tiles of one instance whose descriptor is a kernel parameter:
// the tile code reads the instance's constants from the constant bank
// (operands of the arithmetic instructions) instead of loading them from a
// shared-memory copy, 2.6 % more pack-steps/s on the ring stack. Every
// collision launch on grids of at most 64 MB runs this kernel, one launch
// per instance (the launches of a batch run side by side on the context's
// step streams), so an instance gives the same results alone and in any
// batch. Only the step clock, advanced on the device between graph replays,
// is read from the descriptor array.
template <bool kExtras, int kW>
__global__ void __launch_bounds__(256, 4)
    step_f32_one_kernel(const __grid_constant__ GridF32 G, const __grid_constant__ InstF32 P,
                        const InstF32 *inst, int total_tiles, int nsteps, int esc_cache)
{
    extern __shared__ __align__(16) float s_rf[];
    float4 *s_esc = esc_cache ? reinterpret_cast<float4 *>(s_rf + ((2 * nsteps + 1 + 3) & ~3)) : nullptr;
    for (int k = threadIdx.x; k <= 2 * nsteps; k += blockDim.x) s_rf[k] = P.rf[k];
    const int64_t step0 = *reinterpret_cast<const volatile long long *>(&inst->step0);
    __syncthreads();
    for (int t = blockIdx.x; t < total_tiles; t += gridDim.x)
        run_tile_coll<kExtras, true, kW>(G, P, s_rf, (int64_t)t * blockDim.x, nsteps, s_esc, step0);
}

// Streamed single step over the tiles of one instance (see above). Warp 4
// is the producer: its first lane waits until stage k has been read (the
// "empty" barrier of the stage, one arrival per consumer warp) and refills it
// with the state of the block's next full tile (the "full" barrier counts the
// bytes in). Warps 0-3 consume: each waits for the stage of its tile, reads
// its two packs per thread, releases the stage and computes, so no warp waits
// for another. A partial last tile is read directly. The instance descriptor
// is a kernel parameter (constant bank); only the step clock, advanced on the
// device between graph replays, is read from the descriptor array. A wait
// that gives up raises counters[3]; the producer then waits (bounded) for its
// copies in flight before the block ends.
constexpr int kStreamConsumers = 128;

__global__ void __launch_bounds__(kStreamConsumers + 32, 6)
    step_f32_stream_kernel(const __grid_constant__ GridF32 G, const __grid_constant__ InstF32 P, InstF32 *insts,
                           int total_tiles, unsigned *ticket)
{
    __shared__ __align__(128) StreamStage stage[kStreamStages];
    __shared__ __align__(8) uint64_t full_bar[kStreamStages];
    __shared__ __align__(8) uint64_t empty_bar[kStreamStages];
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int k = 0; k < kStreamStages; ++k) {
            mbar_init(&full_bar[k], 1);
            mbar_init(&empty_bar[k], kStreamConsumers / 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int64_t n_full = P.n_slots / kStreamTile; // tiles [0, n_full) are full
    if (tid >= kStreamConsumers) {
        // producer warp
        if (tid != kStreamConsumers) return;
        int issued[kStreamStages] = {};
        bool failed = false;
        for (int i = 0;; ++i) {
            const int64_t t = blockIdx.x + (int64_t)i * gridDim.x;
            if (t >= n_full) break;
            const int sg = i % kStreamStages;
            if (i >= kStreamStages && !mbar_wait(&empty_bar[sg], (uint32_t)(i / kStreamStages - 1) & 1u)) {
                failed = true;
                break;
            }
            if (i == P.hold_tile) continue; // test hook: this tile's copies are withheld
            stream_prefetch(P, t, stage[sg], &full_bar[sg]);
            ++issued[sg];
        }
        // the copies of this block land before its shared memory is released
        for (int k = 0; k < kStreamStages; ++k)
            if (issued[k] > 0 && !mbar_wait(&full_bar[k], (uint32_t)(issued[k] - 1) & 1u)) failed = true;
        if (failed) atomicAdd(&P.counters[3], 1ull);
        return;
    }
    const int lane = tid & 31;
    const uint32_t hk = pack_key(0u, P);
    // the step clock (advanced on the device between graph replays) and the
    // step's RF scalar, formed by one lane per warp (FP64) and broadcast
    const int64_t step0 = *(volatile const int64_t *)&insts[0].step0;
    const uint32_t n = (uint32_t)step0;
    float srf = 0.0f;
    if (lane == 0) srf = rf_scalar_at(P, step0, 0);
    srf = __shfl_sync(0xffffffffu, srf, 0);
    unsigned n_steps_done = 0;
    bool failed = false;
    for (int i = 0;; ++i) {
        const int64_t t = blockIdx.x + (int64_t)i * gridDim.x;
        if (t >= total_tiles) break;
        const int sg = i % kStreamStages;
        int32_t xq[2], yq[2], zq[2];
        float vx[2], vy[2], vz[2];
        bool own[2];
        if (t < n_full) {
            if (!mbar_wait(&full_bar[sg], (uint32_t)(i / kStreamStages) & 1u)) {
                failed = true;
                break;
            }
            const StreamStage &S = stage[sg];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int j = tid + u * kStreamConsumers;
                own[u] = S.status[j] == MUCITE_ACTIVE;
                xq[u] = S.xq[j]; yq[u] = S.yq[j]; zq[u] = S.zq[j];
                vx[u] = S.vx[j]; vy[u] = S.vy[j]; vz[u] = S.vz[j];
            }
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty_bar[sg]))
                                        : "memory");
        } else {
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int64_t p = t * kStreamTile + tid + u * kStreamConsumers;
                const int64_t q = p < P.n_slots ? p : 0;
                own[u] = p < P.n_slots && P.status[q] == MUCITE_ACTIVE;
                xq[u] = P.xq[q]; yq[u] = P.yq[q]; zq[u] = P.zq[q];
                vx[u] = P.vx[q]; vy[u] = P.vy[q]; vz[u] = P.vz[q];
            }
        }
        const int64_t base = t * kStreamTile;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int j = tid + u * kStreamConsumers;
            const float fx = (float)xq[u], fy = (float)yq[u];
            Local L;
            gather(G, P, fx, fy, lattice_r(fx, fy), zq[u], L);
            float kx, ky, kz;
            kick_of(P, L, srf, kx, ky, kz);
            const uint32_t h1 = dither_word((uint32_t)(base + j) ^ hk, n), h2 = remix32(h1);
            float gx, gy, gr;
            const int s2 = push<false>(G, P, &srf, 0, h1, h2, kx, ky, kz, xq[u], yq[u], zq[u], vx[u], vy[u],
                                       vz[u], gx, gy, gr);
            if (own[u]) {
                n_steps_done += 1u;
                P.xq[base + j] = xq[u]; P.yq[base + j] = yq[u]; P.zq[base + j] = zq[u];
                P.vx[base + j] = vx[u]; P.vy[base + j] = vy[u]; P.vz[base + j] = vz[u];
                if (s2 != MUCITE_ACTIVE) {
                    P.status[base + j] = (uint8_t)s2;
                    P.t_term[base + j] = (int32_t)(step0 + 1);
                } else if (P.dep_q != nullptr) {
                    deposit_at_end(P, xq[u], yq[u], zq[u]);
                }
            }
        }
    }
    if (failed && lane == 0) atomicAdd(&P.counters[3], 1ull);
    // the counters of the warps that left their loop early are still added
    add_counters(P, n_steps_done, 0u, 0u);
    // the last block to arrive advances the instance clock by the step (every
    // block has read it at its start) and re-arms the ticket
    asm volatile("bar.sync 1, %0;" ::"n"(kStreamConsumers) : "memory");
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(ticket, 1u) == gridDim.x - 1) {
            insts[0].step0 = step0 + 1;
            *ticket = 0u;
            __threadfence();
        }
    }
}

// RF scalars of Eq. 4 for the next `nsteps` steps of every instance at
// half-step spacing (entry j is time step0 + j/2): the phase
// frac(phase0 + (n - seg0) dt f) is taken in FP64 from the integer step count.
__global__ void rf_table_kernel(const InstF32 *insts, int nsteps)
{
    const InstF32 &P = insts[blockIdx.x];
    for (int j = threadIdx.x; j <= 2 * nsteps; j += blockDim.x) P.rf[j] = rf_scalar_at(P, P.step0, j);
}

// Instance clocks advanced on the device (graph replays).
__global__ void advance_clock_kernel(InstF32 *insts, int n_inst, int nsteps)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_inst) insts[i].step0 += nsteps;
}

// Register budget of the collision kernel: 64 per thread (4 blocks of 256
// per SM) while the static node table stays in L2, 80 (3 blocks) when it is
// larger (the paper-sized grid): its gathers then wait on HBM, and the wider
// budget keeps all eight node loads of a gather in flight (5 % faster there,
// 5.6 % slower in the 10-step launches of a 1e6-pack run with an L2-resident
// table).
static bool wide_gather(const GridF32 &G)
{
    return (size_t)G.nr * (size_t)G.nz * sizeof(NodeF) > ((size_t)64 << 20);
}

// kCollide: the collision code is compiled in; kExtras: dissociation (Eq. 7)
// and the hybrid Langevin branch are compiled in.
// Dynamic shared memory of a step launch: the 2 nsteps + 1 RF scalars
// (padded to 16 bytes), then with esc_cache two float4 per thread.
static size_t step_f32_smem(int threads, int nsteps, bool esc_cache)
{
    const size_t rf = sizeof(float) * (size_t)((2 * nsteps + 1 + 3) & ~3);
    return rf + (esc_cache ? 2 * sizeof(float4) * (size_t)threads : 0);
}

void launch_step_f32(const GridF32 &G, InstF32 *d_insts, const int32_t *d_tile_start, int n_inst,
                     int total_tiles, int threads, int nsteps, int grid, bool collide, bool extras,
                     bool esc_cache, cudaStream_t s)
{
    rf_table_kernel<<<n_inst, 128, 0, s>>>(d_insts, nsteps);
    const int ec = esc_cache && collide ? 1 : 0;
    const size_t smem = step_f32_smem(threads, nsteps, ec != 0);
    const bool wide = wide_gather(G);
    if (collide && extras && wide)
        step_f32_kernel<true, true, 3><<<grid, threads, smem, s>>>(G, d_insts, d_tile_start, n_inst, total_tiles,
                                                                   nsteps, ec);
    else if (collide && extras)
        step_f32_kernel<true, true, 4><<<grid, threads, smem, s>>>(G, d_insts, d_tile_start, n_inst, total_tiles,
                                                                   nsteps, ec);
    else if (collide && wide)
        step_f32_kernel<true, false, 3><<<grid, threads, smem, s>>>(G, d_insts, d_tile_start, n_inst, total_tiles,
                                                                    nsteps, ec);
    else if (collide)
        step_f32_kernel<true, false, 4><<<grid, threads, smem, s>>>(G, d_insts, d_tile_start, n_inst, total_tiles,
                                                                    nsteps, ec);
    else if (extras)
        step_f32_kernel<false, true, 6><<<grid, threads / kFreeU, smem, s>>>(G, d_insts, d_tile_start, n_inst,
                                                                              total_tiles, nsteps, ec);
    else
        step_f32_kernel<false, false, 6><<<grid, threads / kFreeU, smem, s>>>(G, d_insts, d_tile_start, n_inst,
                                                                               total_tiles, nsteps, ec);
}

bool step_f32_large_grid(const GridF32 &G)
{
    return wide_gather(G);
}

void launch_rf_table(InstF32 *d_insts, int n_inst, int nsteps, cudaStream_t s)
{
    rf_table_kernel<<<n_inst, 128, 0, s>>>(d_insts, nsteps);
}

void launch_step_f32_one(const GridF32 &G, const InstF32 &h_inst, const InstF32 *d_inst, int total_tiles,
                         int threads, int nsteps, int grid, bool extras, bool esc_cache, int cand_weight,
                         cudaStream_t s)
{
    if (total_tiles <= 0) return;
    const size_t smem = step_f32_smem(threads, nsteps, esc_cache);
    const int ec = esc_cache ? 1 : 0;
    const bool eager = cand_weight == kEagerWeight;
    if (extras && eager)
        step_f32_one_kernel<true, kEagerWeight><<<grid, threads, smem, s>>>(G, h_inst, d_inst, total_tiles, nsteps, ec);
    else if (extras)
        step_f32_one_kernel<true, 1><<<grid, threads, smem, s>>>(G, h_inst, d_inst, total_tiles, nsteps, ec);
    else if (eager)
        step_f32_one_kernel<false, kEagerWeight><<<grid, threads, smem, s>>>(G, h_inst, d_inst, total_tiles, nsteps,
                                                                           ec);
    else
        step_f32_one_kernel<false, 1><<<grid, threads, smem, s>>>(G, h_inst, d_inst, total_tiles, nsteps, ec);
}

void launch_step_f32_stream(const GridF32 &G, const InstF32 &P, InstF32 *d_insts, int total_tiles, int grid,
                            unsigned *ticket, cudaStream_t s)
{
    step_f32_stream_kernel<<<grid, kStreamConsumers + 32, 0, s>>>(G, P, d_insts, total_tiles, ticket);
}

int step_f32_stream_blocks_per_sm()
{
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, step_f32_stream_kernel, kStreamConsumers + 32, 0);
    return b;
}

void launch_advance_clock(InstF32 *d_insts, int n_inst, int nsteps, cudaStream_t s)
{
    advance_clock_kernel<<<(n_inst + 127) / 128, 128, 0, s>>>(d_insts, n_inst, nsteps);
}

int step_f32_blocks_per_sm(const GridF32 &G, int threads, int nsteps, bool collide, bool extras, bool esc_cache)
{
    int b = 0;
    const size_t smem = step_f32_smem(threads, nsteps, esc_cache && collide);
    const bool wide = wide_gather(G);
    if (collide && extras)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &b, wide ? step_f32_kernel<true, true, 3> : step_f32_kernel<true, true, 4>, threads, smem);
    else if (collide)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &b, wide ? step_f32_kernel<true, false, 3> : step_f32_kernel<true, false, 4>, threads, smem);
    else if (extras)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, step_f32_kernel<false, true, 6>, threads / kFreeU, smem);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, step_f32_kernel<false, false, 6>, threads / kFreeU,
                                                      smem);
    return b;
}

} // namespace mucite

namespace mucite {

namespace {

__device__ __forceinline__ int32_t q32l(double v)
{
    const double r = rint(v);
    if (r < -2147483648.0) return INT32_MIN;
    if (r > 2147483647.0) return INT32_MAX;
    return (int32_t)r;
}

} // namespace

// Per-pack quantities of the Eq. 1 limits, reduced over the active packs:
// largest expected collision rate, largest speed, smallest
// 0.1 max(|v|, v_th) / |a| (positive floats ordered as unsigned integers).
__global__ void __launch_bounds__(256) dt_limits_kernel(GridF32 G, InstF32 P, LimitArgs A)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float lam = 0.0f, vmax = 0.0f, acc = __int_as_float(0x7f800000);
    if (p < A.n && A.status[p] == MUCITE_ACTIVE) {
        int32_t xq, yq, zq;
        float vx, vy, vz;
        if (A.precision == MUCITE_FP32) {
            xq = ((const int32_t *)A.x)[p];
            yq = ((const int32_t *)A.y)[p];
            zq = ((const int32_t *)A.z)[p];
            vx = ((const float *)A.vx)[p];
            vy = ((const float *)A.vy)[p];
            vz = ((const float *)A.vz)[p];
        } else {
            xq = q32l(((const double *)A.x)[p] * A.sx_inv);
            yq = q32l(((const double *)A.y)[p] * A.sx_inv);
            zq = q32l((((const double *)A.z)[p] - A.gz0) * A.sz_inv);
            vx = (float)((const double *)A.vx)[p];
            vy = (float)((const double *)A.vy)[p];
            vz = (float)((const double *)A.vz)[p];
        }
        const float fx = (float)xq, fy = (float)yq;
        Local L;
        gather(G, P, fx, fy, lattice_r(fx, fy), zq, L);
        if (L.nsig > 0.0f && L.T > 0.0f) lam = collision_rate(P, L, vx, vy, vz);
        vmax = sqrtf(vx * vx + vy * vy + vz * vz);
        const float srf = (float)A.srf;
        float ax, ay, az;
        field_kick(L, A.kick_m, P.dc_scale, srf, ax, ay, az);
        const float am = sqrtf(ax * ax + ay * ay + az * az);
        const float vth = L.T > 0.0f ? sqrtf(A.kT_over_M_coef * L.T) : 0.0f;
        if (am > 0.0f) acc = 0.1f * fmaxf(vmax, vth) / am;
    }
    unsigned ul = __float_as_uint(lam), uv = __float_as_uint(vmax), ua = __float_as_uint(acc);
    for (int o = 16; o > 0; o >>= 1) {
        ul = max(ul, __shfl_down_sync(0xffffffffu, ul, o));
        uv = max(uv, __shfl_down_sync(0xffffffffu, uv, o));
        ua = min(ua, __shfl_down_sync(0xffffffffu, ua, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&A.out[0], ul);
        atomicMax(&A.out[1], uv);
        atomicMin(&A.out[2], ua);
    }
}

void launch_dt_limits(const GridF32 &G, const InstF32 &P, const LimitArgs &A, cudaStream_t s)
{
    if (A.n <= 0) return;
    dt_limits_kernel<<<(unsigned)((A.n + 255) / 256), 256, 0, s>>>(G, P, A);
}

} // namespace mucite
