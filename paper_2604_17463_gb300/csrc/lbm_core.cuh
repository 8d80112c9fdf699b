// lbm_core.cuh -- population storage forms and the BGK + Guo collision of
// one cell, shared by the stream-collide kernels of libiblb.
//
// Deviation form of Eq. 1-6 (g_i = f_i - w_i, drho = sum g_i, rho = 1 + drho):
//   u      = (sum c_i g_i + F/2) / rho
//   g_i^eq = w_i (drho + rho (3 c.u + 9/2 (c.u)^2 - 3/2 u.u))
//   g*_i   = g_i + omega (g_i^eq - g_i)
//            + (1 - omega/2) w_i (3 (c_i - u).F + 9 (c_i.u)(c_i.F))
#pragma once

#include "common.cuh"

namespace iblb {

template <int ST> struct StorageT;

template <> struct StorageT<ST_FP64> {
    using S = double;
    using R = double;
    __device__ __forceinline__ static R load(const S* p, long long i, float) { return p[i]; }
    __device__ __forceinline__ static void store(S* p, long long i, R v, float) { p[i] = v; }
    __device__ __forceinline__ static void store_cs(S* p, long long i, R v, float) { __stcs(p + i, v); }
};

template <> struct StorageT<ST_FP32> {
    using S = float;
    using R = float;
    __device__ __forceinline__ static R load(const S* p, long long i, float) { return p[i]; }
    __device__ __forceinline__ static void store(S* p, long long i, R v, float) { p[i] = v; }
    __device__ __forceinline__ static void store_cs(S* p, long long i, R v, float) { __stcs(p + i, v); }
};

template <> struct StorageT<ST_FP16> {
    using S = __half;
    using R = float;
    __device__ __forceinline__ static R load(const S* p, long long i, float inv_scale) {
        return __half2float(p[i]) * inv_scale;
    }
    __device__ __forceinline__ static void store(S* p, long long i, R v, float scale) {
        p[i] = __float2half_rn(v * scale);
    }
    __device__ __forceinline__ static void store_cs(S* p, long long i, R v, float scale) {
        __stcs(reinterpret_cast<unsigned short*>(p) + i, __half_as_ushort(__float2half_rn(v * scale)));
    }
};

// ---------------------------------------------------------------------------
// Stochastic rounding of the binary16 population stores.  Round-to-nearest
// gives every stored population a deterministic error; in a slowly evolving
// flow the same errors recur step after step and act like a small constant
// forcing, which the slow hydrodynamic modes integrate over their long
// relaxation times (the spreading drop then moves measurably slower than in
// FP64).  Rounding up or down at random, with the probability that makes the
// expected stored value exact, turns that error into zero-mean noise that is
// independent between steps.  The conversion is the sm_100-family
// cvt.rs.f16x2.f32 instruction; its random bits come from a counter-based
// hash of (time step, cell, population pair), so runs are deterministic.
//
// mix32 is the 32-bit integer hash "lowbias32" published by C. Wellons
// (xor-shift / multiply rounds with constants 0x7feb352d, 0x846ca68b).
__device__ __forceinline__ unsigned mix32(unsigned x)
{
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

// Per-cell seed for time step `step`.
__device__ __forceinline__ unsigned sr_seed(unsigned step, long long cell)
{
    return mix32((unsigned)cell ^ mix32(step + 0x9e3779b9U));
}

// Random bits for population pair k of a cell (uniform whenever the seed is).
__device__ __forceinline__ unsigned sr_bits(unsigned seed, int k)
{
    return (seed ^ ((unsigned)k * 0x9e3779b9U)) * 0x85ebca6bU;
}

// hi -> bits 31:16, lo -> bits 15:0, stochastically rounded.
__device__ __forceinline__ unsigned cvt_rs_f16x2(float hi, float lo, unsigned rbits)
{
    unsigned d;
    asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rbits));
    return d;
}

// Store all Q populations of one cell (deviation form): binary16 with
// stochastic rounding, population pairs (2k, 2k+1) sharing one conversion;
// FP32 / FP64 as they are.  CS: streaming (evict-first) stores.
template <int Q, int ST, bool CS>
__device__ __forceinline__ void store_cell(typename StorageT<ST>::S* __restrict__ fout,
                                           long long nc, long long cell,
                                           const typename StorageT<ST>::R* g, float scale,
                                           unsigned seed)
{
    using T = StorageT<ST>;
    if constexpr (ST == ST_FP16) {
        unsigned short* o = reinterpret_cast<unsigned short*>(fout);
#pragma unroll
        for (int i = 0; i < Q; i += 2) {
            const float lo = (i + 1 < Q) ? g[i + 1] * scale : 0.0f;
            const unsigned h = cvt_rs_f16x2(g[i] * scale, lo, sr_bits(seed, i >> 1));
            if (CS) {
                __stcs(o + (long long)i * nc + cell, (unsigned short)(h >> 16));
                if (i + 1 < Q) __stcs(o + (long long)(i + 1) * nc + cell, (unsigned short)(h & 0xffffu));
            } else {
                o[(long long)i * nc + cell] = (unsigned short)(h >> 16);
                if (i + 1 < Q) o[(long long)(i + 1) * nc + cell] = (unsigned short)(h & 0xffffu);
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < Q; i++) {
            if (CS)
                T::store_cs(fout, (long long)i * nc + cell, g[i], scale);
            else
                T::store(fout, (long long)i * nc + cell, g[i], scale);
        }
    }
}

// As store_cell, with the cell index in 32 bits on per-plane base pointers
// (the lattice holds fewer than 2^32 cells).
template <int Q, int ST, bool CS>
__device__ __forceinline__ void store_cell32(typename StorageT<ST>::S* __restrict__ fout,
                                             long long nc, unsigned cell,
                                             const typename StorageT<ST>::R* g, float scale,
                                             unsigned seed)
{
    using T = StorageT<ST>;
    if constexpr (ST == ST_FP16) {
        unsigned short* o = reinterpret_cast<unsigned short*>(fout);
#pragma unroll
        for (int i = 0; i < Q; i += 2) {
            const float lo = (i + 1 < Q) ? g[i + 1] * scale : 0.0f;
            const unsigned h = cvt_rs_f16x2(g[i] * scale, lo, sr_bits(seed, i >> 1));
            unsigned short* p0 = o + (size_t)i * nc;
            if (CS) {
                __stcs(p0 + cell, (unsigned short)(h >> 16));
                if (i + 1 < Q) __stcs(p0 + nc + cell, (unsigned short)(h & 0xffffu));
            } else {
                p0[cell] = (unsigned short)(h >> 16);
                if (i + 1 < Q) p0[nc + cell] = (unsigned short)(h & 0xffffu);
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < Q; i++) {
            typename T::S* pl = fout + (size_t)i * nc;
            if (CS)
                T::store_cs(pl, cell, g[i], scale);
            else
                T::store(pl, cell, g[i], scale);
        }
    }
}

// As store_cell, with one 32-bit index i * nc + cell into the buffer (the
// buffer holds fewer than 2^32 elements).
template <int Q, int ST>
__device__ __forceinline__ void store_cell_flat(typename StorageT<ST>::S* __restrict__ fout,
                                                unsigned nc, unsigned cell,
                                                const typename StorageT<ST>::R* g, unsigned seed)
{
    using T = StorageT<ST>;
    if constexpr (ST == ST_FP16) {
        unsigned short* o = reinterpret_cast<unsigned short*>(fout);
#pragma unroll
        for (int i = 0; i < Q; i += 2) {
            const float lo = (i + 1 < Q) ? g[i + 1] : 0.0f;
            const unsigned h = cvt_rs_f16x2(g[i], lo, sr_bits(seed, i >> 1));
            o[(unsigned)i * nc + cell] = (unsigned short)(h >> 16);
            if (i + 1 < Q) o[(unsigned)(i + 1) * nc + cell] = (unsigned short)(h & 0xffffu);
        }
    } else {
#pragma unroll
        for (int i = 0; i < Q; i++) T::store(fout, (unsigned)i * nc + cell, g[i], 1.0f);
    }
}

// Time-step number for the rounding hash: read from the current slot of a
// two-entry device counter; one thread of the launch writes the next value
// into the other slot (read and written entries never coincide in a launch).
__device__ __forceinline__ unsigned sr_step(const unsigned* in, unsigned* out, bool writer)
{
    const unsigned s = in ? __ldg(in) : 0u;
    if (writer && out) *out = s + 1u;
    return s;
}

// ---------------------------------------------------------------------------
// FP32 lattice constants with exact conservation identities.  Rounded to
// FP32, the weights sum to 1 + 7e-9 and 3 sum w c_x^2 comes to 1 + 7e-9, so
// every FP32 collision creates a little mass (in proportion to drho) and
// multiplies the equilibrium momentum by 1 + 7e-9 omega.  The second acts as
// a negative friction on every flow; over 10^5 steps it made a spreading drop
// run ~0.2 % ahead of the FP64 run at tau = 0.6.  The collision therefore
// uses two sets of binary fractions close to the weights:
//   wb_i (zeroth-order terms): sum_i wb_i = 1 exactly,
//   wa_i ~ 3 w_i (first-order terms, c.u and c.F): sum_i wa_i c_ix^2 = 1 exactly,
// chosen as short binary fractions so that these sums hold for the FP32
// values themselves (their distance to w_i, 3 w_i is below 4e-8; it enters
// only the second-order moments, i.e. the viscosity at the 1e-7 level).
// FP64 arithmetic uses w_i and 3 w_i.
template <int Q> struct ExactF32;
template <> struct ExactF32<9> {
    static constexpr float b0 = 0x1.c71c74p-2f, b1 = 0x1.c71c70p-4f, b2 = 0x1.c71c70p-6f;
    static constexpr float a1 = 0x1.555556p-2f, a2 = 0x1.555554p-4f;
};
template <> struct ExactF32<19> {
    static constexpr float b0 = 0x1.555558p-2f, b1 = 0x1.c71c70p-5f, b2 = 0x1.c71c70p-6f;
    static constexpr float a1 = 0x1.555558p-3f, a2 = 0x1.555554p-4f;
};

// |c_i|^2: 0 rest, 1 axis, 2 diagonal
template <int Q>
__host__ __device__ constexpr int speed2(int i)
{
    using L = Stencil<Q>;
    return L::cx(i) * L::cx(i) + L::cy(i) * L::cy(i) + L::cz(i) * L::cz(i);
}

template <int Q, typename R>
__host__ __device__ constexpr R coef_b(int i)
{
    if constexpr (sizeof(R) == 4) {
        using E = ExactF32<Q>;
        return speed2<Q>(i) == 0 ? E::b0 : (speed2<Q>(i) == 1 ? E::b1 : E::b2);
    } else {
        return (R)Stencil<Q>::w(i);
    }
}

template <int Q, typename R>
__host__ __device__ constexpr R coef_a(int i)
{
    if constexpr (sizeof(R) == 4) {
        using E = ExactF32<Q>;
        return speed2<Q>(i) == 0 ? 0.0f : (speed2<Q>(i) == 1 ? E::a1 : E::a2);
    } else {
        return (R)(3.0 * Stencil<Q>::w(i));
    }
}

// Relaxation rate and body force in the compute precision.
template <typename R>
__device__ __forceinline__ R param_omega(const StreamParams& p);
template <>
__device__ __forceinline__ double param_omega<double>(const StreamParams& p) { return p.omega; }
template <>
__device__ __forceinline__ float param_omega<float>(const StreamParams& p) { return p.omega_f; }
template <typename R>
__device__ __forceinline__ R param_body(const StreamParams& p, int k);
template <>
__device__ __forceinline__ double param_body<double>(const StreamParams& p, int k) { return p.body[k]; }
template <>
__device__ __forceinline__ float param_body<float>(const StreamParams& p, int k) { return p.body_f[k]; }

// Moments of the deviations and the velocity with the half-force term.
template <int Q, typename R>
struct CellMoments {
    R drho, rho, ux, uy, uz;
};

template <int Q, typename R>
__device__ __forceinline__ CellMoments<Q, R> cell_moments(const R* g, R Fx, R Fy, R Fz,
                                                          R ginv = R(1))
{
    using L = Stencil<Q>;
    constexpr int D = L::D;
    R drho = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        drho += g[i];
        if (L::cx(i) > 0) jx += g[i];
        if (L::cx(i) < 0) jx -= g[i];
        if (L::cy(i) > 0) jy += g[i];
        if (L::cy(i) < 0) jy -= g[i];
        if (D == 3) {
            if (L::cz(i) > 0) jz += g[i];
            if (L::cz(i) < 0) jz -= g[i];
        }
    }
    // g may be held scaled by a power of two (binary16 storage): ginv undoes it
    drho *= ginv;
    jx *= ginv;
    jy *= ginv;
    jz *= ginv;
    CellMoments<Q, R> m;
    m.drho = drho;
    m.rho = R(1) + drho;
    const R inv_rho = R(1) / m.rho;
    m.ux = (jx + R(0.5) * Fx) * inv_rho;
    m.uy = (jy + R(0.5) * Fy) * inv_rho;
    m.uz = (D == 3) ? (jz + R(0.5) * Fz) * inv_rho : R(0);
    return m;
}

// BGK relaxation with the Guo source; g is overwritten with g*.
// Written per pair of opposite directions (i, opp(i)): c.u and c.F change
// sign between the two, so omega g^eq + S splits into a part common to both
// and a part of opposite sign:
//   sym  = w [omega (drho - rho 3/2 u.u + 9/2 rho (c.u)^2) - 3 pref u.F + 9 pref (c.u)(c.F)]
//   asym = 3 w [omega rho (c.u) + pref (c.F)]
//   g*_i = (1 - omega) g_i + sym + asym,   g*_opp = (1 - omega) g_opp + sym - asym
// with pref = 1 - omega/2; the rest direction has c = 0.  w and 3 w are
// coef_b and coef_a (exact mass and momentum identities in FP32).
template <int Q, typename R>
__device__ __forceinline__ void cell_collide(R* g, const CellMoments<Q, R>& m, R omega, R Fx, R Fy,
                                             R Fz, R gscale = R(1))
{
    using L = Stencil<Q>;
    constexpr int D = L::D;
    const R pref = R(1) - R(0.5) * omega;
    const R om1 = R(1) - omega;
    const R uF = m.ux * Fx + m.uy * Fy + m.uz * Fz;
    const R base = omega * (m.drho - m.rho * (R(1.5) * (m.ux * m.ux + m.uy * m.uy + m.uz * m.uz)));
    const R sym0 = base - R(3) * pref * uF;     // common part without the (c.u) terms
    const R k2 = omega * R(4.5) * m.rho;        // coefficient of (c.u)^2
    const R k1 = omega * m.rho;                 // coefficient of (c.u), over 3
    const R p9 = R(9) * pref;
    // g held scaled by gscale (a power of two): the new terms take the same scale
    g[0] = om1 * g[0] + (coef_b<Q, R>(0) * gscale) * sym0;
#pragma unroll
    for (int i = 1; i < Q; i++) {
        if (L::opp(i) < i) continue;  // each pair once
        const int o = L::opp(i);
        const R w = coef_b<Q, R>(i) * gscale;
        const R w3 = coef_a<Q, R>(i) * gscale;
        const R cu = (R)L::cx(i) * m.ux + (R)L::cy(i) * m.uy + (D == 3 ? (R)L::cz(i) * m.uz : R(0));
        const R cF = (R)L::cx(i) * Fx + (R)L::cy(i) * Fy + (D == 3 ? (R)L::cz(i) * Fz : R(0));
        const R sym = w * (sym0 + cu * (k2 * cu + p9 * cF));
        const R asym = w3 * (k1 * cu + pref * cF);
        const R gi = g[i], go = g[o];
        g[i] = om1 * gi + sym + asym;
        g[o] = om1 * go + sym - asym;
    }
}

// Band force of a cell: added to (Fx, Fy, Fz) and cleared in the buffer
// (float4 per cell in FP32, [component][cell] in FP64).
template <int D, typename R>
__device__ __forceinline__ void take_band_force(R* __restrict__ F, long long nc, long long cell,
                                                R& Fx, R& Fy, R& Fz)
{
    if constexpr (sizeof(R) == 4) {
        float4* F4 = reinterpret_cast<float4*>(F);
        const float4 f = F4[cell];
        Fx += f.x;
        Fy += f.y;
        if (D == 3) Fz += f.z;
        F4[cell] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
        Fx += F[cell];
        Fy += F[nc + cell];
        F[cell] = 0;
        F[nc + cell] = 0;
        if (D == 3) {
            Fz += F[2 * nc + cell];
            F[2 * nc + cell] = 0;
        }
    }
}

// Moments of a cell (drho, u) into the moment buffer.
template <int D, typename R>
__device__ __forceinline__ void put_moments(R* __restrict__ mom, long long nc, long long cell,
                                            R drho, R ux, R uy, R uz)
{
    if constexpr (sizeof(R) == 4) {
        reinterpret_cast<float4*>(mom)[cell] = make_float4(drho, ux, uy, D == 3 ? uz : 0.f);
    } else {
        mom[cell] = drho;
        mom[nc + cell] = ux;
        mom[2 * nc + cell] = uy;
        if (D == 3) mom[3 * nc + cell] = uz;
    }
}

// ------------------------------------------------------------------ packed pairs
// Two cells at once in packed FP32x2 arithmetic (Blackwell FFMA2 / FADD2 /
// FMUL2): the same moments and pair-symmetric collision as above, with the
// fused multiply-adds written out.
__device__ __forceinline__ float2 p2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, p2(-1.0f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

struct CellMoments2 {
    float2 drho, rho, ux, uy, uz;
};

template <int Q>
__device__ __forceinline__ CellMoments2 cell_moments2(const float2* g, float2 Fx, float2 Fy,
                                                      float2 Fz, float ginv = 1.0f)
{
    using L = Stencil<Q>;
    constexpr int D = L::D;
    float2 drho = g[0], jx = p2(0.f), jy = p2(0.f), jz = p2(0.f);
#pragma unroll
    for (int i = 1; i < Q; i++) {
        drho = add2(drho, g[i]);
        if (L::cx(i) > 0) jx = add2(jx, g[i]);
        if (L::cx(i) < 0) jx = sub2(jx, g[i]);
        if (L::cy(i) > 0) jy = add2(jy, g[i]);
        if (L::cy(i) < 0) jy = sub2(jy, g[i]);
        if (D == 3) {
            if (L::cz(i) > 0) jz = add2(jz, g[i]);
            if (L::cz(i) < 0) jz = sub2(jz, g[i]);
        }
    }
    if (ginv != 1.0f) {  // g held scaled by a power of two (binary16 storage)
        drho = mul2(drho, p2(ginv));
        jx = mul2(jx, p2(ginv));
        jy = mul2(jy, p2(ginv));
        jz = mul2(jz, p2(ginv));
    }
    CellMoments2 m;
    m.drho = drho;
    m.rho = add2(p2(1.f), drho);
    const float2 inv_rho = make_float2(1.0f / m.rho.x, 1.0f / m.rho.y);
    m.ux = mul2(fma2(p2(0.5f), Fx, jx), inv_rho);
    m.uy = mul2(fma2(p2(0.5f), Fy, jy), inv_rho);
    m.uz = (D == 3) ? mul2(fma2(p2(0.5f), Fz, jz), inv_rho) : p2(0.f);
    return m;
}

template <int Q>
__device__ __forceinline__ void cell_collide2(float2* g, const CellMoments2& m, float omega,
                                              float2 Fx, float2 Fy, float2 Fz,
                                              float gscale = 1.0f)
{
    using L = Stencil<Q>;
    constexpr int D = L::D;
    const float pref = 1.0f - 0.5f * omega;
    const float2 om1 = p2(1.0f - omega);
    const float2 uF = fma2(m.uz, Fz, fma2(m.uy, Fy, mul2(m.ux, Fx)));
    const float2 usq = fma2(m.uz, m.uz, fma2(m.uy, m.uy, mul2(m.ux, m.ux)));
    const float2 base = mul2(p2(omega), fma2(mul2(p2(-1.5f), m.rho), usq, m.drho));
    const float2 sym0 = fma2(p2(-3.0f * pref), uF, base);
    const float2 k2 = mul2(p2(omega * 4.5f), m.rho);
    const float2 k1 = mul2(p2(omega), m.rho);
    const float2 p1 = p2(pref), p9 = p2(9.0f * pref);
    // g held scaled by gscale (a power of two): the new terms take the same scale
    g[0] = fma2(om1, g[0], mul2(p2(coef_b<Q, float>(0) * gscale), sym0));
#pragma unroll
    for (int i = 1; i < Q; i++) {
        if (L::opp(i) < i) continue;
        const int o = L::opp(i);
        const float2 w = p2(coef_b<Q, float>(i) * gscale);
        const float2 w3 = p2(coef_a<Q, float>(i) * gscale);
        float2 cu = p2(0.f), cF = p2(0.f);
        if (L::cx(i) > 0) { cu = add2(cu, m.ux); cF = add2(cF, Fx); }
        if (L::cx(i) < 0) { cu = sub2(cu, m.ux); cF = sub2(cF, Fx); }
        if (L::cy(i) > 0) { cu = add2(cu, m.uy); cF = add2(cF, Fy); }
        if (L::cy(i) < 0) { cu = sub2(cu, m.uy); cF = sub2(cF, Fy); }
        if (D == 3) {
            if (L::cz(i) > 0) { cu = add2(cu, m.uz); cF = add2(cF, Fz); }
            if (L::cz(i) < 0) { cu = sub2(cu, m.uz); cF = sub2(cF, Fz); }
        }
        const float2 t = fma2(k2, cu, mul2(p9, cF));
        const float2 sym = mul2(w, fma2(cu, t, sym0));
        const float2 asym = mul2(w3, fma2(k1, cu, mul2(p1, cF)));
        const float2 gi = g[i], go = g[o];
        g[i] = fma2(om1, gi, add2(sym, asym));
        g[o] = fma2(om1, go, sub2(sym, asym));
    }
}

// Pull streaming of one fluid cell (x, y, z) with halfway bounce-back at the
// solid first/last layer of the wall axis (y in 2D, z in 3D) when walls != 0
// and periodic wrap elsewhere: g_i = g*_i(x - c_i), or g*_opp(i)(x) when
// x - c_i is solid.
template <int Q, int ST>
__device__ __forceinline__ void pull_cell(const typename StorageT<ST>::S* __restrict__ fin,
                                          const GridParams& g, int x, int y, int z,
                                          long long cell, float inv_scale,
                                          typename StorageT<ST>::R* out)
{
    using L = Stencil<Q>;
    constexpr int D = L::D;
    const int nx = g.nx, ny = g.ny;
    const long long nc = g.ncell;
    const int xm = (x == 0) ? nx - 1 : x - 1;
    const int xp = (x == nx - 1) ? 0 : x + 1;
    const int Lw = (D == 2) ? ny : g.nz;
    const int a = (D == 2) ? y : z;
    int am = a - 1, ap = a + 1;
    bool solid_m = false, solid_p = false;
    if (g.walls) {
        solid_m = (am == 0);
        solid_p = (ap == Lw - 1);
    } else {
        if (am < 0) am = Lw - 1;
        if (ap >= Lw) ap = 0;
    }
    int ym = y, yp = y;
    if (D == 3) {
        ym = (y == 0) ? ny - 1 : y - 1;
        yp = (y == ny - 1) ? 0 : y + 1;
    }
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const int cx = L::cx(i), cy = L::cy(i);
        const int sx = cx == 0 ? x : (cx > 0 ? xm : xp);
        const int cw = (D == 2) ? cy : L::cz(i);
        const int sa = cw == 0 ? a : (cw > 0 ? am : ap);
        const bool solid = cw == 0 ? false : (cw > 0 ? solid_m : solid_p);
        long long src;
        if (D == 2) {
            src = (long long)sa * nx + sx;
        } else {
            const int sy = cy == 0 ? y : (cy > 0 ? ym : yp);
            src = ((long long)sa * ny + sy) * nx + sx;
        }
        out[i] = solid ? StorageT<ST>::load(fin, (long long)L::opp(i) * nc + cell, inv_scale)
                       : StorageT<ST>::load(fin, (long long)i * nc + src, inv_scale);
    }
}

}  // namespace iblb
