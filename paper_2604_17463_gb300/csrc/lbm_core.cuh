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

// Moments of the deviations and the velocity with the half-force term.
template <int Q, typename R>
struct CellMoments {
    R drho, rho, ux, uy, uz;
};

template <int Q, typename R>
__device__ __forceinline__ CellMoments<Q, R> cell_moments(const R* g, R Fx, R Fy, R Fz)
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
template <int Q, typename R>
__device__ __forceinline__ void cell_collide(R* g, const CellMoments<Q, R>& m, R omega, R Fx, R Fy,
                                             R Fz)
{
    using L = Stencil<Q>;
    constexpr int D = L::D;
    const R usq15 = R(1.5) * (m.ux * m.ux + m.uy * m.uy + m.uz * m.uz);
    const R pref = R(1) - R(0.5) * omega;
    const R uF = m.ux * Fx + m.uy * Fy + m.uz * Fz;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const R cx = (R)L::cx(i), cy = (R)L::cy(i), cz = (R)L::cz(i);
        const R w = (R)L::w(i);
        const R cu = cx * m.ux + cy * m.uy + (D == 3 ? cz * m.uz : R(0));
        const R cF = cx * Fx + cy * Fy + (D == 3 ? cz * Fz : R(0));
        const R geq = w * (m.drho + m.rho * (R(3) * cu + R(4.5) * cu * cu - usq15));
        const R src = pref * w * (R(3) * (cF - uF) + R(9) * cu * cF);
        g[i] = g[i] + omega * (geq - g[i]) + src;
    }
}

}  // namespace iblb
