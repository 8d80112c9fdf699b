// ib_core.cuh -- device functions of the immersed-boundary coupling shared by
// the single-simulation kernels (ib.cu) and the batched kernels (batch.cu).
//
// Paper, Sec. 2: Eq. 7-8 (interpolation / spreading with a discrete delta),
// Eq. 10 (wetting potential Pi).  The delta is the tensor product of
// Peskin's 4-point kernel.
#pragma once

#include "common.cuh"

namespace iblb {

__device__ __forceinline__ double ipow(double x, int k)
{
    double r = 1.0;
    for (int i = 0; i < k; i++) r *= x;
    return r;
}

// Eq. 10
__device__ __forceinline__ double wetting_pi(const ForceParams& fp, double d)
{
    const double s = fp.xi / d;
    return fp.A * (ipow(s, fp.n) - ipow(s, fp.m));
}

// ------------------------------------------------------------------ stencil
// Peskin's 4-point kernel in the weight precision R (FP64 for FP64 storage,
// FP32 otherwise).
template <typename R>
__device__ __forceinline__ R delta4r(R r)
{
    const R a = fabs(r);
    if (a <= R(1)) return (R(3) - R(2) * a + sqrt(R(1) + R(4) * a - R(4) * a * a)) * R(0.125);
    if (a <= R(2)) return (R(5) - R(2) * a - sqrt(R(-7) + R(12) * a - R(4) * a * a)) * R(0.125);
    return R(0);
}

// One warp per node.  Lanes 0 .. D-1 split the node coordinate of their axis
// into floor and fraction (FP64, once per axis); lanes 0 .. 4*D-1 then
// evaluate the 1D weights of the node (axis = lane / 4, offset o = lane % 4,
// distance to the stencil line = fraction + 1 - o) in the weight precision R,
// with the lattice index of that stencil line (wrapped on periodic axes, -1
// on a solid layer or outside the lattice along the wall axis).  Every lane
// then forms the tensor-product weights of its stencil points from warp
// shuffles.  All lanes must call it.
template <int D, typename R>
__device__ __forceinline__ void node_weights(const GridParams& g, const double* __restrict__ q,
                                             int node, int lane, R& wk, int& ik)
{
    int base = 0, ok = 0;
    R frac = R(0);
    if (lane < D) {
        const double qk = q[D * node + lane];
        if (fabs(qk) < 1.0e9) {   // a diverged node touches nothing
            const double fl = floor(qk);
            base = (int)fl - 1;
            frac = (R)(qk - fl);
            ok = 1;
        }
    }
    const int k = lane >> 2;
    const int src = k < D ? k : 0;
    const int b = __shfl_sync(0xffffffffu, base, src);
    const R fr = __shfl_sync(0xffffffffu, frac, src);
    const int okk = __shfl_sync(0xffffffffu, ok, src);
    wk = R(0);
    ik = -1;
    if (lane < 4 * D && okk) {
        const int o = lane & 3;
        const int ext = k == 0 ? g.nx : (k == 1 ? g.ny : g.nz);
        const int i = b + o;
        wk = delta4r<R>(fr + (R)(1 - o));
        if (k == D - 1 && g.walls) {
            ik = (i <= 0 || i >= ext - 1) ? -1 : i;
        } else {
            const int r = i % ext;
            ik = r < 0 ? r + ext : r;
        }
    }
}

// Weight and cell of stencil point s; all lanes must call it (shuffles).
template <int D, typename R>
__device__ __forceinline__ bool point_of(const GridParams& g, R wk, int ik, int s, R& w,
                                         long long& row, int& ix)
{
    const int o0 = s & 3, o1 = (s >> 2) & 3, o2 = (s >> 4) & 3;
    const R w0 = __shfl_sync(0xffffffffu, wk, o0);
    const int i0 = __shfl_sync(0xffffffffu, ik, o0);
    const R w1 = __shfl_sync(0xffffffffu, wk, 4 + o1);
    const int i1 = __shfl_sync(0xffffffffu, ik, 4 + o1);
    R w2 = R(1);
    int i2 = 0;
    if (D == 3) {
        w2 = __shfl_sync(0xffffffffu, wk, 8 + o2);
        i2 = __shfl_sync(0xffffffffu, ik, 8 + o2);
    }
    w = w0 * w1 * w2;
    row = (long long)i2 * g.ny + i1;
    ix = i0;
    return i0 >= 0 && i1 >= 0 && i2 >= 0;
}

// ------------------------------------------------------------------ A1 pieces
// 2D ring, node j of a ring of N nodes (segment j joins node j and j+1):
// phi_j = sigma (t_j - t_{j-1}) - chi_j Pi(d_j) n_j / 2 with t the unit
// tangents, n_j the normalised sum of the outward segment normals (t_y, -t_x)
// of a counter-clockwise ring, chi_j = l_{j-1} + l_j.
__device__ __forceinline__ void ring_node_force(const double* __restrict__ q, int N, int j,
                                                const ForceParams& fp, double* __restrict__ phi,
                                                double* nrm, double* chi, int* err)
{
    const int jm = (j == 0) ? N - 1 : j - 1;
    const int jp = (j == N - 1) ? 0 : j + 1;
    const double ax = q[2 * jm], ay = q[2 * jm + 1];
    const double bx = q[2 * j], by = q[2 * j + 1];
    const double cx = q[2 * jp], cy = q[2 * jp + 1];
    const double s0x = bx - ax, s0y = by - ay;   // segment j-1
    const double s1x = cx - bx, s1y = cy - by;   // segment j
    const double l0 = sqrt(s0x * s0x + s0y * s0y);
    const double l1 = sqrt(s1x * s1x + s1y * s1y);
    const double fsx = fp.sigma * (s1x / l1) - fp.sigma * (s0x / l0);
    const double fsy = fp.sigma * (s1y / l1) - fp.sigma * (s0y / l0);
    const double nsx = s0y / l0 + s1y / l1;
    const double nsy = -s0x / l0 - s1x / l1;
    const double nl = sqrt(nsx * nsx + nsy * nsy);
    const double nhx = nsx / nl, nhy = nsy / nl;
    const double ch = l0 + l1;
    double pi = 0.0;
    if (fp.wetting) {
        const double d = by - fp.wall_plane;
        if (!(d > 0.0)) atomicOr(err, ERR_NODE_IN_WALL);
        pi = wetting_pi(fp, d);
    }
    phi[2 * j] = fsx + (-ch * pi * nhx) / 2.0;
    phi[2 * j + 1] = fsy + (-ch * pi * nhy) / 2.0;
    if (nrm) {
        nrm[2 * j] = nhx;
        nrm[2 * j + 1] = nhy;
    }
    if (chi) chi[j] = ch;
}

// 3D mesh, face f: unit normal nu_f, area A_f and for each corner v
// g_v = nu_f x (prev - next) (so d(A_f)/d(corner v) = g_v / 2), written as one
// 8-double record (g_v[3], nu[3], A, pad) per corner at its CSR position.
constexpr int ENTRY_REC = 8;

__device__ __forceinline__ void face_records(const double* __restrict__ q,
                                             const int* __restrict__ tri, int f,
                                             const int* __restrict__ entry_pos,
                                             double* __restrict__ rec)
{
    double P[3][3];
    for (int c = 0; c < 3; c++) {
        const int node = tri[3 * f + c];
        for (int k = 0; k < 3; k++) P[c][k] = q[3 * node + k];
    }
    const double ab[3] = {P[1][0] - P[0][0], P[1][1] - P[0][1], P[1][2] - P[0][2]};
    const double ac[3] = {P[2][0] - P[0][0], P[2][1] - P[0][1], P[2][2] - P[0][2]};
    const double nf[3] = {ab[1] * ac[2] - ab[2] * ac[1], ab[2] * ac[0] - ab[0] * ac[2],
                          ab[0] * ac[1] - ab[1] * ac[0]};
    const double nlen = sqrt(nf[0] * nf[0] + nf[1] * nf[1] + nf[2] * nf[2]);
    const double inv = 1.0 / nlen;
    const double nu[3] = {nf[0] * inv, nf[1] * inv, nf[2] * inv};
    const double area = 0.5 * nlen;
    for (int v = 0; v < 3; v++) {
        const double* nxt = P[(v + 1) % 3];
        const double* prv = P[(v + 2) % 3];
        const double e3[3] = {prv[0] - nxt[0], prv[1] - nxt[1], prv[2] - nxt[2]};
        double* r = rec + (long long)ENTRY_REC * entry_pos[3 * f + v];
        r[0] = nu[1] * e3[2] - nu[2] * e3[1];
        r[1] = nu[2] * e3[0] - nu[0] * e3[2];
        r[2] = nu[0] * e3[1] - nu[1] * e3[0];
        r[3] = nu[0];
        r[4] = nu[1];
        r[5] = nu[2];
        r[6] = area;
    }
}

// 3D mesh, node j: sum of its contiguous records (faces in increasing order),
// phi_j = tension - chi_j Pi(d_j) n_j / 3.
__device__ __forceinline__ void mesh_node_force(const double* __restrict__ q, int j,
                                                const double* __restrict__ rec,
                                                const int* __restrict__ csr_ptr,
                                                const ForceParams& fp, double* __restrict__ phi,
                                                double* nrm, double* chi, int* err)
{
    double fs[3] = {0, 0, 0}, ns[3] = {0, 0, 0}, area = 0.0;
    const int e0 = csr_ptr[j], e1 = csr_ptr[j + 1];
    for (int e = e0; e < e1; e++) {
        const double* r = rec + (long long)ENTRY_REC * e;
        for (int k = 0; k < 3; k++) {
            fs[k] -= fp.sigma * 0.5 * r[k];
            ns[k] += r[3 + k];
        }
        area += r[6];
    }
    const double nl = sqrt(ns[0] * ns[0] + ns[1] * ns[1] + ns[2] * ns[2]);
    const double nh[3] = {ns[0] / nl, ns[1] / nl, ns[2] / nl};
    double pi = 0.0;
    if (fp.wetting) {
        const double d = q[3 * j + 2] - fp.wall_plane;
        if (!(d > 0.0)) atomicOr(err, ERR_NODE_IN_WALL);
        pi = wetting_pi(fp, d);
    }
    for (int k = 0; k < 3; k++) {
        phi[3 * j + k] = fs[k] + (-area * pi * nh[k]) / 3.0;
        if (nrm) nrm[3 * j + k] = nh[k];
    }
    if (chi) chi[j] = area;
}

}  // namespace iblb
