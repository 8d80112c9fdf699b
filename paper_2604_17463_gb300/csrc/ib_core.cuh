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
// Elastic interface: Skalak's strain energy per unit reference area,
//   W = Gs/4 [I1^2 + 2 I1 - 2 I2 + C I2^2],  I1 = tr(Cg) - 2,  I2 = det(Cg) - 1,
// Cg = F^T F the in-plane right Cauchy-Green tensor of a linear triangle,
// F = [e1 e2] Mr with e1, e2 the current edges b - a, c - a and Mr the
// inverse of the reference edges written in an orthonormal frame of the
// reference triangle.  dW/dCg = W1 Id + W2 cof(Cg) (W1 = dW/dI1, W2 =
// dW/dI2), dW/dF = 2 F dW/dCg, and the corner forces are -A0 dW/de1 (b),
// -A0 dW/de2 (c) and their negated sum (a).  2D rings take the plane-strain
// reduction (second stretch 1): segment tension T = Gs (1 + C) lam (lam^2 - 1),
// lam = length / reference length.

// Reference data of face f: Mr (row major) and the reference area.
__device__ __forceinline__ void face_elastic_reference(const double* __restrict__ q,
                                                       const int* __restrict__ tri, int f,
                                                       double* __restrict__ ref)
{
    double a[3], E1[3], E2[3];
    for (int k = 0; k < 3; k++) {
        a[k] = q[3 * tri[3 * f] + k];
        E1[k] = q[3 * tri[3 * f + 1] + k] - a[k];
        E2[k] = q[3 * tri[3 * f + 2] + k] - a[k];
    }
    const double nx = E1[1] * E2[2] - E1[2] * E2[1];
    const double ny = E1[2] * E2[0] - E1[0] * E2[2];
    const double nz = E1[0] * E2[1] - E1[1] * E2[0];
    const double twice_area = sqrt(nx * nx + ny * ny + nz * nz);
    const double L1 = sqrt(E1[0] * E1[0] + E1[1] * E1[1] + E1[2] * E1[2]);
    // frame: u along E1; the height of E2 above E1 is twice the area / L1,
    // its projection on u is E2 . E1 / L1
    const double p = (E2[0] * E1[0] + E2[1] * E1[1] + E2[2] * E1[2]) / L1;
    const double h = twice_area / L1;
    const double inv_det = 1.0 / (L1 * h);
    ref[0] = h * inv_det;
    ref[1] = -p * inv_det;
    ref[2] = 0.0;
    ref[3] = L1 * inv_det;
    ref[4] = 0.5 * twice_area;
}

// Elastic corner forces of face f (out[v][k], v = corner a, b, c).
__device__ __forceinline__ void face_elastic_force(const double* __restrict__ P0,
                                                   const double* __restrict__ P1,
                                                   const double* __restrict__ P2,
                                                   const double* __restrict__ ref, double Gs,
                                                   double Cs, double out[3][3])
{
    const double m00 = ref[0], m01 = ref[1], m10 = ref[2], m11 = ref[3], A0 = ref[4];
    double f0[3], f1[3];
    for (int k = 0; k < 3; k++) {
        const double e1 = P1[k] - P0[k], e2 = P2[k] - P0[k];
        f0[k] = e1 * m00 + e2 * m10;
        f1[k] = e1 * m01 + e2 * m11;
    }
    const double c00 = f0[0] * f0[0] + f0[1] * f0[1] + f0[2] * f0[2];
    const double c01 = f0[0] * f1[0] + f0[1] * f1[1] + f0[2] * f1[2];
    const double c11 = f1[0] * f1[0] + f1[1] * f1[1] + f1[2] * f1[2];
    const double I1 = c00 + c11 - 2.0;
    const double I2 = c00 * c11 - c01 * c01 - 1.0;
    const double W1 = 0.5 * Gs * (I1 + 1.0);
    const double W2 = 0.5 * Gs * (Cs * I2 - 1.0);
    const double s00 = W1 + W2 * c11, s01 = -W2 * c01, s11 = W1 + W2 * c00;
    for (int k = 0; k < 3; k++) {
        const double g0 = 2.0 * (f0[k] * s00 + f1[k] * s01);
        const double g1 = 2.0 * (f0[k] * s01 + f1[k] * s11);
        const double d1 = g0 * m00 + g1 * m01;
        const double d2 = g0 * m10 + g1 * m11;
        out[1][k] = -A0 * d1;
        out[2][k] = -A0 * d2;
        out[0][k] = A0 * (d1 + d2);
    }
}

// 2D ring, node j of a ring of N nodes (segment j joins node j and j+1):
// phi_j = sigma (t_j - t_{j-1}) - chi_j Pi(d_j) n_j / 2 with t the unit
// tangents, n_j the normalised sum of the outward segment normals (t_y, -t_x)
// of a counter-clockwise ring, chi_j = l_{j-1} + l_j; with an elastic
// interface also T_j t_j - T_{j-1} t_{j-1}.
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
    double fsx = fp.sigma * (s1x / l1) - fp.sigma * (s0x / l0);
    double fsy = fp.sigma * (s1y / l1) - fp.sigma * (s0y / l0);
    if (fp.eref) {
        const double la0 = l0 / fp.eref[jm], la1 = l1 / fp.eref[j];
        const double T0 = fp.Gs * (1.0 + fp.Cs) * la0 * (la0 * la0 - 1.0);
        const double T1 = fp.Gs * (1.0 + fp.Cs) * la1 * (la1 * la1 - 1.0);
        fsx += T1 * (s1x / l1) - T0 * (s0x / l0);
        fsy += T1 * (s1y / l1) - T0 * (s0y / l0);
    }
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

// 3D mesh, face f: unit normal nu_f, area A_f and for each corner v the
// surface-tension force -sigma/2 nu_f x (prev - next) = -sigma d(A_f)/d(v)
// (plus the elastic corner force of an elastic interface), written as one
// 8-double record (force[3], nu[3], A, pad) per corner at its CSR position.
constexpr int ENTRY_REC = 8;

__device__ __forceinline__ void face_records(const double* __restrict__ q,
                                             const int* __restrict__ tri, int f,
                                             const int* __restrict__ entry_pos,
                                             const ForceParams& fp, double* __restrict__ rec)
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
    double fel[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    if (fp.eref) face_elastic_force(P[0], P[1], P[2], fp.eref + 5 * (long long)f, fp.Gs, fp.Cs, fel);
    for (int v = 0; v < 3; v++) {
        const double* nxt = P[(v + 1) % 3];
        const double* prv = P[(v + 2) % 3];
        const double e3[3] = {prv[0] - nxt[0], prv[1] - nxt[1], prv[2] - nxt[2]};
        const double hs = 0.5 * fp.sigma;
        double* r = rec + (long long)ENTRY_REC * entry_pos[3 * f + v];
        r[0] = fel[v][0] - hs * (nu[1] * e3[2] - nu[2] * e3[1]);
        r[1] = fel[v][1] - hs * (nu[2] * e3[0] - nu[0] * e3[2]);
        r[2] = fel[v][2] - hs * (nu[0] * e3[1] - nu[1] * e3[0]);
        r[3] = nu[0];
        r[4] = nu[1];
        r[5] = nu[2];
        r[6] = area;
    }
}

// 3D mesh, node j: sum of its contiguous records (faces in increasing order),
// phi_j = tension (+ elastic) - chi_j Pi(d_j) n_j / 3.
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
            fs[k] += r[k];
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
