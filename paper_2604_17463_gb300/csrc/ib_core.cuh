// ib_core.cuh -- device functions of the immersed-boundary coupling shared by
// the single-simulation kernels (ib.cu) and the batched kernels (batch.cu).
//
// Paper, Sec. 2: Eq. 7-8 (interpolation / spreading with a discrete delta),
// Eq. 10 (wetting potential Pi).  The delta is the tensor product of
// Peskin's 4-point kernel.
#pragma once

#include "common.cuh"

namespace iblb {

// x^k, k >= 0, by repeated squaring (FP64 products are costly on this GPU)
__device__ __forceinline__ double ipow(double x, int k)
{
    double r = 1.0;
    while (k > 0) {
        if (k & 1) r *= x;
        k >>= 1;
        if (k) x *= x;
    }
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

// One thread per node: the node's 4 stencil lines per axis, their 1D
// weights in the weight precision R (from an FP64 floor / fraction split of
// the node coordinate, once per axis) and lattice indices (wrapped on periodic axes, -1 on
// a solid layer or outside the lattice along the wall axis).  Returns false
// for a diverged node (it touches nothing).
template <int D, typename R>
__device__ __forceinline__ bool node_lines(const GridParams& g, const double* __restrict__ q,
                                           int node, R (&w)[3][4], int (&ix)[3][4])
{
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 3; k++)
#pragma unroll
        for (int o = 0; o < 4; o++) {
            w[k][o] = (k < D) ? R(0) : (o == 0 ? R(1) : R(0));
            ix[k][o] = (k < D) ? -1 : (o == 0 ? 0 : -1);
        }
#pragma unroll
    for (int k = 0; k < D; k++) {
        const double qk = q[D * node + k];
        if (!(fabs(qk) < 1.0e9)) {
            ok = false;
            continue;
        }
        const double fl = floor(qk);
        const int base = (int)fl - 1;
        const R fr = (R)(qk - fl);
        const int ext = k == 0 ? g.nx : (k == 1 ? g.ny : g.nz);
#pragma unroll
        for (int o = 0; o < 4; o++) {
            w[k][o] = delta4r<R>(fr + (R)(1 - o));
            const int i = base + o;
            if (k == D - 1 && g.walls) {
                ix[k][o] = (i <= 0 || i >= ext - 1) ? -1 : i;
            } else {
                const int r = i % ext;
                ix[k][o] = r < 0 ? r + ext : r;
            }
        }
    }
    return ok;
}

// Spread of node j by one thread: its 16 (2D) / 64 (3D) stencil points in
// turn, one fire-and-forget vector addition per point in FP32 (a thread
// never waits on its additions, so many are in flight per SM); the band
// segments of the stencil rows are flagged once per row and segment, and,
// when `fine` is given, the 8-cell quarters of them that the stencil touches
// (fine[4 seg + quarter] = 1; the band pass of the overlapped step redoes
// only those).
template <int D, typename R>
__device__ __forceinline__ void spread_node(const GridParams& g, const double* __restrict__ q,
                                            const double* __restrict__ phi, int j,
                                            R* __restrict__ F, uint8_t* __restrict__ flags,
                                            uint8_t* __restrict__ fine = nullptr)
{
    R w[3][4];
    int ix[3][4];
    if (!node_lines<D, R>(g, q, j, w, ix)) return;
    R ph[3] = {R(0), R(0), R(0)};
    for (int k = 0; k < D; k++) ph[k] = (R)phi[D * j + k];
    const int n2 = (D == 3) ? 4 : 1;
    for (int o2 = 0; o2 < n2; o2++) {
        const int i2 = ix[2][o2];
        if (i2 < 0) continue;
#pragma unroll
        for (int o1 = 0; o1 < 4; o1++) {
            const int i1 = ix[1][o1];
            if (i1 < 0) continue;
            const long long row = (long long)i2 * g.ny + i1;
            const R w12 = w[1][o1] * w[2][o2];
            int last_seg = -1, last_q = -1;
#pragma unroll
            for (int o0 = 0; o0 < 4; o0++) {
                const R ww = w[0][o0] * w12;
                if (ww == R(0)) continue;
                const int i0 = ix[0][o0];
                const long long cell = row * g.nx + i0;
                if constexpr (sizeof(R) == 4)
                    atomicAdd(reinterpret_cast<float4*>(F) + cell,
                              make_float4(ph[0] * ww, ph[1] * ww, D == 3 ? ph[2] * ww : 0.f, 0.f));
                else
                    for (int k = 0; k < D; k++) atomicAdd(&F[k * g.ncell + cell], ph[k] * ww);
                if ((i0 >> 5) != last_seg) {
                    last_seg = i0 >> 5;
                    flags[row * g.nseg_x + last_seg] = 1;
                }
                if (fine && (i0 >> 3) != last_q) {
                    last_q = i0 >> 3;
                    fine[row * g.nseg_x * 4 + last_q] = 1;
                }
            }
        }
    }
}

// Interpolated velocity at node j by one thread: the 16 / 64 velocity reads
// of its stencil, 16 issued at a time (one 4 x 4 plane of points) before any
// is used.
template <int D, typename R>
__device__ __forceinline__ void interp_node(const GridParams& g, const double* __restrict__ q,
                                            const R* __restrict__ mom, int j, R (&acc)[3])
{
    R w[3][4];
    int ix[3][4];
    acc[0] = acc[1] = acc[2] = R(0);
    if (!node_lines<D, R>(g, q, j, w, ix)) return;
    const int n2 = (D == 3) ? 4 : 1;
    for (int o2 = 0; o2 < n2; o2++) {
        const int i2 = ix[2][o2];
        if (i2 < 0) continue;
        R ux[16], uy[16], uz[16];
#pragma unroll
        for (int p = 0; p < 16; p++) {
            const int o1 = p >> 2, o0 = p & 3;
            const int i1 = ix[1][o1], i0 = ix[0][o0];
            ux[p] = uy[p] = uz[p] = R(0);
            if (i1 < 0) continue;
            const long long cell = ((long long)i2 * g.ny + i1) * g.nx + i0;
            if constexpr (sizeof(R) == 4) {
                const float4 m = reinterpret_cast<const float4*>(mom)[cell];
                ux[p] = m.y;
                uy[p] = m.z;
                uz[p] = m.w;
            } else {
                ux[p] = mom[g.ncell + cell];
                uy[p] = mom[2 * g.ncell + cell];
                if (D == 3) uz[p] = mom[3 * g.ncell + cell];
            }
        }
#pragma unroll
        for (int p = 0; p < 16; p++) {
            const R ww = w[0][p & 3] * w[1][p >> 2] * w[2][o2];
            acc[0] += ww * ux[p];
            acc[1] += ww * uy[p];
            acc[2] += ww * uz[p];
        }
    }
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
    // FP64 divisions are costly on this GPU: one reciprocal per length,
    // then products
    const double l0 = sqrt(s0x * s0x + s0y * s0y);
    const double l1 = sqrt(s1x * s1x + s1y * s1y);
    const double il0 = 1.0 / l0, il1 = 1.0 / l1;
    const double t0x = s0x * il0, t0y = s0y * il0, t1x = s1x * il1, t1y = s1y * il1;
    double fsx = fp.sigma * t1x - fp.sigma * t0x;
    double fsy = fp.sigma * t1y - fp.sigma * t0y;
    if (fp.eref) {
        const double la0 = l0 / fp.eref[jm], la1 = l1 / fp.eref[j];
        const double T0 = fp.Gs * (1.0 + fp.Cs) * la0 * (la0 * la0 - 1.0);
        const double T1 = fp.Gs * (1.0 + fp.Cs) * la1 * (la1 * la1 - 1.0);
        fsx += T1 * t1x - T0 * t0x;
        fsy += T1 * t1y - T0 * t0y;
    }
    const double nsx = t0y + t1y;
    const double nsy = -t0x - t1x;
    const double inl = 1.0 / sqrt(nsx * nsx + nsy * nsy);
    const double nhx = nsx * inl, nhy = nsy * inl;
    const double ch = l0 + l1;
    double pi = 0.0;
    if (fp.wetting) {
        const double d = by - fp.wall_plane;
        if (!(d > 0.0)) atomicOr(err, ERR_NODE_IN_WALL);
        pi = wetting_pi(fp, d);
    }
    phi[2 * j] = fsx - 0.5 * (ch * pi * nhx);
    phi[2 * j + 1] = fsy - 0.5 * (ch * pi * nhy);
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
    // one reciprocal square root gives both the unit normal and the area
    const double n2 = nf[0] * nf[0] + nf[1] * nf[1] + nf[2] * nf[2];
    const double inv = rsqrt(n2);
    const double nu[3] = {nf[0] * inv, nf[1] * inv, nf[2] * inv};
    const double area = 0.5 * (n2 * inv);
    // tension at corner v: -sigma/2 nu x (prev - next); the opposite edges
    // of corners b and c are -ac and ab, and the three corner forces sum to
    // zero, so corner a takes minus the other two
    const double hs = 0.5 * fp.sigma;
    const double hn[3] = {hs * nu[0], hs * nu[1], hs * nu[2]};
    double ft[3][3];
    ft[1][0] = hn[1] * ac[2] - hn[2] * ac[1];
    ft[1][1] = hn[2] * ac[0] - hn[0] * ac[2];
    ft[1][2] = hn[0] * ac[1] - hn[1] * ac[0];
    ft[2][0] = ab[1] * hn[2] - ab[2] * hn[1];
    ft[2][1] = ab[2] * hn[0] - ab[0] * hn[2];
    ft[2][2] = ab[0] * hn[1] - ab[1] * hn[0];
    for (int k = 0; k < 3; k++) ft[0][k] = -(ft[1][k] + ft[2][k]);
    if (fp.eref) {
        double fel[3][3];
        face_elastic_force(P[0], P[1], P[2], fp.eref + 5 * (long long)f, fp.Gs, fp.Cs, fel);
        for (int v = 0; v < 3; v++)
            for (int k = 0; k < 3; k++) ft[v][k] += fel[v][k];
    }
    for (int v = 0; v < 3; v++) {  // 16-byte stores of the 64-byte record
        double2* r = reinterpret_cast<double2*>(rec + (long long)ENTRY_REC * entry_pos[3 * f + v]);
        r[0] = make_double2(ft[v][0], ft[v][1]);
        r[1] = make_double2(ft[v][2], nu[0]);
        r[2] = make_double2(nu[1], nu[2]);
        r[3] = make_double2(area, 0.0);
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
        const double2* r = reinterpret_cast<const double2*>(rec + (long long)ENTRY_REC * e);
        const double2 a = r[0], b = r[1], c = r[2], d = r[3];
        fs[0] += a.x;
        fs[1] += a.y;
        fs[2] += b.x;
        ns[0] += b.y;
        ns[1] += c.x;
        ns[2] += c.y;
        area += d.x;
    }
    const double inl = rsqrt(ns[0] * ns[0] + ns[1] * ns[1] + ns[2] * ns[2]);
    const double nh[3] = {ns[0] * inl, ns[1] * inl, ns[2] * inl};
    double pi = 0.0;
    if (fp.wetting) {
        const double d = q[3 * j + 2] - fp.wall_plane;
        if (!(d > 0.0)) atomicOr(err, ERR_NODE_IN_WALL);
        pi = wetting_pi(fp, d);
    }
    const double c = (area * pi) * (1.0 / 3.0);
    for (int k = 0; k < 3; k++) {
        phi[3 * j + k] = fs[k] - c * nh[k];
        if (nrm) nrm[3 * j + k] = nh[k];
    }
    if (chi) chi[j] = area;
}

}  // namespace iblb
