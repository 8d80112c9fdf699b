// ib.cu -- immersed-boundary kernels of libiblb: nodal forces (A1), force
// spreading with band marking (A2 + A3), velocity interpolation with forward
// Euler advection (A5 + A6), and the FP64 observables (A7).
//
// Paper, Sec. 2:
//   Eq. 7  qdot_j = sum_x u(x) Delta(q_j - x)           (interpolation)
//   Eq. 8  F(x)   = sum_j phi_j Delta(q_j - x)           (spreading)
//   Eq. 9  interface force = surface tension + wetting term along n
//   Eq. 10 Pi(d)  = A [(xi/d)^n - (xi/d)^m]
//   nodal wetting force phi_Pi,j = -chi_j Pi(d_j) n_j / 3 (3D), / 2 for the
//   2D ring (each segment is shared by two nodes); n_j is the normalised mean
//   of the unit normals of the faces sharing node j, chi_j their total area.
//   The surface-tension force is -sigma times the gradient of the interface
//   area (3D) / length (2D) with linear elements.
// Delta is the tensor product of Peskin's 4-point kernel; stencil points on a
// solid layer (or outside the lattice along the wall axis) take no force and
// give zero velocity.
#include "common.cuh"

namespace iblb {

// Peskin's 4-point kernel, one axis.
__device__ __forceinline__ double delta4(double r)
{
    const double a = fabs(r);
    if (a <= 1.0) return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a)) * 0.125;
    if (a <= 2.0) return (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) * 0.125;
    return 0.0;
}

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

// ------------------------------------------------------------------ A1 forces
// 2D ring: one thread per node; segment j joins node j and node j+1.
__global__ void k_forces_ring(const double* __restrict__ q, int N, ForceParams fp,
                              double* __restrict__ phi, double* __restrict__ nrm,
                              double* __restrict__ chi, int* err)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const int jm = (j == 0) ? N - 1 : j - 1;
    const int jp = (j == N - 1) ? 0 : j + 1;
    const double ax = q[2 * jm], ay = q[2 * jm + 1];
    const double bx = q[2 * j], by = q[2 * j + 1];
    const double cx = q[2 * jp], cy = q[2 * jp + 1];
    const double s0x = bx - ax, s0y = by - ay;   // segment j-1
    const double s1x = cx - bx, s1y = cy - by;   // segment j
    const double l0 = sqrt(s0x * s0x + s0y * s0y);
    const double l1 = sqrt(s1x * s1x + s1y * s1y);
    // -sigma d(length)/dq_j = sigma (t_j - t_{j-1})
    const double fsx = fp.sigma * (s1x / l1) - fp.sigma * (s0x / l0);
    const double fsy = fp.sigma * (s1y / l1) - fp.sigma * (s0y / l0);
    // outward unit normals of a counter-clockwise ring: (t_y, -t_x)
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

// 3D mesh, pass 1: one thread per face computes the unit normal nu_f, the
// area A_f and, for each corner v, g_v = nu_f x (prev - next), so that
// d(A_f)/d(corner v) = g_v / 2.  It writes one record per (face, corner) at
// the position of that pair in the node -> face CSR list (entry_pos), so that
// each node's records are contiguous: g_v[3], nu[3], A, pad (8 doubles).
constexpr int ENTRY_REC = 8;

__global__ void k_face_geometry(const double* __restrict__ q, const int* __restrict__ tri, int M,
                                const int* __restrict__ entry_pos, double* __restrict__ rec)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= M) return;
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

// 3D mesh, pass 2: one thread per node sums its contiguous records (faces in
// increasing order, the summation order of a face loop; no atomics).
__global__ void k_node_forces(const double* __restrict__ q, int N, const double* __restrict__ rec,
                              const int* __restrict__ csr_ptr, ForceParams fp,
                              double* __restrict__ phi, double* __restrict__ nrm,
                              double* __restrict__ chi, int* err)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
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

void launch_forces(int dim, const double* q, int N, int M, const int* tri, const int* csr_ptr,
                   const int* entry_pos, double* entry_rec, const ForceParams& fp, double* phi,
                   double* normal, double* chi, int* err, cudaStream_t s)
{
    if (dim == 2) {
        const int b = 128, g = (N + b - 1) / b;
        k_forces_ring<<<g, b, 0, s>>>(q, N, fp, phi, normal, chi, err);
    } else {
        const int b = 64;
        k_face_geometry<<<(M + b - 1) / b, b, 0, s>>>(q, tri, M, entry_pos, entry_rec);
        k_node_forces<<<(N + b - 1) / b, b, 0, s>>>(q, N, entry_rec, csr_ptr, fp, phi, normal,
                                                    chi, err);
    }
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

// ------------------------------------------------------------------ A2 + A3 spread
// One warp per node: weighted scatter-add of phi_j into the force density
// (fire-and-forget atomics) and marking of the 32-cell row segments touched.
template <int D, typename R>
__global__ void k_spread(const double* __restrict__ q, const double* __restrict__ phi, int N,
                         R* __restrict__ F, uint8_t* __restrict__ flags, GridParams g)
{
    constexpr int S = (D == 2) ? 16 : 64;
    constexpr int PPL = (S + 31) / 32;
    const int node = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (node >= N) return;  // uniform per warp
    R wk;
    int ik;
    node_weights<D, R>(g, q, node, lane, wk, ik);
    R phl = R(0);
    if (lane < D) phl = (R)phi[D * node + lane];
    R ph[3];
    for (int k = 0; k < D; k++) ph[k] = __shfl_sync(0xffffffffu, phl, k);
#pragma unroll
    for (int p = 0; p < PPL; p++) {
        const int s = lane + 32 * p;
        R w;
        long long row;
        int ix;
        const bool ok = point_of<D, R>(g, wk, ik, s < S ? s : 0, w, row, ix);
        if (s < S && ok && w != R(0)) {
            const long long cell = row * g.nx + ix;
            for (int k = 0; k < D; k++) atomicAdd(&F[k * g.ncell + cell], ph[k] * w);
            flags[row * g.nseg_x + (ix >> 5)] = 1;
        }
    }
}

void launch_spread(int storage, int dim, const double* q, const double* phi, int N, void* F,
                   uint8_t* flags, const GridParams& g, cudaStream_t s)
{
    const int b = 128;
    const long long threads = (long long)N * 32;
    const int grid = (int)((threads + b - 1) / b);
    if (grid == 0) return;
    if (storage == ST_FP64) {
        if (dim == 2) k_spread<2, double><<<grid, b, 0, s>>>(q, phi, N, (double*)F, flags, g);
        else k_spread<3, double><<<grid, b, 0, s>>>(q, phi, N, (double*)F, flags, g);
    } else {
        if (dim == 2) k_spread<2, float><<<grid, b, 0, s>>>(q, phi, N, (float*)F, flags, g);
        else k_spread<3, float><<<grid, b, 0, s>>>(q, phi, N, (float*)F, flags, g);
    }
}

// ------------------------------------------------------------------ A5 + A6 interpolate, advect
// One warp per node; lanes share the stencil points and reduce by shuffles.
template <int D, typename R>
__global__ void k_interp(double* __restrict__ q, const R* __restrict__ mom, int N,
                         double* __restrict__ qdot, int advect, GridParams g)
{
    constexpr int S = (D == 2) ? 16 : 64;
    constexpr int PPL = (S + 31) / 32;
    const int node = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (node >= N) return;  // uniform per warp
    R wk;
    int ik;
    node_weights<D, R>(g, q, node, lane, wk, ik);
    R acc[3] = {R(0), R(0), R(0)};
#pragma unroll
    for (int p = 0; p < PPL; p++) {
        const int s = lane + 32 * p;
        R w;
        long long row;
        int ix;
        const bool ok = point_of<D, R>(g, wk, ik, s < S ? s : 0, w, row, ix);
        if (s < S && ok) {
            const long long cell = row * g.nx + ix;
            for (int k = 0; k < D; k++) acc[k] += w * mom[(k + 1) * g.ncell + cell];
        }
    }
    for (int k = 0; k < D; k++)
        for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
    if (lane < D) {
        const R a = lane == 0 ? acc[0] : (lane == 1 ? acc[1] : acc[D == 3 ? 2 : 1]);
        if (qdot) qdot[D * node + lane] = (double)a;
        if (advect) q[D * node + lane] += (double)a;
    }
}

void launch_interp(int storage, int dim, double* q, const void* moments, int N, double* qdot,
                   bool advect, const GridParams& g, cudaStream_t s)
{
    const int b = 128;
    const long long threads = (long long)N * 32;
    const int grid = (int)((threads + b - 1) / b);
    if (grid == 0) return;
    if (storage == ST_FP64) {
        if (dim == 2) k_interp<2, double><<<grid, b, 0, s>>>(q, (const double*)moments, N, qdot, advect, g);
        else k_interp<3, double><<<grid, b, 0, s>>>(q, (const double*)moments, N, qdot, advect, g);
    } else {
        if (dim == 2) k_interp<2, float><<<grid, b, 0, s>>>(q, (const float*)moments, N, qdot, advect, g);
        else k_interp<3, float><<<grid, b, 0, s>>>(q, (const float*)moments, N, qdot, advect, g);
    }
}

// ------------------------------------------------------------------ A7 observables
// Single block, fixed thread -> item assignment and reduction tree, so the
// result is deterministic.  Contact-angle estimator: algebraic least-squares
// circle (2D) / sphere (3D) through the nodes with d > 3 xi, centred on their
// mean, intersected with the plane d = min_j d_j.
constexpr int OBS_BLOCK = 1024;
constexpr int OBS_MAXV = 20;

// Reduce nv values per thread to thread 0 (sum), in a fixed order.
__device__ void block_sum(double* v, int nv, double (*sh)[OBS_BLOCK / 32])
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < nv; k++) {
        double x = v[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) sh[k][wid] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < nv; k++) {
            double t = 0.0;
            for (int w = 0; w < OBS_BLOCK / 32; w++) t += sh[k][w];
            v[k] = t;
        }
    }
    __syncthreads();
}

__device__ void block_minmax(double& mn, double& mx, double (*sh)[OBS_BLOCK / 32])
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if (lane == 0) {
        sh[0][wid] = mn;
        sh[1][wid] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 0; w < OBS_BLOCK / 32; w++) {
            mn = fmin(mn, sh[0][w]);
            mx = fmax(mx, sh[1][w]);
        }
    }
    __syncthreads();
}

__device__ bool solve_small(int n, double* A, double* b)
{
    for (int col = 0; col < n; col++) {
        int piv = col;
        for (int r = col + 1; r < n; r++)
            if (fabs(A[r * n + col]) > fabs(A[piv * n + col])) piv = r;
        if (A[piv * n + col] == 0.0) return false;
        if (piv != col) {
            for (int k = 0; k < n; k++) {
                const double t = A[col * n + k];
                A[col * n + k] = A[piv * n + k];
                A[piv * n + k] = t;
            }
            const double t = b[col];
            b[col] = b[piv];
            b[piv] = t;
        }
        for (int r = col + 1; r < n; r++) {
            const double f = A[r * n + col] / A[col * n + col];
            for (int k = col; k < n; k++) A[r * n + k] -= f * A[col * n + k];
            b[r] -= f * b[col];
        }
    }
    for (int r = n - 1; r >= 0; r--) {
        double acc = b[r];
        for (int k = r + 1; k < n; k++) acc -= A[r * n + k] * b[k];
        b[r] = acc / A[r * n + r];
    }
    return true;
}

__global__ void __launch_bounds__(OBS_BLOCK)
k_observables(int dim, const double* __restrict__ q, int N, const int* __restrict__ tri, int M,
              const double* __restrict__ mass_partial, int n_partial, double xi, double wp,
              double* out)
{
    __shared__ double sh[OBS_MAXV][OBS_BLOCK / 32];
    __shared__ double bc[8];
    const int t = threadIdx.x;
    const int wax = dim - 1;
    // phase 1: mass, volume, extremes, mean of the fit set
    double v[OBS_MAXV];
    for (int k = 0; k < OBS_MAXV; k++) v[k] = 0.0;
    for (int b = t; b < n_partial; b += OBS_BLOCK) v[0] += mass_partial[b];
    if (dim == 2) {
        for (int j = t; j < N; j += OBS_BLOCK) {
            const int jn = (j + 1 == N) ? 0 : j + 1;
            v[1] += q[2 * j] * q[2 * jn + 1] - q[2 * jn] * q[2 * j + 1];
        }
    } else {
        for (int f = t; f < M; f += OBS_BLOCK) {
            const double* a = q + 3 * tri[3 * f];
            const double* b = q + 3 * tri[3 * f + 1];
            const double* c = q + 3 * tri[3 * f + 2];
            v[1] += a[0] * (b[1] * c[2] - b[2] * c[1]) + a[1] * (b[2] * c[0] - b[0] * c[2]) +
                    a[2] * (b[0] * c[1] - b[1] * c[0]);
        }
    }
    double hmin = 1e300, hmax = -1e300;
    for (int j = t; j < N; j += OBS_BLOCK) {
        const double h = q[dim * j + wax];
        hmin = fmin(hmin, h);
        hmax = fmax(hmax, h);
        if (h - wp > 3.0 * xi) {
            for (int k = 0; k < dim; k++) v[2 + k] += q[dim * j + k];
            v[5] += 1.0;
        }
    }
    block_sum(v, 6, sh);
    block_minmax(hmin, hmax, sh);
    if (t == 0) {
        out[0] = v[0];
        out[1] = (dim == 2) ? 0.5 * v[1] : v[1] / 6.0;
        out[2] = hmax - hmin;
        out[6] = hmin - wp;
        bc[0] = v[5];
        for (int k = 0; k < dim; k++) bc[1 + k] = v[5] > 0 ? v[2 + k] / v[5] : 0.0;
    }
    __syncthreads();
    const double cnt = bc[0];
    const double mean[3] = {bc[1], bc[2], dim == 3 ? bc[3] : 0.0};
    __syncthreads();
    // phase 2: normal equations of the algebraic fit
    const int np = dim + 1;
    for (int k = 0; k < OBS_MAXV; k++) v[k] = 0.0;
    for (int j = t; j < N; j += OBS_BLOCK) {
        if (!(q[dim * j + wax] - wp > 3.0 * xi)) continue;
        double vv[4], r2 = 0.0;
        for (int k = 0; k < dim; k++) {
            vv[k] = q[dim * j + k] - mean[k];
            r2 += vv[k] * vv[k];
        }
        vv[dim] = 1.0;
        for (int a = 0; a < np; a++) {
            for (int b = 0; b < np; b++) v[a * np + b] += vv[a] * vv[b];
            v[16 + a] -= vv[a] * r2;
        }
    }
    block_sum(v, OBS_MAXV, sh);
    if (t == 0) {
        bool ok = cnt >= dim + 1;
        double Am[16], rhs[4];
        for (int k = 0; k < np * np; k++) Am[k] = v[k];
        for (int k = 0; k < np; k++) rhs[k] = v[16 + k];
        if (ok) ok = solve_small(np, Am, rhs);
        if (!ok) {
            out[3] = out[4] = out[5] = out[11] = nan("");
            out[7] = out[8] = out[9] = 0.0;
            bc[4] = -1.0;
        } else {
            double cen[3] = {0, 0, 0}, R2 = 0.0;
            for (int k = 0; k < dim; k++) {
                cen[k] = -0.5 * rhs[k];
                R2 += cen[k] * cen[k];
            }
            R2 -= rhs[dim];
            const double R = sqrt(R2);
            for (int k = 0; k < dim; k++) cen[k] += mean[k];
            const double plane = wp + out[6];
            const double dz = plane - cen[dim - 1];
            double cth = dz / R;
            cth = fmin(1.0, fmax(-1.0, cth));
            out[3] = acos(cth) * (180.0 / 3.141592653589793);
            const double rc2 = R * R - dz * dz;
            out[4] = rc2 > 0.0 ? sqrt(rc2) : 0.0;
            out[7] = cen[0];
            out[8] = cen[1];
            out[9] = cen[2];
            out[10] = R;
            bc[4] = out[4];
            bc[5] = cen[0];
            bc[6] = cen[1];
        }
    }
    __syncthreads();
    const double rcl = bc[4];
    const double c0 = bc[5], c1 = bc[6];
    __syncthreads();
    // phase 3: film thickness under the drop
    for (int k = 0; k < OBS_MAXV; k++) v[k] = 0.0;
    if (rcl >= 0.0) {
        for (int j = t; j < N; j += OBS_BLOCK) {
            const double d = q[dim * j + wax] - wp;
            double rr = 0.0;
            const double t0 = q[dim * j] - c0;
            rr += t0 * t0;
            if (dim == 3) {
                const double t1 = q[dim * j + 1] - c1;
                rr += t1 * t1;
            }
            if (sqrt(rr) < 0.5 * rcl && d <= 3.0 * xi) {
                v[0] += d;
                v[1] += 1.0;
            }
        }
    }
    block_sum(v, 2, sh);
    if (t == 0) {
        if (rcl >= 0.0) out[5] = v[1] > 0 ? v[0] / v[1] : nan("");
        if (N == 0) {
            for (int k = 1; k < 12; k++) out[k] = 0.0;
        }
    }
}

void launch_observables(int dim, const double* q, int N, const int* tri, int M,
                        const double* mass_partial, int n_partial, double xi, double wall_plane,
                        double* out, cudaStream_t s)
{
    k_observables<<<1, OBS_BLOCK, 0, s>>>(dim, q, N, tri, M, mass_partial, n_partial, xi,
                                          wall_plane, out);
}

}  // namespace iblb
