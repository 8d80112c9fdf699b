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
//   area (3D) / length (2D) with linear elements; an elastic interface adds
//   minus the gradient of Skalak's strain energy (ib_core.cuh).
// Delta is the tensor product of Peskin's 4-point kernel; stencil points on a
// solid layer (or outside the lattice along the wall axis) take no force and
// give zero velocity.
#include "ib_core.cuh"

namespace iblb {

// ------------------------------------------------------------------ A1 forces
// 2D ring: one thread per node.
__global__ void k_forces_ring(const double* __restrict__ q, int N, ForceParams fp,
                              double* __restrict__ phi, double* __restrict__ nrm,
                              double* __restrict__ chi, int* err)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    ring_node_force(q, N, j, fp, phi, nrm, chi, err);
}

// 3D mesh, pass 1: one thread per face writes its three corner records.
__global__ void k_face_geometry(const double* __restrict__ q, const int* __restrict__ tri, int M,
                                const int* __restrict__ entry_pos, ForceParams fp,
                                double* __restrict__ rec)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= M) return;
    face_records(q, tri, f, entry_pos, fp, rec);
}

// Elastic reference of the interface as it is now: per face (3D) the inverse
// reference edge matrix and area, per segment (2D) the length.
__global__ void k_elastic_reference(int dim, const double* __restrict__ q, int N, int M,
                                    const int* __restrict__ tri, double* __restrict__ eref)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (dim == 3) {
        if (t < M) face_elastic_reference(q, tri, t, eref + 5 * (long long)t);
    } else if (t < N) {
        const int tn = (t + 1 == N) ? 0 : t + 1;
        const double sx = q[2 * tn] - q[2 * t], sy = q[2 * tn + 1] - q[2 * t + 1];
        eref[t] = sqrt(sx * sx + sy * sy);
    }
}

void launch_elastic_reference(int dim, const double* q, int N, int M, const int* tri, double* eref,
                              cudaStream_t s)
{
    const int n = dim == 3 ? M : N;
    if (n > 0) k_elastic_reference<<<(n + 127) / 128, 128, 0, s>>>(dim, q, N, M, tri, eref);
}

// 3D mesh, pass 2: one thread per node sums its records (no atomics).
__global__ void k_node_forces(const double* __restrict__ q, int N, const double* __restrict__ rec,
                              const int* __restrict__ csr_ptr, ForceParams fp,
                              double* __restrict__ phi, double* __restrict__ nrm,
                              double* __restrict__ chi, int* err)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    mesh_node_force(q, j, rec, csr_ptr, fp, phi, nrm, chi, err);
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
        k_face_geometry<<<(M + b - 1) / b, b, 0, s>>>(q, tri, M, entry_pos, fp, entry_rec);
        k_node_forces<<<(N + b - 1) / b, b, 0, s>>>(q, N, entry_rec, csr_ptr, fp, phi, normal,
                                                    chi, err);
    }
}

// ------------------------------------------------------------------ A2 + A3 spread
// One thread per node (spread_node in ib_core.cuh): one vector atomic per
// stencil point, the touched 32-cell row segments marked.  Measured against
// one warp per node (lanes sharing the stencil points) on the 59 292-node
// paper-scale mesh: 45 us against 44 us per step, so the simpler form stays.
template <int D, typename R>
__global__ void __launch_bounds__(128)
k_spread_t(const double* __restrict__ q, const double* __restrict__ phi, int N,
           R* __restrict__ F, uint8_t* __restrict__ flags, uint8_t* __restrict__ fine,
           GridParams g)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < N) spread_node<D, R>(g, q, phi, j, F, flags, fine);
}

void launch_spread(int storage, int dim, const double* q, const double* phi, int N, void* F,
                   uint8_t* flags, uint8_t* fine, const GridParams& g, cudaStream_t s)
{
    if (N <= 0) return;
    const int b = 128, grid = (N + b - 1) / b;
    if (storage == ST_FP64) {
        if (dim == 2) k_spread_t<2, double><<<grid, b, 0, s>>>(q, phi, N, (double*)F, flags, fine, g);
        else k_spread_t<3, double><<<grid, b, 0, s>>>(q, phi, N, (double*)F, flags, fine, g);
    } else {
        if (dim == 2) k_spread_t<2, float><<<grid, b, 0, s>>>(q, phi, N, (float*)F, flags, fine, g);
        else k_spread_t<3, float><<<grid, b, 0, s>>>(q, phi, N, (float*)F, flags, fine, g);
    }
}

// ------------------------------------------------------------------ A5 + A6 interpolate, advect
// One thread per node (interp_node in ib_core.cuh): 16 velocity reads in
// flight per thread; on the 59 292-node mesh 16 us per step against 35 us
// for one warp per node with two reads per lane and a shuffle reduction.
template <int D, typename R>
__global__ void __launch_bounds__(128)
k_interp_t(double* __restrict__ q, const R* __restrict__ mom, int N, double* __restrict__ qdot,
           int advect, GridParams g)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    R acc[3];
    interp_node<D, R>(g, q, mom, j, acc);
    for (int k = 0; k < D; k++) {
        if (qdot) qdot[D * j + k] = (double)acc[k];
        if (advect) q[D * j + k] += (double)acc[k];
    }
}

void launch_interp(int storage, int dim, double* q, const void* moments, int N, double* qdot,
                   bool advect, const GridParams& g, cudaStream_t s)
{
    if (N <= 0) return;
    const int b = 128, grid = (N + b - 1) / b;
    if (storage == ST_FP64) {
        if (dim == 2) k_interp_t<2, double><<<grid, b, 0, s>>>(q, (const double*)moments, N, qdot, advect, g);
        else k_interp_t<3, double><<<grid, b, 0, s>>>(q, (const double*)moments, N, qdot, advect, g);
    } else {
        if (dim == 2) k_interp_t<2, float><<<grid, b, 0, s>>>(q, (const float*)moments, N, qdot, advect, g);
        else k_interp_t<3, float><<<grid, b, 0, s>>>(q, (const float*)moments, N, qdot, advect, g);
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

// Deformation index (Sec. 4, Eq. 15): the enclosed region is split into
// simplices from the node mean p0 (triangles of the ring in 2D, tetrahedra of
// the mesh in 3D).  Over a simplex with vertices v_k relative to p0 and
// signed measure |K|: int x = |K| sum(v_k) / (d + 1) and
// int x x^T = |K| (sum v_k v_k^T + s s^T) / ((d + 1)(d + 2)), s = sum v_k.
// The central second moments in the shear plane (x and the wall axis) give
// the semi-axes sqrt(4 lambda / area) (2D) or sqrt(5 lambda / volume) (3D).
__global__ void __launch_bounds__(OBS_BLOCK)
k_deformation(int dim, const double* __restrict__ q, int N, const int* __restrict__ tri, int M,
              double* out)
{
    __shared__ double sh[6][OBS_BLOCK / 32];
    __shared__ double p0s[3];
    const int t = threadIdx.x;
    const int w = dim - 1;
    double v[6];
    for (int k = 0; k < 6; k++) v[k] = 0.0;
    for (int j = t; j < N; j += OBS_BLOCK)
        for (int k = 0; k < dim; k++) v[k] += q[dim * j + k];
    block_sum(v, 3, sh);
    if (t == 0)
        for (int k = 0; k < 3; k++) p0s[k] = k < dim ? v[k] / N : 0.0;
    __syncthreads();
    const double p0[3] = {p0s[0], p0s[1], p0s[2]};
    for (int k = 0; k < 6; k++) v[k] = 0.0;
    const int nsimp = dim == 2 ? N : M;
    for (int e = t; e < nsimp; e += OBS_BLOCK) {
        double a[3] = {0, 0, 0}, b[3] = {0, 0, 0}, c[3] = {0, 0, 0};
        double meas;
        if (dim == 2) {
            const int jn = (e + 1 == N) ? 0 : e + 1;
            for (int k = 0; k < 2; k++) {
                a[k] = q[2 * e + k] - p0[k];
                b[k] = q[2 * jn + k] - p0[k];
            }
            meas = 0.5 * (a[0] * b[1] - a[1] * b[0]);
        } else {
            const double* A = q + 3 * tri[3 * e];
            const double* B = q + 3 * tri[3 * e + 1];
            const double* C = q + 3 * tri[3 * e + 2];
            for (int k = 0; k < 3; k++) {
                a[k] = A[k] - p0[k];
                b[k] = B[k] - p0[k];
                c[k] = C[k] - p0[k];
            }
            meas = (a[0] * (b[1] * c[2] - b[2] * c[1]) + a[1] * (b[2] * c[0] - b[0] * c[2]) +
                    a[2] * (b[0] * c[1] - b[1] * c[0])) / 6.0;
        }
        const double sx = a[0] + b[0] + c[0], sw = a[w] + b[w] + c[w];
        const double f2 = meas / ((dim + 1) * (dim + 2));
        v[0] += meas;
        v[1] += meas * sx / (dim + 1);
        v[2] += meas * sw / (dim + 1);
        v[3] += f2 * (a[0] * a[0] + b[0] * b[0] + c[0] * c[0] + sx * sx);
        v[4] += f2 * (a[w] * a[w] + b[w] * b[w] + c[w] * c[w] + sw * sw);
        v[5] += f2 * (a[0] * a[w] + b[0] * b[w] + c[0] * c[w] + sx * sw);
    }
    block_sum(v, 6, sh);
    if (t == 0) {
        const double vol = v[0];
        const double gx = v[1] / vol, gw = v[2] / vol;
        const double sxx = v[3] - vol * gx * gx;
        const double sww = v[4] - vol * gw * gw;
        const double sxw = v[5] - vol * gx * gw;
        const double mean = 0.5 * (sxx + sww);
        const double rad = sqrt(0.25 * (sxx - sww) * (sxx - sww) + sxw * sxw);
        const double kk = dim == 2 ? 4.0 : 5.0;
        const double r1 = sqrt(kk * (mean + rad) / vol), r3 = sqrt(kk * (mean - rad) / vol);
        out[0] = (r1 - r3) / (r1 + r3);
        out[1] = r1;
        out[2] = r3;
        out[3] = 0.5 * atan2(2.0 * sxw, sxx - sww) * (180.0 / 3.141592653589793);
        out[4] = vol;
    }
}

void launch_deformation(int dim, const double* q, int N, const int* tri, int M, double* out,
                        cudaStream_t s)
{
    k_deformation<<<1, OBS_BLOCK, 0, s>>>(dim, q, N, tri, M, out);
}

void launch_observables(int dim, const double* q, int N, const int* tri, int M,
                        const double* mass_partial, int n_partial, double xi, double wall_plane,
                        double* out, cudaStream_t s)
{
    k_observables<<<1, OBS_BLOCK, 0, s>>>(dim, q, N, tri, M, mass_partial, n_partial, xi,
                                          wall_plane, out);
}

}  // namespace iblb
