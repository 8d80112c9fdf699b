// classify.cu -- inside / outside classification of the lattice by the
// interface, for the viscosity ratio (Sec. 2: fluid nodes inside and outside
// the drop are identified by ray tracing and relax with tau_in / tau_out).
//
// Rays run along the wall axis through every lattice column (x in 2D;
// (x, y) in 3D).  Each ring segment / mesh face appends its crossings with
// the column lines it covers to a per-column table of at most COL_MAX
// heights; a cell is inside when an odd number of crossings lie below it
// (the stream-collide kernel evaluates that parity, so no sort is needed).
// Ties follow fixed rules so that a column line through a shared vertex or
// edge of a closed interface counts once:
//   2D segment (a, b) crosses column X when min(a_x, b_x) <= X < max(a_x, b_x);
//   3D face, projected on the xy plane and made counter-clockwise, covers
//   column (X, Y) when each edge function is positive, or zero on a top-left
//   edge (horizontal going -x, or going -y).
// Column indices wrap periodically; a column with more than COL_MAX
// crossings sets ERR_CLASSIFY.  Every product and sum is rounded on its own
// (no fused multiply-add), so a crossing height and the sign of an edge
// function are the IEEE FP64 values of the formulas as written.
#include "common.cuh"

namespace iblb {

namespace {

__device__ __forceinline__ int wrapi(long long i, int L)
{
    long long r = i % L;
    return (int)(r < 0 ? r + L : r);
}

__device__ __forceinline__ void add_crossing(int col, double z, int* cnt, double* cz, int* err)
{
    const int k = atomicAdd(&cnt[col], 1);
    if (k < COL_MAX)
        cz[(long long)col * COL_MAX + k] = z;
    else
        atomicOr(err, ERR_CLASSIFY);
}

constexpr long long MAX_SPAN = 4096;  // columns one segment / face may cover

__global__ void k_classify_ring(const double* __restrict__ q, int N, GridParams g, int* cnt,
                                double* cz, int* err)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const int jn = (j + 1 == N) ? 0 : j + 1;
    const double ax = q[2 * j], ay = q[2 * j + 1];
    const double bx = q[2 * jn], by = q[2 * jn + 1];
    if (!(fabs(ax) < 1e9 && fabs(bx) < 1e9 && fabs(ay) < 1e9 && fabs(by) < 1e9)) return;
    const double lo = ax < bx ? ax : bx, hi = ax < bx ? bx : ax;
    const long long X0 = (long long)ceil(lo);
    for (long long X = X0; (double)X < hi && X - X0 < MAX_SPAN; X++) {
        const double y =
            __dadd_rn(ay, __ddiv_rn(__dmul_rn(__dsub_rn((double)X, ax), __dsub_rn(by, ay)),
                                    __dsub_rn(bx, ax)));
        add_crossing(wrapi(X, g.nx), y, cnt, cz, err);
    }
}

__device__ __forceinline__ double edge_fn(double ax, double ay, double bx, double by, double px,
                                          double py)
{
    return __dsub_rn(__dmul_rn(__dsub_rn(bx, ax), __dsub_rn(py, ay)),
                     __dmul_rn(__dsub_rn(by, ay), __dsub_rn(px, ax)));
}

__device__ __forceinline__ bool top_left(double ax, double ay, double bx, double by)
{
    return (ay == by && bx < ax) || (by < ay);
}

__global__ void k_classify_mesh(const double* __restrict__ q, const int* __restrict__ tri, int M,
                                GridParams g, int* cnt, double* cz, int* err)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= M) return;
    const double* P[3] = {q + 3 * tri[3 * f], q + 3 * tri[3 * f + 1], q + 3 * tri[3 * f + 2]};
    for (int k = 0; k < 3; k++)
        for (int c = 0; c < 3; c++)
            if (!(fabs(P[k][c]) < 1e9)) return;
    double area = edge_fn(P[0][0], P[0][1], P[1][0], P[1][1], P[2][0], P[2][1]);
    if (area == 0.0) return;  // vertical face: no column crosses it
    if (area < 0.0) {
        const double* t = P[1];
        P[1] = P[2];
        P[2] = t;
    }
    double xmin = P[0][0], xmax = P[0][0], ymin = P[0][1], ymax = P[0][1];
    for (int k = 1; k < 3; k++) {
        xmin = fmin(xmin, P[k][0]);
        xmax = fmax(xmax, P[k][0]);
        ymin = fmin(ymin, P[k][1]);
        ymax = fmax(ymax, P[k][1]);
    }
    const long long X0 = (long long)ceil(xmin), Y0 = (long long)ceil(ymin);
    for (long long Y = Y0; (double)Y <= ymax && Y - Y0 < MAX_SPAN; Y++)
        for (long long X = X0; (double)X <= xmax && X - X0 < MAX_SPAN; X++) {
            const double px = (double)X, py = (double)Y;
            double w[3];
            bool in = true;
            for (int k = 0; k < 3; k++) {
                const double* a = P[(k + 1) % 3];
                const double* b = P[(k + 2) % 3];
                w[k] = edge_fn(a[0], a[1], b[0], b[1], px, py);
                if (!(w[k] > 0.0 || (w[k] == 0.0 && top_left(a[0], a[1], b[0], b[1])))) in = false;
            }
            if (!in) continue;
            const double num = __dadd_rn(__dadd_rn(__dmul_rn(w[0], P[0][2]), __dmul_rn(w[1], P[1][2])),
                                         __dmul_rn(w[2], P[2][2]));
            const double z = __ddiv_rn(num, __dadd_rn(__dadd_rn(w[0], w[1]), w[2]));
            add_crossing(wrapi(X, g.nx) + g.nx * wrapi(Y, g.ny), z, cnt, cz, err);
        }
}

__global__ void k_inside_mask(GridParams g, const int* __restrict__ cnt,
                              const double* __restrict__ cz, unsigned char* mask)
{
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.ncell;
         c += (long long)gridDim.x * blockDim.x) {
        const long long plane = (long long)g.nx * g.ny;
        int col, a;
        if (g.dim == 2) {
            col = (int)(c % g.nx);
            a = (int)((c / g.nx) % g.ny);
        } else {
            col = (int)(c % plane);
            a = (int)(c / plane);
        }
        mask[c] = inside_cell(cnt, cz, col, a) ? 1 : 0;
    }
}

}  // namespace

void launch_classify(int dim, const double* q, int N, const int* tri, int M, const GridParams& g,
                     int* cnt, double* cz, int* err, cudaStream_t s)
{
    const int ncol = dim == 2 ? g.nx : g.nx * g.ny;
    cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)ncol, s);
    if (N == 0) return;
    if (dim == 2)
        k_classify_ring<<<(N + 127) / 128, 128, 0, s>>>(q, N, g, cnt, cz, err);
    else
        k_classify_mesh<<<(M + 127) / 128, 128, 0, s>>>(q, tri, M, g, cnt, cz, err);
}

void launch_inside_mask(const GridParams& g, const int* cnt, const double* cz,
                        unsigned char* mask, cudaStream_t s)
{
    long long b = (g.ncell + 255) / 256;
    if (b > 152 * 32) b = 152 * 32;
    k_inside_mask<<<(int)b, 256, 0, s>>>(g, cnt, cz, mask);
}

}  // namespace iblb
