// classify_core.cuh -- device functions of the inside / outside
// classification (Sec. 2, viscosity ratio), shared by the single-simulation
// kernels (classify.cu) and the batched engine (batch.cu).  The rules (ray
// casting along the wall axis, tie-breaking, no fused multiply-add) are
// described in classify.cu.
#pragma once

#include "common.cuh"

namespace iblb {

__device__ __forceinline__ int classify_wrap(long long i, int L)
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

constexpr long long CLASSIFY_MAX_SPAN = 4096;  // columns one segment / face may cover

// 2D ring segment j (nodes j, j + 1): its crossings with the column lines
// x = X, min(a_x, b_x) <= X < max(a_x, b_x).
__device__ __forceinline__ void classify_segment(const double* __restrict__ q, int N, int j,
                                                 const GridParams& g, int* cnt, double* cz,
                                                 int* err)
{
    const int jn = (j + 1 == N) ? 0 : j + 1;
    const double ax = q[2 * j], ay = q[2 * j + 1];
    const double bx = q[2 * jn], by = q[2 * jn + 1];
    if (!(fabs(ax) < 1e9 && fabs(bx) < 1e9 && fabs(ay) < 1e9 && fabs(by) < 1e9)) return;
    const double lo = ax < bx ? ax : bx, hi = ax < bx ? bx : ax;
    const long long X0 = (long long)ceil(lo);
    for (long long X = X0; (double)X < hi && X - X0 < CLASSIFY_MAX_SPAN; X++) {
        const double y =
            __dadd_rn(ay, __ddiv_rn(__dmul_rn(__dsub_rn((double)X, ax), __dsub_rn(by, ay)),
                                    __dsub_rn(bx, ax)));
        add_crossing(classify_wrap(X, g.nx), y, cnt, cz, err);
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

// 3D mesh face f: the columns (X, Y) its xy projection covers and the
// height of the face above each.
__device__ __forceinline__ void classify_face(const double* __restrict__ q,
                                              const int* __restrict__ tri, int f,
                                              const GridParams& g, int* cnt, double* cz, int* err)
{
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
    for (long long Y = Y0; (double)Y <= ymax && Y - Y0 < CLASSIFY_MAX_SPAN; Y++)
        for (long long X = X0; (double)X <= xmax && X - X0 < CLASSIFY_MAX_SPAN; X++) {
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
            add_crossing(classify_wrap(X, g.nx) + g.nx * classify_wrap(Y, g.ny), z, cnt, cz, err);
        }
}

}  // namespace iblb
