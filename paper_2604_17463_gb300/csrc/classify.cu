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
#include "classify_core.cuh"

namespace iblb {

namespace {

__global__ void k_classify_ring(const double* __restrict__ q, int N, GridParams g, int* cnt,
                                double* cz, int* err)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < N) classify_segment(q, N, j, g, cnt, cz, err);
}

__global__ void k_classify_mesh(const double* __restrict__ q, const int* __restrict__ tri, int M,
                                GridParams g, int* cnt, double* cz, int* err)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f < M) classify_face(q, tri, f, g, cnt, cz, err);
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
