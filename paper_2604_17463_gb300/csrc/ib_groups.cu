// ib_groups.cu -- spreading (Eq. 8) and interpolation (Eq. 7) of a 3D
// interface by spatial groups of nodes, with the stencils of a group summed
// in (or read from) a box of the lattice held in shared memory.
//
// On a paper-scale mesh (59 292 nodes of a hemispherical cap) every lattice
// cell near the surface receives ~50 stencil contributions; the nodes of
// one 8 x 8 x 8 tile touch ~14x fewer cells than they have stencil points,
// so summing a group's stencils in shared memory adds each touched cell once
// to global memory, and interpolation reads each cell of the box once.  On
// GB300 both measured slower than one thread per node with global vector
// additions (spread 61 against 44 us, interpolation 21 against 18 us per
// step on that mesh): the per-node additions are fire-and-forget, while a
// group waits on its box at every barrier and its shared-memory additions
// collide or cost shuffles.  Selected with iblb_tuning.ib_grouped.
//
// Grouping (regroup, three kernels): each node is counted in the tile of its
// cell (periodic axes wrapped), the tiles are scanned (one block) into node
// offsets and groups of at most GROUP_NODES nodes, and the nodes are placed
// in a list.  Positions move slowly, so the engine regroups once per chunk
// of steps; a group's box is recomputed from its nodes' positions at every
// use, so a stale grouping costs only box size.  A group whose box exceeds
// the shared-memory capacity (box_cap) falls back to the per-node kernels
// (ib_core.cuh).  Results equal the per-node kernels' up to the order of
// the additions.
#include "ib_core.cuh"

#include <algorithm>
#include <climits>

namespace iblb {

namespace {

__device__ __forceinline__ int wrap_mod(int i, int n)
{
    const int r = i % n;
    return r < 0 ? r + n : r;
}

// Cell of a node, wrapped on periodic axes, clamped to the lattice along the
// wall axis; -1 for a diverged node.
__device__ __forceinline__ int node_tile(const GridParams& g, const double* __restrict__ q, int j)
{
    int c[3];
    const int ext[3] = {g.nx, g.ny, g.nz};
    for (int k = 0; k < 3; k++) {
        const double x = q[3 * j + k];
        if (!(fabs(x) < 1.0e9)) return -1;
        const int i = (int)floor(x);
        c[k] = (k == 2 && g.walls) ? min(max(i, 0), ext[k] - 1) : wrap_mod(i, ext[k]);
    }
    const int tx = (g.nx + GROUP_TILE - 1) / GROUP_TILE;
    const int ty = (g.ny + GROUP_TILE - 1) / GROUP_TILE;
    return ((c[2] / GROUP_TILE) * ty + c[1] / GROUP_TILE) * tx + c[0] / GROUP_TILE;
}

__global__ void k_group_count(const double* __restrict__ q, int N, GridParams g,
                              NodeGroups ng)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    int t = node_tile(g, q, j);
    if (t < 0) t = 0;  // a diverged node touches nothing: any group will do
    ng.key[j] = t;
    ng.rank[j] = atomicAdd(&ng.tile_cnt[t], 1);
}

// One block: exclusive scans of the node counts and of the group counts per
// tile; writes tile_off, the group descriptors (first list position, nodes)
// and the number of groups, and clears tile_cnt for the next regroup.
constexpr int SCAN_THREADS = 1024;

__global__ void __launch_bounds__(SCAN_THREADS) k_group_scan(NodeGroups ng)
{
    __shared__ int s_nodes[SCAN_THREADS], s_groups[SCAN_THREADS];
    const int t = threadIdx.x;
    const int per = (ng.ntiles + SCAN_THREADS - 1) / SCAN_THREADS;
    const int t0 = min(t * per, ng.ntiles), t1 = min(t0 + per, ng.ntiles);
    int sn = 0, sg = 0;
    for (int i = t0; i < t1; i++) {
        const int c = ng.tile_cnt[i];
        sn += c;
        sg += (c + GROUP_NODES - 1) / GROUP_NODES;
    }
    s_nodes[t] = sn;
    s_groups[t] = sg;
    __syncthreads();
    // Hillis-Steele inclusive scan of both arrays
    for (int o = 1; o < SCAN_THREADS; o <<= 1) {
        const int a = t >= o ? s_nodes[t - o] : 0;
        const int b = t >= o ? s_groups[t - o] : 0;
        __syncthreads();
        s_nodes[t] += a;
        s_groups[t] += b;
        __syncthreads();
    }
    int off = s_nodes[t] - sn, goff = s_groups[t] - sg;
    for (int i = t0; i < t1; i++) {
        const int c = ng.tile_cnt[i];
        ng.tile_off[i] = off;
        for (int k = 0; k * GROUP_NODES < c; k++)
            ng.desc[goff++] = make_int2(off + k * GROUP_NODES, min(GROUP_NODES, c - k * GROUP_NODES));
        off += c;
        ng.tile_cnt[i] = 0;
    }
    if (t == SCAN_THREADS - 1) *ng.ngroups = s_groups[t];
}

__global__ void k_group_place(int N, NodeGroups ng)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < N) ng.list[ng.tile_off[ng.key[j]] + ng.rank[j]] = j;
}

// The box of one group: per-axis offsets of each node's stencil origin from
// the group's reference origin (the first node's), their minimum m and the
// box extents E (4 cells beyond the largest offset).  Periodic offsets are
// taken in (-n/2, n/2].
struct GroupBox {
    int r[3];   // reference origin (wrapped on periodic axes)
    int m[3];   // smallest offset
    int E[3];   // box extent
    int vol;    // cells; INT_MAX above the capacity, 0 for no node
    float inv_e0, inv_e01;  // 1 / E0 and 1 / (E0 E1), for box_cell
};

// floor(c / d) for 0 <= c < 2048 from a correctly rounded 1 / d: the
// relative error of (c + 1/2) (1/d) is below 2^-22, less than the distance
// (1/2) / d of (c + 1/2) / d from the nearest integer.
__device__ __forceinline__ int small_div(int c, float inv_d)
{
    return (int)(((float)c + 0.5f) * inv_d);
}

__device__ __forceinline__ int origin_of(const GridParams& g, double x, int k)
{
    const int b = (int)floor(x) - 1;
    const int ext = k == 0 ? g.nx : (k == 1 ? g.ny : g.nz);
    return (k == 2 && g.walls) ? b : wrap_mod(b, ext);
}

__device__ __forceinline__ int rel_offset(const GridParams& g, int b, int r, int k)
{
    int d = b - r;
    if (!(k == 2 && g.walls)) {
        const int ext = k == 0 ? g.nx : (k == 1 ? g.ny : g.nz);
        if (d > ext / 2) d -= ext;
        else if (d < -((ext - 1) / 2)) d += ext;
    }
    return d;
}

// Block-wide: every thread passes its node (j < 0: none); all get the box
// and their own offsets d; vol is INT_MAX above cap cells.  Contains
// __syncthreads.
__device__ __forceinline__ void group_box(const GridParams& g, const double* __restrict__ q,
                                          int j0, int j, int cap, GroupBox& bx, int (&d)[3],
                                          int (*s_red)[GROUP_NODES / 32])
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    bool valid = j >= 0;
    double x[3] = {0, 0, 0};
    if (valid)
        for (int k = 0; k < 3; k++) {
            x[k] = q[3 * j + k];
            valid = valid && fabs(x[k]) < 1.0e9;
        }
    double x0[3];
    bool ok0 = true;
    for (int k = 0; k < 3; k++) {
        x0[k] = q[3 * j0 + k];
        ok0 = ok0 && fabs(x0[k]) < 1.0e9;
    }
    for (int k = 0; k < 3; k++) {
        bx.r[k] = ok0 ? origin_of(g, x0[k], k) : 0;
        d[k] = valid ? rel_offset(g, origin_of(g, x[k], k), bx.r[k], k) : 0;
        const int lo = __reduce_min_sync(0xffffffffu, valid ? d[k] : INT_MAX);
        const int hi = __reduce_max_sync(0xffffffffu, valid ? d[k] : INT_MIN);
        if (lane == 0) {
            s_red[k][wid] = lo;
            s_red[3 + k][wid] = hi;
        }
    }
    __syncthreads();
    long long vol = 1;
    bool empty = false;
    for (int k = 0; k < 3; k++) {
        int lo = INT_MAX, hi = INT_MIN;
        for (int w = 0; w < GROUP_NODES / 32; w++) {
            lo = min(lo, s_red[k][w]);
            hi = max(hi, s_red[3 + k][w]);
        }
        empty = empty || lo > hi;
        bx.m[k] = lo;
        bx.E[k] = empty ? 0 : hi - lo + 4;
        vol *= empty ? 0 : (long long)bx.E[k];
    }
    bx.vol = (empty || vol > cap) ? INT_MAX : (int)vol;
    if (empty) bx.vol = 0;
    bx.inv_e0 = empty ? 0.f : 1.0f / (float)bx.E[0];
    bx.inv_e01 = empty ? 0.f : 1.0f / (float)(bx.E[0] * bx.E[1]);
    if (!valid) d[0] = INT_MIN;  // marks "no node" for the caller
}

// Global cell of box cell c < vol <= 2048 (-1: outside the lattice along
// the wall axis).
__device__ __forceinline__ long long box_cell(const GridParams& g, const GroupBox& bx, int c)
{
    const int lz = small_div(c, bx.inv_e01), rem = c - lz * (bx.E[0] * bx.E[1]);
    const int ly = small_div(rem, bx.inv_e0), lx = rem - ly * bx.E[0];
    const int gx = wrap_mod(bx.r[0] + bx.m[0] + lx, g.nx);
    const int gy = wrap_mod(bx.r[1] + bx.m[1] + ly, g.ny);
    int gz = bx.r[2] + bx.m[2] + lz;
    if (g.walls) {
        if (gz <= 0 || gz >= g.nz - 1) return -1;
    } else {
        gz = wrap_mod(gz, g.nz);
    }
    return ((long long)gz * g.ny + gy) * g.nx + gx;
}

// 1D weights of node j along each axis (as node_lines: FP64 floor /
// fraction split, weights in R).
template <typename R>
__device__ __forceinline__ void node_weights3(const double* __restrict__ q, int j, R (&w)[3][4])
{
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const double qk = q[3 * j + k];
        const double fl = floor(qk);
        const R fr = (R)(qk - fl);
#pragma unroll
        for (int o = 0; o < 4; o++) w[k][o] = delta4r<R>(fr + (R)(1 - o));
    }
}

// Select a[i], i in 0..3 (register arrays stay in registers).
template <typename R>
__device__ __forceinline__ R sel4(const R (&a)[4], int i)
{
    return i == 0 ? a[0] : (i == 1 ? a[1] : (i == 2 ? a[2] : a[3]));
}

__device__ __forceinline__ int wrap_once(int i, int n)
{
    while (i >= n) i -= n;
    return i;
}

// Spread: one CTA per group (persistent over the groups).  Each thread
// computes its node's 1D weights; then each warp adds the stencils of its
// 32 nodes one node at a time, lane k taking stencil points k and k + 32
// (x offset k & 3, y offset (k >> 2) & 3, z offset k >> 4 and 2 + (k >> 4)),
// so the 32 shared-memory additions of an instruction go to 32 different
// cells.  Then every touched cell of the box is added once to F.
template <typename R>
__global__ void __launch_bounds__(GROUP_NODES)
k_spread_grouped(const double* __restrict__ q, const double* __restrict__ phi,
                 NodeGroups ng, R* __restrict__ F, uint8_t* __restrict__ flags, GridParams g)
{
    constexpr int cap = box_cap<R>();
    __shared__ R sb[3][cap];
    __shared__ int s_red[6][GROUP_NODES / 32];
    const int lane = threadIdx.x & 31;
    const int o0 = lane & 3, o1 = (lane >> 2) & 3, o2a = lane >> 4;
    const int ngroups = *ng.ngroups;
    for (int gi = blockIdx.x; gi < ngroups; gi += gridDim.x) {
        const int2 dsc = ng.desc[gi];
        const int j0 = ng.list[dsc.x];
        const int j = (int)threadIdx.x < dsc.y ? ng.list[dsc.x + threadIdx.x] : -1;
        GroupBox bx;
        int d[3];
        group_box(g, q, j0, j, cap, bx, d, s_red);
        const bool has = d[0] != INT_MIN;
        if (bx.vol == INT_MAX) {  // box too large: per-node additions
            if (has) spread_node<3, R>(g, q, phi, j, F, flags);
            __syncthreads();
            continue;
        }
        for (int c = threadIdx.x; c < bx.vol; c += GROUP_NODES) sb[0][c] = sb[1][c] = sb[2][c] = R(0);
        // this thread's node: weights, force, box offsets and lattice origin
        R w[3][4] = {};
        R ph[3] = {R(0), R(0), R(0)};
        int ob[3] = {0, 0, 0}, go[3] = {0, 0, 0};
        if (has) {
            node_weights3<R>(q, j, w);
            for (int k = 0; k < 3; k++) {
                ph[k] = (R)phi[3 * j + k];
                ob[k] = d[k] - bx.m[k];
            }
            go[0] = wrap_mod(bx.r[0] + d[0], g.nx);
            go[1] = wrap_mod(bx.r[1] + d[1], g.ny);
            go[2] = (g.walls) ? bx.r[2] + d[2] : wrap_mod(bx.r[2] + d[2], g.nz);
        }
        __syncthreads();
        const unsigned hasm = __ballot_sync(0xffffffffu, has);
        for (int n = 0; n < 32; n++) {
            if (!((hasm >> n) & 1u)) continue;
            R s0[4], s1[4], s2[4];
#pragma unroll
            for (int o = 0; o < 4; o++) {
                s0[o] = __shfl_sync(0xffffffffu, w[0][o], n);
                s1[o] = __shfl_sync(0xffffffffu, w[1][o], n);
                s2[o] = __shfl_sync(0xffffffffu, w[2][o], n);
            }
            const R p0 = __shfl_sync(0xffffffffu, ph[0], n);
            const R p1 = __shfl_sync(0xffffffffu, ph[1], n);
            const R p2 = __shfl_sync(0xffffffffu, ph[2], n);
            const int bxo = __shfl_sync(0xffffffffu, ob[0], n);
            const int byo = __shfl_sync(0xffffffffu, ob[1], n);
            const int bzo = __shfl_sync(0xffffffffu, ob[2], n);
            const int gx = wrap_once(__shfl_sync(0xffffffffu, go[0], n) + o0, g.nx);
            const int gy = wrap_once(__shfl_sync(0xffffffffu, go[1], n) + o1, g.ny);
            const int gz0 = __shfl_sync(0xffffffffu, go[2], n);
            const R w0 = sel4(s0, o0), w1 = sel4(s1, o1);
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int o2 = o2a + 2 * h;
                const R ww = w0 * (w1 * sel4(s2, o2));
                int gz = gz0 + o2;
                if (g.walls) {
                    if (gz <= 0 || gz >= g.nz - 1) continue;
                } else {
                    gz = wrap_once(gz, g.nz);
                }
                if (ww == R(0)) continue;
                const int l = ((bzo + o2) * bx.E[1] + (byo + o1)) * bx.E[0] + bxo + o0;
                atomicAdd(&sb[0][l], p0 * ww);
                atomicAdd(&sb[1][l], p1 * ww);
                atomicAdd(&sb[2][l], p2 * ww);
                flags[((long long)gz * g.ny + gy) * g.nseg_x + (gx >> 5)] = 1;
            }
        }
        __syncthreads();
        for (int c = threadIdx.x; c < bx.vol; c += GROUP_NODES) {
            const R a = sb[0][c], b = sb[1][c], e = sb[2][c];
            if (a == R(0) && b == R(0) && e == R(0)) continue;
            const long long cell = box_cell(g, bx, c);
            if (cell < 0) continue;
            if constexpr (sizeof(R) == 4)
                atomicAdd(reinterpret_cast<float4*>(F) + cell, make_float4(a, b, e, 0.f));
            else {
                atomicAdd(&F[cell], a);
                atomicAdd(&F[g.ncell + cell], b);
                atomicAdd(&F[2 * g.ncell + cell], e);
            }
        }
        __syncthreads();
    }
}

// Interpolation (+ advection): the group's box of velocities is read once
// into shared memory (float4 (drho, ux, uy, uz) per cell in FP32, as the
// moments are stored; three FP64 arrays otherwise), four cells per thread in
// flight, then each thread sums its node's 64 stencil points from there.
template <typename R>
__global__ void __launch_bounds__(GROUP_NODES)
k_interp_grouped(double* __restrict__ q, const R* __restrict__ mom, NodeGroups ng,
                 double* __restrict__ qdot, int advect, GridParams g)
{
    constexpr int cap = box_cap<R>();
    constexpr bool F32 = sizeof(R) == 4;
    __shared__ __align__(16) unsigned char smem[F32 ? cap * 16 : cap * 3 * 8];
    float4* sb4 = reinterpret_cast<float4*>(smem);
    double* sbd = reinterpret_cast<double*>(smem);
    __shared__ int s_red[6][GROUP_NODES / 32];
    const int ngroups = *ng.ngroups;
    for (int gi = blockIdx.x; gi < ngroups; gi += gridDim.x) {
        const int2 dsc = ng.desc[gi];
        const int j0 = ng.list[dsc.x];
        const int j = (int)threadIdx.x < dsc.y ? ng.list[dsc.x + threadIdx.x] : -1;
        GroupBox bx;
        int d[3];
        group_box(g, q, j0, j, cap, bx, d, s_red);
        const bool has = d[0] != INT_MIN;
        R acc[3] = {R(0), R(0), R(0)};
        if (bx.vol == INT_MAX) {
            if (has) interp_node<3, R>(g, q, mom, j, acc);
        } else {
            constexpr int U = 4;
            for (int c0 = threadIdx.x; c0 < bx.vol; c0 += U * GROUP_NODES) {
                long long cell[U];
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const int c = c0 + u * GROUP_NODES;
                    cell[u] = c < bx.vol ? box_cell(g, bx, c) : -1;
                }
                if constexpr (F32) {
                    float4 v[U];
#pragma unroll
                    for (int u = 0; u < U; u++)
                        v[u] = cell[u] >= 0 ? reinterpret_cast<const float4*>(mom)[cell[u]]
                                            : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int u = 0; u < U; u++)
                        if (c0 + u * GROUP_NODES < bx.vol) sb4[c0 + u * GROUP_NODES] = v[u];
                } else {
                    double v[U][3];
#pragma unroll
                    for (int u = 0; u < U; u++)
                        for (int k = 0; k < 3; k++)
                            v[u][k] = cell[u] >= 0 ? mom[(k + 1) * g.ncell + cell[u]] : 0.0;
#pragma unroll
                    for (int u = 0; u < U; u++)
                        if (c0 + u * GROUP_NODES < bx.vol)
                            for (int k = 0; k < 3; k++) sbd[k * cap + c0 + u * GROUP_NODES] = v[u][k];
                }
            }
            __syncthreads();
            if (has) {
                R w[3][4];
                node_weights3<R>(q, j, w);
                const int ox = d[0] - bx.m[0], oy = d[1] - bx.m[1], oz = d[2] - bx.m[2];
                for (int o2 = 0; o2 < 4; o2++) {
#pragma unroll
                    for (int p = 0; p < 16; p++) {
                        const int o1 = p >> 2, o0 = p & 3;
                        const int l = ((oz + o2) * bx.E[1] + (oy + o1)) * bx.E[0] + ox + o0;
                        const R ww = w[0][o0] * w[1][o1] * w[2][o2];
                        if constexpr (F32) {
                            const float4 m = sb4[l];
                            acc[0] += ww * m.y;
                            acc[1] += ww * m.z;
                            acc[2] += ww * m.w;
                        } else {
                            acc[0] += ww * sbd[l];
                            acc[1] += ww * sbd[cap + l];
                            acc[2] += ww * sbd[2 * cap + l];
                        }
                    }
                }
            }
        }
        __syncthreads();  // the box is reused, and q[j0] is read before any advection
        if (has)
            for (int k = 0; k < 3; k++) {
                if (qdot) qdot[3 * j + k] = (double)acc[k];
                if (advect) q[3 * j + k] += (double)acc[k];
            }
    }
}

int grouped_grid(const NodeGroups& ng, int sm_count)
{
    return std::max(1, std::min(ng.max_groups, 8 * sm_count));
}

}  // namespace

void launch_regroup(const double* q, int N, const GridParams& g, const NodeGroups& ng,
                    cudaStream_t s)
{
    if (N <= 0) return;
    const int b = 256, grid = (N + b - 1) / b;
    k_group_count<<<grid, b, 0, s>>>(q, N, g, ng);
    k_group_scan<<<1, SCAN_THREADS, 0, s>>>(ng);
    k_group_place<<<grid, b, 0, s>>>(N, ng);
}

void launch_spread_grouped(int storage, const double* q, const double* phi, const NodeGroups& ng,
                           void* F, uint8_t* flags, const GridParams& g, int sm_count,
                           cudaStream_t s)
{
    const int grid = grouped_grid(ng, sm_count);
    if (storage == ST_FP64)
        k_spread_grouped<double><<<grid, GROUP_NODES, 0, s>>>(q, phi, ng, (double*)F, flags, g);
    else
        k_spread_grouped<float><<<grid, GROUP_NODES, 0, s>>>(q, phi, ng, (float*)F, flags, g);
}

void launch_interp_grouped(int storage, double* q, const void* moments, const NodeGroups& ng,
                           double* qdot, bool advect, const GridParams& g, int sm_count,
                           cudaStream_t s)
{
    const int grid = grouped_grid(ng, sm_count);
    if (storage == ST_FP64)
        k_interp_grouped<double><<<grid, GROUP_NODES, 0, s>>>(q, (const double*)moments, ng, qdot,
                                                              advect ? 1 : 0, g);
    else
        k_interp_grouped<float><<<grid, GROUP_NODES, 0, s>>>(q, (const float*)moments, ng, qdot,
                                                             advect ? 1 : 0, g);
}

}  // namespace iblb
