// spread_det.cu -- order-deterministic spreading (A2 + A3) of libiblb.
//
// Eq. 8 of the paper, F(x) = sum_j phi_j Delta(q_j - x), written as a gather:
// every cell sums the contributions of the nodes whose stencils cover it in
// a fixed order, so that FP64 runs are bitwise reproducible (the scatter
// with atomics in ib.cu adds in whatever order the hardware serves them).
//
// Per step:
//   1. k_det_bin     per node: the 1D delta weights (as node_lines), the
//                    stencil origin o = floor(q) - 1 per axis, the node's
//                    bin (a tile of DT^D stencil origins), a count per bin,
//                    and the cell tiles its stencil touches (each appended
//                    once to a list of active cell tiles);
//   2. k_det_scan    exclusive prefix sum of the bin counts (one block);
//   3. k_det_place   node items into their bins' ranges;
//   4. k_det_sort    each bin's items into increasing order;
//   5. k_det_gather  per fluid cell of an active cell tile: the bins that can
//                    hold a covering node, in a fixed order, and their nodes
//                    in increasing order; F(x) is written (not added: the
//                    band buffer is zero there) and the cell's band segment
//                    flagged.
// Only the order of the additions differs from the scatter: the weights are
// the same numbers, formed the same way.  The same kernels serve the
// single-simulation engine (one slot, node item = node id) and the batched
// engine (items = (slot, node) pairs in slot order, bins and cell tiles
// numbered globally across slots).
#include "ib_core.cuh"
#include "spread_det.cuh"

namespace iblb {
namespace {

constexpr int DT = DET_TILE;     // tile edge in cells (bins and cell tiles)
constexpr int GATHER_BLOCK = 64;
constexpr int SCAN_BLOCK = 1024;

__device__ __forceinline__ int2 item_of(const int2* __restrict__ items, int it)
{
    return items ? items[it] : make_int2(0, it);
}

__device__ __forceinline__ int wrap(int v, int n)
{
    const int r = v % n;
    return r < 0 ? r + n : r;
}

// Axis k of a slot is periodic unless it is the wall axis with walls.
__device__ __forceinline__ bool periodic_axis(const GridParams& g, int k)
{
    return !(g.walls && k == g.dim - 1);
}

__device__ __forceinline__ int extent(const GridParams& g, int k)
{
    return k == 0 ? g.nx : (k == 1 ? g.ny : g.nz);
}

// Bin coordinate of stencil origin o along axis k: o mod n on periodic axes,
// o + 3 along the wall axis (origins -2 .. n-2 reach a fluid layer, bins
// 1 .. n+1).
__device__ __forceinline__ int bin_coord(const GridParams& g, int k, int o)
{
    return periodic_axis(g, k) ? wrap(o, extent(g, k)) : o + 3;
}

template <int D, typename R>
__global__ void k_det_bin(const DetSlot* __restrict__ slots, const int2* __restrict__ items,
                          int nitems, int* __restrict__ bin_of, int* __restrict__ org,
                          R* __restrict__ wts, int* __restrict__ cnt, int* __restrict__ active,
                          int2* __restrict__ act_list, int* __restrict__ nact)
{
    const int it = blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= nitems) return;
    const int2 sj = item_of(items, it);
    const DetSlot& d = slots[sj.x];
    const GridParams g = d.g;
    const double* q = d.q + (long long)D * sj.y;
    int o[3] = {0, 0, 0};
    bool ok = true;
    for (int k = 0; k < D; k++) {
        const double qk = q[k];
        if (!(fabs(qk) < 1.0e9)) {  // a diverged node touches nothing
            ok = false;
            break;
        }
        const double fl = floor(qk);
        o[k] = (int)fl - 1;
        const R fr = (R)(qk - fl);  // as node_lines: FP64 split, weights in R
        for (int s = 0; s < 4; s++) wts[(long long)it * 12 + 4 * k + s] = delta4r<R>(fr + (R)(1 - s));
        org[3 * it + k] = o[k];
    }
    int b[3] = {0, 0, 0};
    if (ok) {
        for (int k = 0; k < D; k++) {
            b[k] = bin_coord(g, k, o[k]);
            if (!periodic_axis(g, k) && (b[k] < 1 || b[k] > extent(g, k) + 1)) ok = false;
        }
    }
    if (!ok) {
        bin_of[it] = -1;
        return;
    }
    const int bin = d.bin_base + b[0] / DT +
                    d.nb[0] * (b[1] / DT + (D == 3 ? d.nb[1] * (b[2] / DT) : 0));
    bin_of[it] = bin;
    atomicAdd(&cnt[bin], 1);
    // cell tiles touched by the stencil lines o .. o+3 (fluid layers only
    // along the wall axis); each is appended to the active list once
    int tl[3][4], nt[3] = {0, 0, 1};
    tl[2][0] = 0;
    for (int k = 0; k < D; k++) {
        const int n = extent(g, k);
        for (int s = 0; s < 4; s++) {
            int c = o[k] + s;
            if (periodic_axis(g, k)) {
                c = wrap(c, n);
            } else if (c < 1 || c > n - 2) {
                continue;
            }
            const int t = c / DT;
            bool seen = false;
            for (int u = 0; u < nt[k]; u++) seen |= (tl[k][u] == t);
            if (!seen) tl[k][nt[k]++] = t;
        }
    }
    for (int a = 0; a < nt[0]; a++)
        for (int c1 = 0; c1 < nt[1]; c1++)
            for (int c2 = 0; c2 < nt[2]; c2++) {
                const int local = tl[0][a] + d.ct[0] * (tl[1][c1] + (D == 3 ? d.ct[1] * tl[2][c2] : 0));
                if (atomicExch(&active[d.cell_base + local], 1) == 0)
                    act_list[atomicAdd(nact, 1)] = make_int2(sj.x, local);
            }
}

// Exclusive prefix sum of cnt[0 .. n) into start and cur (one block).
__global__ void __launch_bounds__(SCAN_BLOCK)
k_det_scan(const int* __restrict__ cnt, int n, int* __restrict__ start, int* __restrict__ cur)
{
    __shared__ int part[SCAN_BLOCK];
    const int t = threadIdx.x;
    const int lo = (int)((long long)t * n / SCAN_BLOCK);
    const int hi = (int)((long long)(t + 1) * n / SCAN_BLOCK);
    int s = 0;
    for (int i = lo; i < hi; i++) s += cnt[i];
    part[t] = s;
    __syncthreads();
    // Hillis-Steele inclusive scan of the per-thread sums
    for (int off = 1; off < SCAN_BLOCK; off <<= 1) {
        const int v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = part[t] - s;
    for (int i = lo; i < hi; i++) {
        start[i] = run;
        cur[i] = run;
        run += cnt[i];
    }
}

__global__ void k_det_place(const int* __restrict__ bin_of, int nitems, int* __restrict__ cur,
                            int* __restrict__ list)
{
    const int it = blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= nitems) return;
    const int b = bin_of[it];
    if (b >= 0) list[atomicAdd(&cur[b], 1)] = it;
}

// Insertion sort of each bin's range (bins hold few nodes).
__global__ void k_det_sort(const int* __restrict__ cnt, const int* __restrict__ start, int nbins,
                           int* __restrict__ list)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbins) return;
    const int c = cnt[b];
    if (c < 2) return;
    int* l = list + start[b];
    for (int i = 1; i < c; i++) {
        const int v = l[i];
        int k = i - 1;
        while (k >= 0 && l[k] > v) {
            l[k + 1] = l[k];
            k--;
        }
        l[k + 1] = v;
    }
}

// Bin tiles along axis k whose origins can cover cell coordinate x, in a
// fixed order (origins x, x-1, x-2, x-3), without repeats.
__device__ __forceinline__ int source_bins(const GridParams& g, int k, int x, int* out)
{
    int n = 0;
    for (int s = 0; s < 4; s++) {
        const int b = bin_coord(g, k, x - s) / DT;
        bool seen = false;
        for (int u = 0; u < n; u++) seen |= (out[u] == b);
        if (!seen) out[n++] = b;
    }
    return n;
}

// Sum of the 1D weights of a node (origin o) on axis k at cell coordinate
// x; *hit tells whether any stencil line lands on x.
template <typename R>
__device__ __forceinline__ R axis_weight(const GridParams& g, int k, int o, const R* w, int x,
                                         bool* hit)
{
    R s = R(0);
    bool h = false;
    const int n = extent(g, k);
    const bool per = periodic_axis(g, k);
    for (int t = 0; t < 4; t++) {
        const int c = per ? wrap(o + t, n) : o + t;
        if (c == x) {
            s = h ? s + w[t] : w[t];
            h = true;
        }
    }
    *hit = h;
    return s;
}

template <int D, typename R>
__global__ void __launch_bounds__(GATHER_BLOCK)
k_det_gather(const DetSlot* __restrict__ slots, const int2* __restrict__ items,
             const int2* __restrict__ act_list, const int* __restrict__ nact,
             const int* __restrict__ cnt, const int* __restrict__ start,
             const int* __restrict__ list, const int* __restrict__ org, const R* __restrict__ wts)
{
    constexpr int CELLS = (D == 3) ? DT * DT * DT : DT * DT;
    constexpr int PER = GATHER_BLOCK / CELLS;  // cell tiles per block iteration
    const int n_act = *nact;
    const int sub = threadIdx.x / CELLS, ci = threadIdx.x % CELLS;
    for (int a0 = blockIdx.x * PER; a0 < n_act; a0 += gridDim.x * PER) {
        const int a = a0 + sub;
        if (a >= n_act) continue;
        const int2 st = act_list[a];
        const DetSlot& d = slots[st.x];
        const GridParams g = d.g;
        int tc[3];
        tc[0] = st.y % d.ct[0];
        tc[1] = (st.y / d.ct[0]) % d.ct[1];
        tc[2] = (D == 3) ? st.y / (d.ct[0] * d.ct[1]) : 0;
        int x[3] = {tc[0] * DT + ci % DT, tc[1] * DT + (ci / DT) % DT, 0};
        if (D == 3) x[2] = tc[2] * DT + ci / (DT * DT);
        bool inside = true;
        for (int k = 0; k < D; k++) {
            const int n = extent(g, k);
            if (x[k] >= n) inside = false;
            if (!periodic_axis(g, k) && (x[k] < 1 || x[k] > n - 2)) inside = false;
        }
        if (!inside) continue;
        int sb[3][4], ns[3] = {1, 1, 1};
        sb[2][0] = 0;
        for (int k = 0; k < D; k++) ns[k] = source_bins(g, k, x[k], sb[k]);
        R acc[3] = {R(0), R(0), R(0)};
        bool touched = false;
        for (int i2 = 0; i2 < ns[2]; i2++)
            for (int i1 = 0; i1 < ns[1]; i1++)
                for (int i0 = 0; i0 < ns[0]; i0++) {
                    const int bin = d.bin_base + sb[0][i0] +
                                    d.nb[0] * (sb[1][i1] + (D == 3 ? d.nb[1] * sb[2][i2] : 0));
                    const int c = cnt[bin], s0 = start[bin];
                    for (int e = s0; e < s0 + c; e++) {
                        const int it = list[e];
                        const R* w = wts + (long long)it * 12;
                        bool h0, h1, h2 = true;
                        const R w0 = axis_weight<R>(g, 0, org[3 * it], w, x[0], &h0);
                        const R w1 = axis_weight<R>(g, 1, org[3 * it + 1], w + 4, x[1], &h1);
                        R w2 = R(1);
                        if (D == 3) w2 = axis_weight<R>(g, 2, org[3 * it + 2], w + 8, x[2], &h2);
                        if (!(h0 && h1 && h2)) continue;
                        const R ww = (D == 3) ? w0 * w1 * w2 : w0 * w1;
                        const int j = item_of(items, it).y;
                        for (int k = 0; k < D; k++) acc[k] += (R)d.phi[(long long)D * j + k] * ww;
                        touched = true;
                    }
                }
        if (!touched) continue;
        const long long cell = ((long long)x[2] * g.ny + x[1]) * g.nx + x[0];
        R* F = (R*)d.F;
        if constexpr (sizeof(R) == 4)  // float4 per cell
            reinterpret_cast<float4*>(F)[cell] = make_float4(acc[0], acc[1], D == 3 ? acc[2] : 0.f, 0.f);
        else
            for (int k = 0; k < D; k++) F[(long long)k * g.ncell + cell] = acc[k];
        const long long row = (long long)x[2] * g.ny + x[1];
        d.flags[row * g.nseg_x + (x[0] >> 5)] = 1;
    }
}

template <int D, typename R>
void launch_det_t(const DetSlot* slots, const int2* items, int nitems, const DetBuffers& b,
                  int nbins, int ncelltiles, int sm_count, cudaStream_t s)
{
    cudaMemsetAsync(b.cnt, 0, sizeof(int) * (size_t)nbins, s);
    cudaMemsetAsync(b.active, 0, sizeof(int) * (size_t)ncelltiles, s);
    cudaMemsetAsync(b.nact, 0, sizeof(int), s);
    const int nb = (nitems + 127) / 128;
    k_det_bin<D, R><<<nb, 128, 0, s>>>(slots, items, nitems, b.bin_of, b.org, (R*)b.wts, b.cnt,
                                       b.active, b.act_list, b.nact);
    k_det_scan<<<1, SCAN_BLOCK, 0, s>>>(b.cnt, nbins, b.start, b.cur);
    k_det_place<<<nb, 128, 0, s>>>(b.bin_of, nitems, b.cur, b.list);
    k_det_sort<<<(nbins + 127) / 128, 128, 0, s>>>(b.cnt, b.start, nbins, b.list);
    k_det_gather<D, R><<<sm_count * 8, GATHER_BLOCK, 0, s>>>(slots, items, b.act_list, b.nact,
                                                            b.cnt, b.start, b.list, b.org,
                                                            (const R*)b.wts);
}

}  // namespace

void launch_spread_det(int storage, int dim, const DetSlot* slots, const int2* items, int nitems,
                       const DetBuffers& b, int nbins, int ncelltiles, int sm_count,
                       cudaStream_t s)
{
    if (nitems <= 0) return;
    if (storage == ST_FP64) {
        if (dim == 2) launch_det_t<2, double>(slots, items, nitems, b, nbins, ncelltiles, sm_count, s);
        else launch_det_t<3, double>(slots, items, nitems, b, nbins, ncelltiles, sm_count, s);
    } else {
        if (dim == 2) launch_det_t<2, float>(slots, items, nitems, b, nbins, ncelltiles, sm_count, s);
        else launch_det_t<3, float>(slots, items, nitems, b, nbins, ncelltiles, sm_count, s);
    }
}

void det_tiles(const GridParams& g, int nb[3], int ct[3])
{
    for (int k = 0; k < 3; k++) {
        nb[k] = 1;
        ct[k] = 1;
    }
    for (int k = 0; k < g.dim; k++) {
        const int n = k == 0 ? g.nx : (k == 1 ? g.ny : g.nz);
        const bool per = !(g.walls && k == g.dim - 1);
        nb[k] = ((per ? n : n + 2) + DT - 1) / DT;
        ct[k] = (n + DT - 1) / DT;
    }
}

}  // namespace iblb
