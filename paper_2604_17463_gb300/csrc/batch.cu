// batch.cu -- batched engine (many independent droplet simulations advanced
// by shared launches) and the admission side of the serving loop.
//
// A batch holds simulations ("slots") of one lattice type and one population
// storage form.  Each time step runs the same phases as a single simulation
// (nodal forces, spread, stream-collide, interpolate + advect; Sec. 2 of the
// paper), but every phase is ONE launch over all active slots:
//   - stream-collide: a persistent kernel whose warps walk contiguous ranges
//     of a (slot, row, x0) work list; an item is cpt 32-cell segments of one
//     lattice row of one slot, cpt chosen per slot by the tile autotuner;
//   - IB phases: one thread (forces) or one warp (spread, interpolation) per
//     (slot, node) item of a concatenated node list.
// Slot state lives in one device arena (the batch's HBM budget) carved by a
// first-fit allocator; a request is admitted when its footprint fits, else
// the call returns IBLB_EAGAIN.  Slots advance together; a run stops at each
// slot's last step, marks it done and drops it from the work lists.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/iblb.h"
#include "classify_core.cuh"
#include "ib_core.cuh"
#include "lbm_core.cuh"
#include "spread_det.cuh"

namespace iblb {

struct SlotDev {
    void* f[2];
    void* mom;
    void* F;
    uint8_t* flags;        // band flags, one byte per 32-cell row segment
    int* err;
    GridParams g;
    long long nfluid;      // fluid cells
    double omega;
    float omega_f, scale, inv_scale;
    int cur_base;          // current buffer = cur_base ^ batch parity
    unsigned* rng;         // two-entry step counter for binary16 stochastic rounding
    int cpt;               // 32-cell row segments per stream-collide work item
    double* q;
    double* phi;
    int N, M;
    int* tri;
    int* csr_ptr;
    int* entry_pos;
    double* entry_rec;
    ForceParams fp;
    double uw_lo[3], uw_hi[3];  // tangential velocities of the lower / upper wall
    int moving;                 // either wall moves
    // viscosity ratio: cells outside the interface relax with omega_out;
    // per-column crossing table of the inside / outside classification
    int two_tau;
    int ncol;                   // columns: nx (2D), nx * ny (3D)
    double omega_out;
    float omega_out_f;
    int* col_cnt;               // [ncol]
    double* col_z;              // [ncol][COL_MAX]
};

namespace {

constexpr int BT = 128;  // threads per stream-collide block

// 32-cell segments a warp of the batched stream-collide works on at once
// (their loads are all issued before any of them is collided, so that
// enough bytes are in flight per SM for the HBM bound), and the resident
// blocks per SM asked of the register allocator; chosen by measurement on
// the 256-drop set (D2Q9 FP32: 3 segments at 5 blocks beat 2 at 6 or 8 and
// 4 at 4; D2Q9 binary16: 2 at 6) and on 40 D3Q19 requests of the serving
// mix (FP32: 2 segments at 4 blocks with the next item prefetched, 1.89 ms
// per launch, beat 1 segment at 5, 6, 7 or 8 blocks, 2.99-3.71 ms, and 2 at
// 3 blocks, 1.96 ms; binary16: 2 at 4, 1.63 ms, beat 1 at 6 or 8, 2.5 ms).
// FP64 is bound by its arithmetic.  A slot's work items hold cpt segments,
// a multiple of this.
constexpr int b_ilp_of(int Q, int ST)
{
    return ST == ST_FP64 ? 1 : (Q == 9 ? (ST == ST_FP32 ? 3 : 2) : 2);
}
template <int Q, int ST> struct BIlp {
    static constexpr int value = b_ilp_of(Q, ST);
};
int b_ilp(int Q, int storage) { return b_ilp_of(Q, storage); }

template <int Q, int ST> struct BMinBlocks {
    static constexpr int value = ST == ST_FP64 ? (Q == 9 ? 5 : 4) : (Q == 9 ? (ST == ST_FP32 ? 5 : 6) : 4);
};
// The next work item is loaded while the current one is processed (D3Q19
// FP32; measured slower for binary16).
template <int Q, int ST> struct BPrefetch {
    static constexpr bool value = Q == 19 && ST == ST_FP32;
};

// One stream-collide work item: cpt consecutive 32-cell segments x0 ..
// x0 + 32 segs - 1 of one lattice row of one slot, with the slot's
// parameters the kernel needs on every item (96 bytes, read as six 16-byte
// loads, so that an item costs one memory round trip).
struct __align__(16) BItem {
    const void* f[2];      // the slot's population buffers
    uint8_t* flags;        // the slot's band flags (per 32-cell row segment)
    void* F;               // the slot's force density [dim][ncell]
    void* mom;             // the slot's moments [1 + dim][ncell]
    int slot, row;         // slot index; full row index (y, or y + ny z)
    int x0, nx, ny, Lw;    // first cell of the item; extent; wall-axis length
    unsigned nc;           // cells of the slot's lattice
    int segs;              // segments in this item
    float omega_f;         // 1 / tau
    int cur_base;          // bit 0: current buffer = bit 0 ^ batch parity; bit 1: moving
                           // walls; bit 2: viscosity ratio
    float scale, inv_scale;  // binary16 storage scale
    unsigned* rng;         // binary16 rounding step counter
};
static_assert(sizeof(BItem) == 96, "work item layout");

// An item as six 16-byte words held in registers; fields by their place
// in BItem (little-endian).
struct BItemRegs {
    int4 a, b, c, d, e, f;
};

__device__ __forceinline__ BItemRegs load_item(const BItem* __restrict__ items, int i)
{
    const int4* p = reinterpret_cast<const int4*>(items + i);
    return BItemRegs{__ldg(p), __ldg(p + 1), __ldg(p + 2), __ldg(p + 3), __ldg(p + 4),
                     __ldg(p + 5)};
}

__device__ __forceinline__ void* ptr_of(int lo, int hi)
{
    return reinterpret_cast<void*>(((unsigned long long)(unsigned)hi << 32) | (unsigned)lo);
}

// Batched stream-collide.  Warp w of the persistent grid (W warps) takes the
// items w, w + W, w + 2W, ... of the work list, which is ordered by slot,
// row and x0: at any time the warps of the GPU work on one window of
// consecutive items, so each population plane is read and written in a
// compact region (DRAM pages are reused across warps) whatever the slot
// sizes.  Lane k of a warp takes x = x0 + 32 j + k of segment j, so a warp
// reads and writes 32 consecutive cells of a row per plane and every
// segment is one band flag (laid out per row as in the single-simulation
// engine).  Everything but the x wrap depends on the row only.  In band
// segments the force density is loaded right after the populations, so that
// its latency overlaps theirs.  Populations are addressed by one 32-bit index
// i * ncell + cell from the slot's buffer (Q * ncell < 2^32).  Arithmetic is
// FP32 for the FP32 and binary16 forms, FP64 for FP64.  EXT: the
// instantiation that adds the moving-wall term and the viscosity ratio
// (per item, as its slot asks; launched only while some active slot has
// either, the other instantiation carries no trace of them).
template <int Q, int ST, bool WRITE_ALL, bool EXT>
__global__ void __launch_bounds__(BT, (BMinBlocks<Q, ST>::value))
k_b_stream_collide(const SlotDev* __restrict__ slots, const BItem* __restrict__ items,
                   int nitems, int par)
{
    using T = StorageT<ST>;
    using S = typename T::S;
    using R = typename T::R;
    using L = Stencil<Q>;
    constexpr int D = L::D;
    constexpr int ILP = BIlp<Q, ST>::value;
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * (BT / 32);
    const int wid = blockIdx.x * (BT / 32) + (threadIdx.x >> 5);
    if (wid >= nitems) return;

    constexpr bool PF = BPrefetch<Q, ST>::value;
    BItemRegs nxt;
    if constexpr (PF) nxt = load_item(items, wid);
    for (int it = wid; it < nitems; it += nwarps) {
        BItemRegs item;
        if constexpr (PF) {
            item = nxt;
            if (it + nwarps < nitems) nxt = load_item(items, it + nwarps);
        } else {
            item = load_item(items, it);
        }
        const int cur = (item.e.w & 1) ^ par;  // cur_base ^ parity
        const bool moving = EXT && (item.e.w & 2) != 0;
        const bool two_tau = EXT && (item.e.w & 4) != 0;
        const S* __restrict__ fin =
            (const S*)(cur ? ptr_of(item.a.z, item.a.w) : ptr_of(item.a.x, item.a.y));
        S* __restrict__ fout =
            (S*)(cur ? ptr_of(item.a.x, item.a.y) : ptr_of(item.a.z, item.a.w));
        uint8_t* __restrict__ flags = (uint8_t*)ptr_of(item.b.x, item.b.y);
        R* __restrict__ F = (R*)ptr_of(item.b.z, item.b.w);
        R* __restrict__ mom = (R*)ptr_of(item.c.x, item.c.y);
        const int slot = item.c.z, row = item.c.w;
        const int x0 = item.d.x, nx = item.d.y, ny = item.d.z, Lw = item.d.w;
        const unsigned nc = (unsigned)item.e.x;
        const int segs = item.e.y;
        const int nseg = (nx + 31) >> 5;
        R omega, gsc = R(1), ginv = R(1);
        if constexpr (sizeof(R) == 4)
            omega = __int_as_float(item.e.z);
        else
            omega = slots[slot].omega;
        // viscosity ratio: cells outside the interface (an even number of
        // crossings of their column below them) relax with omega_out
        R omega_out = omega;
        const int* col_cnt = nullptr;
        const double* col_z = nullptr;
        if constexpr (EXT) {
            if (two_tau) {
                omega_out = sizeof(R) == 4 ? (R)slots[slot].omega_out_f : (R)slots[slot].omega_out;
                col_cnt = slots[slot].col_cnt;
                col_z = slots[slot].col_z;
            }
        }
        unsigned step = 0;
        if constexpr (ST == ST_FP16) {  // populations stay in their stored scale
            unsigned* rng = (unsigned*)ptr_of(item.f.z, item.f.w);
            gsc = __int_as_float(item.f.x);
            ginv = __int_as_float(item.f.y);
            step = sr_step(rng + cur, nullptr, false);
            // the slot's first item advances its rounding step counter
            if (row == (D == 2 ? 1 : ny) && x0 == 0 && lane == 0) rng[cur ^ 1] = step + 1u;
        }
        int y, a;  // a: coordinate along the wall axis
        if (D == 2) {
            y = row;
            a = row;
        } else {
            a = row / ny;
            y = row - a * ny;
        }
        const unsigned rowbase = (unsigned)row * (unsigned)nx;
        unsigned dym = 0u, dyp = 0u;
        if (D == 3) {
            dym = (y == 0) ? (unsigned)(ny - 1) * (unsigned)nx : 0u - (unsigned)nx;
            dyp = (y == ny - 1) ? 0u - (unsigned)(ny - 1) * (unsigned)nx : (unsigned)nx;
        }
        const unsigned dwm = (D == 2) ? 0u - (unsigned)nx : 0u - (unsigned)nx * (unsigned)ny;
        const bool solid_m = (a == 1), solid_p = (a == Lw - 2);
        // moving walls (Ladd): a population bounced back at a wall of
        // tangential velocity u_w gains 2 w_i rho_w (c_i . u_w) / c_s^2 with
        // rho_w = 1, as in the single engine; only the rows next to a wall
        // read the slot's wall velocities
        double uwm[3] = {0.0, 0.0, 0.0}, uwp[3] = {0.0, 0.0, 0.0};
        if constexpr (EXT) {
            if (moving && (solid_m || solid_p))
                for (int k = 0; k < 3; k++) {
                    uwm[k] = slots[slot].uw_lo[k];
                    uwp[k] = slots[slot].uw_hi[k];
                }
        }
        for (int j0 = 0; j0 < segs; j0 += ILP) {
            R g[ILP][Q];
            R fxk[ILP], fyk[ILP], fzk[ILP];
            unsigned cellk[ILP];
            int bandk[ILP];
            bool validk[ILP];
            // pass 1: the band flags and every population load, then the
            // force density of the band segments
#pragma unroll
            for (int k = 0; k < ILP; k++) {
                const int x = x0 + 32 * (j0 + k) + lane;
                const bool valid = (j0 + k < segs) && x < nx;
                validk[k] = valid;
                const int xv = valid ? x : 0;  // idle lanes read cell 0's sources
                bandk[k] = (j0 + k < segs) ? flags[(unsigned)row * (unsigned)nseg + (xv >> 5)] : 0;
                const unsigned cell = rowbase + (unsigned)xv;
                cellk[k] = cell;
                const unsigned dxm = (xv == 0) ? (unsigned)(nx - 1) : 0u - 1u;       // c_x = +1
                const unsigned dxp = (xv == nx - 1) ? 0u - (unsigned)(nx - 1) : 1u;  // c_x = -1
#pragma unroll
                for (int i = 0; i < Q; i++) {
                    const int cx = L::cx(i), cy = L::cy(i);
                    const int cw = (D == 2) ? cy : L::cz(i);
                    const bool solid = cw == 0 ? false : (cw > 0 ? solid_m : solid_p);
                    unsigned off = (cx > 0 ? dxm : (cx < 0 ? dxp : 0u)) +
                                   (cw > 0 ? dwm : (cw < 0 ? 0u - dwm : 0u));
                    if (D == 3) off += (cy > 0 ? dym : (cy < 0 ? dyp : 0u));
                    if (solid) {
                        g[k][i] = T::load(fin, (unsigned)L::opp(i) * nc + cell, R(1));
                        if (EXT && moving) {
                            const double* uw = cw > 0 ? uwm : uwp;
                            const double cu = (D == 2) ? L::cx(i) * uw[0] + cy * uw[1]
                                                       : L::cx(i) * uw[0] + cy * uw[1] + cw * uw[2];
                            g[k][i] += (R)(6.0 * L::w(i) * cu) * gsc;
                        }
                    } else {
                        g[k][i] = T::load(fin, (unsigned)i * nc + cell + off, R(1));
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < ILP; k++) {
                fxk[k] = R(0);
                fyk[k] = R(0);
                fzk[k] = R(0);
                if (bandk[k] && validk[k]) {
                    if constexpr (sizeof(R) == 4) {  // float4 per cell
                        const float4 f = reinterpret_cast<const float4*>(F)[cellk[k]];
                        fxk[k] = f.x;
                        fyk[k] = f.y;
                        fzk[k] = f.z;
                    } else {
                        fxk[k] = F[cellk[k]];
                        fyk[k] = F[nc + cellk[k]];
                        if (D == 3) fzk[k] = F[2 * nc + cellk[k]];
                    }
                }
            }
            // pass 2: collide and store each cell
#pragma unroll
            for (int k = 0; k < ILP; k++) {
                if (!validk[k]) continue;
                const unsigned cell = cellk[k];
                const int band = bandk[k];
                const R Fx = fxk[k], Fy = fyk[k], Fz = fzk[k];
                if (band) {  // the band buffer is left zero for the next spread
                    if constexpr (sizeof(R) == 4) {
                        reinterpret_cast<float4*>(F)[cell] = make_float4(0.f, 0.f, 0.f, 0.f);
                    } else {
                        F[cell] = 0;
                        F[nc + cell] = 0;
                        if (D == 3) F[2 * nc + cell] = 0;
                    }
                }
                const CellMoments<Q, R> mo = cell_moments<Q, R>(g[k], Fx, Fy, Fz, ginv);
                R om = omega;
                if constexpr (EXT) {
                    if (two_tau) {
                        const int xc = (int)(cell - rowbase);
                        if (!inside_cell(col_cnt, col_z, D == 2 ? xc : xc + nx * y, a))
                            om = omega_out;
                    }
                }
                cell_collide<Q, R>(g[k], mo, om, Fx, Fy, Fz, gsc);
                store_cell_flat<Q, ST>(fout, nc, cell, g[k],
                                       ST == ST_FP16 ? sr_seed(step, (long long)cell) : 0u);
                if (WRITE_ALL || band) put_moments<D, R>(mom, nc, cell, mo.drho, mo.ux, mo.uy, mo.uz);
                if (!isfinite(mo.drho)) atomicOr(slots[slot].err, ERR_NONFINITE);
            }
            // clear the flags of the segments just read (after every lane of
            // the warp has read its flag)
            __syncwarp();
#pragma unroll
            for (int k = 0; k < ILP; k++)
                if (lane == 0 && j0 + k < segs && bandk[k])
                    flags[(unsigned)row * (unsigned)nseg + (unsigned)((x0 >> 5) + j0 + k)] = 0;
        }
    }
}

__global__ void k_b_forces_ring(const SlotDev* __restrict__ slots, const int2* __restrict__ nodes,
                                int nnodes)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nnodes) return;
    const int2 nd = nodes[t];
    const SlotDev& sd = slots[nd.x];
    ring_node_force(sd.q, sd.N, nd.y, sd.fp, sd.phi, nullptr, nullptr, sd.err);
}

__global__ void k_b_face_geometry(const SlotDev* __restrict__ slots,
                                  const int2* __restrict__ faces, int nfaces)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nfaces) return;
    const int2 fd = faces[t];
    const SlotDev& sd = slots[fd.x];
    face_records(sd.q, sd.tri, fd.y, sd.entry_pos, sd.fp, sd.entry_rec);
}

__global__ void k_b_node_forces(const SlotDev* __restrict__ slots, const int2* __restrict__ nodes,
                                int nnodes)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nnodes) return;
    const int2 nd = nodes[t];
    const SlotDev& sd = slots[nd.x];
    mesh_node_force(sd.q, nd.y, sd.entry_rec, sd.csr_ptr, sd.fp, sd.phi, nullptr, nullptr, sd.err);
}

// One thread per (slot, node): spread into the slot's force density and mark
// its band segments (as the single-simulation kernel, spread_node).
template <int D, typename R>
__global__ void __launch_bounds__(128)
k_b_spread(const SlotDev* __restrict__ slots, const int2* __restrict__ nodes, int nnodes)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nnodes) return;
    const int2 nd = nodes[t];
    const SlotDev& sd = slots[nd.x];
    spread_node<D, R>(sd.g, sd.q, sd.phi, nd.y, (R*)sd.F, sd.flags);
}

// One thread per (slot, node): interpolate and advect (interp_node).
template <int D, typename R>
__global__ void __launch_bounds__(128)
k_b_interp(const SlotDev* __restrict__ slots, const int2* __restrict__ nodes, int nnodes)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nnodes) return;
    const int2 nd = nodes[t];
    const SlotDev& sd = slots[nd.x];
    R acc[3];
    interp_node<D, R>(sd.g, sd.q, (const R*)sd.mom, nd.y, acc);
    for (int k = 0; k < D; k++) sd.q[D * nd.y + k] += (double)acc[k];
}

}  // namespace

// ------------------------------------------------------------------ launchers
static void launch_b_sc(int Q, int storage, bool write_all, bool moving, const SlotDev* slots,
                        const BItem* tiles, int ntiles, int par, int grid, cudaStream_t s)
{
#define IBLB_BSC(QQ, SS)                                                                             \
    do {                                                                                             \
        if (moving) {                                                                                \
            if (write_all)                                                                           \
                k_b_stream_collide<QQ, SS, true, true><<<grid, BT, 0, s>>>(slots, tiles, ntiles, par);  \
            else                                                                                     \
                k_b_stream_collide<QQ, SS, false, true><<<grid, BT, 0, s>>>(slots, tiles, ntiles, par); \
        } else {                                                                                     \
            if (write_all)                                                                           \
                k_b_stream_collide<QQ, SS, true, false><<<grid, BT, 0, s>>>(slots, tiles, ntiles, par); \
            else                                                                                     \
                k_b_stream_collide<QQ, SS, false, false><<<grid, BT, 0, s>>>(slots, tiles, ntiles, par);\
        }                                                                                            \
    } while (0)
    if (Q == 9) {
        if (storage == ST_FP64) IBLB_BSC(9, ST_FP64);
        else if (storage == ST_FP32) IBLB_BSC(9, ST_FP32);
        else IBLB_BSC(9, ST_FP16);
    } else {
        if (storage == ST_FP64) IBLB_BSC(19, ST_FP64);
        else if (storage == ST_FP32) IBLB_BSC(19, ST_FP32);
        else IBLB_BSC(19, ST_FP16);
    }
#undef IBLB_BSC
}

// Resident blocks per SM of the batched stream-collide instantiation used by
// (Q, storage): the persistent grid is this times the SM count.
static int b_sc_blocks_per_sm(int Q, int storage)
{
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
#define IBLB_OCC(QQ, SS) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_b_stream_collide<QQ, SS, false, false>, BT, 0)
    if (Q == 9) {
        if (storage == ST_FP64) IBLB_OCC(9, ST_FP64);
        else if (storage == ST_FP32) IBLB_OCC(9, ST_FP32);
        else IBLB_OCC(9, ST_FP16);
    } else {
        if (storage == ST_FP64) IBLB_OCC(19, ST_FP64);
        else if (storage == ST_FP32) IBLB_OCC(19, ST_FP32);
        else IBLB_OCC(19, ST_FP16);
    }
#undef IBLB_OCC
    if (e != cudaSuccess || n < 1) {
        (void)cudaGetLastError();
        n = 4;
    }
    return n;
}

// Viscosity ratio: the column crossing tables of the slots that have one,
// cleared and rebuilt from the current interface (classify_core.cuh), one
// thread per (slot, column), then per (slot, segment) / (slot, face).
__global__ void k_b_col_clear(const SlotDev* __restrict__ slots, const int* __restrict__ tt)
{
    const SlotDev& sd = slots[tt[blockIdx.y]];
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col < sd.ncol) sd.col_cnt[col] = 0;
}

__global__ void k_b_classify(const SlotDev* __restrict__ slots, const int2* __restrict__ items,
                             int n, int dim)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int2 it = items[t];
    const SlotDev& sd = slots[it.x];
    if (!sd.two_tau) return;
    if (dim == 2)
        classify_segment(sd.q, sd.N, it.y, sd.g, sd.col_cnt, sd.col_z, sd.err);
    else
        classify_face(sd.q, sd.tri, it.y, sd.g, sd.col_cnt, sd.col_z, sd.err);
}

static void launch_b_ib(int dim, int storage, int phase, const SlotDev* slots, const int2* nodes,
                        int nnodes, const int2* faces, int nfaces, cudaStream_t s)
{
    const int wb = 128;
    const int node_grid = (nnodes + wb - 1) / wb;  // one thread per (slot, node)
    if (phase == 0) {  // nodal forces
        if (dim == 2) {
            k_b_forces_ring<<<(nnodes + 127) / 128, 128, 0, s>>>(slots, nodes, nnodes);
        } else {
            if (nfaces > 0) k_b_face_geometry<<<(nfaces + 63) / 64, 64, 0, s>>>(slots, faces, nfaces);
            k_b_node_forces<<<(nnodes + 63) / 64, 64, 0, s>>>(slots, nodes, nnodes);
        }
    } else if (phase == 1) {  // spread
        if (storage == ST_FP64) {
            if (dim == 2) k_b_spread<2, double><<<node_grid, wb, 0, s>>>(slots, nodes, nnodes);
            else k_b_spread<3, double><<<node_grid, wb, 0, s>>>(slots, nodes, nnodes);
        } else {
            if (dim == 2) k_b_spread<2, float><<<node_grid, wb, 0, s>>>(slots, nodes, nnodes);
            else k_b_spread<3, float><<<node_grid, wb, 0, s>>>(slots, nodes, nnodes);
        }
    } else {  // interpolate + advect
        if (storage == ST_FP64) {
            if (dim == 2) k_b_interp<2, double><<<node_grid, wb, 0, s>>>(slots, nodes, nnodes);
            else k_b_interp<3, double><<<node_grid, wb, 0, s>>>(slots, nodes, nnodes);
        } else {
            if (dim == 2) k_b_interp<2, float><<<node_grid, wb, 0, s>>>(slots, nodes, nnodes);
            else k_b_interp<3, float><<<node_grid, wb, 0, s>>>(slots, nodes, nnodes);
        }
    }
}

}  // namespace iblb

using namespace iblb;

// ------------------------------------------------------------------ host side
namespace {

constexpr size_t ALIGN = 256;

size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

// First-fit allocator over the batch arena (offsets), coalescing on free.
struct Arena {
    size_t size = 0;
    std::map<size_t, size_t> free_blocks;  // offset -> length
    void reset(size_t n)
    {
        size = n;
        free_blocks.clear();
        free_blocks[0] = n;
    }
    bool alloc(size_t n, size_t* off)
    {
        for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n;
                const size_t noff = it->first + n;
                free_blocks.erase(it);
                if (rest) free_blocks[noff] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n)
    {
        auto it = free_blocks.emplace(off, n).first;
        auto next = std::next(it);
        if (next != free_blocks.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_blocks.erase(next);
        }
        if (it != free_blocks.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_blocks.erase(it);
            }
        }
    }
    size_t free_bytes() const
    {
        size_t t = 0;
        for (auto& kv : free_blocks) t += kv.second;
        return t;
    }
};

struct Layout {
    size_t pop[2], mom, F, flags, err, rng, q, phi, tri, csr, epos, erec, eref, cols, colz, total;
};

Layout slot_layout(int Q, int dim, size_t elt, size_t relt, long long ncell, int rowlen, int N,
                   int M, bool elastic, int ncol)
{
    Layout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += align_up(bytes > 0 ? bytes : 1);
        return at;
    };
    L.pop[0] = take((size_t)Q * ncell * elt);
    L.pop[1] = take((size_t)Q * ncell * elt);
    const int storage = relt == 8 ? 0 : 1;
    L.mom = take(moments_bytes(storage, dim, ncell));
    L.F = take(force_bytes(storage, dim, ncell));
    L.flags = take((size_t)(ncell / rowlen) * (size_t)((rowlen + 31) / 32));
    L.err = take(sizeof(int));
    L.rng = take(2 * sizeof(unsigned));
    L.q = take(sizeof(double) * (size_t)N * dim);
    L.phi = take(sizeof(double) * (size_t)N * dim);
    if (dim == 3) {
        L.tri = take(sizeof(int) * 3 * (size_t)M);
        L.csr = take(sizeof(int) * (size_t)(N + 1));
        L.epos = take(sizeof(int) * 3 * (size_t)M);
        L.erec = take(sizeof(double) * ENTRY_REC * 3 * (size_t)M);
    }
    if (elastic) L.eref = take(sizeof(double) * (dim == 3 ? 5 * (size_t)M : (size_t)N));
    if (ncol > 0) {
        L.cols = take(sizeof(int) * (size_t)ncol);
        L.colz = take(sizeof(double) * COL_MAX * (size_t)ncol);
    }
    L.total = o;
    return L;
}

struct Slot {
    bool used = false, active = false, done = false;
    iblb_config cfg{};
    long long steps_total = 0, steps_done = 0;
    size_t off = 0, bytes = 0;
    int buf = 0;          // buffer holding the current state
    int cpt = 1;
    int status = 0;       // device error bits seen at completion
    SlotDev dev{};
};

double wetting_A(const iblb_config& c)
{
    const double th = c.theta_eq_deg * (M_PI / 180.0);
    return c.sigma * ((double)(c.pi_m - 1) * (double)(c.pi_n - 1)) /
           ((double)(c.pi_n - c.pi_m) * c.xi) * (1.0 + std::cos(th));
}

}  // namespace

struct iblb_batch_s {
    int Q = 9, dim = 2, storage = 0;
    size_t elt = 8, relt = 8;
    cudaStream_t stream = nullptr, cap = nullptr;
    unsigned char* arena_ptr = nullptr;
    Arena arena;
    std::vector<Slot> slots;
    SlotDev* d_slots = nullptr;
    BItem* d_tiles = nullptr;  // stream-collide work items
    int2* d_nodes = nullptr;
    int2* d_faces = nullptr;
    size_t cap_tiles = 0, cap_nodes = 0, cap_faces = 0;
    int* d_tt = nullptr;      // active slots with a viscosity ratio
    size_t cap_tt = 0;
    int ntt = 0, max_ncol = 0;
    int ntiles = 0, nnodes = 0, nfaces = 0, nactive = 0;
    bool any_ext = false;     // an active slot has moving walls or a viscosity ratio
    double* d_partial = nullptr;
    double* d_obs = nullptr;
    int par = 0;
    bool dirty = true;
    int sm_count = 0;
    int sc_blocks_per_sm = 4;  // resident blocks per SM of the stream-collide kernel
    std::map<std::tuple<int, int, int>, cudaGraphExec_t> graphs;
    std::map<int, int> tile_cache;  // width bucket -> cells per thread
    // order-deterministic spreading (when any active slot asks for it)
    bool det = false;
    DetSlot* d_detslots = nullptr;
    size_t cap_detslots = 0;
    DetBuffers detb{};
    size_t cap_cnt = 0, cap_start = 0, cap_cur = 0, cap_active = 0, cap_actlist = 0;
    size_t cap_binof = 0, cap_org = 0, cap_list = 0, cap_wts = 0;
    int det_nbins = 0, det_ncelltiles = 0;
    std::string msg;
    long long launches = 0;
};

namespace {

iblb_status bfail(iblb_batch_s* b, iblb_status st, const std::string& m)
{
    if (b) b->msg = m;
    return st;
}

#define BCK(b, call)                                                                     \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return bfail(b, IBLB_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

void clear_graphs(iblb_batch_s* b)
{
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
}

template <typename T>
cudaError_t ensure(T** p, size_t* cap, size_t n)
{
    if (n <= *cap && *p) return cudaSuccess;
    if (*p) cudaFree(*p);
    *p = nullptr;
    size_t c = std::max<size_t>(n, 64);
    c = c + c / 2;
    cudaError_t e = cudaMalloc(p, sizeof(T) * c);
    if (e == cudaSuccess) *cap = c;
    return e;
}

// Stream-collide work items of one slot (descriptor d, index `slot`): every
// fluid row (2D: y = 1 .. ny-2; 3D: rows z * ny + y with z = 1 .. nz-2) in
// pieces of cpt 32-cell segments from x0 = 0.
void slot_items(const SlotDev& d, int slot, int cpt, std::vector<BItem>& out)
{
    const GridParams& g = d.g;
    const int step = 32 * cpt;
    const int r0 = g.dim == 2 ? 1 : g.ny;
    const int r1 = g.dim == 2 ? g.ny - 1 : g.ny * (g.nz - 1);
    BItem it{};
    it.f[0] = d.f[0];
    it.f[1] = d.f[1];
    it.flags = d.flags;
    it.F = d.F;
    it.mom = d.mom;
    it.slot = slot;
    it.nx = g.nx;
    it.ny = g.ny;
    it.Lw = g.dim == 2 ? g.ny : g.nz;
    it.nc = (unsigned)g.ncell;
    it.omega_f = d.omega_f;
    it.cur_base = (d.cur_base & 1) | (d.moving ? 2 : 0) | (d.two_tau ? 4 : 0);
    it.scale = d.scale;
    it.inv_scale = d.inv_scale;
    it.rng = d.rng;
    for (int r = r0; r < r1; r++)
        for (int x0 = 0; x0 < g.nx; x0 += step) {
            it.row = r;
            it.x0 = x0;
            it.segs = std::min(cpt, (g.nx - x0 + 31) / 32);
            out.push_back(it);
        }
}

// Rebuild the slot descriptors and the work lists of the active slots.
iblb_status rebuild(iblb_batch_s* b)
{
    std::vector<BItem> tiles;
    std::vector<int2> nodes, faces;
    std::vector<SlotDev> devs(b->slots.size());
    for (size_t s = 0; s < b->slots.size(); s++) {
        Slot& sl = b->slots[s];
        if (!sl.used) continue;
        sl.dev.cur_base = sl.buf ^ b->par;
        sl.dev.cpt = sl.cpt;
        devs[s] = sl.dev;
        if (!sl.active) continue;
        slot_items(sl.dev, (int)s, sl.cpt, tiles);
        for (int j = 0; j < sl.dev.N; j++) nodes.push_back(make_int2((int)s, j));
        for (int f = 0; f < (b->dim == 3 ? sl.dev.M : 0); f++) faces.push_back(make_int2((int)s, f));
    }
    BCK(b, cudaStreamSynchronize(b->stream));
    BCK(b, ensure(&b->d_tiles, &b->cap_tiles, tiles.size()));
    BCK(b, ensure(&b->d_nodes, &b->cap_nodes, nodes.size()));
    BCK(b, ensure(&b->d_faces, &b->cap_faces, faces.size()));
    if (!devs.empty())
        BCK(b, cudaMemcpy(b->d_slots, devs.data(), sizeof(SlotDev) * devs.size(),
                          cudaMemcpyHostToDevice));
    if (!tiles.empty())
        BCK(b, cudaMemcpy(b->d_tiles, tiles.data(), sizeof(BItem) * tiles.size(), cudaMemcpyHostToDevice));
    if (!nodes.empty())
        BCK(b, cudaMemcpy(b->d_nodes, nodes.data(), sizeof(int2) * nodes.size(), cudaMemcpyHostToDevice));
    if (!faces.empty())
        BCK(b, cudaMemcpy(b->d_faces, faces.data(), sizeof(int2) * faces.size(), cudaMemcpyHostToDevice));
    b->ntiles = (int)tiles.size();
    b->nnodes = (int)nodes.size();
    b->nfaces = (int)faces.size();
    b->any_ext = false;
    b->ntt = 0;
    b->max_ncol = 0;
    std::vector<int> tt;
    for (size_t k = 0; k < b->slots.size(); k++) {
        const Slot& sl = b->slots[k];
        if (!sl.active) continue;
        if (sl.dev.moving || sl.dev.two_tau) b->any_ext = true;
        if (sl.dev.two_tau) {
            tt.push_back((int)k);
            b->max_ncol = std::max(b->max_ncol, sl.dev.ncol);
        }
    }
    b->ntt = (int)tt.size();
    if (!tt.empty()) {
        BCK(b, ensure(&b->d_tt, &b->cap_tt, tt.size()));
        BCK(b, cudaMemcpy(b->d_tt, tt.data(), sizeof(int) * tt.size(), cudaMemcpyHostToDevice));
    }
    // deterministic spread: bins and cell tiles of the active slots, numbered
    // globally in slot order
    b->det = false;
    for (auto& sl : b->slots)
        if (sl.active && sl.cfg.deterministic_spread) b->det = true;
    if (b->det && !nodes.empty()) {
        std::vector<DetSlot> ds(b->slots.size());
        int nbins = 0, ncell = 0;
        for (size_t k = 0; k < b->slots.size(); k++) {
            const Slot& sl = b->slots[k];
            if (!sl.active) continue;
            DetSlot& d = ds[k];
            d.g = sl.dev.g;
            det_tiles(d.g, d.nb, d.ct);
            d.bin_base = nbins;
            d.cell_base = ncell;
            nbins += d.nb[0] * d.nb[1] * d.nb[2];
            ncell += d.ct[0] * d.ct[1] * d.ct[2];
            d.q = sl.dev.q;
            d.phi = sl.dev.phi;
            d.F = sl.dev.F;
            d.flags = sl.dev.flags;
        }
        const size_t ni = nodes.size();
        BCK(b, ensure(&b->d_detslots, &b->cap_detslots, ds.size()));
        BCK(b, ensure(&b->detb.cnt, &b->cap_cnt, (size_t)nbins));
        BCK(b, ensure(&b->detb.start, &b->cap_start, (size_t)nbins));
        BCK(b, ensure(&b->detb.cur, &b->cap_cur, (size_t)nbins));
        BCK(b, ensure(&b->detb.active, &b->cap_active, (size_t)ncell));
        BCK(b, ensure(&b->detb.act_list, &b->cap_actlist, (size_t)ncell));
        BCK(b, ensure(&b->detb.bin_of, &b->cap_binof, ni));
        BCK(b, ensure(&b->detb.org, &b->cap_org, 3 * ni));
        BCK(b, ensure(&b->detb.list, &b->cap_list, ni));
        double* w = (double*)b->detb.wts;  // FP64 room serves both precisions
        BCK(b, ensure(&w, &b->cap_wts, 12 * ni));
        b->detb.wts = w;
        if (!b->detb.nact) BCK(b, cudaMalloc(&b->detb.nact, sizeof(int)));
        BCK(b, cudaMemcpy(b->d_detslots, ds.data(), sizeof(DetSlot) * ds.size(), cudaMemcpyHostToDevice));
        b->det_nbins = nbins;
        b->det_ncelltiles = ncell;
    }
    int na = 0;
    for (auto& sl : b->slots) na += sl.active ? 1 : 0;
    b->nactive = na;
    clear_graphs(b);
    b->dirty = false;
    return IBLB_OK;
}

int kernels_per_step(const iblb_batch_s* b)
{
    if (b->nnodes == 0) return 1;
    return (b->dim == 3 ? 2 : 1) + 2 + (b->det ? DET_KERNELS : 1) + (b->ntt > 0 ? 2 : 0);
}

// Viscosity ratio: inside / outside of every slot that has one, from the
// interface at the start of the step (before its stream-collide).
void enqueue_classify(iblb_batch_s* b, cudaStream_t s)
{
    if (b->ntt == 0 || b->nnodes == 0) return;
    k_b_col_clear<<<dim3((b->max_ncol + 255) / 256, b->ntt), 256, 0, s>>>(b->d_slots, b->d_tt);
    const int2* items = b->dim == 2 ? b->d_nodes : b->d_faces;
    const int n = b->dim == 2 ? b->nnodes : b->nfaces;
    k_b_classify<<<(n + 127) / 128, 128, 0, s>>>(b->d_slots, items, n, b->dim);
}

// A2/A3 over all active slots: atomics, or the ordered gather.
void enqueue_spread(iblb_batch_s* b, cudaStream_t s)
{
    if (b->det)
        launch_spread_det(b->storage, b->dim, b->d_detslots, b->d_nodes, b->nnodes, b->detb,
                          b->det_nbins, b->det_ncelltiles, b->sm_count, s);
    else
        launch_b_ib(b->dim, b->storage, 1, b->d_slots, b->d_nodes, b->nnodes, b->d_faces,
                    b->nfaces, s);
}

// One batched step at parity `par` (all phases over all active slots).
void enqueue_step(iblb_batch_s* b, cudaStream_t s, int par, bool write_all)
{
    if (b->nnodes > 0) {
        launch_b_ib(b->dim, b->storage, 0, b->d_slots, b->d_nodes, b->nnodes, b->d_faces,
                    b->nfaces, s);
        enqueue_spread(b, s);
        enqueue_classify(b, s);
    }
    const int grid = std::max(1, std::min(b->ntiles, b->sm_count * b->sc_blocks_per_sm));
    launch_b_sc(b->Q, b->storage, write_all, b->any_ext, b->d_slots, b->d_tiles, b->ntiles, par,
                grid, s);
    if (b->nnodes > 0)
        launch_b_ib(b->dim, b->storage, 2, b->d_slots, b->d_nodes, b->nnodes, b->d_faces,
                    b->nfaces, s);
}

iblb_status get_graph(iblb_batch_s* b, int steps, bool last, cudaGraphExec_t* out)
{
    auto key = std::make_tuple(b->par, steps, last ? 1 : 0);
    auto it = b->graphs.find(key);
    if (it != b->graphs.end()) {
        *out = it->second;
        return IBLB_OK;
    }
    BCK(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    int par = b->par;
    for (int k = 0; k < steps; k++) {
        enqueue_step(b, b->cap, par, last && k == steps - 1);
        par ^= 1;
    }
    cudaGraph_t graph;
    cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
    if (e != cudaSuccess) return bfail(b, IBLB_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
    cudaGraphExec_t exec;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return bfail(b, IBLB_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e));
    b->graphs[key] = exec;
    *out = exec;
    return IBLB_OK;
}

int width_bucket(const iblb_config& c)
{
    int w = c.nx, k = 0;
    while (w > 1) {
        w >>= 1;
        k++;
    }
    return k * 4 + (c.lattice == IBLB_D3Q19 ? 2 : 0);
}

// Tile autotuner: time the batched stream-collide over the new slot alone
// with 1, 2 and 4 cells per thread (trial launches read the slot's current
// buffer and write only its second buffer; its band flags are all clear, so
// nothing else changes) and keep the fastest; cached per width bucket.
iblb_status tune_slot(iblb_batch_s* b, int s)
{
    Slot& sl = b->slots[s];
    const int key = width_bucket(sl.cfg);
    auto it = b->tile_cache.find(key);
    if (it != b->tile_cache.end()) {
        sl.cpt = it->second;
        return IBLB_OK;
    }
    SlotDev* d_one = nullptr;
    BItem* d_t = nullptr;
    std::vector<BItem> probe;
    {
        SlotDev d = sl.dev;
        d.cur_base = sl.buf;
        slot_items(d, 0, b_ilp(b->Q, b->storage), probe);
    }
    const long long maxt = (long long)probe.size();
    BCK(b, cudaMalloc(&d_one, sizeof(SlotDev)));
    BCK(b, cudaMalloc(&d_t, sizeof(BItem) * (size_t)maxt));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int pick = 4 * b_ilp(b->Q, b->storage);
    const int trials = 5;
    const int ilp = b_ilp(b->Q, b->storage);
    for (int cpt : {2 * ilp, 4 * ilp, 8 * ilp}) {
        SlotDev d = sl.dev;
        d.cpt = cpt;
        d.cur_base = sl.buf;
        std::vector<BItem> tl;
        slot_items(d, 0, cpt, tl);
        cudaMemcpy(d_one, &d, sizeof(SlotDev), cudaMemcpyHostToDevice);
        cudaMemcpy(d_t, tl.data(), sizeof(BItem) * tl.size(), cudaMemcpyHostToDevice);
        const int grid = std::max(1, std::min((int)tl.size(), b->sm_count * b->sc_blocks_per_sm));
        const bool mw = d.moving != 0 || d.two_tau != 0;
        launch_b_sc(b->Q, b->storage, false, mw, d_one, d_t, (int)tl.size(), 0, grid, b->stream);
        cudaEventRecord(e0, b->stream);
        for (int t = 0; t < trials; t++)
            launch_b_sc(b->Q, b->storage, false, mw, d_one, d_t, (int)tl.size(), 0, grid, b->stream);
        cudaEventRecord(e1, b->stream);
        b->launches += trials + 1;
        add_launches(trials + 1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            pick = cpt;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d_one);
    cudaFree(d_t);
    BCK(b, cudaGetLastError());
    sl.cpt = pick;
    b->tile_cache[key] = pick;
    return IBLB_OK;
}

iblb_status check_cfg(const iblb_batch_s* b, const iblb_config& c)
{
    if (c.lattice != b->Q || c.storage != b->storage) return IBLB_EINVAL;
    const int dim = c.lattice == IBLB_D2Q9 ? 2 : 3;
    const int nz = dim == 2 ? 1 : c.nz;
    if (c.nx < 1 || c.ny < 1 || nz < 1) return IBLB_EINVAL;
    if (!c.walls) return IBLB_EINVAL;  // droplets at a wall
    if ((dim == 2 ? c.ny : nz) < 3) return IBLB_EINVAL;
    if (!(c.tau > 0.5)) return IBLB_EINVAL;
    if (c.wetting && (!(c.xi > 0.0) || !(c.pi_n > c.pi_m) || c.pi_m < 2)) return IBLB_EINVAL;
    // the stream-collide kernel indexes a slot's populations with 32 bits
    if ((double)c.lattice * c.nx * c.ny * nz >= 4294967296.0) return IBLB_EINVAL;
    if (c.body_force[0] != 0.0 || c.body_force[1] != 0.0 || c.body_force[2] != 0.0)
        return IBLB_EINVAL;  // the batched kernel has no body force
    if (c.tau_out != 0.0 && !(c.tau_out > 0.5)) return IBLB_EINVAL;
    if (!(c.shear_modulus >= 0.0) || !std::isfinite(c.shear_modulus) || !(c.skalak_c > -0.5) ||
        !std::isfinite(c.skalak_c))
        return IBLB_EINVAL;
    for (int k = 0; k < 3; k++)  // as iblb_create: |u_w| <= 0.3
        for (double u : {c.wall_u_lo[k], c.wall_u_hi[k]})
            if (!std::isfinite(u) || std::fabs(u) > 0.3) return IBLB_EINVAL;
    // moving walls are tangential: no velocity along the wall axis
    if (c.wall_u_lo[dim - 1] != 0.0 || c.wall_u_hi[dim - 1] != 0.0) return IBLB_EINVAL;
    if (dim == 2 && (c.wall_u_lo[2] != 0.0 || c.wall_u_hi[2] != 0.0)) return IBLB_EINVAL;
    return IBLB_OK;
}

}  // namespace

extern "C" {

size_t iblb_batch_footprint(const iblb_config* c, int n_nodes, int n_faces)
{
    if (!c) return 0;
    const int dim = c->lattice == IBLB_D2Q9 ? 2 : 3;
    const int nz = dim == 2 ? 1 : c->nz;
    const size_t elt = c->storage == IBLB_FP64 ? 8 : (c->storage == IBLB_FP32_DEV ? 4 : 2);
    const size_t relt = c->storage == IBLB_FP64 ? 8 : 4;
    const long long ncell = (long long)c->nx * c->ny * nz;
    const bool two_tau = c->tau_out != 0.0 && c->tau_out != c->tau;
    const int ncol = two_tau ? (dim == 2 ? c->nx : c->nx * c->ny) : 0;
    return slot_layout(c->lattice, dim, elt, relt, ncell, c->nx, n_nodes, n_faces,
                       c->shear_modulus != 0.0, ncol).total;
}

iblb_status iblb_batch_create(int lattice, int storage, size_t hbm_budget_bytes, int max_slots,
                              void* cuda_stream, iblb_batch* out)
{
    if (!out) return IBLB_EINVAL;
    *out = nullptr;
    if (lattice != IBLB_D2Q9 && lattice != IBLB_D3Q19) return IBLB_EINVAL;
    if (storage < IBLB_FP64 || storage > IBLB_FP16_DEV) return IBLB_EINVAL;
    if (max_slots < 1 || max_slots > (1 << 20) || hbm_budget_bytes < ALIGN) return IBLB_EINVAL;
    (void)cudaGetLastError();
    iblb_batch_s* b = new iblb_batch_s();
    b->Q = lattice;
    b->dim = lattice == IBLB_D2Q9 ? 2 : 3;
    b->storage = storage;
    b->elt = storage == IBLB_FP64 ? 8 : (storage == IBLB_FP32_DEV ? 4 : 2);
    b->relt = storage == IBLB_FP64 ? 8 : 4;
    b->stream = (cudaStream_t)cuda_stream;
    b->slots.resize(max_slots);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) b->sc_blocks_per_sm = b_sc_blocks_per_sm(lattice, storage);
    const size_t budget = hbm_budget_bytes / ALIGN * ALIGN;
    if (e == cudaSuccess) e = cudaMalloc(&b->arena_ptr, budget);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_slots, sizeof(SlotDev) * max_slots);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_partial, sizeof(double) * 1024);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_obs, sizeof(double) * 12);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        iblb_batch_destroy(b);
        return e == cudaErrorMemoryAllocation ? IBLB_ENOMEM : IBLB_ECUDA;
    }
    b->arena.reset(budget);
    *out = b;
    return IBLB_OK;
}

void iblb_batch_destroy(iblb_batch b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    clear_graphs(b);
    cudaFree(b->arena_ptr);
    cudaFree(b->d_slots);
    cudaFree(b->d_tiles);
    cudaFree(b->d_nodes);
    cudaFree(b->d_faces);
    cudaFree(b->d_tt);
    cudaFree(b->d_detslots);
    cudaFree(b->detb.cnt);
    cudaFree(b->detb.start);
    cudaFree(b->detb.cur);
    cudaFree(b->detb.active);
    cudaFree(b->detb.act_list);
    cudaFree(b->detb.nact);
    cudaFree(b->detb.bin_of);
    cudaFree(b->detb.org);
    cudaFree(b->detb.list);
    cudaFree(b->detb.wts);
    cudaFree(b->d_partial);
    cudaFree(b->d_obs);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
}

const char* iblb_batch_last_error(iblb_batch b) { return b ? b->msg.c_str() : "null batch"; }

iblb_status iblb_batch_admit(iblb_batch b, const iblb_config* cfg, const double* xyz, int n_nodes,
                             const int* tri, int n_faces, long long n_steps, int* slot_out)
{
    if (!b || !cfg || !slot_out) return IBLB_EINVAL;
    *slot_out = -1;
    if (check_cfg(b, *cfg) != IBLB_OK) return bfail(b, IBLB_EINVAL, "configuration not valid for this batch");
    if (n_steps < 1 || n_nodes < 3 || !xyz) return bfail(b, IBLB_EINVAL, "bad steps or nodes");
    const int dim = b->dim;
    if (dim == 3 && (!tri || n_faces < 1)) return bfail(b, IBLB_EINVAL, "3D interfaces need triangles");
    if (dim == 2 && tri) return bfail(b, IBLB_EINVAL, "2D interfaces are rings: tri must be NULL");
    for (long long k = 0; k < (long long)n_nodes * dim; k++)
        if (!std::isfinite(xyz[k])) return bfail(b, IBLB_EINVAL, "non-finite node coordinate");
    if (cfg->wetting)
        for (int j = 0; j < n_nodes; j++)
            if (!(xyz[dim * j + dim - 1] - 0.5 > 0.0))
                return bfail(b, IBLB_ENODE_IN_WALL, "a node lies at or below the wall plane");
    std::vector<int> ptr, epos;
    if (dim == 3) {
        for (long long k = 0; k < 3LL * n_faces; k++)
            if (tri[k] < 0 || tri[k] >= n_nodes) return bfail(b, IBLB_EINVAL, "triangle index out of range");
        ptr.assign(n_nodes + 1, 0);
        for (long long k = 0; k < 3LL * n_faces; k++) ptr[tri[k] + 1]++;
        for (int j = 0; j < n_nodes; j++) ptr[j + 1] += ptr[j];
        for (int j = 0; j < n_nodes; j++)
            if (ptr[j + 1] == ptr[j]) return bfail(b, IBLB_EINVAL, "a node belongs to no face");
        epos.resize(3LL * n_faces);
        std::vector<int> fill(ptr.begin(), ptr.end() - 1);
        for (int f = 0; f < n_faces; f++)
            for (int v = 0; v < 3; v++) epos[3 * f + v] = fill[tri[3 * f + v]]++;
    }
    int s = -1;
    for (size_t k = 0; k < b->slots.size(); k++)
        if (!b->slots[k].used) {
            s = (int)k;
            break;
        }
    if (s < 0) return bfail(b, IBLB_EAGAIN, "no free slot");
    const int nz = dim == 2 ? 1 : cfg->nz;
    GridParams g{};
    g.nx = cfg->nx;
    g.ny = cfg->ny;
    g.nz = nz;
    g.dim = dim;
    g.walls = 1;
    g.nseg_x = (cfg->nx + 31) / 32;
    g.ncell = (long long)cfg->nx * cfg->ny * nz;
    const long long nfluid = dim == 2 ? (long long)cfg->nx * (cfg->ny - 2)
                                      : (long long)cfg->nx * cfg->ny * (nz - 2);
    const bool elastic = cfg->shear_modulus != 0.0;
    const bool two_tau = cfg->tau_out != 0.0 && cfg->tau_out != cfg->tau;
    const int ncol = two_tau ? (dim == 2 ? cfg->nx : cfg->nx * cfg->ny) : 0;
    const Layout L = slot_layout(b->Q, dim, b->elt, b->relt, g.ncell, cfg->nx, n_nodes,
                                 dim == 3 ? n_faces : 0, elastic, ncol);
    size_t off = 0;
    if (!b->arena.alloc(L.total, &off)) return bfail(b, IBLB_EAGAIN, "no room in the HBM budget");
    Slot& sl = b->slots[s];
    sl = Slot();
    sl.used = true;
    sl.cfg = *cfg;
    sl.cfg.nz = nz;
    sl.steps_total = n_steps;
    sl.off = off;
    sl.bytes = L.total;
    unsigned char* base = b->arena_ptr + off;
    SlotDev& d = sl.dev;
    d.f[0] = base + L.pop[0];
    d.f[1] = base + L.pop[1];
    d.mom = base + L.mom;
    d.F = base + L.F;
    d.flags = base + L.flags;
    d.err = (int*)(base + L.err);
    d.rng = (unsigned*)(base + L.rng);
    d.g = g;
    d.nfluid = nfluid;
    d.omega = 1.0 / cfg->tau;
    d.omega_f = (float)d.omega;
    const int sexp = cfg->fp16_scale_exp ? cfg->fp16_scale_exp : 16;
    d.scale = b->storage == IBLB_FP16_DEV ? std::ldexp(1.0f, sexp) : 1.0f;
    d.inv_scale = 1.0f / d.scale;
    d.q = (double*)(base + L.q);
    d.phi = (double*)(base + L.phi);
    d.N = n_nodes;
    d.M = dim == 3 ? n_faces : n_nodes;
    d.fp.sigma = cfg->sigma;
    d.fp.xi = cfg->xi;
    d.fp.n = cfg->pi_n;
    d.fp.m = cfg->pi_m;
    d.fp.wetting = cfg->wetting ? 1 : 0;
    d.fp.A = cfg->wetting ? wetting_A(*cfg) : 0.0;
    d.fp.wall_plane = 0.5;
    d.fp.Gs = cfg->shear_modulus;
    d.fp.Cs = cfg->skalak_c;
    d.two_tau = two_tau ? 1 : 0;
    d.ncol = ncol;
    d.omega_out = two_tau ? 1.0 / cfg->tau_out : d.omega;
    d.omega_out_f = (float)d.omega_out;
    d.col_cnt = two_tau ? (int*)(base + L.cols) : nullptr;
    d.col_z = two_tau ? (double*)(base + L.colz) : nullptr;
    d.moving = 0;
    for (int k = 0; k < 3; k++) {
        d.uw_lo[k] = k < dim ? cfg->wall_u_lo[k] : 0.0;
        d.uw_hi[k] = k < dim ? cfg->wall_u_hi[k] : 0.0;
        if (d.uw_lo[k] != 0.0 || d.uw_hi[k] != 0.0) d.moving = 1;
    }
    d.fp.eref = elastic ? (const double*)(base + L.eref) : nullptr;
    if (dim == 3) {
        d.tri = (int*)(base + L.tri);
        d.csr_ptr = (int*)(base + L.csr);
        d.entry_pos = (int*)(base + L.epos);
        d.entry_rec = (double*)(base + L.erec);
    }
    // rest state and cleared buffers, then the interface
    cudaError_t e = cudaMemsetAsync(base, 0, L.total, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d.q, xyz, sizeof(double) * (size_t)n_nodes * dim, cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess && dim == 3) {
        e = cudaMemcpyAsync(d.tri, tri, sizeof(int) * 3 * (size_t)n_faces, cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d.csr_ptr, ptr.data(), sizeof(int) * ptr.size(), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d.entry_pos, epos.data(), sizeof(int) * epos.size(), cudaMemcpyHostToDevice, b->stream);
    }
    if (e == cudaSuccess) {
        launch_init_moments(b->storage, g, d.mom, b->stream);
        b->launches++;
        add_launches(1);
        if (elastic) {  // the interface as admitted is the elastic reference shape
            launch_elastic_reference(dim, d.q, n_nodes, dim == 3 ? n_faces : 0, d.tri,
                                     (double*)(base + L.eref), b->stream);
            b->launches++;
            add_launches(1);
        }
        e = cudaStreamSynchronize(b->stream);
    }
    if (e != cudaSuccess) {
        b->arena.release(off, L.total);
        sl = Slot();
        return bfail(b, IBLB_ECUDA, std::string("admit: ") + cudaGetErrorString(e));
    }
    iblb_status st = tune_slot(b, s);
    if (st != IBLB_OK) return st;
    sl.active = true;
    b->dirty = true;
    *slot_out = s;
    return IBLB_OK;
}

}  // extern "C"

namespace {

// Algorithmic HBM bytes of one batched stream-collide launch over the active
// slots: populations read once and written once per fluid cell.
double active_stream_bytes(const iblb_batch_s* b)
{
    double t = 0.0;
    for (const auto& sl : b->slots)
        if (sl.active) t += 2.0 * b->Q * (double)b->elt * (double)sl.dev.nfluid;
    return t;
}

// Advance every active slot by up to max_steps steps.  Without `kernel_ms`
// the steps run as CUDA-graph chunks; with it, one launch at a time with a
// CUDA event pair around each phase (forces, spread, stream-collide,
// interpolate + advect), summed into kernel_ms, and the algorithmic bytes of
// the stream-collide launches summed into *sc_bytes.
iblb_status batch_run(iblb_batch_s* b, int max_steps, int* n_completed, double* kernel_ms,
                      double* sc_bytes)
{
    int completed = 0;
    int left = max_steps;
    constexpr int PHASES = 4;  // forces, spread, stream-collide, interpolation
    cudaEvent_t ev[PHASES + 1] = {};
    if (kernel_ms) {
        for (int k = 0; k < IBLB_K_COUNT; k++) kernel_ms[k] = 0.0;
        if (sc_bytes) *sc_bytes = 0.0;
        for (auto& e : ev) BCK(b, cudaEventCreate(&e));
    }
    iblb_status st = IBLB_OK;
    while (left > 0 && st == IBLB_OK) {
        if (b->dirty) {
            st = rebuild(b);
            if (st != IBLB_OK) break;
        }
        if (b->nactive == 0) break;
        long long r = left;
        for (auto& sl : b->slots)
            if (sl.active) r = std::min(r, sl.steps_total - sl.steps_done);
        int seg = (int)r;
        // segment of `seg` steps, the last one writing every cell's moments
        if (!kernel_ms) {
            int done_here = 0;
            while (done_here < seg) {
                const int k = std::min(32, seg - done_here);
                const bool last = (done_here + k == seg);
                cudaGraphExec_t ge;
                st = get_graph(b, k, last, &ge);
                if (st != IBLB_OK) break;
                cudaError_t e = cudaGraphLaunch(ge, b->stream);
                if (e != cudaSuccess) {
                    st = bfail(b, IBLB_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
                    break;
                }
                b->launches += (long long)k * kernels_per_step(b);
                add_launches((long long)k * kernels_per_step(b));
                b->par ^= (k & 1);
                done_here += k;
            }
            if (st != IBLB_OK) break;
        } else {
            const double bytes = active_stream_bytes(b);
            const int grid = std::max(1, std::min(b->ntiles, b->sm_count * b->sc_blocks_per_sm));
            for (int k = 0; k < seg; k++) {
                const bool last = (k == seg - 1);
                cudaEventRecord(ev[0], b->stream);
                if (b->nnodes > 0)
                    launch_b_ib(b->dim, b->storage, 0, b->d_slots, b->d_nodes, b->nnodes,
                                b->d_faces, b->nfaces, b->stream);
                cudaEventRecord(ev[1], b->stream);
                if (b->nnodes > 0) {
                    enqueue_spread(b, b->stream);
                    enqueue_classify(b, b->stream);
                }
                cudaEventRecord(ev[2], b->stream);
                launch_b_sc(b->Q, b->storage, last, b->any_ext, b->d_slots, b->d_tiles,
                            b->ntiles, b->par, grid, b->stream);
                cudaEventRecord(ev[3], b->stream);
                if (b->nnodes > 0)
                    launch_b_ib(b->dim, b->storage, 2, b->d_slots, b->d_nodes, b->nnodes,
                                b->d_faces, b->nfaces, b->stream);
                cudaEventRecord(ev[4], b->stream);
                b->par ^= 1;
                b->launches += kernels_per_step(b);
                add_launches(kernels_per_step(b));
                cudaError_t e = cudaEventSynchronize(ev[4]);
                if (e != cudaSuccess) {
                    st = bfail(b, IBLB_ECUDA, std::string("profiled step: ") + cudaGetErrorString(e));
                    break;
                }
                for (int q = 0; q < PHASES; q++) {
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, ev[q], ev[q + 1]);
                    kernel_ms[q] += ms;
                }
                if (sc_bytes) *sc_bytes += bytes;
            }
            if (st != IBLB_OK) break;
        }
        for (auto& sl : b->slots) {
            if (!sl.active) continue;
            sl.steps_done += seg;
            sl.buf ^= (seg & 1);
            if (sl.steps_done >= sl.steps_total) {
                sl.active = false;
                sl.done = true;
                b->dirty = true;
                completed++;
            }
        }
        left -= seg;
    }
    if (kernel_ms)
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
    if (n_completed) *n_completed = completed;
    if (st != IBLB_OK) return st;
    BCK(b, cudaGetLastError());
    return IBLB_OK;
}

}  // namespace

extern "C" {

iblb_status iblb_batch_run(iblb_batch b, int max_steps, int* n_completed)
{
    if (!b || max_steps < 0) return IBLB_EINVAL;
    return batch_run(b, max_steps, n_completed, nullptr, nullptr);
}

iblb_status iblb_batch_run_profiled(iblb_batch b, int max_steps, int* n_completed,
                                    double* kernel_ms, double* stream_collide_bytes)
{
    if (!b || max_steps < 0 || !kernel_ms) return IBLB_EINVAL;
    return batch_run(b, max_steps, n_completed, kernel_ms, stream_collide_bytes);
}

iblb_status iblb_batch_sync(iblb_batch b)
{
    if (!b) return IBLB_EINVAL;
    BCK(b, cudaStreamSynchronize(b->stream));
    return IBLB_OK;
}

iblb_status iblb_batch_poll(iblb_batch b, int* done_slots, int cap, int* n_done)
{
    if (!b || !n_done || (cap > 0 && !done_slots)) return IBLB_EINVAL;
    int n = 0;
    for (size_t s = 0; s < b->slots.size(); s++)
        if (b->slots[s].used && b->slots[s].done) {
            if (n < cap) done_slots[n] = (int)s;
            n++;
        }
    *n_done = n;
    return IBLB_OK;
}

iblb_status iblb_batch_slot_status(iblb_batch b, int slot, long long* steps_done)
{
    if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].used) return IBLB_EINVAL;
    Slot& sl = b->slots[slot];
    if (steps_done) *steps_done = sl.steps_done;
    int e = 0;
    BCK(b, cudaMemcpyAsync(&e, sl.dev.err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    if (e & ERR_NODE_IN_WALL) return bfail(b, IBLB_ENODE_IN_WALL, "slot: node in the wall");
    if (e & ERR_NONFINITE) return bfail(b, IBLB_ENONFINITE, "slot: non-finite density");
    return IBLB_OK;
}

iblb_status iblb_batch_observables(iblb_batch b, int slot, iblb_obs* out)
{
    if (!b || !out || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].used)
        return IBLB_EINVAL;
    Slot& sl = b->slots[slot];
    const SlotDev& d = sl.dev;
    launch_mass_partials(b->Q, b->storage, d.f[sl.buf], d.g, d.inv_scale, b->d_partial, b->stream);
    launch_observables(b->dim, d.q, d.N, b->dim == 3 ? d.tri : nullptr, d.M, b->d_partial,
                       mass_partial_blocks(d.g), sl.cfg.xi, 0.5, b->d_obs, b->stream);
    b->launches += 2;
    add_launches(2);
    BCK(b, cudaGetLastError());
    double v[12];
    BCK(b, cudaMemcpyAsync(v, b->d_obs, sizeof(v), cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    out->mass = v[0];
    out->volume = v[1];
    out->height = v[2];
    out->theta_deg = v[3];
    out->r_cl = v[4];
    out->film = v[5];
    out->d_min = v[6];
    out->centre[0] = v[7];
    out->centre[1] = v[8];
    out->centre[2] = v[9];
    out->radius = v[10];
    return iblb_batch_slot_status(b, slot, nullptr);
}

iblb_status iblb_batch_read_fields(iblb_batch b, int slot, double* rho, double* u, double* xyz)
{
    if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].used) return IBLB_EINVAL;
    Slot& sl = b->slots[slot];
    const SlotDev& d = sl.dev;
    const long long nc = d.g.ncell;
    if (rho || u) {
        double* tmp = nullptr;
        BCK(b, cudaMalloc(&tmp, sizeof(double) * (size_t)(1 + b->dim) * nc));
        launch_unpack_moments(b->storage, d.g, d.mom, tmp, tmp + nc, b->stream);
        b->launches++;
        add_launches(1);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess && rho)
            e = cudaMemcpyAsync(rho, tmp, sizeof(double) * nc, cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess && u)
            e = cudaMemcpyAsync(u, tmp + nc, sizeof(double) * b->dim * nc, cudaMemcpyDeviceToHost,
                                b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        cudaFree(tmp);
        if (e != cudaSuccess) return bfail(b, IBLB_ECUDA, cudaGetErrorString(e));
    }
    if (xyz)
        BCK(b, cudaMemcpyAsync(xyz, d.q, sizeof(double) * d.N * b->dim, cudaMemcpyDeviceToHost,
                               b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    return iblb_batch_slot_status(b, slot, nullptr);
}

iblb_status iblb_batch_release(iblb_batch b, int slot)
{
    if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].used) return IBLB_EINVAL;
    BCK(b, cudaStreamSynchronize(b->stream));
    Slot& sl = b->slots[slot];
    b->arena.release(sl.off, sl.bytes);
    const bool was_active = sl.active;
    sl = Slot();
    if (was_active) b->dirty = true;
    return IBLB_OK;
}

iblb_status iblb_batch_stats(iblb_batch b, iblb_batch_info* info)
{
    if (!b || !info) return IBLB_EINVAL;
    int used = 0, active = 0, done = 0;
    for (auto& sl : b->slots) {
        used += sl.used;
        active += sl.active;
        done += sl.done;
    }
    info->slots_used = used;
    info->slots_active = active;
    info->slots_done = done;
    info->arena_bytes = b->arena.size;
    info->free_bytes = b->arena.free_bytes();
    info->kernel_launches = b->launches;
    return IBLB_OK;
}

long long iblb_batch_steps_to_next_completion(iblb_batch b)
{
    if (!b) return -1;
    long long r = -1;
    for (const auto& sl : b->slots)
        if (sl.active) {
            const long long left = sl.steps_total - sl.steps_done;
            if (r < 0 || left < r) r = left;
        }
    return r;
}

int iblb_batch_slot_tile(iblb_batch b, int slot)
{
    if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].used) return -1;
    return b->slots[slot].cpt;
}

}  // extern "C"
