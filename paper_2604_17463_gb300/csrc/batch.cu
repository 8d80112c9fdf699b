// batch.cu -- batched engine (many independent droplet simulations advanced
// by shared launches) and the admission side of the serving loop.
//
// A batch holds simulations ("slots") of one lattice type and one population
// storage form.  Each time step runs the same phases as a single simulation
// (nodal forces, spread, stream-collide, interpolate + advect; Sec. 2 of the
// paper), but every phase is ONE launch over all active slots:
//   - stream-collide: a persistent kernel whose blocks fetch (slot, tile) work
//     items from a list with an atomic counter; a tile is 128 x cpt consecutive
//     fluid cells of one slot, cpt (cells per thread) chosen per slot by the
//     tile autotuner;
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
#include "ib_core.cuh"
#include "lbm_core.cuh"

namespace iblb {

struct SlotDev {
    void* f[2];
    void* mom;
    void* F;
    uint8_t* flags;        // one byte per 32 fluid cells (fluid-cell index)
    int* err;
    GridParams g;
    long long nfluid;      // fluid cells
    long long fluid_off;   // cell index of the first fluid cell
    double omega;
    float omega_f, scale, inv_scale;
    int cur_base;          // current buffer = cur_base ^ batch parity
    unsigned* rng;         // two-entry step counter for binary16 stochastic rounding
    int cpt;               // cells per thread of this slot's tiles
    double* q;
    double* phi;
    int N, M;
    int* tri;
    int* csr_ptr;
    int* entry_pos;
    double* entry_rec;
    ForceParams fp;
};

namespace {

constexpr int BT = 128;  // threads per stream-collide block

template <int Q, int ST, bool WRITE_ALL>
__global__ void __launch_bounds__(BT)
k_b_stream_collide(const SlotDev* __restrict__ slots, const int2* __restrict__ tiles, int ntiles,
                   int par, unsigned* counter)
{
    using T = StorageT<ST>;
    using S = typename T::S;
    using R = typename T::R;
    using L = Stencil<Q>;
    constexpr int D = L::D;
    __shared__ int s_tile;
    const int lane = threadIdx.x & 31;
    for (;;) {
        if (threadIdx.x == 0) s_tile = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int t = s_tile;
        __syncthreads();
        if (t >= ntiles) break;
        const int2 td = tiles[t];
        const SlotDev& sd = slots[td.x];
        const int cur = sd.cur_base ^ par;
        unsigned step = 0;
        if constexpr (ST == ST_FP16)  // the slot's first tile advances its counter
            step = sr_step(sd.rng + cur, sd.rng + (cur ^ 1), td.y == 0 && threadIdx.x == 0);
        const S* fin = (const S*)sd.f[cur];
        S* fout = (S*)sd.f[cur ^ 1];
        R* mom = (R*)sd.mom;
        R* F = (R*)sd.F;
        const GridParams g = sd.g;
        const long long nc = g.ncell;
        for (int c = 0; c < sd.cpt; c++) {
            const long long f = (long long)td.y + (long long)c * BT + threadIdx.x;
            const bool valid = f < sd.nfluid;
            const long long seg = f >> 5;
            int band = 0;
            if (lane == 0 && valid) band = sd.flags[seg];
            band = __shfl_sync(0xffffffffu, band, 0);
            if (!valid) continue;
            const long long cell = sd.fluid_off + f;
            const long long row = cell / g.nx;
            const int x = (int)(cell - row * g.nx);
            int y, z;
            if (D == 2) {
                y = (int)row;
                z = 0;
            } else {
                y = (int)(row % g.ny);
                z = (int)(row / g.ny);
            }
            R gv[Q];
            pull_cell<Q, ST>(fin, g, x, y, z, cell, sd.inv_scale, gv);
            R Fx = 0, Fy = 0, Fz = 0;
            if (band) {
                Fx = F[cell];
                Fy = F[nc + cell];
                F[cell] = 0;
                F[nc + cell] = 0;
                if (D == 3) {
                    Fz = F[2 * nc + cell];
                    F[2 * nc + cell] = 0;
                }
            }
            const R omega = (R)sd.omega;
            const CellMoments<Q, R> mo = cell_moments<Q, R>(gv, Fx, Fy, Fz);
            cell_collide<Q, R>(gv, mo, omega, Fx, Fy, Fz);
            store_cell<Q, ST, false>(fout, nc, cell, gv, sd.scale,
                                     ST == ST_FP16 ? sr_seed(step, cell) : 0u);
            if (WRITE_ALL || band) {
                mom[cell] = mo.drho;
                mom[nc + cell] = mo.ux;
                mom[2 * nc + cell] = mo.uy;
                if (D == 3) mom[3 * nc + cell] = mo.uz;
            }
            if (!isfinite(mo.drho)) atomicOr(sd.err, ERR_NONFINITE);
            if (lane == 0 && band) sd.flags[seg] = 0;
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
    face_records(sd.q, sd.tri, fd.y, sd.entry_pos, sd.entry_rec);
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

// One warp per (slot, node): scatter-add into the slot's force density and
// mark its fluid-cell segments.
template <int D, typename R>
__global__ void k_b_spread(const SlotDev* __restrict__ slots, const int2* __restrict__ nodes,
                           int nnodes)
{
    constexpr int S = (D == 2) ? 16 : 64;
    constexpr int PPL = (S + 31) / 32;
    const int item = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (item >= nnodes) return;  // uniform per warp
    const int2 nd = nodes[item];
    const SlotDev& sd = slots[nd.x];
    const GridParams g = sd.g;
    R wk;
    int ik;
    node_weights<D, R>(g, sd.q, nd.y, lane, wk, ik);
    R phl = R(0);
    if (lane < D) phl = (R)sd.phi[D * nd.y + lane];
    R ph[3];
    for (int k = 0; k < D; k++) ph[k] = __shfl_sync(0xffffffffu, phl, k);
    R* F = (R*)sd.F;
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
            sd.flags[(cell - sd.fluid_off) >> 5] = 1;
        }
    }
}

template <int D, typename R>
__global__ void k_b_interp(const SlotDev* __restrict__ slots, const int2* __restrict__ nodes,
                           int nnodes)
{
    constexpr int S = (D == 2) ? 16 : 64;
    constexpr int PPL = (S + 31) / 32;
    const int item = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (item >= nnodes) return;
    const int2 nd = nodes[item];
    const SlotDev& sd = slots[nd.x];
    const GridParams g = sd.g;
    R wk;
    int ik;
    node_weights<D, R>(g, sd.q, nd.y, lane, wk, ik);
    const R* mom = (const R*)sd.mom;
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
        sd.q[D * nd.y + lane] += (double)a;
    }
}

}  // namespace

// ------------------------------------------------------------------ launchers
static void launch_b_sc(int Q, int storage, bool write_all, const SlotDev* slots,
                        const int2* tiles, int ntiles, int par, unsigned* counter, int grid,
                        cudaStream_t s)
{
#define IBLB_BSC(QQ, SS)                                                                       \
    do {                                                                                       \
        if (write_all)                                                                         \
            k_b_stream_collide<QQ, SS, true><<<grid, BT, 0, s>>>(slots, tiles, ntiles, par, counter); \
        else                                                                                   \
            k_b_stream_collide<QQ, SS, false><<<grid, BT, 0, s>>>(slots, tiles, ntiles, par, counter); \
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

static void launch_b_ib(int dim, int storage, int phase, const SlotDev* slots, const int2* nodes,
                        int nnodes, const int2* faces, int nfaces, cudaStream_t s)
{
    const int wb = 128;
    const int warps_grid = (int)(((long long)nnodes * 32 + wb - 1) / wb);
    if (phase == 0) {  // nodal forces
        if (dim == 2) {
            k_b_forces_ring<<<(nnodes + 127) / 128, 128, 0, s>>>(slots, nodes, nnodes);
        } else {
            if (nfaces > 0) k_b_face_geometry<<<(nfaces + 63) / 64, 64, 0, s>>>(slots, faces, nfaces);
            k_b_node_forces<<<(nnodes + 63) / 64, 64, 0, s>>>(slots, nodes, nnodes);
        }
    } else if (phase == 1) {  // spread
        if (storage == ST_FP64) {
            if (dim == 2) k_b_spread<2, double><<<warps_grid, wb, 0, s>>>(slots, nodes, nnodes);
            else k_b_spread<3, double><<<warps_grid, wb, 0, s>>>(slots, nodes, nnodes);
        } else {
            if (dim == 2) k_b_spread<2, float><<<warps_grid, wb, 0, s>>>(slots, nodes, nnodes);
            else k_b_spread<3, float><<<warps_grid, wb, 0, s>>>(slots, nodes, nnodes);
        }
    } else {  // interpolate + advect
        if (storage == ST_FP64) {
            if (dim == 2) k_b_interp<2, double><<<warps_grid, wb, 0, s>>>(slots, nodes, nnodes);
            else k_b_interp<3, double><<<warps_grid, wb, 0, s>>>(slots, nodes, nnodes);
        } else {
            if (dim == 2) k_b_interp<2, float><<<warps_grid, wb, 0, s>>>(slots, nodes, nnodes);
            else k_b_interp<3, float><<<warps_grid, wb, 0, s>>>(slots, nodes, nnodes);
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
    size_t pop[2], mom, F, flags, err, rng, q, phi, tri, csr, epos, erec, total;
};

Layout slot_layout(int Q, int dim, size_t elt, size_t relt, long long ncell, long long nfluid,
                   int N, int M)
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
    L.mom = take((size_t)(1 + dim) * ncell * relt);
    L.F = take((size_t)dim * ncell * relt);
    L.flags = take((size_t)((nfluid + 31) / 32));
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
    int2* d_tiles = nullptr;
    int2* d_nodes = nullptr;
    int2* d_faces = nullptr;
    size_t cap_tiles = 0, cap_nodes = 0, cap_faces = 0;
    int ntiles = 0, nnodes = 0, nfaces = 0, nactive = 0;
    unsigned* d_counter = nullptr;
    double* d_partial = nullptr;
    double* d_obs = nullptr;
    int par = 0;
    bool dirty = true;
    int sm_count = 0;
    std::map<std::tuple<int, int, int>, cudaGraphExec_t> graphs;
    std::map<int, int> tile_cache;  // width bucket -> cells per thread
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

// Rebuild the slot descriptors and the work lists of the active slots.
iblb_status rebuild(iblb_batch_s* b)
{
    std::vector<int2> tiles, nodes, faces;
    std::vector<SlotDev> devs(b->slots.size());
    for (size_t s = 0; s < b->slots.size(); s++) {
        Slot& sl = b->slots[s];
        if (!sl.used) continue;
        sl.dev.cur_base = sl.buf ^ b->par;
        sl.dev.cpt = sl.cpt;
        devs[s] = sl.dev;
        if (!sl.active) continue;
        const long long tile = (long long)BT * sl.cpt;
        for (long long f0 = 0; f0 < sl.dev.nfluid; f0 += tile) tiles.push_back(make_int2((int)s, (int)f0));
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
        BCK(b, cudaMemcpy(b->d_tiles, tiles.data(), sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice));
    if (!nodes.empty())
        BCK(b, cudaMemcpy(b->d_nodes, nodes.data(), sizeof(int2) * nodes.size(), cudaMemcpyHostToDevice));
    if (!faces.empty())
        BCK(b, cudaMemcpy(b->d_faces, faces.data(), sizeof(int2) * faces.size(), cudaMemcpyHostToDevice));
    b->ntiles = (int)tiles.size();
    b->nnodes = (int)nodes.size();
    b->nfaces = (int)faces.size();
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
    return (b->dim == 3 ? 2 : 1) + 3;
}

// One batched step at parity `par` (all phases over all active slots).
void enqueue_step(iblb_batch_s* b, cudaStream_t s, int par, bool write_all)
{
    if (b->nnodes > 0) {
        launch_b_ib(b->dim, b->storage, 0, b->d_slots, b->d_nodes, b->nnodes, b->d_faces,
                    b->nfaces, s);
        launch_b_ib(b->dim, b->storage, 1, b->d_slots, b->d_nodes, b->nnodes, b->d_faces,
                    b->nfaces, s);
    }
    cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned), s);
    const int grid = std::max(1, std::min(b->ntiles, b->sm_count * 16));
    launch_b_sc(b->Q, b->storage, write_all, b->d_slots, b->d_tiles, b->ntiles, par, b->d_counter,
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
    int2* d_t = nullptr;
    unsigned* d_c = nullptr;
    const long long maxt = (sl.dev.nfluid + BT - 1) / BT;
    BCK(b, cudaMalloc(&d_one, sizeof(SlotDev)));
    BCK(b, cudaMalloc(&d_t, sizeof(int2) * (size_t)maxt));
    BCK(b, cudaMalloc(&d_c, sizeof(unsigned)));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int pick = 1;
    const int trials = 5;
    for (int cpt : {1, 2, 4}) {
        SlotDev d = sl.dev;
        d.cpt = cpt;
        d.cur_base = sl.buf;
        std::vector<int2> tl;
        for (long long f0 = 0; f0 < d.nfluid; f0 += (long long)BT * cpt) tl.push_back(make_int2(0, (int)f0));
        cudaMemcpy(d_one, &d, sizeof(SlotDev), cudaMemcpyHostToDevice);
        cudaMemcpy(d_t, tl.data(), sizeof(int2) * tl.size(), cudaMemcpyHostToDevice);
        const int grid = std::max(1, std::min((int)tl.size(), b->sm_count * 16));
        cudaMemsetAsync(d_c, 0, sizeof(unsigned), b->stream);
        launch_b_sc(b->Q, b->storage, false, d_one, d_t, (int)tl.size(), 0, d_c, grid, b->stream);
        cudaEventRecord(e0, b->stream);
        for (int t = 0; t < trials; t++) {
            cudaMemsetAsync(d_c, 0, sizeof(unsigned), b->stream);
            launch_b_sc(b->Q, b->storage, false, d_one, d_t, (int)tl.size(), 0, d_c, grid,
                        b->stream);
        }
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
    cudaFree(d_c);
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
    if (c.body_force[0] != 0.0 || c.body_force[1] != 0.0 || c.body_force[2] != 0.0)
        return IBLB_EINVAL;  // the batched kernel has no body force
    if (c.tau_out != 0.0 && c.tau_out != c.tau)
        return IBLB_EINVAL;  // nor a viscosity ratio
    for (int k = 0; k < 3; k++)
        if (c.wall_u_lo[k] != 0.0 || c.wall_u_hi[k] != 0.0)
            return IBLB_EINVAL;  // nor moving walls
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
    const long long nfluid = dim == 2 ? (long long)c->nx * (c->ny - 2)
                                      : (long long)c->nx * c->ny * (nz - 2);
    return slot_layout(c->lattice, dim, elt, relt, ncell, nfluid, n_nodes, n_faces).total;
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
    const size_t budget = hbm_budget_bytes / ALIGN * ALIGN;
    if (e == cudaSuccess) e = cudaMalloc(&b->arena_ptr, budget);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_slots, sizeof(SlotDev) * max_slots);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, sizeof(unsigned));
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
    cudaFree(b->d_counter);
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
    const Layout L = slot_layout(b->Q, dim, b->elt, b->relt, g.ncell, nfluid, n_nodes,
                                 dim == 3 ? n_faces : 0);
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
    d.fluid_off = dim == 2 ? (long long)cfg->nx : (long long)cfg->nx * cfg->ny;
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

iblb_status iblb_batch_run(iblb_batch b, int max_steps, int* n_completed)
{
    if (!b || max_steps < 0) return IBLB_EINVAL;
    int completed = 0;
    int left = max_steps;
    while (left > 0) {
        if (b->dirty) {
            iblb_status st = rebuild(b);
            if (st != IBLB_OK) return st;
        }
        if (b->nactive == 0) break;
        long long r = left;
        for (auto& sl : b->slots)
            if (sl.active) r = std::min(r, sl.steps_total - sl.steps_done);
        int seg = (int)r;
        // segment of `seg` steps, the last one writing every cell's moments
        int done_here = 0;
        while (done_here < seg) {
            const int k = std::min(32, seg - done_here);
            const bool last = (done_here + k == seg);
            cudaGraphExec_t ge;
            iblb_status st = get_graph(b, k, last, &ge);
            if (st != IBLB_OK) return st;
            BCK(b, cudaGraphLaunch(ge, b->stream));
            b->launches += (long long)k * kernels_per_step(b);
            add_launches((long long)k * kernels_per_step(b));
            b->par ^= (k & 1);
            done_here += k;
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
    if (n_completed) *n_completed = completed;
    BCK(b, cudaGetLastError());
    return IBLB_OK;
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

int iblb_batch_slot_tile(iblb_batch b, int slot)
{
    if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].used) return -1;
    return b->slots[slot].cpt;
}

}  // extern "C"
