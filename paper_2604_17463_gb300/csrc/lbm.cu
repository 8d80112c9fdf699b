// lbm.cu -- fused lattice Boltzmann stream-collide kernel (A4) and the
// population / moment conversion kernels of libiblb.
//
// One time step of the lattice Boltzmann equation (Eq. 1) in pull form:
//   f_i(x, t+1)  = f*_i(x - c_i, t)                 (exact streaming)
//                  f*_opp(i)(x, t)  if x - c_i is a solid layer (halfway
//                                   bounce-back at the flat walls)
//   rho = sum_i f_i,  u = (sum_i c_i f_i + F/2) / rho          (Eq. 5-6)
//   f*_i(x, t+1) = f_i - (f_i - f_i^eq(rho, u)) / tau + S_i(u, F)
// with the second-order equilibrium (Eq. 3) and the Guo source (Eq. 4).
//
// Populations are stored as deviations from the rest state, g_i = f_i - w_i,
// in FP64, FP32 or scaled binary16; the collision is written for deviations:
//   g_i^eq = w_i (drho + rho (3 c.u + 9/2 (c.u)^2 - 3/2 u.u)),  drho = sum g_i
//   g*_i   = g_i + omega (g_i^eq - g_i) + (1 - omega/2) w_i (3 (c_i - u).F + 9 (c_i.u)(c_i.F))
// which is algebraically the same update as above (sum w_i = 1, sum w_i c_i = 0).
//
// Layout: structure of arrays, plane i at offset i * ncell, x fastest, so a
// warp reads and writes 32 consecutive cells of one row per plane.  The force
// density F is read (and cleared) only in 32-cell row segments flagged by the
// spread kernel; elsewhere F is the uniform body force.  The moments are
// written only in flagged segments (for the interpolation) or everywhere on
// the last step of a call.
#include "lbm_core.cuh"

namespace iblb {

// One cell (x, y, z) of the plain kernel: pull, moments, collision, store;
// band != 0: the force density of the cell is added (and cleared) and the
// moments written.  Shared by the plain kernel and the band-cell kernel of
// the overlapped step.
template <int Q, int ST, bool WRITE_ALL, bool CS, bool EXT>
__device__ __forceinline__ void sc_cell(const typename StorageT<ST>::S* __restrict__ fin,
                                        typename StorageT<ST>::S* __restrict__ fout,
                                        typename StorageT<ST>::R* __restrict__ mom,
                                        typename StorageT<ST>::R* __restrict__ F,
                                        const StreamParams& p, int x, int y, int z, int band,
                                        unsigned step)
{
    using T = StorageT<ST>;
    using R = typename T::R;
    using L = Stencil<Q>;
    constexpr int D = L::D;
    const int nx = p.g.nx, ny = p.g.ny;
    const long long nc = p.g.ncell;
    const int walls = p.g.walls;
    const long long row = (long long)z * ny + y;
    const long long cell = row * nx + x;

    const int Lw = (D == 2) ? ny : p.g.nz;
    const int a = (D == 2) ? y : z;  // coordinate along the wall axis
    // binary16 populations stay in their stored scale (x 2^k) through the
    // collision: the moments undo the scale, the new terms take it on, and
    // no per-population rescaling is needed on load or store
    const float lsc = (ST == ST_FP16) ? 1.0f : p.inv_scale;
    const unsigned c32 = (unsigned)cell;
    R g[Q];
    R Fx, Fy, Fz;
    if constexpr (D == 2) {
        // Sources of the pull as 32-bit offsets from the cell on per-plane
        // base pointers: periodic along x, solid first/last rows when walls
        // != 0 (else periodic along y); everything but the x wrap depends on
        // the block's row only.  Offsets are unsigned and wrap modulo 2^32
        // (cell indices stay below 2^32).
        const unsigned wstride = (unsigned)nx;
        bool solid_m = false, solid_p = false;
        unsigned dwm = 0u - wstride, dwp = wstride;  // sources a - 1, a + 1
        if (walls) {
            solid_m = (a - 1 == 0);
            solid_p = (a + 1 == Lw - 1);
        } else {
            if (a == 0) dwm = (unsigned)(Lw - 1) * wstride;
            if (a == Lw - 1) dwp = 0u - (unsigned)(Lw - 1) * wstride;
        }
        const unsigned dxm = (x == 0) ? (unsigned)(nx - 1) : 0u - 1u;
        const unsigned dxp = (x == nx - 1) ? 0u - (unsigned)(nx - 1) : 1u;
#pragma unroll
        for (int i = 0; i < Q; i++) {
            const int cx = L::cx(i), cy = L::cy(i);
            const bool solid = cy == 0 ? false : (cy > 0 ? solid_m : solid_p);
            const unsigned off = (cx > 0 ? dxm : (cx < 0 ? dxp : 0u)) + (cy > 0 ? dwm : (cy < 0 ? dwp : 0u));
            if (solid) {
                g[i] = T::load(fin + (size_t)L::opp(i) * nc, c32, lsc);
                if (EXT && p.moving) {  // moving wall: + 2 w_i (c_i . u_w) / c_s^2 (rho_w = 1)
                    const double* uw = cy > 0 ? p.uw_lo : p.uw_hi;
                    g[i] += (R)(6.0 * L::w(i) * (cx * uw[0] + cy * uw[1])) *
                            (ST == ST_FP16 ? (R)p.scale : R(1));
                }
            } else {
                g[i] = T::load(fin + (size_t)i * nc, c32 + off, lsc);
            }
        }
        Fx = param_body<R>(p, 0);
        Fy = param_body<R>(p, 1);
        Fz = R(0);
    } else {
        // 3D: neighbour coordinates per axis (periodic along x and y; solid
        // first/last layers along z when walls != 0), the source index formed
        // per direction; this form measured faster than the offset form above
        // on the 3D workload
        const int xm = (x == 0) ? nx - 1 : x - 1;
        const int xp = (x == nx - 1) ? 0 : x + 1;
        int am = a - 1, ap = a + 1;
        bool solid_m = false, solid_p = false;
        if (walls) {
            solid_m = (am == 0);
            solid_p = (ap == Lw - 1);
        } else {
            if (am < 0) am = Lw - 1;
            if (ap >= Lw) ap = 0;
        }
        const int ym = (y == 0) ? ny - 1 : y - 1;
        const int yp = (y == ny - 1) ? 0 : y + 1;
#pragma unroll
        for (int i = 0; i < Q; i++) {
            const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
            const int sx = cx == 0 ? x : (cx > 0 ? xm : xp);
            const int sa = cz == 0 ? a : (cz > 0 ? am : ap);
            const int sy = cy == 0 ? y : (cy > 0 ? ym : yp);
            const bool solid = cz == 0 ? false : (cz > 0 ? solid_m : solid_p);
            if constexpr (ST == ST_FP16) {
                // binary16: 32-bit cell index on a per-plane base pointer
                const unsigned src32 =
                    ((unsigned)sa * (unsigned)ny + (unsigned)sy) * (unsigned)nx + (unsigned)sx;
                if (solid)
                    g[i] = T::load(fin + (long long)L::opp(i) * nc, c32, lsc);
                else
                    g[i] = T::load(fin + (long long)i * nc, src32, lsc);
                if (EXT && p.moving && solid) {
                    const double* uw = cz > 0 ? p.uw_lo : p.uw_hi;
                    g[i] += (R)(6.0 * L::w(i) * (cx * uw[0] + cy * uw[1] + cz * uw[2])) * p.scale;
                }
                continue;
            }
            const long long src = ((long long)sa * ny + sy) * nx + sx;
            if (solid) {
                g[i] = T::load(fin, (long long)L::opp(i) * nc + cell, p.inv_scale);
                if (EXT && p.moving) {  // moving wall: + 2 w_i (c_i . u_w) / c_s^2 (rho_w = 1)
                    const double* uw = cz > 0 ? p.uw_lo : p.uw_hi;
                    g[i] += (R)(6.0 * L::w(i) * (cx * uw[0] + cy * uw[1] + cz * uw[2]));
                }
            } else {
                g[i] = T::load(fin, (long long)i * nc + src, p.inv_scale);
            }
        }
        // FP32 copies of the parameters: no FP64 conversion per thread (the
        // same values as converting the FP64 ones)
        Fx = param_body<R>(p, 0);
        Fy = param_body<R>(p, 1);
        Fz = param_body<R>(p, 2);
    }

    if (band) take_band_force<D, R>(F, nc, cell, Fx, Fy, Fz);
    CellMoments<Q, R> mo;
    if constexpr (ST == ST_FP16)
        mo = cell_moments<Q, R>(g, Fx, Fy, Fz, (R)p.inv_scale);
    else
        mo = cell_moments<Q, R>(g, Fx, Fy, Fz);
    R om = param_omega<R>(p);
    if (EXT && p.two_tau) {  // viscosity ratio: outside the interface relax with omega_out
        const int col = (D == 2) ? x : x + nx * y;
        if (!inside_cell(p.col_cnt, p.col_z, col, a)) om = (R)p.omega_out;
    }
    if constexpr (ST == ST_FP16) {
        cell_collide<Q, R>(g, mo, om, Fx, Fy, Fz, (R)p.scale);
        if constexpr (D == 2)
            store_cell32<Q, ST, CS>(fout, nc, c32, g, 1.0f, sr_seed(step, cell));
        else
            store_cell<Q, ST, CS>(fout, nc, cell, g, 1.0f, sr_seed(step, cell));
    } else {
        cell_collide<Q, R>(g, mo, om, Fx, Fy, Fz);
        if constexpr (D == 2)
            store_cell32<Q, ST, CS>(fout, nc, c32, g, p.scale, 0u);
        else
            store_cell<Q, ST, CS>(fout, nc, cell, g, p.scale, 0u);
    }

    if (WRITE_ALL || band) put_moments<D, R>(mom, nc, cell, mo.drho, mo.ux, mo.uy, mo.uz);
    if (!isfinite(mo.drho)) atomicOr(p.err, ERR_NONFINITE);
}

// The plain kernel: one cell per thread, blocks of BLOCK cells along x.
// flags == nullptr: every cell takes the body force only (the bulk pass of
// the overlapped step; the band cells are redone by k_band_sc).
template <int Q, int ST, bool WRITE_ALL, int BLOCK, bool CS, bool EXT = false>
__global__ void __launch_bounds__(BLOCK)
k_stream_collide(const typename StorageT<ST>::S* __restrict__ fin,
                 typename StorageT<ST>::S* __restrict__ fout,
                 typename StorageT<ST>::R* __restrict__ mom,
                 typename StorageT<ST>::R* __restrict__ F,
                 uint8_t* __restrict__ flags, const StreamParams p)
{
    constexpr int D = Stencil<Q>::D;
    const int woff = p.g.walls ? 1 : 0;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y, z;
    if (D == 2) {
        y = blockIdx.y + woff;
        z = 0;
    } else {
        y = blockIdx.y;
        z = blockIdx.z + woff;
    }
    const int lane = threadIdx.x & 31;
    const long long seg = ((long long)z * p.g.ny + y) * p.g.nseg_x + (x >> 5);
    int band = 0;
    if (lane == 0 && flags && (x >> 5) < p.g.nseg_x) band = flags[seg];
    band = __shfl_sync(0xffffffffu, band, 0);
    unsigned step = 0;
    if constexpr (ST == ST_FP16)
        step = sr_step(p.rng_in, p.rng_out,
                       blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0);
    if (x >= p.g.nx) return;
    sc_cell<Q, ST, WRITE_ALL, CS, EXT>(fin, fout, mom, F, p, x, y, z, band, step);
    if (lane == 0 && band) flags[seg] = 0;
}

template <int Q, int ST, int BLOCK, bool CS>
static void launch_sc_b(bool write_all, const void* fin, void* fout, void* mom, void* F,
                        uint8_t* flags, const StreamParams& p, cudaStream_t s)
{
    using T = StorageT<ST>;
    const int woff = p.g.walls ? 1 : 0;
    dim3 block(BLOCK);
    dim3 grid((p.g.nx + BLOCK - 1) / BLOCK, 1, 1);
    if (Q == 9) {
        grid.y = p.g.ny - 2 * woff;
    } else {
        grid.y = p.g.ny;
        grid.z = p.g.nz - 2 * woff;
    }
    auto* a = (const typename T::S*)fin;
    auto* b = (typename T::S*)fout;
    auto* m = (typename T::R*)mom;
    auto* f = (typename T::R*)F;
    if (write_all)
        k_stream_collide<Q, ST, true, BLOCK, CS><<<grid, block, 0, s>>>(a, b, m, f, flags, p);
    else
        k_stream_collide<Q, ST, false, BLOCK, CS><<<grid, block, 0, s>>>(a, b, m, f, flags, p);
}

template <int Q, int ST>
static void launch_sc_ext(bool write_all, const void* fin, void* fout, void* mom, void* F,
                              uint8_t* flags, const StreamParams& p, cudaStream_t s)
{
    using T = StorageT<ST>;
    const int woff = p.g.walls ? 1 : 0;
    dim3 grid((p.g.nx + 127) / 128, 1, 1);
    if (Q == 9) {
        grid.y = p.g.ny - 2 * woff;
    } else {
        grid.y = p.g.ny;
        grid.z = p.g.nz - 2 * woff;
    }
    auto* a = (const typename T::S*)fin;
    auto* b = (typename T::S*)fout;
    auto* m = (typename T::R*)mom;
    auto* f = (typename T::R*)F;
    if (write_all)
        k_stream_collide<Q, ST, true, 128, false, true><<<grid, 128, 0, s>>>(a, b, m, f, flags, p);
    else
        k_stream_collide<Q, ST, false, 128, false, true><<<grid, 128, 0, s>>>(a, b, m, f, flags, p);
}

template <int Q, int ST>
static void launch_sc_t(bool write_all, const void* fin, void* fout, void* mom, void* F,
                        uint8_t* flags, const StreamParams& p, const Tuning& tu, cudaStream_t s)
{
    if (p.two_tau || p.moving) {  // the variant with per-cell tau and moving walls
        launch_sc_ext<Q, ST>(write_all, fin, fout, mom, F, flags, p, s);
        return;
    }
    const bool cs = tu.streaming_stores != 0;
    switch (tu.block_x) {
        case 64:
            if (cs) launch_sc_b<Q, ST, 64, true>(write_all, fin, fout, mom, F, flags, p, s);
            else launch_sc_b<Q, ST, 64, false>(write_all, fin, fout, mom, F, flags, p, s);
            break;
        case 256:
            if (cs) launch_sc_b<Q, ST, 256, true>(write_all, fin, fout, mom, F, flags, p, s);
            else launch_sc_b<Q, ST, 256, false>(write_all, fin, fout, mom, F, flags, p, s);
            break;
        default:
            if (cs) launch_sc_b<Q, ST, 128, true>(write_all, fin, fout, mom, F, flags, p, s);
            else launch_sc_b<Q, ST, 128, false>(write_all, fin, fout, mom, F, flags, p, s);
            break;
    }
}

// ------------------------------------------------------------------ band cells
// Overlapped step: the bulk pass (any variant, flags == nullptr) updates
// every cell with the body force only; k_band_list then lists the 8-cell
// quarters of the flagged 32-cell row segments that a stencil touched (all
// four quarters of a flagged segment whose quarters carry no marks, as from
// the ordered or the grouped spread), and k_band_sc updates their cells
// again from the same sources, with the force density and the moments: each
// warp takes four listed quarters, 8 lanes per quarter.  Outside the marked
// quarters F is zero, so the bulk pass's result is already exact there.  The
// cell arithmetic is the plain kernel's, so the result is that of one pass.
// With whole segments, one warp each, the band kernel took 14.4 us per step
// on the 256 x 256 x 128 drop (~16 600 segments, three to four rounds of
// memory latency); a quarter-listed pass needs a quarter of the warps.  (A
// variant in which the bulk pass left out the previous step's band, and the
// band pass took the union, measured no faster: the plain kernel then has to
// read the mark before its loads.)
// One atomic per block of BAND_LIST_THREADS segments: the warps' counts
// are summed in shared memory, thread 0 reserves the block's range.
constexpr int BAND_LIST_THREADS = 256;

__global__ void __launch_bounds__(BAND_LIST_THREADS)
k_band_list(const uint8_t* __restrict__ flags, const uint8_t* __restrict__ fine, long long nseg,
            int* __restrict__ list, int* __restrict__ count)
{
    __shared__ int s_cnt[BAND_LIST_THREADS / 32];
    __shared__ int s_base;
    // one thread per segment: its marked quarters (all four when flagged
    // without marks), written as quarter ids 4 s + k
    const long long sg = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned qm = 0u;
    if (sg < nseg && flags[sg] != 0) {
        const unsigned fw = reinterpret_cast<const unsigned*>(fine)[sg];
        qm = fw == 0u ? 0xfu
                      : ((fw & 0xffu) ? 1u : 0u) | ((fw & 0xff00u) ? 2u : 0u) |
                            ((fw & 0xff0000u) ? 4u : 0u) | ((fw & 0xff000000u) ? 8u : 0u);
    }
    const int c = __popc(qm);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = c;  // inclusive warp scan of the counts
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) s_cnt[wid] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int w = 0; w < BAND_LIST_THREADS / 32; w++) {
            const int t = s_cnt[w];
            s_cnt[w] = tot;
            tot += t;
        }
        s_base = tot ? atomicAdd(count, tot) : 0;
    }
    __syncthreads();
    int pos = s_base + s_cnt[wid] + incl - c;
    for (int k = 0; k < 4; k++)
        if (qm & (1u << k)) list[pos++] = (int)(4 * sg + k);
}

template <int Q, int ST, bool EXT>
__global__ void __launch_bounds__(128)
k_band_sc(const typename StorageT<ST>::S* __restrict__ fin,
          typename StorageT<ST>::S* __restrict__ fout, typename StorageT<ST>::R* __restrict__ mom,
          typename StorageT<ST>::R* __restrict__ F, uint8_t* __restrict__ flags,
          uint8_t* __restrict__ fine, const int* __restrict__ list,
          const int* __restrict__ count, const StreamParams p)
{
    constexpr int D = Stencil<Q>::D;
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    const int n = *count;
    unsigned step = 0;
    if constexpr (ST == ST_FP16) step = sr_step(p.rng_in, nullptr, false);
    for (int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); 4 * w < n; w += nw) {
        const int e = 4 * w + (lane >> 3);
        if (e < n) {
            const int qd = list[e];
            const int sg = qd >> 2;
            const int row = sg / p.g.nseg_x;
            const int x = (sg - row * p.g.nseg_x) * 32 + (qd & 3) * 8 + (lane & 7);
            const int y = (D == 2) ? row : row % p.g.ny;
            const int z = (D == 2) ? 0 : row / p.g.ny;
            if (x < p.g.nx) sc_cell<Q, ST, false, false, EXT>(fin, fout, mom, F, p, x, y, z, 1, step);
            if ((lane & 7) == 0) {
                fine[qd] = 0;
                flags[sg] = 0;
            }
        }
    }
}

template <int Q, int ST>
static void launch_band_t(const void* fin, void* fout, void* mom, void* F, uint8_t* flags,
                          uint8_t* fine, int* list, int* count, const StreamParams& p,
                          int sm_count, cudaStream_t s)
{
    using T = StorageT<ST>;
    const long long nseg = (long long)p.g.ny * p.g.nz * p.g.nseg_x;
    cudaMemsetAsync(count, 0, sizeof(int), s);
    k_band_list<<<(unsigned)((nseg + BAND_LIST_THREADS - 1) / BAND_LIST_THREADS),
                  BAND_LIST_THREADS, 0, s>>>(flags, fine, nseg, list, count);
    auto* a = (const typename T::S*)fin;
    auto* b = (typename T::S*)fout;
    auto* m = (typename T::R*)mom;
    auto* f = (typename T::R*)F;
    // four listed quarters per warp, 16 blocks of 4 warps per SM
    const int grid = 16 * sm_count;
    if (p.moving)
        k_band_sc<Q, ST, true><<<grid, 128, 0, s>>>(a, b, m, f, flags, fine, list, count, p);
    else
        k_band_sc<Q, ST, false><<<grid, 128, 0, s>>>(a, b, m, f, flags, fine, list, count, p);
}

void launch_band_cells(int Q, int storage, const void* fin, void* fout, void* moments, void* F,
                       uint8_t* flags, uint8_t* fine, int* list, int* count,
                       const StreamParams& p, int sm_count, cudaStream_t s)
{
#define IBLB_BAND(QQ, SS) \
    launch_band_t<QQ, SS>(fin, fout, moments, F, flags, fine, list, count, p, sm_count, s)
    if (Q == 9) {
        if (storage == ST_FP64) IBLB_BAND(9, ST_FP64);
        else if (storage == ST_FP32) IBLB_BAND(9, ST_FP32);
        else IBLB_BAND(9, ST_FP16);
    } else {
        if (storage == ST_FP64) IBLB_BAND(19, ST_FP64);
        else if (storage == ST_FP32) IBLB_BAND(19, ST_FP32);
        else IBLB_BAND(19, ST_FP16);
    }
#undef IBLB_BAND
}

void launch_stream_collide(int Q, int storage, bool write_all, const void* fin, void* fout,
                           void* moments, void* F, uint8_t* flags, const StreamParams& p,
                           const Tuning& tu, cudaStream_t s)
{
    if (Q == 9) {
        if (storage == ST_FP64) launch_sc_t<9, ST_FP64>(write_all, fin, fout, moments, F, flags, p, tu, s);
        else if (storage == ST_FP32) launch_sc_t<9, ST_FP32>(write_all, fin, fout, moments, F, flags, p, tu, s);
        else launch_sc_t<9, ST_FP16>(write_all, fin, fout, moments, F, flags, p, tu, s);
    } else {
        if (storage == ST_FP64) launch_sc_t<19, ST_FP64>(write_all, fin, fout, moments, F, flags, p, tu, s);
        else if (storage == ST_FP32) launch_sc_t<19, ST_FP32>(write_all, fin, fout, moments, F, flags, p, tu, s);
        else launch_sc_t<19, ST_FP16>(write_all, fin, fout, moments, F, flags, p, tu, s);
    }
}

// ------------------------------------------------------------------ pairs
// Variant 2: two x-adjacent cells per thread.  Populations move as float2 /
// half2 (8 / 4 bytes per thread and plane); for the directions with c_x = +1
// (-1) the source pair (x-1, x) ((x+1, x+2)) is assembled from the aligned
// pair of the same source row and the neighbouring lane's value by a warp
// shuffle, with one scalar load at warp and row ends (periodic wrap in x).
// Moments and collision run in packed FP32x2 arithmetic.  Needs an even nx.
template <int ST> struct Pair;

template <> struct Pair<ST_FP32> {
    __device__ __forceinline__ static float2 load2(const float* p, long long i, float)
    {
        return *reinterpret_cast<const float2*>(p + i);
    }
    __device__ __forceinline__ static float load1(const float* p, long long i, float) { return p[i]; }
    __device__ __forceinline__ static void store2(float* p, long long i, float2 v, float, unsigned)
    {
        *reinterpret_cast<float2*>(p + i) = v;
    }
};

template <> struct Pair<ST_FP16> {
    __device__ __forceinline__ static float2 load2(const __half* p, long long i, float inv_scale)
    {
        return mul2(__half22float2(*reinterpret_cast<const __half2*>(p + i)), p2(inv_scale));
    }
    __device__ __forceinline__ static float load1(const __half* p, long long i, float inv_scale)
    {
        return __half2float(p[i]) * inv_scale;
    }
    // two neighbouring cells of one population, stochastically rounded
    // (cell x in the low half, x + 1 in the high half of the stored pair)
    __device__ __forceinline__ static void store2(__half* p, long long i, float2 v, float scale,
                                                  unsigned rbits)
    {
        const float2 w = mul2(v, p2(scale));
        *reinterpret_cast<unsigned*>(p + i) = cvt_rs_f16x2(w.y, w.x, rbits);
    }
};

template <int Q, int ST, bool WRITE_ALL, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
k_stream_collide2(const typename StorageT<ST>::S* __restrict__ fin,
                  typename StorageT<ST>::S* __restrict__ fout, float* __restrict__ mom,
                  float* __restrict__ F, uint8_t* __restrict__ flags, const StreamParams p)
{
    using L = Stencil<Q>;
    using P = Pair<ST>;
    constexpr int D = L::D;
    const int nx = p.g.nx, ny = p.g.ny;
    const long long nc = p.g.ncell;
    const int walls = p.g.walls;
    const int woff = walls ? 1 : 0;
    const float inv = p.inv_scale;

    const int x0 = 2 * (blockIdx.x * BLOCK + threadIdx.x);
    int y, z;
    if (D == 2) {
        y = blockIdx.y + woff;
        z = 0;
    } else {
        y = blockIdx.y;
        z = blockIdx.z + woff;
    }
    const int lane = threadIdx.x & 31;
    const bool active = x0 < nx;
    const long long row = (long long)z * ny + y;
    const long long cell = row * nx + x0;
    // band flags: lanes 0-15 share one 32-cell segment, lanes 16-31 the next
    const long long seg = row * p.g.nseg_x + (x0 >> 5);
    int fl = 0;
    if ((lane & 15) == 0 && active && flags) fl = flags[seg];
    const int band = __shfl_sync(0xffffffffu, fl, lane & 16);
    unsigned step = 0;
    if constexpr (ST == ST_FP16)
        step = sr_step(p.rng_in, p.rng_out,
                       blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0);

    const int Lw = (D == 2) ? ny : p.g.nz;
    const int a = (D == 2) ? y : z;
    int am = a - 1, ap = a + 1;
    bool solid_m = false, solid_p = false;
    if (walls) {
        solid_m = (am == 0);
        solid_p = (ap == Lw - 1);
    } else {
        if (am < 0) am = Lw - 1;
        if (ap >= Lw) ap = 0;
    }
    int ym = y, yp = y;
    if (D == 3) {
        ym = (y == 0) ? ny - 1 : y - 1;
        yp = (y == ny - 1) ? 0 : y + 1;
    }

    // pass 1: every load of the thread (aligned pairs and the edge values)
    // is issued before any shuffle, so that the loads overlap
    float2 g[Q];
    float edge[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const int cx = L::cx(i), cy = L::cy(i);
        const int cw = (D == 2) ? cy : L::cz(i);
        const bool solid = cw == 0 ? false : (cw > 0 ? solid_m : solid_p);  // uniform per row
        edge[i] = 0.f;
        if (solid) {
            g[i] = active ? P::load2(fin, (long long)L::opp(i) * nc + cell, inv) : p2(0.f);
            continue;
        }
        const int sa = cw == 0 ? a : (cw > 0 ? am : ap);
        long long srow;
        if (D == 2) {
            srow = sa;
        } else {
            const int sy = cy == 0 ? y : (cy > 0 ? ym : yp);
            srow = (long long)sa * ny + sy;
        }
        const long long base = (long long)i * nc + srow * nx;
        g[i] = active ? P::load2(fin, base + x0, inv) : p2(0.f);
        if (cx > 0 && (lane == 0 || x0 == 0) && active)
            edge[i] = P::load1(fin, base + (x0 == 0 ? nx - 1 : x0 - 1), inv);
        if (cx < 0 && (lane == 31 || x0 + 2 >= nx) && active)
            edge[i] = P::load1(fin, base + (x0 + 2 >= nx ? 0 : x0 + 2), inv);
    }
    // pass 2: the x-shifted directions take one value from the neighbouring
    // lane (or the edge load at warp and row ends)
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const int cx = L::cx(i);
        const int cw = (D == 2) ? L::cy(i) : L::cz(i);
        const bool solid = cw == 0 ? false : (cw > 0 ? solid_m : solid_p);
        if (solid || cx == 0) continue;
        const float2 A = g[i];
        if (cx > 0) {  // source x - 1
            float left = __shfl_up_sync(0xffffffffu, A.y, 1);
            if (lane == 0 || x0 == 0) left = edge[i];
            g[i] = make_float2(left, A.x);
        } else {       // source x + 1
            float right = __shfl_down_sync(0xffffffffu, A.x, 1);
            if (lane == 31 || x0 + 2 >= nx) right = edge[i];
            g[i] = make_float2(A.y, right);
        }
    }
    if (!active) return;

    float2 Fx = p2(p.body_f[0]), Fy = p2(p.body_f[1]), Fz = p2(p.body_f[2]);
    if (band) {  // float4 per cell: (Fx, Fy, Fz, 0)
        float4* F4 = reinterpret_cast<float4*>(F);
        const float4 a = F4[cell], b = F4[cell + 1];
        Fx = add2(Fx, make_float2(a.x, b.x));
        Fy = add2(Fy, make_float2(a.y, b.y));
        if (D == 3) Fz = add2(Fz, make_float2(a.z, b.z));
        F4[cell] = make_float4(0.f, 0.f, 0.f, 0.f);
        F4[cell + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const CellMoments2 mo = cell_moments2<Q>(g, Fx, Fy, Fz);
    cell_collide2<Q>(g, mo, p.omega_f, Fx, Fy, Fz);
    const unsigned seed = ST == ST_FP16 ? sr_seed(step, cell) : 0u;
#pragma unroll
    for (int i = 0; i < Q; i++) P::store2(fout, (long long)i * nc + cell, g[i], p.scale, sr_bits(seed, i));
    if (WRITE_ALL || band) {  // float4 per cell: (drho, ux, uy, uz)
        float4* m4 = reinterpret_cast<float4*>(mom);
        m4[cell] = make_float4(mo.drho.x, mo.ux.x, mo.uy.x, D == 3 ? mo.uz.x : 0.f);
        m4[cell + 1] = make_float4(mo.drho.y, mo.ux.y, mo.uy.y, D == 3 ? mo.uz.y : 0.f);
    }
    if (!isfinite(mo.drho.x) || !isfinite(mo.drho.y)) atomicOr(p.err, ERR_NONFINITE);
    if ((lane & 15) == 0 && band) flags[seg] = 0;
}

template <int Q, int ST, int BLOCK>
static void launch_sc2_b(bool write_all, const void* fin, void* fout, void* mom, void* F,
                         uint8_t* flags, const StreamParams& p, cudaStream_t s)
{
    using T = StorageT<ST>;
    const int woff = p.g.walls ? 1 : 0;
    dim3 grid((p.g.nx / 2 + BLOCK - 1) / BLOCK, 1, 1);
    if (Q == 9) {
        grid.y = p.g.ny - 2 * woff;
    } else {
        grid.y = p.g.ny;
        grid.z = p.g.nz - 2 * woff;
    }
    auto* a = (const typename T::S*)fin;
    auto* b = (typename T::S*)fout;
    if (write_all)
        k_stream_collide2<Q, ST, true, BLOCK><<<grid, BLOCK, 0, s>>>(a, b, (float*)mom, (float*)F, flags, p);
    else
        k_stream_collide2<Q, ST, false, BLOCK><<<grid, BLOCK, 0, s>>>(a, b, (float*)mom, (float*)F, flags, p);
}

template <int Q, int ST>
static void launch_sc2_t(bool write_all, const void* fin, void* fout, void* mom, void* F,
                         uint8_t* flags, const StreamParams& p, const Tuning& tu, cudaStream_t s)
{
    switch (tu.block_x) {
        case 64: launch_sc2_b<Q, ST, 64>(write_all, fin, fout, mom, F, flags, p, s); break;
        case 256: launch_sc2_b<Q, ST, 256>(write_all, fin, fout, mom, F, flags, p, s); break;
        default: launch_sc2_b<Q, ST, 128>(write_all, fin, fout, mom, F, flags, p, s); break;
    }
}

bool pair_kernel_ok(int storage, const GridParams& g)
{
    return storage != ST_FP64 && g.nx % 2 == 0;
}

void launch_stream_collide_pairs(int Q, int storage, bool write_all, const void* fin, void* fout,
                                 void* moments, void* F, uint8_t* flags, const StreamParams& p,
                                 const Tuning& tu, cudaStream_t s)
{
    if (Q == 9) {
        if (storage == ST_FP32) launch_sc2_t<9, ST_FP32>(write_all, fin, fout, moments, F, flags, p, tu, s);
        else launch_sc2_t<9, ST_FP16>(write_all, fin, fout, moments, F, flags, p, tu, s);
    } else {
        if (storage == ST_FP32) launch_sc2_t<19, ST_FP32>(write_all, fin, fout, moments, F, flags, p, tu, s);
        else launch_sc2_t<19, ST_FP16>(write_all, fin, fout, moments, F, flags, p, tu, s);
    }
}

// ------------------------------------------------------------------ row pairs
// Variant 3 (D3Q19, FP32 / binary16 storage): two cells per thread, (x, y0, z)
// and (x, y0 + 1, z), in adjacent rows of one layer.  Loads and stores stay
// scalar and coalesced along x; the two cells share the neighbour indices
// along x and z and the per-thread set-up, and their moments and collision
// run in packed FP32x2 arithmetic (one instruction for both cells).  binary16
// stores convert the two cells' values of a population with one stochastic
// rounding instruction.  A last odd row is computed by its own lane pair
// with the second cell masked off.
template <int ST> struct RowPair;
template <> struct RowPair<ST_FP32> {
    __device__ __forceinline__ static float load(const float* p, unsigned i) { return p[i]; }
};
template <> struct RowPair<ST_FP16> {
    __device__ __forceinline__ static float load(const __half* p, unsigned i) { return __half2float(p[i]); }
};

template <int ST, bool WRITE_ALL, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
k_stream_collide_y2(const typename StorageT<ST>::S* __restrict__ fin,
                    typename StorageT<ST>::S* __restrict__ fout, float* __restrict__ mom,
                    float* __restrict__ F, uint8_t* __restrict__ flags, const StreamParams p)
{
    using L = Stencil<19>;
    using P = RowPair<ST>;
    constexpr int Q = 19;
    const int nx = p.g.nx, ny = p.g.ny, nz = p.g.nz;
    const unsigned nc = (unsigned)p.g.ncell;
    const int walls = p.g.walls;
    const int woff = walls ? 1 : 0;
    const int x = blockIdx.x * BLOCK + threadIdx.x;
    const int y0 = 2 * blockIdx.y;
    const int z = blockIdx.z + woff;
    const bool hasB = y0 + 1 < ny;
    const int lane = threadIdx.x & 31;
    const unsigned rowA = (unsigned)z * (unsigned)ny + (unsigned)y0;
    const unsigned rowB = hasB ? rowA + 1u : rowA;
    int fa = 0, fb = 0;
    if (lane == 0 && flags && (x >> 5) < p.g.nseg_x) {
        fa = flags[rowA * (unsigned)p.g.nseg_x + (x >> 5)];
        fb = hasB ? flags[rowB * (unsigned)p.g.nseg_x + (x >> 5)] : 0;
    }
    const int bandA = __shfl_sync(0xffffffffu, fa, 0);
    const int bandB = __shfl_sync(0xffffffffu, fb, 0);
    unsigned step = 0;
    if constexpr (ST == ST_FP16)
        step = sr_step(p.rng_in, p.rng_out,
                       blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0);
    if (x >= nx) return;
    const unsigned cellA = rowA * (unsigned)nx + (unsigned)x;
    const unsigned cellB = rowB * (unsigned)nx + (unsigned)x;

    const int xm = (x == 0) ? nx - 1 : x - 1;
    const int xp = (x == nx - 1) ? 0 : x + 1;
    int am = z - 1, ap = z + 1;
    bool solid_m = false, solid_p = false;
    if (walls) {
        solid_m = (am == 0);
        solid_p = (ap == nz - 1);
    } else {
        if (am < 0) am = nz - 1;
        if (ap >= nz) ap = 0;
    }
    const int yB = hasB ? y0 + 1 : y0;
    const int ymA = (y0 == 0) ? ny - 1 : y0 - 1;
    const int ypA = (y0 + 1 == ny) ? 0 : y0 + 1;
    const int ymB = (yB == 0) ? ny - 1 : yB - 1;
    const int ypB = (yB + 1 == ny) ? 0 : yB + 1;

    float2 g[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
        const bool solid = cz == 0 ? false : (cz > 0 ? solid_m : solid_p);
        if (solid) {
            const typename StorageT<ST>::S* pl = fin + (size_t)L::opp(i) * nc;
            g[i] = make_float2(P::load(pl, cellA), P::load(pl, cellB));
            continue;
        }
        const int sx = cx == 0 ? x : (cx > 0 ? xm : xp);
        const int sz = cz == 0 ? z : (cz > 0 ? am : ap);
        const int syA = cy == 0 ? y0 : (cy > 0 ? ymA : ypA);
        const int syB = cy == 0 ? yB : (cy > 0 ? ymB : ypB);
        const unsigned zb = (unsigned)sz * (unsigned)ny;
        const typename StorageT<ST>::S* pl = fin + (size_t)i * nc;
        g[i] = make_float2(P::load(pl, (zb + (unsigned)syA) * (unsigned)nx + (unsigned)sx),
                           P::load(pl, (zb + (unsigned)syB) * (unsigned)nx + (unsigned)sx));
    }
    float2 Fx = p2(p.body_f[0]), Fy = p2(p.body_f[1]), Fz = p2(p.body_f[2]);
    if (bandA) take_band_force<3, float>(F, nc, cellA, Fx.x, Fy.x, Fz.x);
    if (bandB && hasB) take_band_force<3, float>(F, nc, cellB, Fx.y, Fy.y, Fz.y);
    const float ginv = (ST == ST_FP16) ? p.inv_scale : 1.0f;
    const float gsc = (ST == ST_FP16) ? p.scale : 1.0f;
    const CellMoments2 mo = cell_moments2<Q>(g, Fx, Fy, Fz, ginv);
    cell_collide2<Q>(g, mo, p.omega_f, Fx, Fy, Fz, gsc);
    if constexpr (ST == ST_FP16) {
        unsigned short* o = reinterpret_cast<unsigned short*>(fout);
        const unsigned seed = sr_seed(step, (long long)cellA);
#pragma unroll
        for (int i = 0; i < Q; i++) {
            // cell B in the high half, cell A in the low half
            const unsigned h = cvt_rs_f16x2(g[i].y, g[i].x, sr_bits(seed, i));
            unsigned short* pl = o + (size_t)i * nc;
            pl[cellA] = (unsigned short)(h & 0xffffu);
            if (hasB) pl[cellB] = (unsigned short)(h >> 16);
        }
    } else {
#pragma unroll
        for (int i = 0; i < Q; i++) {
            float* pl = fout + (size_t)i * nc;
            pl[cellA] = g[i].x;
            if (hasB) pl[cellB] = g[i].y;
        }
    }
    if (WRITE_ALL || bandA) put_moments<3, float>(mom, nc, cellA, mo.drho.x, mo.ux.x, mo.uy.x, mo.uz.x);
    if (hasB && (WRITE_ALL || bandB))
        put_moments<3, float>(mom, nc, cellB, mo.drho.y, mo.ux.y, mo.uy.y, mo.uz.y);
    if (!isfinite(mo.drho.x) || (hasB && !isfinite(mo.drho.y))) atomicOr(p.err, ERR_NONFINITE);
    if (lane == 0) {
        if (bandA) flags[rowA * (unsigned)p.g.nseg_x + (x >> 5)] = 0;
        if (bandB && hasB) flags[rowB * (unsigned)p.g.nseg_x + (x >> 5)] = 0;
    }
}

template <int ST, int BLOCK>
static void launch_y2_b(bool write_all, const void* fin, void* fout, void* mom, void* F,
                        uint8_t* flags, const StreamParams& p, cudaStream_t s)
{
    using T = StorageT<ST>;
    const int woff = p.g.walls ? 1 : 0;
    dim3 grid((p.g.nx + BLOCK - 1) / BLOCK, (p.g.ny + 1) / 2, p.g.nz - 2 * woff);
    auto* a = (const typename T::S*)fin;
    auto* b = (typename T::S*)fout;
    if (write_all)
        k_stream_collide_y2<ST, true, BLOCK><<<grid, BLOCK, 0, s>>>(a, b, (float*)mom, (float*)F, flags, p);
    else
        k_stream_collide_y2<ST, false, BLOCK><<<grid, BLOCK, 0, s>>>(a, b, (float*)mom, (float*)F, flags, p);
}

bool rowpair_kernel_ok(int Q, int storage, const GridParams& g)
{
    return Q == 19 && storage != ST_FP64 && g.ny >= 2;
}

void launch_stream_collide_rowpairs(int storage, bool write_all, const void* fin, void* fout,
                                    void* moments, void* F, uint8_t* flags, const StreamParams& p,
                                    const Tuning& tu, cudaStream_t s)
{
#define IBLB_Y2(SS)                                                                           \
    switch (tu.block_x) {                                                                    \
        case 64: launch_y2_b<SS, 64>(write_all, fin, fout, moments, F, flags, p, s); break;  \
        case 256: launch_y2_b<SS, 256>(write_all, fin, fout, moments, F, flags, p, s); break; \
        default: launch_y2_b<SS, 128>(write_all, fin, fout, moments, F, flags, p, s); break; \
    }
    if (storage == ST_FP32) {
        IBLB_Y2(ST_FP32)
    } else {
        IBLB_Y2(ST_FP16)
    }
#undef IBLB_Y2
}

// ------------------------------------------------------------------ conversions
__device__ double weight_q(int Q, int i)
{
    return Q == 9 ? Stencil<9>::w(i) : Stencil<19>::w(i);
}

template <int ST>
__global__ void k_pack(int Q, const double* __restrict__ f, typename StorageT<ST>::S* dst,
                       long long ncell, float scale)
{
    const long long n = (long long)Q * ncell;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t / ncell);
        const double dev = f[t] - weight_q(Q, i);
        StorageT<ST>::store(dst, t, (typename StorageT<ST>::R)dev, scale);
    }
}

template <int ST>
__global__ void k_unpack(int Q, const typename StorageT<ST>::S* src, double* __restrict__ f,
                         long long ncell, float inv_scale)
{
    const long long n = (long long)Q * ncell;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t / ncell);
        f[t] = weight_q(Q, i) + (double)StorageT<ST>::load(src, t, inv_scale);
    }
}

static int grid_for(long long n, int block = 256)
{
    long long b = (n + block - 1) / block;
    if (b > 152 * 32) b = 152 * 32;
    if (b < 1) b = 1;
    return (int)b;
}

void launch_pack_populations(int Q, int storage, const double* f, void* dst, long long ncell,
                             float scale, cudaStream_t s)
{
    const int gb = grid_for((long long)Q * ncell);
    if (storage == ST_FP64) k_pack<ST_FP64><<<gb, 256, 0, s>>>(Q, f, (double*)dst, ncell, scale);
    else if (storage == ST_FP32) k_pack<ST_FP32><<<gb, 256, 0, s>>>(Q, f, (float*)dst, ncell, scale);
    else k_pack<ST_FP16><<<gb, 256, 0, s>>>(Q, f, (__half*)dst, ncell, scale);
}

void launch_unpack_populations(int Q, int storage, const void* src, double* f, long long ncell,
                               float inv_scale, cudaStream_t s)
{
    const int gb = grid_for((long long)Q * ncell);
    if (storage == ST_FP64) k_unpack<ST_FP64><<<gb, 256, 0, s>>>(Q, (const double*)src, f, ncell, inv_scale);
    else if (storage == ST_FP32) k_unpack<ST_FP32><<<gb, 256, 0, s>>>(Q, (const float*)src, f, ncell, inv_scale);
    else k_unpack<ST_FP16><<<gb, 256, 0, s>>>(Q, (const __half*)src, f, ncell, inv_scale);
}

template <int Q, int ST>
__global__ void k_set_equilibrium(int dim, const double* __restrict__ rho,
                                  const double* __restrict__ u, typename StorageT<ST>::S* dst,
                                  long long ncell, float scale)
{
    using L = Stencil<Q>;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * blockDim.x) {
        const double r = rho ? rho[c] : 1.0;
        const double ux = u[c], uy = u[ncell + c], uz = dim == 3 ? u[2 * ncell + c] : 0.0;
        const double uu = ux * ux + uy * uy + uz * uz;
#pragma unroll
        for (int i = 0; i < Q; i++) {
            const double cu = L::cx(i) * ux + L::cy(i) * uy + L::cz(i) * uz;
            // f_eq - w_i (Eq. 3 written for the deviation)
            const double dev = L::w(i) * ((r - 1.0) + r * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu));
            StorageT<ST>::store(dst, (long long)i * ncell + c, (typename StorageT<ST>::R)dev, scale);
        }
    }
}

template <int Q>
static void launch_set_eq_q(int storage, int dim, const double* rho, const double* u, void* dst,
                            long long ncell, float scale, cudaStream_t s)
{
    const int gb = grid_for(ncell);
    if (storage == ST_FP64)
        k_set_equilibrium<Q, ST_FP64><<<gb, 256, 0, s>>>(dim, rho, u, (double*)dst, ncell, scale);
    else if (storage == ST_FP32)
        k_set_equilibrium<Q, ST_FP32><<<gb, 256, 0, s>>>(dim, rho, u, (float*)dst, ncell, scale);
    else
        k_set_equilibrium<Q, ST_FP16><<<gb, 256, 0, s>>>(dim, rho, u, (__half*)dst, ncell, scale);
}

void launch_set_equilibrium(int Q, int storage, int dim, const double* rho, const double* u,
                            void* dst, long long ncell, float scale, cudaStream_t s)
{
    if (Q == 9) launch_set_eq_q<9>(storage, dim, rho, u, dst, ncell, scale, s);
    else launch_set_eq_q<19>(storage, dim, rho, u, dst, ncell, scale, s);
}

__device__ __forceinline__ bool is_solid_cell(const GridParams& g, long long c)
{
    if (!g.walls) return false;
    const long long plane = (long long)g.nx * g.ny;
    const int a = (g.dim == 2) ? (int)((c / g.nx) % g.ny) : (int)(c / plane);
    const int Lw = (g.dim == 2) ? g.ny : g.nz;
    return a == 0 || a == Lw - 1;
}

template <typename R>
__global__ void k_unpack_moments(GridParams g, const R* __restrict__ mom, double* rho, double* u)
{
    const long long ncell = g.ncell;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * blockDim.x) {
        const bool solid = is_solid_cell(g, c);
        R m[4];
        if constexpr (sizeof(R) == 4) {
            const float4 v = reinterpret_cast<const float4*>(mom)[c];
            m[0] = v.x;
            m[1] = v.y;
            m[2] = v.z;
            m[3] = v.w;
        } else {
            for (int k = 0; k <= g.dim; k++) m[k] = mom[k * ncell + c];
        }
        if (rho) rho[c] = solid ? 0.0 : 1.0 + (double)m[0];
        if (u)
            for (int k = 0; k < g.dim; k++) u[k * ncell + c] = solid ? 0.0 : (double)m[k + 1];
    }
}

void launch_unpack_moments(int storage, const GridParams& g, const void* moments, double* rho,
                           double* u, cudaStream_t s)
{
    const int gb = grid_for(g.ncell);
    if (storage == ST_FP64)
        k_unpack_moments<double><<<gb, 256, 0, s>>>(g, (const double*)moments, rho, u);
    else
        k_unpack_moments<float><<<gb, 256, 0, s>>>(g, (const float*)moments, rho, u);
}

template <typename R>
__global__ void k_init_moments(GridParams g, R* mom)
{
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.ncell;
         c += (long long)gridDim.x * blockDim.x) {
        const R d0 = is_solid_cell(g, c) ? R(-1) : R(0);
        if constexpr (sizeof(R) == 4) {
            reinterpret_cast<float4*>(mom)[c] = make_float4(d0, 0.f, 0.f, 0.f);
        } else {  // [1 + dim][cell]: only the components the buffer holds
            mom[c] = d0;
            for (int k = 0; k < g.dim; k++) mom[(k + 1) * g.ncell + c] = R(0);
        }
    }
}

void launch_init_moments(int storage, const GridParams& g, void* moments, cudaStream_t s)
{
    const int gb = grid_for(g.ncell);
    if (storage == ST_FP64) k_init_moments<double><<<gb, 256, 0, s>>>(g, (double*)moments);
    else k_init_moments<float><<<gb, 256, 0, s>>>(g, (float*)moments);
}

template <typename R>
__global__ void k_load_velocity(int dim, const double* __restrict__ u, R* mom, long long ncell)
{
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * blockDim.x)
        if constexpr (sizeof(R) == 4)
            reinterpret_cast<float4*>(mom)[c] =
                make_float4(0.f, (float)u[c], (float)u[ncell + c], dim == 3 ? (float)u[2 * ncell + c] : 0.f);
        else
            for (int k = 0; k < dim; k++) mom[(k + 1) * ncell + c] = (R)u[k * ncell + c];
}

void launch_load_velocity(int storage, int dim, const double* u, void* moments, long long ncell,
                          cudaStream_t s)
{
    const int gb = grid_for(ncell);
    if (storage == ST_FP64) k_load_velocity<double><<<gb, 256, 0, s>>>(dim, u, (double*)moments, ncell);
    else k_load_velocity<float><<<gb, 256, 0, s>>>(dim, u, (float*)moments, ncell);
}

template <typename R>
__global__ void k_unpack_force(GridParams g, const R* __restrict__ F, double b0, double b1,
                               double b2, double* out)
{
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.ncell;
         c += (long long)gridDim.x * blockDim.x) {
        const bool solid = is_solid_cell(g, c);
        const double body[3] = {b0, b1, b2};
        R f[3];
        if constexpr (sizeof(R) == 4) {
            const float4 v = reinterpret_cast<const float4*>(F)[c];
            f[0] = v.x;
            f[1] = v.y;
            f[2] = v.z;
        } else {
            for (int k = 0; k < g.dim; k++) f[k] = F[k * g.ncell + c];
        }
        for (int k = 0; k < g.dim; k++) out[k * g.ncell + c] = solid ? 0.0 : (double)f[k] + body[k];
    }
}

void launch_unpack_force(int storage, const GridParams& g, const void* F, const double* body,
                         double* out, cudaStream_t s)
{
    const int gb = grid_for(g.ncell);
    if (storage == ST_FP64)
        k_unpack_force<double><<<gb, 256, 0, s>>>(g, (const double*)F, body[0], body[1], body[2], out);
    else
        k_unpack_force<float><<<gb, 256, 0, s>>>(g, (const float*)F, body[0], body[1], body[2], out);
}

__global__ void k_fill_flags(uint8_t* flags, long long n, uint8_t v)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x)
        flags[t] = v;
}

void launch_clear_flags(uint8_t* flags, long long n, cudaStream_t s)
{
    k_fill_flags<<<grid_for(n), 256, 0, s>>>(flags, n, 0);
}

void launch_set_all_flags(uint8_t* flags, long long n, cudaStream_t s)
{
    k_fill_flags<<<grid_for(n), 256, 0, s>>>(flags, n, 1);
}

// ------------------------------------------------------------------ mass
constexpr int MASS_BLOCK = 256;

int mass_partial_blocks(const GridParams& g)
{
    long long b = (g.ncell + MASS_BLOCK - 1) / MASS_BLOCK;
    if (b > 1024) b = 1024;
    if (b < 1) b = 1;
    return (int)b;
}

template <int ST>
__global__ void __launch_bounds__(MASS_BLOCK)
k_mass_partials(int Q, const typename StorageT<ST>::S* __restrict__ f, GridParams g,
                float inv_scale, double* partial)
{
    double acc = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.ncell;
         c += (long long)gridDim.x * blockDim.x) {
        if (is_solid_cell(g, c)) continue;
        double dev = 0.0;
        for (int i = 0; i < Q; i++)
            dev += (double)StorageT<ST>::load(f, (long long)i * g.ncell + c, inv_scale);
        acc += 1.0 + dev;
    }
    __shared__ double red[MASS_BLOCK / 32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < MASS_BLOCK / 32; k++) t += red[k];
        partial[blockIdx.x] = t;
    }
}

void launch_mass_partials(int Q, int storage, const void* f, const GridParams& g, float inv_scale,
                          double* partial, cudaStream_t s)
{
    const int nb = mass_partial_blocks(g);
    if (storage == ST_FP64)
        k_mass_partials<ST_FP64><<<nb, MASS_BLOCK, 0, s>>>(Q, (const double*)f, g, inv_scale, partial);
    else if (storage == ST_FP32)
        k_mass_partials<ST_FP32><<<nb, MASS_BLOCK, 0, s>>>(Q, (const float*)f, g, inv_scale, partial);
    else
        k_mass_partials<ST_FP16><<<nb, MASS_BLOCK, 0, s>>>(Q, (const __half*)f, g, inv_scale, partial);
}

}  // namespace iblb
