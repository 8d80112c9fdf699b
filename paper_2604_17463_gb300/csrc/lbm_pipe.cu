// lbm_pipe.cu -- pipelined stream-collide kernel (A4) for GB300.
//
// Same update as the plain kernel in lbm.cu (pull streaming with halfway
// bounce-back, moments with the half-force term, BGK + Guo, Eq. 1-6), with
// the loads decoupled from the arithmetic:
//   - persistent CTAs (a few per SM) walk the tiles round-robin;
//   - a producer warp stages, for each of the Q directions, the source rows
//     of a tile into shared memory with bulk asynchronous copies
//     (cp.async.bulk, completion counted in bytes on an mbarrier), several
//     tiles ahead of the consumers.  Two tile shapes:
//       rows mode:    R whole rows (nx <= 1024, nx % 32 == 0); the periodic
//                     x-shift wraps inside shared memory and consecutive
//                     source rows of a direction go in one copy;
//       segment mode: one x-segment of W cells (W a multiple of 256) of one
//                     row plus a 16-byte halo on each side;
//   - eight consumer warps read the shifted populations from shared memory,
//     collide and store the new populations with coalesced stores, then
//     release the stage on a second mbarrier.
// For a direction whose source row is a solid layer (bounce-back) the
// producer stages the opposite direction of the current row instead, and the
// consumer reads it unshifted.
// Every wait is bounded: after a limit (by default ~2 s; a launch-shape
// parameter) a waiting thread latches ERR_TIMEOUT and the CTA stops; the
// producer always waits (bounded by ~2 s) for the copies it issued before it
// exits.
#include "lbm_core.cuh"

namespace iblb {

namespace {

template <int Q> struct StencilTable {
    int8_t v[Q][4];  // cx, cy, cz, opp
};

template <int Q>
constexpr StencilTable<Q> make_table()
{
    StencilTable<Q> t{};
    for (int i = 0; i < Q; i++) {
        t.v[i][0] = (int8_t)Stencil<Q>::cx(i);
        t.v[i][1] = (int8_t)Stencil<Q>::cy(i);
        t.v[i][2] = (int8_t)Stencil<Q>::cz(i);
        t.v[i][3] = (int8_t)Stencil<Q>::opp(i);
    }
    return t;
}

__constant__ StencilTable<9> c_tab9 = make_table<9>();
__constant__ StencilTable<19> c_tab19 = make_table<19>();

template <int Q>
__device__ __forceinline__ const StencilTable<Q>& tab();
template <>
__device__ __forceinline__ const StencilTable<9>& tab<9>() { return c_tab9; }
template <>
__device__ __forceinline__ const StencilTable<19>& tab<19>() { return c_tab19; }

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Non-blocking test of the phase (mbarrier.test_wait never suspends the
// thread, unlike try_wait, which may wait inside the instruction).
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

constexpr long long PIPE_TIMEOUT_CYCLES = 4000000000LL;  // ~2 s at 2 GHz

// Bounded wait for the phase of `bar` with the given parity, at most `limit`
// clock cycles.  Returns false (and stops the CTA) on timeout or when another
// thread of the CTA gave up.
// Limits below WAIT_POLL_BELOW cycles are enforced by polling with the
// non-blocking test (a suspended try_wait could outlast them); longer ones
// wait in try_wait between clock checks.
constexpr long long WAIT_POLL_BELOW = 1000000LL;

__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t parity, int* err,
                                           volatile int* abort_flag, long long limit)
{
    if (limit < WAIT_POLL_BELOW) {
        const long long t0 = clock64();
        while (!mbar_test_wait(bar, parity)) {
            if (*abort_flag) return false;
            if (clock64() - t0 > limit) {
                atomicOr(err, ERR_TIMEOUT);
                *abort_flag = 1;
                return false;
            }
        }
        return true;
    }
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > limit) {
            atomicOr(err, ERR_TIMEOUT);
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}

}  // namespace


// Tile t -> first lattice row (y0, z) and first cell x0, with R_t rows.
template <int D>
__device__ __forceinline__ void decode_tile(const PipeShape& ps, const GridParams& g, long long t,
                                            int& y0, int& z, int& x0, int& rows)
{
    const int woff = g.walls ? 1 : 0;
    if (ps.mode == PIPE_ROWS) {
        const int ny_f = (D == 2) ? g.ny - 2 * woff : g.ny;   // rows stacked along y
        const int yb = (int)(t % ps.yblocks);
        const long long zi = t / ps.yblocks;
        const int ylo = (D == 2) ? woff : 0;
        y0 = ylo + yb * ps.R;
        rows = min(ps.R, ylo + ny_f - y0);
        z = (D == 2) ? 0 : (int)zi + woff;
        x0 = 0;
    } else {
        const long long row_idx = t / ps.nseg;
        x0 = (int)(t - row_idx * ps.nseg) * ps.W;
        rows = 1;
        if (D == 2) {
            y0 = (int)row_idx + woff;
            z = 0;
        } else {
            z = (int)(row_idx / g.ny) + woff;
            y0 = (int)(row_idx % g.ny);
        }
    }
}

// Source of direction i for the destination row (y, z): the plane and row to
// stage (the opposite direction of the same row under bounce-back).
template <int D>
__device__ __forceinline__ void source_row(const GridParams& g, int y, int z, int cy, int cz, int i,
                                           int op, int& plane, int& sy, int& sz)
{
    plane = i;
    bool bb = false;
    if (D == 2) {
        int sa = y - cy;
        if (g.walls) bb = (sa <= 0 || sa >= g.ny - 1);
        else sa = (sa + g.ny) % g.ny;
        sy = sa;
        sz = 0;
    } else {
        sy = (y - cy + g.ny) % g.ny;
        int sa = z - cz;
        if (g.walls) bb = (sa <= 0 || sa >= g.nz - 1);
        else sa = (sa + g.nz) % g.nz;
        sz = sa;
    }
    if (bb) {
        plane = op;
        sy = y;
        sz = z;
    }
}

// NC consumer warps per CTA: 8 with two CTAs per SM, 16 or 24 with one.
template <int Q, int ST, bool WRITE_ALL, int NC>
__global__ void __launch_bounds__(32 * (NC + 1), NC == 8 ? 2 : 1)
k_sc_pipe(const typename StorageT<ST>::S* __restrict__ fin,
          typename StorageT<ST>::S* __restrict__ fout, typename StorageT<ST>::R* __restrict__ mom,
          typename StorageT<ST>::R* __restrict__ F, uint8_t* __restrict__ flags,
          const StreamParams p, const PipeShape ps)
{
    using T = StorageT<ST>;
    using S = typename T::S;
    using R = typename T::R;
    using L = Stencil<Q>;
    constexpr int D = L::D;
    constexpr int ELT = (int)sizeof(S);
    constexpr int HALO = 16 / ELT;

    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)ps.stages * ps.stage_bytes);
    uint64_t* empty = full + ps.stages;
    __shared__ volatile int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nx = p.g.nx, ny = p.g.ny;
    const long long nc = p.g.ncell;
    const int walls = p.g.walls;
    const bool rows_mode = ps.mode == PIPE_ROWS;
    unsigned step = 0;
    if constexpr (ST == ST_FP16)
        step = sr_step(p.rng_in, p.rng_out, blockIdx.x == 0 && threadIdx.x == 0);

    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < ps.stages; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NC);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == 0) {
        // ---------------- producer
        long long k = 0;
        for (long long t = blockIdx.x; t < ps.ntiles; t += gridDim.x, ++k) {
            const int s = (int)(k % ps.stages);
            if (k >= ps.stages) {
                const uint32_t par = (uint32_t)(((k / ps.stages) - 1) & 1);
                if (!wait_phase(&empty[s], par, p.err, &abort_flag, ps.wait_limit)) break;
            }
            int y0, z, x0, rows;
            decode_tile<D>(ps, p.g, t, y0, z, x0, rows);
            unsigned char* stage = smem + (size_t)s * ps.stage_bytes;
            const uint32_t tx = rows_mode ? (uint32_t)(Q * rows * nx * ELT) : (uint32_t)ps.tx_bytes;
            if (lane == 0) mbar_arrive_expect_tx(&full[s], tx);
            __syncwarp();
            if (lane < Q) {
                const int cy = tab<Q>().v[lane][1], cz = tab<Q>().v[lane][2];
                const int op = tab<Q>().v[lane][3];
                unsigned char* dst = stage + (size_t)lane * ps.plane_bytes;
                if (rows_mode) {
                    // merge consecutive source rows of this direction into runs
                    const size_t row_bytes = (size_t)nx * ELT;
                    int r = 0;
                    while (r < rows) {
                        int plane, sy, sz;
                        source_row<D>(p.g, y0 + r, z, cy, cz, lane, op, plane, sy, sz);
                        int len = 1;
                        while (r + len < rows) {
                            int pl2, sy2, sz2;
                            source_row<D>(p.g, y0 + r + len, z, cy, cz, lane, op, pl2, sy2, sz2);
                            if (pl2 != plane || sz2 != sz || sy2 != sy + len) break;
                            ++len;
                        }
                        const S* src = fin + (long long)plane * nc + ((long long)sz * ny + sy) * nx;
                        bulk_g2s(dst + (size_t)r * row_bytes, src, (uint32_t)(len * row_bytes),
                                 &full[s]);
                        r += len;
                    }
                } else {
                    const int W = ps.W;
                    int plane, sy, sz;
                    source_row<D>(p.g, y0, z, cy, cz, lane, op, plane, sy, sz);
                    const S* row = fin + (long long)plane * nc + ((long long)sz * ny + sy) * nx;
                    bulk_g2s(dst + HALO * ELT, row + x0, (uint32_t)(W * ELT), &full[s]);
                    bulk_g2s(dst, row + (x0 > 0 ? x0 - HALO : nx - HALO), 16u, &full[s]);
                    bulk_g2s(dst + (size_t)(HALO + W) * ELT, row + (x0 + W < nx ? x0 + W : 0),
                             16u, &full[s]);
                }
            }
            __syncwarp();
        }
        // drain: the copies of the last issued tiles must land before exit
        // (with the fixed ~2 s bound whatever the tuned wait limit: copies
        // in flight complete in microseconds)
        const long long issued = k;
        const long long first = issued > ps.stages ? issued - ps.stages : 0;
        for (long long j = first; j < issued; j++) {
            const int s = (int)(j % ps.stages);
            const uint32_t par = (uint32_t)((j / ps.stages) & 1);
            if (mbar_try_wait(&full[s], par)) continue;
            const long long t0 = clock64();
            while (!mbar_try_wait(&full[s], par)) {
                if (clock64() - t0 > PIPE_TIMEOUT_CYCLES) {
                    atomicOr(p.err, ERR_TIMEOUT);
                    break;
                }
            }
        }
        return;
    }

    // ---------------- consumers: warp c takes chunks c, c + NC, ... of every
    // tile (a chunk is 32 consecutive cells of one row) and arrives on the
    // stage's empty barrier once per tile, with or without work.
    const int cwarp = warp - 1;
    const R omega = param_omega<R>(p);
    long long k = 0;
    for (long long t = blockIdx.x; t < ps.ntiles; t += gridDim.x, ++k) {
        const int s = (int)(k % ps.stages);
        if (!wait_phase(&full[s], (uint32_t)((k / ps.stages) & 1), p.err, &abort_flag,
                        ps.wait_limit))
            break;
        int y0, z, x0, rows;
        decode_tile<D>(ps, p.g, t, y0, z, x0, rows);
        const unsigned char* stage = smem + (size_t)s * ps.stage_bytes;
        const int width = rows_mode ? nx : ps.W;
        const int chunks = rows * (width >> 5);
        for (int c = cwarp; c < chunks; c += NC) {
            const int r = c / (width >> 5);
            const int lx = (c - r * (width >> 5)) * 32 + lane;
            const int y = y0 + r;
            const int x = x0 + lx;
            const int a = (D == 2) ? y : z;
            const int Lw = (D == 2) ? ny : p.g.nz;
            const bool solid_m = walls && (a - 1 == 0);
            const bool solid_p = walls && (a + 1 == Lw - 1);
            const long long rowl = (long long)z * ny + y;
            const long long cell = rowl * nx + x;
            const long long seg = rowl * p.g.nseg_x + (x >> 5);
            int band = 0;
            if (lane == 0 && flags) band = flags[seg];
            band = __shfl_sync(0xffffffffu, band, 0);

            R g[Q];
#pragma unroll
            for (int i = 0; i < Q; i++) {
                const int cwl = (D == 2) ? L::cy(i) : L::cz(i);
                const bool bb = cwl == 0 ? false : (cwl > 0 ? solid_m : solid_p);
                const int shift = bb ? 0 : L::cx(i);
                const S* pl = reinterpret_cast<const S*>(stage + (size_t)i * ps.plane_bytes);
                int idx;
                if (rows_mode) {
                    int xs = lx - shift;
                    xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
                    idx = r * nx + xs;
                } else {
                    idx = HALO + lx - shift;
                }
                g[i] = T::load(pl, idx, p.inv_scale);
            }
            R Fx = param_body<R>(p, 0), Fy = param_body<R>(p, 1), Fz = param_body<R>(p, 2);
            if (band) take_band_force<D, R>(F, nc, cell, Fx, Fy, Fz);
            const CellMoments<Q, R> mo = cell_moments<Q, R>(g, Fx, Fy, Fz);
            cell_collide<Q, R>(g, mo, omega, Fx, Fy, Fz);
            store_cell<Q, ST, false>(fout, nc, cell, g, p.scale,
                                     ST == ST_FP16 ? sr_seed(step, cell) : 0u);
            if (WRITE_ALL || band) put_moments<D, R>(mom, nc, cell, mo.drho, mo.ux, mo.uy, mo.uz);
            if (!isfinite(mo.drho)) atomicOr(p.err, ERR_NONFINITE);
            if (lane == 0 && band) flags[seg] = 0;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }
}

// ------------------------------------------------------------------ host side
static int elt_of(int storage) { return storage == ST_FP64 ? 8 : (storage == ST_FP32 ? 4 : 2); }

// Dynamic shared memory a CTA may request: the opt-in maximum for one CTA per
// SM, half the SM's capacity for two; each less the static shared memory and
// the per-CTA reservation.
static int dyn_smem_limit(const SmemLimits& lim, int ctas_per_sm)
{
    const int one = lim.per_block_optin - 512;
    const int two = (lim.per_sm - 2 * 1024) / 2 - 512;
    return ctas_per_sm == 1 ? one : (two < one ? two : one);
}

bool pipe_shape(int Q, int storage, const GridParams& g, int sm_count, const SmemLimits& lim,
                int rows_per_tile, int ctas_per_sm, int consumer_warps, PipeShape& ps)
{
    if (ctas_per_sm == 2 && consumer_warps != 8) return false;
    if (ctas_per_sm == 1 && consumer_warps != 16 && consumer_warps != 24) return false;
    ps.consumer_warps = consumer_warps;
    ps.wait_limit = PIPE_TIMEOUT_CYCLES;
    const int elt = elt_of(storage);
    const int halo = 16 / elt;
    const int woff = g.walls ? 1 : 0;
    if (ctas_per_sm < 1 || ctas_per_sm > 2) return false;
    ps.ctas_per_sm = ctas_per_sm;
    const int budget = dyn_smem_limit(lim, ctas_per_sm) - 2 * 8 * 8;  // less the barriers
    if (g.nx % 32 == 0 && g.nx <= 1024) {
        ps.mode = PIPE_ROWS;
        const int ny_f = (g.dim == 2) ? g.ny - 2 * woff : g.ny;
        const long long nz_f = (g.dim == 2) ? 1 : (long long)(g.nz - 2 * woff);
        int R = rows_per_tile > 0 ? rows_per_tile : 1;
        // at least 2 stages
        while (R > 1 && 2LL * Q * R * g.nx * elt > budget) R--;
        if (R > ny_f) R = ny_f;
        ps.R = R;
        ps.W = g.nx;
        ps.nseg = 1;
        ps.yblocks = (ny_f + R - 1) / R;
        ps.ntiles = nz_f * ps.yblocks;
        ps.plane_bytes = R * g.nx * elt;
        ps.tx_bytes = (long long)Q * ps.plane_bytes;
    } else {
        if (g.nx % 256 != 0 || g.nx % halo != 0) return false;
        ps.mode = PIPE_SEGMENTS;
        int W = g.nx;
        while (W > 1024 || 2LL * Q * (W * elt + 32) > budget) {
            if (W % 2 != 0 || (W / 2) % 256 != 0) return false;
            W /= 2;
        }
        const long long rows = (g.dim == 2) ? (long long)(g.ny - 2 * woff)
                                            : (long long)g.ny * (g.nz - 2 * woff);
        ps.R = 1;
        ps.W = W;
        ps.nseg = g.nx / W;
        ps.yblocks = 0;
        ps.ntiles = rows * ps.nseg;
        ps.plane_bytes = (W + 2 * halo) * elt;
        ps.tx_bytes = (long long)Q * (W * elt + 32);
    }
    ps.stage_bytes = Q * ps.plane_bytes;
    ps.stages = budget / ps.stage_bytes;
    if (ps.stages > 8) ps.stages = 8;
    if (ps.stages < 2) return false;
    ps.smem_bytes = ps.stages * ps.stage_bytes + 2 * ps.stages * 8;
    ps.grid = sm_count * ps.ctas_per_sm;
    if (ps.ntiles < ps.grid) ps.grid = (int)ps.ntiles;
    return ps.tx_bytes < (1 << 20) && ps.ntiles > 0;
}

template <int Q, int ST, int NC>
static void launch_pipe_nc(bool write_all, const typename StorageT<ST>::S* a,
                           typename StorageT<ST>::S* b, typename StorageT<ST>::R* m,
                           typename StorageT<ST>::R* f, uint8_t* flags, const StreamParams& p,
                           const PipeShape& ps, cudaStream_t s)
{
    if (write_all)
        k_sc_pipe<Q, ST, true, NC><<<ps.grid, 32 * (NC + 1), ps.smem_bytes, s>>>(a, b, m, f, flags, p, ps);
    else
        k_sc_pipe<Q, ST, false, NC><<<ps.grid, 32 * (NC + 1), ps.smem_bytes, s>>>(a, b, m, f, flags, p, ps);
}

template <int Q, int ST>
static cudaError_t launch_pipe_t(bool write_all, const void* fin, void* fout, void* mom, void* F,
                                 uint8_t* flags, const StreamParams& p, const PipeShape& ps,
                                 cudaStream_t s)
{
    using T = StorageT<ST>;
    auto* a = (const typename T::S*)fin;
    auto* b = (typename T::S*)fout;
    auto* m = (typename T::R*)mom;
    auto* f = (typename T::R*)F;
    if (ps.consumer_warps == 24)
        launch_pipe_nc<Q, ST, 24>(write_all, a, b, m, f, flags, p, ps, s);
    else if (ps.consumer_warps == 16)
        launch_pipe_nc<Q, ST, 16>(write_all, a, b, m, f, flags, p, ps, s);
    else
        launch_pipe_nc<Q, ST, 8>(write_all, a, b, m, f, flags, p, ps, s);
    return cudaGetLastError();
}

template <int Q, int ST>
static cudaError_t prepare_t(int bytes)
{
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(k_sc_pipe<Q, ST, true, 8>, a, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sc_pipe<Q, ST, false, 8>, a, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sc_pipe<Q, ST, true, 16>, a, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sc_pipe<Q, ST, false, 16>, a, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sc_pipe<Q, ST, true, 24>, a, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sc_pipe<Q, ST, false, 24>, a, bytes);
    return e;
}

cudaError_t prepare_stream_collide_pipe(const SmemLimits& lim)
{
    static int done_bytes = -1;
    const int bytes = dyn_smem_limit(lim, 1);
    if (done_bytes == bytes) return cudaSuccess;
    cudaError_t e = prepare_t<9, ST_FP64>(bytes);
    if (e == cudaSuccess) e = prepare_t<9, ST_FP32>(bytes);
    if (e == cudaSuccess) e = prepare_t<9, ST_FP16>(bytes);
    if (e == cudaSuccess) e = prepare_t<19, ST_FP64>(bytes);
    if (e == cudaSuccess) e = prepare_t<19, ST_FP32>(bytes);
    if (e == cudaSuccess) e = prepare_t<19, ST_FP16>(bytes);
    if (e == cudaSuccess) done_bytes = bytes;
    return e;
}

cudaError_t launch_stream_collide_pipe(int Q, int storage, bool write_all, const void* fin,
                                       void* fout, void* moments, void* F, uint8_t* flags,
                                       const StreamParams& p, const PipeShape& ps, cudaStream_t s)
{
    if (Q == 9) {
        if (storage == ST_FP64) return launch_pipe_t<9, ST_FP64>(write_all, fin, fout, moments, F, flags, p, ps, s);
        if (storage == ST_FP32) return launch_pipe_t<9, ST_FP32>(write_all, fin, fout, moments, F, flags, p, ps, s);
        return launch_pipe_t<9, ST_FP16>(write_all, fin, fout, moments, F, flags, p, ps, s);
    }
    if (storage == ST_FP64) return launch_pipe_t<19, ST_FP64>(write_all, fin, fout, moments, F, flags, p, ps, s);
    if (storage == ST_FP32) return launch_pipe_t<19, ST_FP32>(write_all, fin, fout, moments, F, flags, p, ps, s);
    return launch_pipe_t<19, ST_FP16>(write_all, fin, fout, moments, F, flags, p, ps, s);
}

}  // namespace iblb
