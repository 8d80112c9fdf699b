// lbm_pipe.cu -- pipelined stream-collide kernel (A4) for GB300.
//
// Same update as the plain kernel in lbm.cu (pull streaming with halfway
// bounce-back, moments with the half-force term, BGK + Guo, Eq. 1-6), with
// the loads decoupled from the arithmetic:
//   - persistent CTAs (a few per SM) walk the tiles round-robin; a tile is one
//     x-segment of W cells (W a multiple of 256) of one fluid row;
//   - a producer warp stages, for each of the Q directions, the source-row
//     segment of the tile plus a 16-byte halo on each side into shared memory
//     with bulk asynchronous copies (cp.async.bulk, completion counted in
//     bytes on an mbarrier), several tiles ahead of the consumers;
//   - eight consumer warps read the shifted populations from shared memory,
//     collide and store the new populations with coalesced stores, then
//     release the stage on a second mbarrier.
// For a direction whose source row is a solid layer (bounce-back) the
// producer stages the opposite direction of the current row instead, and the
// consumer reads it unshifted.
// Every wait is bounded: after ~2 s a waiting thread latches ERR_TIMEOUT and
// the CTA stops; the producer always waits (bounded) for the copies it issued
// before it exits.
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

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

constexpr long long PIPE_TIMEOUT_CYCLES = 4000000000LL;  // ~2 s at 2 GHz

// Bounded wait for the phase of `bar` with the given parity.  Returns false
// (and stops the CTA) on timeout or when another thread of the CTA gave up.
__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t parity, int* err,
                                           volatile int* abort_flag)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > PIPE_TIMEOUT_CYCLES) {
            atomicOr(err, ERR_TIMEOUT);
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}

}  // namespace

constexpr int PIPE_CONSUMER_WARPS = 8;
constexpr int PIPE_THREADS = 32 * (1 + PIPE_CONSUMER_WARPS);

template <int Q, int ST, bool WRITE_ALL>
__global__ void __launch_bounds__(PIPE_THREADS, 2)
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
    const int woff = walls ? 1 : 0;
    const int W = ps.W;

    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < ps.stages; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], PIPE_CONSUMER_WARPS);
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
                if (!wait_phase(&empty[s], par, p.err, &abort_flag)) break;
            }
            const long long row_idx = t / ps.nseg;
            const int x0 = (int)(t - row_idx * ps.nseg) * W;
            int y, z;
            if (D == 2) {
                y = (int)row_idx + woff;
                z = 0;
            } else {
                z = (int)(row_idx / ny) + woff;
                y = (int)(row_idx % ny);
            }
            unsigned char* stage = smem + (size_t)s * ps.stage_bytes;
            if (lane == 0) mbar_arrive_expect_tx(&full[s], (uint32_t)ps.tx_bytes);
            __syncwarp();
            if (lane < Q) {
                const int cx = tab<Q>().v[lane][0], cy = tab<Q>().v[lane][1];
                const int cz = tab<Q>().v[lane][2], op = tab<Q>().v[lane][3];
                (void)cx;
                int plane = lane, sy = y, sz = z;
                bool bb = false;
                if (D == 2) {
                    int sa = y - cy;
                    if (walls) bb = (sa <= 0 || sa >= ny - 1);
                    else sa = (sa + ny) % ny;
                    sy = sa;
                } else {
                    sy = (y - cy + ny) % ny;
                    int sa = z - cz;
                    const int nz = p.g.nz;
                    if (walls) bb = (sa <= 0 || sa >= nz - 1);
                    else sa = (sa + nz) % nz;
                    sz = sa;
                }
                if (bb) {
                    plane = op;
                    sy = y;
                    sz = z;
                }
                const S* row = fin + (long long)plane * nc + ((long long)sz * ny + sy) * nx;
                unsigned char* dst = stage + (size_t)lane * ps.plane_bytes;
                bulk_g2s(dst + HALO * ELT, row + x0, (uint32_t)(W * ELT), &full[s]);
                bulk_g2s(dst, row + (x0 > 0 ? x0 - HALO : nx - HALO), 16u, &full[s]);
                bulk_g2s(dst + (size_t)(HALO + W) * ELT, row + (x0 + W < nx ? x0 + W : 0), 16u,
                         &full[s]);
            }
            __syncwarp();
        }
        // drain: the copies of the last issued tiles must land before exit
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

    // ---------------- consumers: warp c takes chunks c, c + 8, ... of every tile
    const int cwarp = warp - 1;
    const R omega = (R)p.omega;
    long long k = 0;
    for (long long t = blockIdx.x; t < ps.ntiles; t += gridDim.x, ++k) {
        const int s = (int)(k % ps.stages);
        if (!wait_phase(&full[s], (uint32_t)((k / ps.stages) & 1), p.err, &abort_flag)) break;
        const long long row_idx = t / ps.nseg;
        const int x0 = (int)(t - row_idx * ps.nseg) * W;
        int y, z;
        if (D == 2) {
            y = (int)row_idx + woff;
            z = 0;
        } else {
            z = (int)(row_idx / ny) + woff;
            y = (int)(row_idx % ny);
        }
        const int a = (D == 2) ? y : z;
        const int Lw = (D == 2) ? ny : p.g.nz;
        const bool solid_m = walls && (a - 1 == 0);
        const bool solid_p = walls && (a + 1 == Lw - 1);
        const unsigned char* stage = smem + (size_t)s * ps.stage_bytes;
        const long long rowl = (long long)z * ny + y;

        for (int lx0 = cwarp * 32; lx0 < W; lx0 += PIPE_CONSUMER_WARPS * 32) {
            const int lx = lx0 + lane;
            const int x = x0 + lx;
            const long long cell = rowl * nx + x;
            const long long seg = rowl * p.g.nseg_x + (x >> 5);
            int band = 0;
            if (lane == 0) band = flags[seg];
            band = __shfl_sync(0xffffffffu, band, 0);

            R g[Q];
#pragma unroll
            for (int i = 0; i < Q; i++) {
                const int cwl = (D == 2) ? L::cy(i) : L::cz(i);
                const bool bb = cwl == 0 ? false : (cwl > 0 ? solid_m : solid_p);
                const int shift = bb ? 0 : L::cx(i);
                const S* pl = reinterpret_cast<const S*>(stage + (size_t)i * ps.plane_bytes);
                g[i] = T::load(pl, HALO + lx - shift, p.inv_scale);
            }
            R Fx = (R)p.body[0], Fy = (R)p.body[1], Fz = (R)p.body[2];
            if (band) {
                Fx += F[cell];
                Fy += F[nc + cell];
                F[cell] = 0;
                F[nc + cell] = 0;
                if (D == 3) {
                    Fz += F[2 * nc + cell];
                    F[2 * nc + cell] = 0;
                }
            }
            const CellMoments<Q, R> mo = cell_moments<Q, R>(g, Fx, Fy, Fz);
            cell_collide<Q, R>(g, mo, omega, Fx, Fy, Fz);
#pragma unroll
            for (int i = 0; i < Q; i++) T::store(fout, (long long)i * nc + cell, g[i], p.scale);
            if (WRITE_ALL || band) {
                mom[cell] = mo.drho;
                mom[nc + cell] = mo.ux;
                mom[2 * nc + cell] = mo.uy;
                if (D == 3) mom[3 * nc + cell] = mo.uz;
            }
            if (!isfinite(mo.drho)) atomicOr(p.err, ERR_NONFINITE);
            if (lane == 0 && band) flags[seg] = 0;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }
}

// ------------------------------------------------------------------ host side
bool pipe_shape(int Q, int storage, const GridParams& g, int sm_count, PipeShape& ps)
{
    const int elt = storage == ST_FP64 ? 8 : (storage == ST_FP32 ? 4 : 2);
    const int halo = 16 / elt;
    if (g.nx % 256 != 0 || g.nx % halo != 0) return false;
    int W = g.nx;
    while (W > 1024) {
        if (W % 2 != 0 || (W / 2) % 256 != 0) return false;
        W /= 2;
    }
    const int woff = g.walls ? 1 : 0;
    const long long rows = (g.dim == 2) ? (long long)(g.ny - 2 * woff)
                                        : (long long)g.ny * (g.nz - 2 * woff);
    ps.W = W;
    ps.nseg = g.nx / W;
    ps.ntiles = rows * ps.nseg;
    ps.plane_bytes = (W + 2 * halo) * elt;
    ps.stage_bytes = Q * ps.plane_bytes;
    ps.tx_bytes = (long long)Q * (W * elt + 32);
    ps.ctas_per_sm = 2;
    const int budget = PIPE_SMEM_PER_CTA - 1024;
    ps.stages = budget / ps.stage_bytes;
    if (ps.stages > 8) ps.stages = 8;
    if (ps.stages < 2) return false;
    ps.smem_bytes = ps.stages * ps.stage_bytes + 2 * ps.stages * 8;
    ps.grid = sm_count * ps.ctas_per_sm;
    if (ps.ntiles < ps.grid) ps.grid = (int)ps.ntiles;
    return ps.tx_bytes < (1 << 20);
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
    if (write_all)
        k_sc_pipe<Q, ST, true><<<ps.grid, PIPE_THREADS, ps.smem_bytes, s>>>(a, b, m, f, flags, p, ps);
    else
        k_sc_pipe<Q, ST, false><<<ps.grid, PIPE_THREADS, ps.smem_bytes, s>>>(a, b, m, f, flags, p, ps);
    return cudaGetLastError();
}

template <int Q, int ST>
static cudaError_t prepare_t()
{
    const int bytes = PIPE_SMEM_PER_CTA;
    cudaError_t e = cudaFuncSetAttribute(k_sc_pipe<Q, ST, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sc_pipe<Q, ST, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

cudaError_t prepare_stream_collide_pipe()
{
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = prepare_t<9, ST_FP64>();
    if (e == cudaSuccess) e = prepare_t<9, ST_FP32>();
    if (e == cudaSuccess) e = prepare_t<9, ST_FP16>();
    if (e == cudaSuccess) e = prepare_t<19, ST_FP64>();
    if (e == cudaSuccess) e = prepare_t<19, ST_FP32>();
    if (e == cudaSuccess) e = prepare_t<19, ST_FP16>();
    if (e == cudaSuccess) done = true;
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
