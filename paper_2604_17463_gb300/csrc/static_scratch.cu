// static_scratch.cu -- an entry point that allocates no device memory:
// the FP64 population mass of a caller-owned population array.
//
// Some callers cannot allocate device memory at the time they need this
// number: a host application that reserves all of its GPU memory up front
// (a serving process running from a fixed pool), code running while another
// library holds the device allocator, or an embedding that forbids
// allocations after initialisation.  iblb_mass_static gives them the mass
// reduction of iblb_observables without cudaMalloc: its per-block partial
// sums live in the file-scope device array below (IBLB_STATIC_PARTIALS
// doubles, 512 KiB, held by every GPU that loads the library until the
// process exits).  The caller passes the populations and the output.
#include <atomic>
#include <cmath>

#include "../../include/iblb.h"
#include "lbm_core.cuh"

// Per-block partial sums.  In host code this name is only a stand-in for the
// symbol (not a device address); the device address comes from
// cudaGetSymbolAddress in iblb_mass_static.
static __device__ __align__(256) double g_mass_partials[IBLB_STATIC_PARTIALS];

namespace iblb {
namespace {

constexpr int MS_THREADS = 256;
constexpr int MS_CELLS_PER_THREAD = 64;
constexpr long long MS_CELLS_PER_BLOCK = (long long)MS_THREADS * MS_CELLS_PER_THREAD;
constexpr int MS_MAX_DEVICES = 64;

// Device address of g_mass_partials per device, resolved by the first call on
// that device.  Atomic, so that host threads making their first calls at the
// same time do not race (both resolve the same address).
std::atomic<double*> g_partials_addr[MS_MAX_DEVICES];
constexpr int MS_TOTAL_THREADS = 256;

// Block b sums the fluid cells [b * MS_CELLS_PER_BLOCK, (b+1) * MS_CELLS_PER_BLOCK)
// in a fixed order and overwrites partial[b]: no entry needs clearing.
template <int ST>
__global__ void __launch_bounds__(MS_THREADS)
k_mass_static_partials(int Q, const typename StorageT<ST>::S* __restrict__ f, GridParams g,
                       float inv_scale, double* __restrict__ partial)
{
    const long long first = blockIdx.x * MS_CELLS_PER_BLOCK;
    const long long end = min(first + MS_CELLS_PER_BLOCK, g.ncell);
    const long long plane = (long long)g.nx * g.ny;
    double acc = 0.0;
    for (long long c = first + threadIdx.x; c < end; c += MS_THREADS) {
        if (g.walls) {
            const int a = (g.dim == 2) ? (int)((c / g.nx) % g.ny) : (int)(c / plane);
            const int Lw = (g.dim == 2) ? g.ny : g.nz;
            if (a == 0 || a == Lw - 1) continue;
        }
        double dev = 0.0;
        for (int i = 0; i < Q; i++)
            dev += (double)StorageT<ST>::load(f, (long long)i * g.ncell + c, inv_scale);
        acc += 1.0 + dev;
    }
    __shared__ double red[MS_THREADS / 32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < MS_THREADS / 32; w++) t += red[w];
        partial[blockIdx.x] = t;
    }
}

// One block adds the n partials in a fixed order: thread k sums the
// contiguous range [k * n / T, (k + 1) * n / T), then a fixed shuffle and
// shared-memory tree combines the T sums.  The order depends on n only, so
// the result is deterministic.
__global__ void __launch_bounds__(MS_TOTAL_THREADS)
k_mass_static_total(const double* __restrict__ partial, int n, double* out)
{
    const int k = threadIdx.x;
    const int lo = (int)((long long)k * n / MS_TOTAL_THREADS);
    const int hi = (int)((long long)(k + 1) * n / MS_TOTAL_THREADS);
    double t = 0.0;
    for (int b = lo; b < hi; b++) t += partial[b];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    __shared__ double red[MS_TOTAL_THREADS / 32];
    if ((k & 31) == 0) red[k >> 5] = t;
    __syncthreads();
    if (k == 0) {
        double s = 0.0;
        for (int w = 0; w < MS_TOTAL_THREADS / 32; w++) s += red[w];
        *out = s;
    }
}

}  // namespace
}  // namespace iblb

using namespace iblb;

extern "C" iblb_status iblb_mass_static(const void* f_dev, int lattice, int storage, int nx, int ny,
                                        int nz, int walls, int fp16_scale_exp, double* mass_dev,
                                        void* cuda_stream)
{
    if (!f_dev || !mass_dev) return IBLB_EINVAL;
    if (lattice != IBLB_D2Q9 && lattice != IBLB_D3Q19) return IBLB_EINVAL;
    if (storage < IBLB_FP64 || storage > IBLB_FP16_DEV) return IBLB_EINVAL;
    const int dim = lattice == IBLB_D2Q9 ? 2 : 3;
    if (dim == 2) nz = 1;
    if (nx < 1 || ny < 1 || nz < 1) return IBLB_EINVAL;
    if (walls && (dim == 2 ? ny : nz) < 3) return IBLB_EINVAL;
    if (fp16_scale_exp < 0 || fp16_scale_exp > 24) return IBLB_EINVAL;
    const long long ncell = (long long)nx * ny * nz;
    const long long nblocks = (ncell + MS_CELLS_PER_BLOCK - 1) / MS_CELLS_PER_BLOCK;
    if (nblocks > IBLB_STATIC_PARTIALS) return IBLB_EINVAL;  // lattice beyond the static scratch

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MS_MAX_DEVICES) return IBLB_ECUDA;
    double* partial = g_partials_addr[dev].load(std::memory_order_acquire);
    if (!partial) {
        // first call on this device (with it current): resolve the device
        // address of the static array once
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_mass_partials) != cudaSuccess || !ptr) return IBLB_ECUDA;
        partial = static_cast<double*>(ptr);
        g_partials_addr[dev].store(partial, std::memory_order_release);
    }

    GridParams g{};
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.dim = dim;
    g.walls = walls ? 1 : 0;
    g.nseg_x = (nx + 31) / 32;
    g.ncell = ncell;
    const float inv_scale =
        storage == IBLB_FP16_DEV ? 1.0f / std::ldexp(1.0f, fp16_scale_exp ? fp16_scale_exp : 16) : 1.0f;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int nb = (int)nblocks;
    if (storage == IBLB_FP64)
        k_mass_static_partials<ST_FP64><<<nb, MS_THREADS, 0, s>>>(lattice, (const double*)f_dev, g, inv_scale, partial);
    else if (storage == IBLB_FP32_DEV)
        k_mass_static_partials<ST_FP32><<<nb, MS_THREADS, 0, s>>>(lattice, (const float*)f_dev, g, inv_scale, partial);
    else
        k_mass_static_partials<ST_FP16><<<nb, MS_THREADS, 0, s>>>(lattice, (const __half*)f_dev, g, inv_scale, partial);
    k_mass_static_total<<<1, MS_TOTAL_THREADS, 0, s>>>(partial, nb, mass_dev);
    if (cudaGetLastError() != cudaSuccess) return IBLB_ECUDA;
    add_launches(2);
    return IBLB_OK;
}
