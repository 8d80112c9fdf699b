// common.cuh -- internal declarations shared by the CUDA translation units of
// libiblb (lattice stencils, kernel parameter blocks, launchers).
//
// Lattice: D2Q9 and D3Q19 (the paper uses D3Q19, Sec. 2; D2Q9 is its 2D
// analogue).  The weights are the standard ones for these stencils; the paper
// does not print them.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace iblb {

// ------------------------------------------------------------------ stencils
// Velocity order (shared with the host-visible population layout):
//   D2Q9 : rest, +x, +y, -x, -y, (+x+y), (-x+y), (-x-y), (+x-y)
//   D3Q19: rest, +x, -x, +y, -y, +z, -z, then the 12 edge directions in
//          opposite pairs (2k+1, 2k+2).
template <int Q> struct Stencil;

template <> struct Stencil<9> {
    static constexpr int D = 2;
    __host__ __device__ static constexpr int cx(int i) {
        constexpr int t[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
        return t[i];
    }
    __host__ __device__ static constexpr int cy(int i) {
        constexpr int t[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
        return t[i];
    }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __host__ __device__ static constexpr int opp(int i) {
        constexpr int t[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
        return t[i];
    }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
};

template <> struct Stencil<19> {
    static constexpr int D = 3;
    __host__ __device__ static constexpr int cx(int i) {
        constexpr int t[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 0, 0, 1, -1, 1, -1, 0, 0};
        return t[i];
    }
    __host__ __device__ static constexpr int cy(int i) {
        constexpr int t[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 1, -1};
        return t[i];
    }
    __host__ __device__ static constexpr int cz(int i) {
        constexpr int t[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 1, -1, 1, -1, 0, 0, -1, 1, -1, 1};
        return t[i];
    }
    __host__ __device__ static constexpr int opp(int i) {
        return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1);
    }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
};

// Device error flags (bitwise OR).
enum : int { ERR_NODE_IN_WALL = 1, ERR_NONFINITE = 2, ERR_TIMEOUT = 4, ERR_CLASSIFY = 8 };

// Interface crossings kept per lattice column for the inside / outside test.
constexpr int COL_MAX = 16;

// ------------------------------------------------------------------ params
struct GridParams {
    int nx, ny, nz;        // extent (nz = 1 in 2D)
    int dim;               // 2 or 3
    int walls;             // solid first/last layer along the wall axis
    int nseg_x;            // 32-cell band segments per x row
    long long ncell;       // nx * ny * nz
};

struct StreamParams {
    GridParams g;
    double omega;          // 1 / tau
    double body[3];        // uniform force density
    float omega_f;         // the same in FP32 (no per-thread conversion on the FP32 paths)
    float body_f[3];
    // viscosity ratio: cells outside the interface relax with omega_out
    int two_tau;
    double omega_out;
    const int* col_cnt;    // crossings per column
    const double* col_z;   // [column][COL_MAX] crossing heights
    // moving walls (tangential velocities of the lower / upper wall)
    int moving;
    double uw_lo[3], uw_hi[3];
    // time-step counter for the stochastic rounding of binary16 stores:
    // read rng_in, one thread writes rng_out = rng_in + 1
    const unsigned* rng_in;
    unsigned* rng_out;
    float scale, inv_scale;  // binary16 storage scale (1 for other storage)
    int* err;
};

struct ForceParams {
    double sigma;
    double A, xi;          // wetting amplitude (Eq. 11) and length
    int n, m;              // exponents of Pi
    int wetting;
    double wall_plane;     // 0.5
    // elastic interface (Skalak): shear modulus, area-dilation parameter and
    // the reference data of the interface as set (null when Gs = 0):
    // 3D [M][5] = inverse reference edge matrix (4) and reference area per
    // face; 2D [N] = reference length per segment
    double Gs, Cs;
    const double* eref;
};

// Layout of the force density F and of the moments in device memory: in
// FP32 compute precision one float4 per cell, F = (Fx, Fy, Fz, 0) and
// moments = (drho, ux, uy, uz) (uz = 0 in 2D), so that spreading adds one
// vector per stencil point and interpolation reads one; in FP64,
// [component][cell] arrays (F: dim components, moments: 1 + dim).
inline size_t force_bytes(int storage, int dim, long long ncell)
{
    return storage == 0 ? sizeof(double) * (size_t)dim * (size_t)ncell
                        : sizeof(float) * 4 * (size_t)ncell;
}
inline size_t moments_bytes(int storage, int dim, long long ncell)
{
    return storage == 0 ? sizeof(double) * (size_t)(1 + dim) * (size_t)ncell
                        : sizeof(float) * 4 * (size_t)ncell;
}

// Launch shape of the stream-collide kernel (chosen by the autotuner).
struct Tuning {
    int variant = 1;            // 0: plain kernel; 1: pipelined kernel; 2: cell pairs along x;
                                // 3: row pairs (where the shape allows)
    int block_x = 128;          // plain kernel: threads per block along x (64, 128, 256)
    int streaming_stores = 0;   // plain kernel: evict-first stores of the new populations
    int rows_per_tile = 2;      // pipelined kernel, rows mode: rows per tile
    int ctas_per_sm = 2;        // pipelined kernel: resident CTAs per SM (1 or 2)
    int consumer_warps = 8;     // pipelined kernel: 8 (2 CTAs/SM), 16 or 24 (1 CTA/SM)
    long long wait_limit = 0;   // pipelined kernel: clock cycles a wait may take (0: ~2 s)
    int ib_grouped = 0;         // 3D interfaces: 1 spreads / interpolates by spatial groups of
                                // nodes (ib_groups.cu) instead of one thread per node
    int step_overlap = 0;       // 0: overlapped step on 3D lattices of >= 2^20 cells; 1: always;
                                // 2: never (see enqueue_step_overlapped)
};

// Shape of the pipelined stream-collide launch (see lbm_pipe.cu).
enum : int { PIPE_ROWS = 0, PIPE_SEGMENTS = 1 };
struct PipeShape {
    int mode;              // PIPE_ROWS: R whole rows per tile; PIPE_SEGMENTS: W-cell segments
    int R;                 // rows per tile (rows mode)
    int yblocks;           // tiles along y per layer (rows mode)
    int W;                 // tile width in cells (segment mode: multiple of 256)
    int nseg;              // tiles per row (segment mode)
    long long ntiles;      // tiles in the lattice
    int plane_bytes;       // shared-memory bytes of one staged direction
    int stage_bytes;       // Q * plane_bytes
    long long tx_bytes;    // bytes copied per full stage
    int stages;            // pipeline depth per CTA
    int ctas_per_sm;
    int consumer_warps;    // consumer warps per CTA (8, 16 or 24)
    int smem_bytes;        // dynamic shared memory per CTA
    int grid;              // persistent CTAs
    long long wait_limit;  // clock cycles a pipeline wait may take before it gives up
};
// Shared-memory limits of the device (bytes), read at creation.
struct SmemLimits {
    int per_block_optin;   // cudaDevAttrMaxSharedMemoryPerBlockOptin
    int per_sm;            // cudaDevAttrMaxSharedMemoryPerMultiprocessor
};

// ------------------------------------------------------------------ launchers
// Storage ids match iblb_storage.
enum Storage : int { ST_FP64 = 0, ST_FP32 = 1, ST_FP16 = 2 };

// One fused stream-collide step over every fluid cell (pull, halfway
// bounce-back, Guo forcing).  fin/fout: population deviations [Q][ncell];
// moments: drho [ncell] then u [dim][ncell] (compute precision); F: force
// density [dim][ncell], read and cleared only in flagged band segments.
void launch_stream_collide(int Q, int storage, bool write_all, const void* fin, void* fout,
                           void* moments, void* F, uint8_t* flags, const StreamParams& p,
                           const Tuning& tu, cudaStream_t s);

// Pair variant (lbm.cu): two x-adjacent cells per thread, packed FP32x2
// arithmetic; FP32 / binary16 storage with an even nx.
bool pair_kernel_ok(int storage, const GridParams& g);
void launch_stream_collide_pairs(int Q, int storage, bool write_all, const void* fin, void* fout,
                                 void* moments, void* F, uint8_t* flags, const StreamParams& p,
                                 const Tuning& tu, cudaStream_t s);

// Row-pair variant (lbm.cu): two y-adjacent cells per thread, packed FP32x2
// arithmetic; D3Q19 with FP32 / binary16 storage.
bool rowpair_kernel_ok(int Q, int storage, const GridParams& g);
void launch_stream_collide_rowpairs(int storage, bool write_all, const void* fin, void* fout,
                                    void* moments, void* F, uint8_t* flags, const StreamParams& p,
                                    const Tuning& tu, cudaStream_t s);

// Pipelined variant (lbm_pipe.cu): usable when pipe_shape() returns true.
bool pipe_shape(int Q, int storage, const GridParams& g, int sm_count, const SmemLimits& lim,
                int rows_per_tile, int ctas_per_sm, int consumer_warps, PipeShape& ps);
cudaError_t prepare_stream_collide_pipe(const SmemLimits& lim);
cudaError_t launch_stream_collide_pipe(int Q, int storage, bool write_all, const void* fin,
                                       void* fout, void* moments, void* F, uint8_t* flags,
                                       const StreamParams& p, const PipeShape& ps, cudaStream_t s);

// Band cells of the overlapped step (lbm.cu): after a bulk pass with
// flags == nullptr, list the flagged segments (list: one int per segment at
// most) and update their cells again with the force density and the
// moments, 8-cell quarter by quarter: the quarters marked in `fine` (4 bytes
// per segment, 4-byte aligned), all four of a flagged segment without
// marks.  Flags and marks are cleared.  list: one int per quarter at most;
// count: one int, reset here.  Three operations on stream s (a 4-byte
// memset and two kernels).
void launch_band_cells(int Q, int storage, const void* fin, void* fout, void* moments, void* F,
                       uint8_t* flags, uint8_t* fine, int* list, int* count,
                       const StreamParams& p, int sm_count, cudaStream_t s);
constexpr int BAND_KERNELS = 2;

// Host FP64 <-> device storage conversion of populations ([Q][ncell], f_i).
void launch_pack_populations(int Q, int storage, const double* f, void* dst, long long ncell,
                             float scale, cudaStream_t s);
void launch_unpack_populations(int Q, int storage, const void* src, double* f, long long ncell,
                               float inv_scale, cudaStream_t s);
// Moments (compute precision) -> FP64 rho [ncell] and u [dim][ncell].
void launch_unpack_moments(int storage, const GridParams& g, const void* moments, double* rho,
                           double* u, cudaStream_t s);
// Initialise moments to the rest state (drho = 0 on fluid, -1 on solid).
void launch_init_moments(int storage, const GridParams& g, void* moments, cudaStream_t s);
// Dense FP64 u [dim][ncell] -> moments' u part (compute precision).
void launch_load_velocity(int storage, int dim, const double* u, void* moments, long long ncell,
                          cudaStream_t s);
// F [dim][ncell] (compute precision) plus body force on fluid cells -> FP64.
void launch_unpack_force(int storage, const GridParams& g, const void* F, const double* body,
                         double* out, cudaStream_t s);
void launch_clear_flags(uint8_t* flags, long long n, cudaStream_t s);
void launch_set_all_flags(uint8_t* flags, long long n, cudaStream_t s);
// Mass of the populations: per-block FP64 partial sums into `partial`
// (length mass_partial_blocks(g)); sum them in order afterwards.
int mass_partial_blocks(const GridParams& g);
void launch_mass_partials(int Q, int storage, const void* f, const GridParams& g, float inv_scale,
                          double* partial, cudaStream_t s);

// IB kernels.  q, phi: [N][dim] FP64.
// 2D ring: one kernel; 3D mesh: per-face geometry written as one record per
// (face, corner) at its CSR position entry_pos[3f + corner] (8 doubles per
// record), then a per-node sum over its contiguous records (two kernels).
void launch_forces(int dim, const double* q, int N, int M, const int* tri, const int* csr_ptr,
                   const int* entry_pos, double* entry_rec, const ForceParams& fp, double* phi,
                   double* normal, double* chi, int* err, cudaStream_t s);
constexpr int ENTRY_RECORD_DOUBLES = 8;
// fine (may be null): one byte per 8-cell quarter of each segment (4 per
// segment), set where a stencil touches it, for the band pass.
void launch_spread(int storage, int dim, const double* q, const double* phi, int N, void* F,
                   uint8_t* flags, uint8_t* fine, const GridParams& g, cudaStream_t s);
// qdot [N][dim] = sum u Delta; if advect, q += qdot.
void launch_interp(int storage, int dim, double* q, const void* moments, int N, double* qdot,
                   bool advect, const GridParams& g, cudaStream_t s);

// Spatial groups of 3D interface nodes (ib_groups.cu): nodes of one
// GROUP_TILE^3 tile of the lattice, at most GROUP_NODES per group; the
// grouped spread / interpolation hold a group's box of the lattice in shared
// memory (box_cap cells).
constexpr int GROUP_TILE = 8;
constexpr int GROUP_NODES = 128;
template <typename R>
constexpr int box_cap() { return sizeof(R) == 4 ? 2048 : 1536; }
struct NodeGroups {
    int* tile_cnt = nullptr;   // [ntiles] nodes per tile (zero between regroups)
    int* tile_off = nullptr;   // [ntiles] first list position of each tile
    int* key = nullptr;        // [N] tile of each node
    int* rank = nullptr;       // [N] position of each node within its tile
    int* list = nullptr;       // [N] nodes ordered by tile
    int2* desc = nullptr;      // [max_groups] (first list position, node count)
    int* ngroups = nullptr;    // [1]
    int ntiles = 0, max_groups = 0;
};
// Tiles of a lattice and the bound on the number of groups of N nodes.
inline int group_tiles(const GridParams& g)
{
    return ((g.nx + GROUP_TILE - 1) / GROUP_TILE) * ((g.ny + GROUP_TILE - 1) / GROUP_TILE) *
           ((g.nz + GROUP_TILE - 1) / GROUP_TILE);
}
inline int group_bound(int N, int ntiles)
{
    return (N + GROUP_NODES - 1) / GROUP_NODES + (N < ntiles ? N : ntiles);
}
void launch_regroup(const double* q, int N, const GridParams& g, const NodeGroups& ng,
                    cudaStream_t s);
constexpr int REGROUP_KERNELS = 3;
void launch_spread_grouped(int storage, const double* q, const double* phi, const NodeGroups& ng,
                           void* F, uint8_t* flags, const GridParams& g, int sm_count,
                           cudaStream_t s);
void launch_interp_grouped(int storage, double* q, const void* moments, const NodeGroups& ng,
                           double* qdot, bool advect, const GridParams& g, int sm_count,
                           cudaStream_t s);

// Elastic reference of the interface at its current positions (see
// ForceParams::eref).
void launch_elastic_reference(int dim, const double* q, int N, int M, const int* tri, double* eref,
                              cudaStream_t s);

// Observables (single block, deterministic).  out: 12 doubles, layout of iblb_obs.
void launch_observables(int dim, const double* q, int N, const int* tri, int M,
                        const double* mass_partial, int n_partial, double xi, double wall_plane,
                        double* out, cudaStream_t s);

// f = f_eq(rho, u) in storage form (deviation from w, scaled); rho may be null (1).
void launch_set_equilibrium(int Q, int storage, int dim, const double* rho, const double* u,
                            void* dst, long long ncell, float scale, cudaStream_t s);
// Deformation index of the interface in the shear plane: out[5] =
// {D, r1, r3, inclination (deg), enclosed area / volume}.
void launch_deformation(int dim, const double* q, int N, const int* tri, int M, double* out,
                        cudaStream_t s);

// Inside / outside test of the cell at wall-axis coordinate a in column col:
// an odd number of interface crossings below it.
__device__ __forceinline__ bool inside_cell(const int* __restrict__ cnt,
                                            const double* __restrict__ cz, int col, int a)
{
    int c = cnt[col];
    if (c == 0) return false;
    if (c > COL_MAX) c = COL_MAX;
    bool in = false;
    for (int k = 0; k < c; k++) in ^= (cz[(long long)col * COL_MAX + k] < (double)a);
    return in;
}

// Column crossings of the current interface (classify.cu); the column count
// array is cleared first.
void launch_classify(int dim, const double* q, int N, const int* tri, int M, const GridParams& g,
                     int* cnt, double* cz, int* err, cudaStream_t s);
void launch_inside_mask(const GridParams& g, const int* cnt, const double* cz,
                        unsigned char* mask, cudaStream_t s);

// Kernel-launch accounting shared by the engines (iblb_kernel_launch_count).
void add_launches(long long n);

}  // namespace iblb
