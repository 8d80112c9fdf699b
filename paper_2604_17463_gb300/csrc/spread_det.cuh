// spread_det.cuh -- descriptors and launcher of the order-deterministic
// spreading (spread_det.cu), shared by the single-simulation engine and the
// batched engine.
#pragma once

#include "common.cuh"

namespace iblb {

constexpr int DET_TILE = 4;  // edge of the node bins and cell tiles, in cells

// One simulation as seen by the deterministic spread.
struct DetSlot {
    GridParams g;
    int nb[3];             // node bins per axis (bins of DET_TILE stencil origins)
    int ct[3];             // cell tiles per axis
    int bin_base;          // first global bin of this slot
    int cell_base;         // first global cell tile of this slot
    const double* q;       // node positions [N][dim]
    const double* phi;     // nodal forces [N][dim]
    void* F;               // force density [dim][ncell], compute precision
    uint8_t* flags;        // band flags, one byte per 32-cell row segment
};

// Device work buffers (owned by the engine that launches).
struct DetBuffers {
    int* bin_of;           // [items] global bin of each node item (-1: none)
    int* org;              // [items][3] stencil origin per axis
    void* wts;             // [items][12] 1D weights, compute precision
    int* cnt;              // [bins]
    int* start;            // [bins]
    int* cur;              // [bins]
    int* list;             // [items] node items grouped by bin, increasing
    int* active;           // [cell tiles] 1 when a stencil touches the tile
    int2* act_list;        // [cell tiles] (slot, local cell tile) of the active ones
    int* nact;             // number of active cell tiles
};

// Bins and cell tiles per axis of one lattice (1 on unused axes).
void det_tiles(const GridParams& g, int nb[3], int ct[3]);

// One deterministic spread over `nitems` node items (items == nullptr: one
// slot, item = node id); nbins / ncelltiles: totals over all slots.
void launch_spread_det(int storage, int dim, const DetSlot* slots, const int2* items, int nitems,
                       const DetBuffers& b, int nbins, int ncelltiles, int sm_count,
                       cudaStream_t s);

// Kernel launches of one deterministic spread.
constexpr int DET_KERNELS = 5;

}  // namespace iblb
