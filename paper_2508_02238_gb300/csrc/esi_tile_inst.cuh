// Tile-kernel entry points and their launchers for one row width: included by
// esi_tile_w128.cu (4 pixels per lane) and esi_tile_w32.cu (1 pixel per lane).
#pragma once

#include "esi_tile.cuh"

namespace esi {

// 8-row tiles: at least three blocks per SM (their shared memory allows
// three at the default batch), so the compiler may use up to 85 registers a
// thread; other heights: as many blocks as fill 1024 threads
#define ESI_TILE_BOUNDS(TH) __launch_bounds__(TH * 32, (TH * 32 >= 1024) ? 1 : (TH == 8 ? 3 : 1024 / (TH * 32)))

template <int TH, int PPL, int RD, int DK, bool VEC, bool EV = false>
__global__ void ESI_TILE_BOUNDS(TH) esi_tile_kernel(TileArgs a)
{
    tile_body<TH, PPL, RD, DK, VEC, EV>(a, blockIdx.x);
}

// Batched tiles of a serving tick: a persistent grid walks the work items
// (stream job, tile) of one parameter variant group.
template <int TH, int PPL, int RD, int DK, bool VEC>
__global__ void ESI_TILE_BOUNDS(TH) esi_tile_tab_kernel(const unsigned char *tab, int group)
{
    const TickDir *d = reinterpret_cast<const TickDir *>(tab);
    const int n = d->n_items[group];
    const int2 *items = reinterpret_cast<const int2 *>(tab + d->off_items[group]);
    const TileArgs *jobs = reinterpret_cast<const TileArgs *>(tab + d->off_tilejob);
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const int2 it = items[i];
        tile_body<TH, PPL, RD, DK, VEC>(jobs[it.x], it.y);
        __syncthreads();  // shared memory is reused by the next item
    }
}

cudaError_t allow_dynamic_smem_impl(const void *kernel);

}  // namespace esi
