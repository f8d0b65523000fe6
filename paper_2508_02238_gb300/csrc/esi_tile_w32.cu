// Tile kernels with 32-pixel rows (1 pixel per lane), 16 or 32 rows: four times
// as many independent row walks as 128-pixel rows, for sensors whose pixel
// count leaves the GPU short of warps.
#include "esi_tile_inst.cuh"

namespace esi {

#define ESI_W32_VARIANTS(TH)                                                       \
    X(TH, 0, kDecayGeneral) X(TH, 0, kDecaySquare) X(TH, 0, kDecayNone)            \
    X(TH, 1, kDecayGeneral) X(TH, 1, kDecaySquare) X(TH, 1, kDecayNone)

#define ESI_W32_ALL ESI_W32_VARIANTS(16) ESI_W32_VARIANTS(32)

// per-event output (esi_event_states): no frames, so one render mode and no
// frame-word variant
#define ESI_W32_EV Y(16, kDecayGeneral) Y(16, kDecaySquare) Y(16, kDecayNone) Y(32, kDecayGeneral) Y(32, kDecaySquare) Y(32, kDecayNone)

cudaError_t set_tile_attributes_w32()
{
    cudaError_t e = cudaSuccess;
#define X(TH, RD, DK)                                                                          \
    if (e == cudaSuccess) e = allow_dynamic_smem_impl((const void *)esi_tile_kernel<TH, 1, RD, DK, false>);
    ESI_W32_ALL
#undef X
#define Y(TH, DK)                                                                              \
    if (e == cudaSuccess) e = allow_dynamic_smem_impl((const void *)esi_tile_kernel<TH, 1, 0, DK, false, true>);
    ESI_W32_EV
#undef Y
    return e;
}

cudaError_t launch_tile_w32(const TileArgs &a, int tile_h, cudaStream_t s)
{
    const size_t smem = tile_smem_bytes(tile_h, a.batch, a.n_chunks);
    const int rd = a.mp.render_decay ? 1 : 0;
    const int dk = decay_kind_of(a.dp);
#define X(TH, RD, DK)                                                                 \
    if (tile_h == TH && rd == RD && dk == DK) {                                       \
        esi_tile_kernel<TH, 1, RD, DK, false><<<a.n_tiles, TH * 32, smem, s>>>(a);    \
        return cudaGetLastError();                                                    \
    }
    ESI_W32_ALL
#undef X
    return cudaErrorInvalidValue;
}

cudaError_t launch_tile_ev_w32(const TileArgs &a, int tile_h, cudaStream_t s)
{
    const size_t smem = tile_smem_bytes_ev(tile_h, a.batch, a.n_chunks);
    const int dk = decay_kind_of(a.dp);
#define Y(TH, DK)                                                                       \
    if (tile_h == TH && dk == DK) {                                                     \
        esi_tile_kernel<TH, 1, 0, DK, false, true><<<a.n_tiles, TH * 32, smem, s>>>(a); \
        return cudaGetLastError();                                                      \
    }
    ESI_W32_EV
#undef Y
    return cudaErrorInvalidValue;
}

}  // namespace esi
