// Tile kernels with 64-pixel rows (2 pixels per lane), 4, 8 or 16 rows: twice
// as many independent row walks as 128-pixel rows in half the shared memory.
#include "esi_tile_inst.cuh"

namespace esi {

#define ESI_W64_VARIANTS(TH)                                                      \
    X(TH, 0, kDecayGeneral, false) X(TH, 0, kDecayGeneral, true)                  \
    X(TH, 0, kDecaySquare, false) X(TH, 0, kDecaySquare, true)                    \
    X(TH, 0, kDecayNone, false) X(TH, 0, kDecayNone, true)                        \
    X(TH, 1, kDecayGeneral, false) X(TH, 1, kDecayGeneral, true)                  \
    X(TH, 1, kDecaySquare, false) X(TH, 1, kDecaySquare, true)                    \
    X(TH, 1, kDecayNone, false) X(TH, 1, kDecayNone, true)

#define ESI_W64_ALL ESI_W64_VARIANTS(4) ESI_W64_VARIANTS(8) ESI_W64_VARIANTS(16)

// per-event output (esi_event_states): no frames, so one render mode and no
// frame-word variant
#define ESI_W64_EV Y(4, kDecayGeneral) Y(4, kDecaySquare) Y(4, kDecayNone) Y(8, kDecayGeneral) Y(8, kDecaySquare) Y(8, kDecayNone) Y(16, kDecayGeneral) Y(16, kDecaySquare) Y(16, kDecayNone)

cudaError_t set_tile_attributes_w64()
{
    cudaError_t e = cudaSuccess;
#define X(TH, RD, DK, V)                                                                       \
    if (e == cudaSuccess) e = allow_dynamic_smem_impl((const void *)esi_tile_kernel<TH, 2, RD, DK, V>);
    ESI_W64_ALL
#undef X
#define Y(TH, DK)                                                                              \
    if (e == cudaSuccess) e = allow_dynamic_smem_impl((const void *)esi_tile_kernel<TH, 2, 0, DK, false, true>);
    ESI_W64_EV
#undef Y
    return e;
}

cudaError_t launch_tile_w64(const TileArgs &a, int tile_h, bool vec, cudaStream_t s)
{
    const size_t smem = tile_smem_bytes(tile_h, a.batch, a.n_chunks);
    const int rd = a.mp.render_decay ? 1 : 0;
    const int dk = decay_kind_of(a.dp);
#define X(TH, RD, DK, V)                                                          \
    if (tile_h == TH && rd == RD && dk == DK && vec == V) {                       \
        esi_tile_kernel<TH, 2, RD, DK, V><<<a.n_tiles, TH * 32, smem, s>>>(a);    \
        return cudaGetLastError();                                                \
    }
    ESI_W64_ALL
#undef X
    return cudaErrorInvalidValue;
}

cudaError_t launch_tile_ev_w64(const TileArgs &a, int tile_h, cudaStream_t s)
{
    const size_t smem = tile_smem_bytes_ev(tile_h, a.batch, a.n_chunks);
    const int dk = decay_kind_of(a.dp);
#define Y(TH, DK)                                                                       \
    if (tile_h == TH && dk == DK) {                                                     \
        esi_tile_kernel<TH, 2, 0, DK, false, true><<<a.n_tiles, TH * 32, smem, s>>>(a); \
        return cudaGetLastError();                                                      \
    }
    ESI_W64_EV
#undef Y
    return cudaErrorInvalidValue;
}

}  // namespace esi
