// Split-row tile kernels (128-pixel rows): 4, 8 or 16 rows per tile, both
// render modes, the three decay kinds, aligned or unaligned rows.
#include "esi_tile_inst.cuh"
#include "esi_tile_split.cuh"

namespace esi {

template <int TH, int RD, int DK, bool VEC>
__global__ void ESI_TILE_BOUNDS(TH) esi_tile_split_kernel(TileArgs a)
{
    tile_body_split<TH, RD, DK, VEC>(a, blockIdx.x);
}

#define ESI_SPLIT_VARIANTS(TH)                                                    \
    X(TH, 0, kDecayGeneral, false) X(TH, 0, kDecayGeneral, true)                  \
    X(TH, 0, kDecaySquare, false) X(TH, 0, kDecaySquare, true)                    \
    X(TH, 0, kDecayNone, false) X(TH, 0, kDecayNone, true)                        \
    X(TH, 1, kDecayGeneral, false) X(TH, 1, kDecayGeneral, true)                  \
    X(TH, 1, kDecaySquare, false) X(TH, 1, kDecaySquare, true)                    \
    X(TH, 1, kDecayNone, false) X(TH, 1, kDecayNone, true)

#define ESI_SPLIT_ALL ESI_SPLIT_VARIANTS(4) ESI_SPLIT_VARIANTS(8) ESI_SPLIT_VARIANTS(16)

cudaError_t set_tile_split_attributes()
{
    cudaError_t e = cudaSuccess;
#define X(TH, RD, DK, V)                                                                            \
    if (e == cudaSuccess) e = allow_dynamic_smem_impl((const void *)esi_tile_split_kernel<TH, RD, DK, V>);
    ESI_SPLIT_ALL
#undef X
    return e;
}

cudaError_t launch_tile_split(const TileArgs &a, int tile_h, bool vec, cudaStream_t s)
{
    const size_t smem = tile_smem_bytes(tile_h, a.batch, a.n_chunks);
    const int rd = a.mp.render_decay ? 1 : 0;
    const int dk = decay_kind_of(a.dp);
#define X(TH, RD, DK, V)                                                             \
    if (tile_h == TH && rd == RD && dk == DK && vec == V) {                          \
        esi_tile_split_kernel<TH, RD, DK, V><<<a.n_tiles, TH * 32, smem, s>>>(a);    \
        return cudaGetLastError();                                                   \
    }
    ESI_SPLIT_ALL
#undef X
    return cudaErrorInvalidValue;
}

// Static shared memory of the largest variant (render decay on) per tile
// height, asked of the runtime once.
size_t tile_split_static_smem_bytes(int tile_h)
{
    static size_t cached[3] = {0, 0, 0};
    const int i = tile_h == 4 ? 0 : tile_h == 8 ? 1 : 2;
    if (!cached[i]) {
        cudaFuncAttributes fa{};
        cudaError_t e = cudaErrorInvalidValue;
        if (tile_h == 4) e = cudaFuncGetAttributes(&fa, (const void *)esi_tile_split_kernel<4, 1, kDecayGeneral, true>);
        if (tile_h == 8) e = cudaFuncGetAttributes(&fa, (const void *)esi_tile_split_kernel<8, 1, kDecayGeneral, true>);
        if (tile_h == 16) e = cudaFuncGetAttributes(&fa, (const void *)esi_tile_split_kernel<16, 1, kDecayGeneral, true>);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        cached[i] = fa.sharedSizeBytes;
    }
    return cached[i];
}

}  // namespace esi
