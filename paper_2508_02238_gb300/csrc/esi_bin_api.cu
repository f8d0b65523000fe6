// esi_bin_events: the first level of the render's stable counting sort by
// pixel, on its own, for inspection.  It launches the same binning kernel a
// render launches, on a caller's device ring, and leaves the records and the
// run table in caller buffers, so that their order can be checked against a
// plain stable sort.  Reordering events by pixel is legal because each
// pixel's state depends only on its own events in time order (Alg. 2, Eq. 5);
// stability keeps that order.
#include <climits>

#include "esi_api_impl.h"

using namespace esi;

extern "C" int esi_bin_events(int width, int height, const esi_tuning *shape,
                              const esi_event *ring, uint64_t ring_capacity, uint64_t first,
                              size_t n, int64_t t_base, uint64_t *records, uint32_t *runs,
                              uint64_t *dropped, void *cuda_stream)
{
    if (width < 1 || height < 1 || width > 65535 || height > 65535 || !shape) return ESI_EINVAL;
    if (n == 0) {
        if (dropped) *dropped = 0;
        return ESI_OK;
    }
    if (!ring || !records || !runs) return ESI_EINVAL;
    if (ring_capacity == 0 || (ring_capacity & (ring_capacity - 1)) || n > ring_capacity)
        return ESI_EINVAL;
    if (n > (size_t)INT_MAX) return ESI_ERANGE;
    // the chunks are staged by 16-byte bulk copies (TMA)
    if (reinterpret_cast<uintptr_t>(ring) & 15u) return ESI_EINVAL;
    esi_tuning t = *shape;
    if (!t.tile_w) t.tile_w = kTileW;
    if (!t.tile_h) t.tile_h = t.tile_w == 32 ? 32 : 8;
    if (!t.chunk_events) t.chunk_events = 2048;
    if (!t.batch_records) t.batch_records = 4096;
    if (!t.max_batch_events) t.max_batch_events = t.chunk_events;
    if (!t.scan_chain) t.scan_chain = kScanChainDefault;
    if (!t.split_rows) t.split_rows = 2;
    int rc = validate_tuning(t);
    if (rc) return rc;
    const int tiles_x = (width + t.tile_w - 1) / t.tile_w;
    const int n_tiles = tiles_x * ((height + t.tile_h - 1) / t.tile_h);
    if (bin_smem_bytes(t.chunk_events, n_tiles, false) + 1024 > (size_t)kMaxSmemPerBlock)
        return ESI_ERANGE;
    int th_log2 = 0;
    while ((1 << th_log2) < t.tile_h) ++th_log2;
    const int n_chunks = (int)((n + (size_t)t.chunk_events - 1) / (size_t)t.chunk_events);

    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = set_kernel_attributes();
    DevStatus *st = nullptr;
    if (e == cudaSuccess) e = cudaMalloc((void **)&st, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaMemsetAsync(st, 0, sizeof(DevStatus), s);
    if (e == cudaSuccess) {
        BinArgs ba;
        ba.ring = ring;
        ba.ring_mask = ring_capacity - 1;
        ba.first = first & (ring_capacity - 1);
        ba.n = (int)n;
        ba.chunk = t.chunk_events;
        ba.t_base = t_base;
        ba.W = width;
        ba.H = height;
        ba.tiles_x = tiles_x;
        ba.n_tiles = n_tiles;
        ba.th_log2 = th_log2;
        ba.tw_log2 = t.tile_w == 32 ? 5 : t.tile_w == 64 ? 6 : 7;
        ba.tile_bits = index_bits(n_tiles);
        ba.rec = reinterpret_cast<unsigned long long *>(records);
        ba.hrow = runs;
        ba.use_mask = bin_mask_fits(t.chunk_events, n_tiles) ? 1 : 0;
        ba.status = st;
        e = launch_bin(ba, n_chunks, s);
    }
    DevStatus hs{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (st) cudaFree(st);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? ESI_ENOMEM : ESI_ECUDA;
    if (dropped) *dropped = hs.dropped;
    return hs.err;
}
