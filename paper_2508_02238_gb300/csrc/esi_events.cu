// Continuous-time output: the state of each event's pixel right after the
// event (Alg. 2 per event; Alg. 1 and Eq. 3 by the handle's method).
//
// The pending events go through the render's binning and tile kernels: the
// binning also writes each record's event index beside it, and the tile
// kernel's per-event-output instantiation carries the index through its
// gather and row sort and stores S at it after every event.  No frame is
// rendered, and the state left behind is bit-identical to a render's.
#include <algorithm>
#include <vector>

#include "esi_api_impl.h"

namespace esi {

namespace {

// Records a tile sorts per shared-memory batch here: the index arrays take
// 8 bytes per record on top of the render's layout, so at most 2048 (and
// never more than the tuning's batch, whose layout was checked to fit).
int ev_batch(const esi_handle *h, int max_chunks)
{
    for (int b = std::min(h->tun.batch_records, 2048); b >= 1024; b /= 2)
        if (tile_smem_bytes_ev(h->tun.tile_h, b, max_chunks) + tile_static_smem_bytes(h->tun.tile_h, h->tun.tile_w) <=
            (size_t)kMaxSmemPerBlock)
            return b;
    return 0;
}

}  // namespace

}  // namespace esi

using namespace esi;

extern "C" int esi_event_states(esi_handle *h, float *out, size_t cap, int out_on_device, size_t *n_out)
{
    if (!h || !n_out || (out_on_device != 0 && out_on_device != 1)) return ESI_EINVAL;
    const unsigned long long n = h->tail - h->head;
    *n_out = (size_t)n;
    if (n == 0) return ESI_OK;
    if (!out) return ESI_EINVAL;
    if (cap < n) return ESI_ERANGE;
    const esi_tuning &tu = h->tun;
    const int chunk = tu.chunk_events;
    const unsigned long long maxb = (unsigned long long)tu.max_batch_events;
    const int64_t no_frames = 0;
    const int batch = ev_batch(h, (int)((maxb + chunk - 1) / chunk));
    if (!batch) return ESI_ERANGE;
    std::vector<SubBatch> plan;
    int rc = plan_subbatches(h, n, &no_frames, 0, &plan);
    if (rc) return rc;

    float *dout = out;
    if (!out_on_device) {
        rc = ensure_device(h, &h->diag, &h->diag_cap, (size_t)n * sizeof(float));
        if (rc) return rc;
        dout = reinterpret_cast<float *>(h->diag);
    }
    for (int b = 0; b < 2; ++b) {
        const size_t max_chunks = (size_t)((maxb + chunk - 1) / chunk);
        rc = ensure_device(h, &h->rec[b], &h->rec_cap[b], max_chunks * (size_t)chunk);
        if (!rc) rc = ensure_device(h, &h->rec_idx[b], &h->rec_idx_cap[b], max_chunks * (size_t)chunk);
        if (!rc) rc = ensure_device(h, &h->hrow[b], &h->hrow_cap[b], max_chunks * (size_t)h->n_tiles);
        if (rc) return rc;
    }
    cudaError_t e = cudaSuccess;
    if (h->dev_push_pending) {
        e = cudaEventRecord(h->ev_start, h->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->bin_stream, h->ev_start, 0);
        if (e != cudaSuccess) return cuda_fail(h, e);
        h->dev_push_pending = false;
    }
    // the per-tile walks start after everything queued on the handle's
    // stream (state writes, device pushes)
    e = cudaEventRecord(h->ev_tstart, h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->tile_stream, h->ev_tstart, 0);
    if (e != cudaSuccess) return cuda_fail(h, e);
    for (const SubBatch &sb : plan) {
        const int nb = (int)(sb.i1 - sb.i0);
        if (nb <= 0) continue;
        const int n_chunks = (nb + chunk - 1) / chunk;
        const int buf = h->next_buf;
        h->next_buf ^= 1;
        if (h->tile_pending[buf]) {
            e = cudaStreamWaitEvent(h->bin_stream, h->ev_tile[buf], 0);
            if (e != cudaSuccess) return cuda_fail(h, e);
        }
        BinArgs ba;
        ba.ring = h->ring;
        ba.ring_mask = h->cap - 1;
        ba.first = h->head + sb.i0;
        ba.n = nb;
        ba.chunk = chunk;
        ba.t_base = sb.t_base;
        ba.W = h->W;
        ba.H = h->H;
        ba.tiles_x = h->tiles_x;
        ba.n_tiles = h->n_tiles;
        ba.th_log2 = h->th_log2;
        ba.tw_log2 = h->tw_log2;
        ba.tile_bits = index_bits(h->n_tiles);
        ba.rec = h->rec[buf];
        ba.hrow = h->hrow[buf];
        ba.use_mask = bin_mask_fits(chunk, h->n_tiles) ? 1 : 0;
        ba.status = h->dstatus;
        ba.rec_idx = h->rec_idx[buf];
        ba.ev_out = dout + sb.i0;
        cudaEvent_t ev;
        rc = prof_begin(h, &ev, h->bin_stream);
        if (!rc) rc = cuda_fail(h, launch_bin(ba, n_chunks, h->bin_stream));
        if (!rc) rc = prof_end(h, kKindBin, ev, h->bin_stream);
        if (!rc) rc = cuda_fail(h, cudaEventRecord(h->ev_bin[buf], h->bin_stream));
        if (!rc) rc = cuda_fail(h, cudaStreamWaitEvent(h->tile_stream, h->ev_bin[buf], 0));
        if (rc) return rc;

        TileArgs ta;
        ta.rec = h->rec[buf];
        ta.hrow = h->hrow[buf];
        ta.n_chunks = n_chunks;
        ta.chunk = chunk;
        ta.n_tiles = h->n_tiles;
        ta.t_base = sb.t_base;
        ta.S = h->S;
        ta.T = h->T;
        ta.W = h->W;
        ta.H = h->H;
        ta.tiles_x = h->tiles_x;
        ta.dp = h->dp;
        ta.mp = h->mp;
        ta.win = h->dwin;
        ta.w_begin = 0;
        ta.w_end = 0;
        ta.frames = nullptr;
        ta.frame_outs = nullptr;
        ta.P = h->P;
        ta.batch = batch;
        ta.status = h->dstatus;
        ta.rec_idx = h->rec_idx[buf];
        ta.ev_out = dout + sb.i0;
        ta.scan_chain = h->tun.scan_chain;
        rc = prof_begin(h, &ev, h->tile_stream);
        if (!rc) rc = cuda_fail(h, launch_tile_ev(ta, tu.tile_h, tu.tile_w, h->tile_stream));
        if (!rc) rc = prof_end(h, kKindEvState, ev, h->tile_stream);
        if (!rc) rc = cuda_fail(h, cudaEventRecord(h->ev_tile[buf], h->tile_stream));
        if (rc) return rc;
        h->tile_pending[buf] = true;
    }
    // the binning launches read ring indices [head, tail): later pushes wait
    // for them before overwriting those slots
    auto &sp = h->span[h->span_next];
    e = cudaEventRecord(sp.ev, h->bin_stream);
    if (e != cudaSuccess) return cuda_fail(h, e);
    sp.a0 = h->head;
    sp.a1 = h->head + n;
    sp.live = true;
    h->span_next = (h->span_next + 1) % esi_handle::kSpans;
    h->head += n;
    h->consumed += n;
    while (!h->exact_spans.empty() && h->exact_spans.front().second <= h->head)
        h->exact_spans.erase(h->exact_spans.begin());
    // the state now holds events up to the last one: frames must not be earlier
    h->frame_floor = std::max(h->frame_floor, h->last_event_t);
    h->push_floor = std::max(h->push_floor, h->last_event_t);
    e = cudaEventRecord(h->ev_tdone, h->tile_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->ev_tdone, 0);
    if (e != cudaSuccess) return cuda_fail(h, e);
    if (!out_on_device) {
        e = cudaMemcpyAsync(out, dout, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e);
    }
    return read_status(h);
}
