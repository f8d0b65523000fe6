// Continuous-time output: the state of each event's pixel right after the
// event (Alg. 2 per event; Alg. 1 and Eq. 3 by the handle's method).
//
// The pending events are binned by tile exactly as for a render, with each
// record's event index written beside it.  One warp then walks one tile's
// records in their stable (arrival) order, 32 at a time, with the per-event
// arithmetic of the tile kernel: same-pixel lanes are found with
// __match_any_sync, the pixel's state passes from lane to lane by shuffle,
// and every lane stores its event's S at the event's index.  The final
// state is bit-identical to what a render over the same events leaves.
#include <cmath>
#include <vector>

#include "esi_api_impl.h"
#include "esi_device.cuh"

namespace esi {

namespace {

constexpr int kEvWarps = 4;   // tiles per block

struct EvStateArgs {
    const unsigned long long *rec;   // binned records, block c at rec + c * chunk
    const unsigned *rec_idx;         // event index (in the sub-batch) of each record
    const unsigned *hrow;            // [tile][chunk] (start << 16 | count)
    int n_chunks, chunk, n_tiles;
    long long t_base;
    float *S;
    long long *T;
    int W, tiles_x, th_log2, tw_log2;
    DecayParams dp;
    MapParams mp;
    float *out;                      // S after each event of the sub-batch
};

template <int DK>
__global__ void __launch_bounds__(kEvWarps * 32) esi_event_state_kernel(EvStateArgs a)
{
    const int lane = threadIdx.x & 31;
    const int tile = blockIdx.x * kEvWarps + (threadIdx.x >> 5);
    if (tile >= a.n_tiles) return;   // the whole warp leaves together
    const int twl = a.tw_log2;
    const int x0 = (tile % a.tiles_x) << twl, y0 = (tile / a.tiles_x) << a.th_log2;
    const unsigned *runs = a.hrow + (size_t)tile * a.n_chunks;
    for (int c = 0; c < a.n_chunks; ++c) {
        const unsigned run = runs[c];
        const unsigned start = run >> 16, cnt = run & 0xffffu;
        const size_t base = (size_t)c * a.chunk + start;
        for (unsigned g = 0; g < cnt; g += 32) {
            const bool valid = g + lane < cnt;
            const unsigned long long r = valid ? a.rec[base + g + lane] : 0ull;
            const unsigned idx = valid ? a.rec_idx[base + g + lane] : 0u;
            const unsigned pit = (unsigned)(r >> 33);
            const long long pix = (long long)(y0 + (int)(pit >> twl)) * a.W + x0 +
                                  (int)(pit & ((1u << twl) - 1u));
            const unsigned toff = (unsigned)r;
            // every lane takes part (invalid lanes share a key no record has)
            const unsigned peers = __match_any_sync(kFull, valid ? pit : 0xffffffffu);
            const unsigned mine = valid ? peers : 0u;
            const unsigned below = mine & lanemask_lt();
            const unsigned rank = __popc(below);
            const int prev = below ? 31 - __clz(below) : lane;
            const unsigned t_prev_rec = __shfl_sync(kFull, toff, prev);
            const bool first = valid && rank == 0;
            float s_in = first ? a.S[pix] : 0.0f;
            const long long t_prev = first ? a.T[pix] - a.t_base : (long long)t_prev_rec;
            const float d = valid ? decay_state_k<DK>((long long)toff - t_prev, a.dp) : 0.0f;
            const float cc = ((r >> 32) & 1u) ? a.mp.C : -a.mp.C;
            const unsigned maxr = __reduce_max_sync(kFull, valid ? rank : 0u);
            float s_out = 0.0f;
            for (unsigned k = 0;; ++k) {
                if (valid && rank == k) s_out = event_step<DK>(s_in, cc, d, a.dp, a.mp);
                if (k == maxr) break;
                const float got = __shfl_sync(kFull, s_out, prev);
                if (valid && rank == k + 1) s_in = got;
            }
            if (valid) a.out[idx] = s_out;
            // the pixel's last record in the group writes the state back;
            // the next group reads it after the warp barrier
            if (valid && (mine >> lane) == 1u) {
                a.S[pix] = s_out;
                a.T[pix] = a.t_base + (long long)toff;
            }
            __syncwarp();
        }
    }
}

cudaError_t launch_event_state(const EvStateArgs &a, int dk, cudaStream_t s)
{
    const int grid = (a.n_tiles + kEvWarps - 1) / kEvWarps;
    if (dk == kDecaySquare)
        esi_event_state_kernel<kDecaySquare><<<grid, kEvWarps * 32, 0, s>>>(a);
    else if (dk == kDecayNone)
        esi_event_state_kernel<kDecayNone><<<grid, kEvWarps * 32, 0, s>>>(a);
    else
        esi_event_state_kernel<kDecayGeneral><<<grid, kEvWarps * 32, 0, s>>>(a);
    return cudaGetLastError();
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
    const int dk = decay_kind_of(h->dp);
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
        ba.use_mask = (h->n_tiles <= kBinMaskTiles && bin_mask_fits(chunk, h->n_tiles)) ? 1 : 0;
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

        EvStateArgs ea;
        ea.rec = h->rec[buf];
        ea.rec_idx = h->rec_idx[buf];
        ea.hrow = h->hrow[buf];
        ea.n_chunks = n_chunks;
        ea.chunk = chunk;
        ea.n_tiles = h->n_tiles;
        ea.t_base = sb.t_base;
        ea.S = h->S;
        ea.T = h->T;
        ea.W = h->W;
        ea.tiles_x = h->tiles_x;
        ea.th_log2 = h->th_log2;
        ea.tw_log2 = h->tw_log2;
        ea.dp = h->dp;
        ea.mp = h->mp;
        ea.out = dout + sb.i0;
        rc = prof_begin(h, &ev, h->tile_stream);
        if (!rc) rc = cuda_fail(h, launch_event_state(ea, dk, h->tile_stream));
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
