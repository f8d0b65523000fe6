// Private definition of esi_handle and the host helpers shared by the C ABI
// translation units.
#pragma once

#include <string>
#include <vector>

#include "esi_internal.h"

namespace esi {

enum KernelKind {
    kKindBin = 0, kKindTile = 1, kKindFill = 2, kKindTick = 3, kKindNoise = 4, kKindCount = 5,
    kKindEvState = 6, kNumKernelKinds = 7
};
static const char *const kKernelNames[kNumKernelKinds] = {
    "esi_bin", "esi_tile", "esi_fill", "esi_tick", "esi_noise_map", "esi_count", "esi_tile_ev"};

struct ProfRec {
    int kind;
    cudaEvent_t start;
    cudaEvent_t stop;
};

}  // namespace esi

struct esi_handle {
    int W = 0, H = 0;
    long long P = 0;
    esi_params prm{};
    esi::DecayParams dp{};
    esi::MapParams mp{};
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;

    esi_tuning tun{};
    int tiles_x = 0, tiles_y = 0, n_tiles = 0, th_log2 = 0, tw_log2 = 7;

    float *S = nullptr;           // accumulation matrix (Alg. 2), row-major
    long long *T = nullptr;       // last decay time matrix (Alg. 2)

    // pending events: ring of `cap` events (power of two) on the device;
    // absolute indices head <= i < tail.  Times for planning, pinned:
    // tsparse holds the time of every kSparse-th absolute index (slot
    // (i / kSparse) & (cap / kSparse - 1)), valid for i >= sparse_from until
    // the slot is reused; tmirror holds every time of host-checked pushes,
    // whose index ranges exact_spans lists.  Other times are read back from
    // the ring when planning needs them.
    esi_event *ring = nullptr;
    unsigned long long cap = 0, head = 0, tail = 0;
    long long *tmirror = nullptr;
    long long *tsparse = nullptr;
    unsigned long long sparse_from = 0;
    std::vector<std::pair<unsigned long long, unsigned long long>> exact_spans;
    esi_event *hfetch = nullptr;         // pinned: events read back for planning

    // host pushes run on in_stream, which waits only for renders whose
    // binning still reads ring slots the push overwrites: the last renders'
    // consumed index ranges, each with an event after its last binning launch
    cudaStream_t in_stream = nullptr;
    struct RenderSpan {
        unsigned long long a0 = 0, a1 = 0;   // absolute ring indices consumed
        cudaEvent_t ev = nullptr;             // after the render's last binning launch
        bool live = false;
    };
    static constexpr int kSpans = 4;
    RenderSpan span[kSpans];
    int span_next = 0;                        // oldest entry, reused next
    // large pushes: the device checks the time order and returns the times
    // chunk by chunk on aux_stream while the next chunk is copied in
    cudaStream_t aux_stream = nullptr;
    cudaEvent_t ev_chunk[4] = {nullptr, nullptr, nullptr, nullptr};
    long long *dsparse = nullptr;        // every kSparse-th time of the push being checked
    size_t dsparse_cap = 0;
    // packed host pushes: two device staging buffers of a chunk each, the
    // copy of one overlapping the unpack of the other (ev_unpk: unpack done)
    unsigned long long *pk_stage = nullptr;
    size_t pk_stage_cap = 0;
    cudaEvent_t ev_unpk[2] = {nullptr, nullptr};
    std::vector<esi_event> pk_host;      // small packed host pushes, unpacked
    esi::PushResult *dres = nullptr;
    esi::PushResult *hres = nullptr;     // pinned

    // binning of sub-batch i + 1 overlaps the tile kernel of sub-batch i:
    // it runs on bin_stream into the other half of the double-buffered
    // scratch; events order it against the handle's stream
    cudaStream_t bin_stream = nullptr;
    // tile kernels run on a high-priority stream joined to the handle's
    // stream by events, so their blocks are dispatched before those of a
    // binning launch queued at the same time
    cudaStream_t tile_stream = nullptr;
    cudaEvent_t ev_tstart = nullptr, ev_tdone = nullptr;
    cudaEvent_t ev_start = nullptr;      // render's work may begin (handle stream)
    cudaEvent_t ev_bin[2] = {nullptr, nullptr};
    cudaEvent_t ev_tile[2] = {nullptr, nullptr};
    bool tile_pending[2] = {false, false};
    int next_buf = 0;                    // scratch half of the next sub-batch
    bool dev_push_pending = false;       // a device push queued since the last render
    unsigned long long *rec[2] = {nullptr, nullptr};   // binned records of a sub-batch
    size_t rec_cap[2] = {0, 0};
    unsigned int *hrow[2] = {nullptr, nullptr};        // [chunk][tile] run table
    // split-row tile kernel: whether it runs, the scratch of the tiles'
    // row-sorted records (tile launches run one after another) and the
    // counter handing out the tiles' regions
    bool split = false;
    unsigned long long *srt = nullptr;
    size_t srt_cap = 0;
    unsigned long long *srt_top = nullptr;
    size_t srt_top_cap = 0;
    size_t hrow_cap[2] = {0, 0};
    esi::WinInfo *dwin = nullptr;        // per-frame constants of a render
    size_t dwin_cap = 0;
    esi::WinInfo *hwin = nullptr;        // pinned staging of dwin
    size_t hwin_cap = 0;
    cudaEvent_t hwin_ev = nullptr;       // the last copy out of hwin
    bool hwin_busy = false;
    unsigned char *dframes = nullptr;    // frames staged for host outputs
    size_t dframes_cap = 0;

    unsigned *rec_idx[2] = {nullptr, nullptr};  // event index beside each record (esi_event_states)
    size_t rec_idx_cap[2] = {0, 0};
    unsigned char *diag = nullptr;       // scratch of esi_noise_map / esi_count_events / esi_event_states
    size_t diag_cap = 0;

    esi::DevStatus *dstatus = nullptr;
    esi::DevStatus *hstatus = nullptr;   // pinned

    long long push_floor = 0;     // pushes must not be earlier than this
    long long frame_floor = 0;    // frames must not be earlier than this
    long long last_event_t = 0;
    long long last_frame_t = 0;
    unsigned long long pushed = 0, consumed = 0, dropped = 0, frames = 0, launches = 0;
    unsigned long long ring_grows = 0, push_waits = 0;

    bool prof_on = false;
    std::vector<esi::ProfRec> prof_recs;
    std::vector<cudaEvent_t> ev_pool;
    double prof_ms[esi::kNumKernelKinds] = {};
    unsigned long long prof_n[esi::kNumKernelKinds] = {};

    std::string cuda_msg;
};

namespace esi {

int cuda_fail(esi_handle *h, cudaError_t e);
long long decay_cutoff(double k_per_s);
int validate_params(int W, int H, const esi_params *p);
void prepare_params(const esi_params &p, DecayParams *dp, MapParams *mp);
int validate_tuning(const esi_tuning &t);
esi_tuning default_tuning(int W, int H);
int read_status(esi_handle *h);
int prof_begin(esi_handle *h, cudaEvent_t *ev, cudaStream_t s);
int prof_end(esi_handle *h, int kind, cudaEvent_t start, cudaStream_t s);
int sync_all(esi_handle *h);
int init_state(esi_handle *h);
int render_impl(esi_handle *h, const int64_t *tf, int m, uint8_t *out, int out_on_device);

// One binning + tile launch pair of a render: pending events i0 .. i1
// (relative to head), frames w0 .. w1 completed by it, record times offset
// from t_base.
struct SubBatch {
    unsigned long long i0, i1;
    int w0, w1;
    long long t_base;
};
// Splits the first n_split pending events into sub-batches of at most
// max_batch_events whose record times fit in 32 bits; each completes the
// frames (of tf[0 .. m)) that end before its successor starts.  m may be 0.
int plan_subbatches(esi_handle *h, unsigned long long n_split, const int64_t *tf, int m,
                    std::vector<SubBatch> *plan);

// Grows a device buffer to at least `need` elements (contents are not kept;
// the handle's streams are drained before the old buffer is freed).
template <class T>
int ensure_device(esi_handle *h, T **p, size_t *cap, size_t need)
{
    if (need <= *cap) return ESI_OK;
    size_t nc = need > *cap * 2 ? need : *cap * 2;
    if (*p) {
        int rc = sync_all(h);
        if (rc) return rc;
        cudaFree(*p);
        *p = nullptr;
        *cap = 0;
    }
    cudaError_t e = cudaMalloc((void **)p, nc * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(h, e);
    *cap = nc;
    return ESI_OK;
}
int fill_i64(esi_handle *h, long long *dst, long long n, long long value);
cudaError_t launch_fill_i64(long long *dst, long long n, long long value, cudaStream_t s);
// Checks events a0 + first .. a0 + first + cnt of an n-event push starting at
// ring index a0: each time >= its predecessor's (prev for the push's first),
// res->bad set otherwise; the time of absolute index g (g % kSparse == 0)
// goes to sparse[(g - g0) / kSparse] (g0: the push's first such index); the
// push's last time to res->last.
cudaError_t launch_push_check(const esi_event *ring, unsigned long long mask, unsigned long long a0,
                              unsigned long long first, long long cnt, unsigned long long n,
                              long long prev, unsigned long long g0, long long *sparse,
                              PushResult *res, cudaStream_t s);
// The same for packed events: src[i] (esi.h's 8-byte layout, time
// t_base + offset) is written to ring index a0 + first + i and checked.
cudaError_t launch_push_unpack(const unsigned long long *src, esi_event *ring,
                               unsigned long long mask, unsigned long long a0,
                               unsigned long long first, long long cnt, unsigned long long n,
                               long long t_base, long long prev, unsigned long long g0,
                               long long *sparse, PushResult *res, cudaStream_t s);

// Launch-shape measurement shared by esi_autotune and esi_stream_autotune:
// cache lookup, candidate timing on a scratch handle, cache update.
struct AutotuneKey {
    int W, H, bucket, render_decay, decay_kind, flags;
};
int autotune_shapes(const AutotuneKey &key, const esi_params &prm, cudaStream_t stream,
                    const esi_event *sample, size_t n, const int64_t *t_frames, size_t m,
                    const std::vector<esi_tuning> &cands, bool force, esi_tuning *best);
int autotune_bucket(size_t n, size_t m);

}  // namespace esi
