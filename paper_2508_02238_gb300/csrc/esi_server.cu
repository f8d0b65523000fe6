// Batched serving of many sensors (esi_server_* in esi.h).
//
// A tick gathers, for every stream with a frame due, its pushed events up to
// the tick's time and its due frame times, packs them with per-stream
// descriptors into one pinned staging buffer, copies that to a fixed device
// table, and runs one batched binning launch plus one batched tile launch per
// parameter variant (render mode x decay kind x row alignment).  The kernels
// read their sizes and per-stream descriptors from the device table, so one
// captured CUDA graph serves every tick; frames are written straight into
// mapped host memory.  A host-function node stamps each tick's completion.
#include <time.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "esi_api_impl.h"
#include "esi_internal.h"

using namespace esi;

namespace {

long long wall_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

int rc_of(cudaError_t e)
{
    if (e == cudaSuccess) return ESI_OK;
    return e == cudaErrorMemoryAllocation ? ESI_ENOMEM : ESI_ECUDA;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// First-fit allocator over one device arena (the state budget).
class Arena {
  public:
    void init(size_t size)
    {
        size_ = size;
        free_.clear();
        if (size) free_[0] = size;
    }
    // offset of a block of n bytes, or SIZE_MAX when nothing fits
    size_t alloc(size_t n)
    {
        n = align_up(n, 256);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            const size_t off = it->first, len = it->second;
            free_.erase(it);
            if (len > n) free_[off + n] = len - n;
            return off;
        }
        return SIZE_MAX;
    }
    void release(size_t off, size_t n)
    {
        n = align_up(n, 256);
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }

  private:
    size_t size_ = 0;
    std::map<size_t, size_t> free_;
};

constexpr int kGroups = kTickGroups;
constexpr int kChunk = 2048;
constexpr int kBatch = 2048;
constexpr int kMaxChunksPerStream = 64;
constexpr int kTickSlots = 64;  // completion stamps kept for ticks in flight
constexpr int kMaxSlots = 1 << 20;  // caller stream slots of one esi_server_run

struct Stream {
    bool open = false;
    int W = 0, H = 0;
    long long P = 0;
    esi_params prm{};
    DecayParams dp{};
    MapParams mp{};
    int group = 0;
    int tile_h = 8, th_log2 = 3;
    int tiles_x = 0, n_tiles = 0;
    size_t arena_off = 0, arena_bytes = 0;
    float *S = nullptr;
    long long *T = nullptr;
    std::vector<esi_event> pend;
    size_t pend_head = 0;
    long long last_event_t = 0;
    long long push_floor = 0;
    long long next_frame_t = 0;
    long long watermark = LLONG_MAX;      // events complete up to here
    long long last_push_ns = 0;
    unsigned char *slots_host = nullptr;  // frame_slots * P bytes, mapped
    unsigned char *slots_dev = nullptr;
    unsigned long long seq_issued = 0;    // frames handed to ticks
    unsigned long long seq_done = 0;      // frames finished
    std::vector<long long> slot_t;
    std::vector<double> slot_lat;
    // optional caller buffer that keeps every finished frame (by number)
    unsigned char *sink = nullptr;
    unsigned long long sink_n = 0;
    long long *sink_t = nullptr;
};

struct TickFrame {
    int stream;
    unsigned long long seq;
    long long t_frame;
    long long ref_push_ns;
};

struct TickRec {
    unsigned long long id = 0;
    long long call_ns = 0;
    std::vector<TickFrame> frames;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int stage = 0;
};

// Completion stamps written by the host-function node of each tick.
struct Completion {
    std::atomic<unsigned long long> done{0};
    long long ns[kTickSlots] = {};
};

void CUDART_CB on_tick_done(void *user)
{
    Completion *c = static_cast<Completion *>(user);
    const unsigned long long d = c->done.load(std::memory_order_relaxed);
    c->ns[d % kTickSlots] = wall_ns();
    c->done.store(d + 1, std::memory_order_release);
}

double percentile(std::vector<double> v, double q)
{
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (double)(v.size() - 1);
    const size_t i = (size_t)pos;
    const double f = pos - (double)i;
    return (i + 1 < v.size()) ? v[i] * (1.0 - f) + v[i + 1] * f : v[i];
}

}  // namespace

struct esi_server {
    esi_server_opts opts{};
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t budget = 0, used = 0;
    unsigned char *arena_base = nullptr;
    Arena arena;
    std::vector<Stream> streams;
    int n_open = 0;
    int tile_h = 8;  // tile height of newly opened streams

    // capacities of one tick
    int cap_jobs = 0, cap_chunks = 0, cap_items = 0, cap_frames = 0, max_tiles = 0;
    int tile_grid = 0;  // persistent grid of the batched tile kernel
    int bin_grid = 0;   // persistent grid of the batched binning kernel
    bool bin_mask = false;  // binning finds same-tile lanes by mask words
    long long cap_events = 0;
    size_t off_binjob = 0, off_chunkjob = 0, off_tilejob = 0, off_items = 0, off_win = 0,
           off_fout = 0, off_events = 0, tab_bytes = 0;
    unsigned char *stage[2] = {nullptr, nullptr};  // pinned
    cudaEvent_t stage_ev[2] = {nullptr, nullptr};
    bool stage_busy[2] = {false, false};
    int stage_next = 0;
    unsigned char *dtab = nullptr;
    unsigned long long *rec = nullptr;
    unsigned int *hrow = nullptr;
    size_t hrow_cap = 0;
    DevStatus *dstatus = nullptr;

    cudaGraphExec_t gexec = nullptr;
    unsigned long long graph_groups = 0;  // bit g set: the graph launches group g
    Completion *comp = nullptr;
    unsigned long long ticks_issued = 0;
    std::vector<TickRec *> inflight;
    std::vector<cudaEvent_t> ev_pool;

    // statistics since the last reset
    std::vector<double> frame_lat, pkt_lat, host_tick, gpu_tick;
    unsigned long long n_ticks = 0, n_frames = 0, n_events = 0, n_packets = 0;
    unsigned long long n_admitted = 0, n_refused = 0, n_events_refused = 0;
    double gpu_ms = 0.0;
    unsigned long long gpu_n = 0;
    int launches_per_tick = 0;
};

namespace {

cudaEvent_t take_event(esi_server *s)
{
    if (!s->ev_pool.empty()) {
        cudaEvent_t e = s->ev_pool.back();
        s->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Finish every tick whose completion stamp is in: frames become readable,
// latencies are recorded.
void poll(esi_server *s)
{
    const unsigned long long done = s->comp->done.load(std::memory_order_acquire);
    size_t k = 0;
    for (; k < s->inflight.size(); ++k) {
        TickRec *t = s->inflight[k];
        if (t->id >= done) break;
        const long long ready = s->comp->ns[t->id % kTickSlots];
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, t->ev0, t->ev1) == cudaSuccess) {
            s->gpu_ms += ms;
            s->gpu_n += 1;
            s->gpu_tick.push_back(ms);
        }
        s->ev_pool.push_back(t->ev0);
        s->ev_pool.push_back(t->ev1);
        for (const TickFrame &f : t->frames) {
            Stream &st = s->streams[f.stream];
            const double lat = (double)(ready - t->call_ns) * 1e-6;
            s->frame_lat.push_back(lat);
            if (f.ref_push_ns) s->pkt_lat.push_back((double)(ready - f.ref_push_ns) * 1e-6);
            s->n_frames += 1;
            if (!st.open) continue;
            const int slot = (int)(f.seq % (unsigned long long)s->opts.frame_slots);
            st.slot_t[slot] = f.t_frame;
            st.slot_lat[slot] = lat;
            st.seq_done = std::max(st.seq_done, f.seq + 1);
            if (st.sink && f.seq < st.sink_n) {
                std::memcpy(st.sink + (size_t)f.seq * (size_t)st.P,
                            st.slots_host + (size_t)slot * (size_t)st.P, (size_t)st.P);
                if (st.sink_t) st.sink_t[f.seq] = f.t_frame;
            }
        }
        delete t;
    }
    s->inflight.erase(s->inflight.begin(), s->inflight.begin() + k);
}

int wait_all(esi_server *s)
{
    cudaError_t e = cudaStreamSynchronize(s->stream);
    // the host-function node may still be finishing its store
    while (e == cudaSuccess && s->comp->done.load(std::memory_order_acquire) < s->ticks_issued) {
    }
    poll(s);
    return rc_of(e);
}

// Variant group g: tile height index g / 12 (4, 8, 16 rows), then render
// mode, decay kind and row alignment.
int group_tile_h(int g) { return 4 << (g / 12); }
int group_rd(int g) { return (g % 12) / 6; }
int group_dk(int g) { return (g % 6) / 2; }
bool group_vec(int g) { return g % 2 == 1; }

cudaError_t launch_group(esi_server *s, int g, cudaStream_t cs)
{
    return launch_tile_batch_tab(s->dtab, g, s->tile_grid, group_tile_h(g), group_rd(g),
                                 group_dk(g), group_vec(g), kBatch, kMaxChunksPerStream, cs);
}

// Capture the per-tick graph for the variant groups in `groups`.
int build_graph(esi_server *s, unsigned long long groups)
{
    if (s->gexec) {
        cudaGraphExecDestroy(s->gexec);
        s->gexec = nullptr;
    }
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return rc_of(e);
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess)
        e = launch_bin_batch_tab(s->dtab, s->bin_grid, kChunk, s->max_tiles, s->bin_mask, cs);
    for (int gi = 0; gi < kGroups && e == cudaSuccess; ++gi)
        if (groups & (1ull << gi)) e = launch_group(s, gi, cs);
    if (e == cudaSuccess) e = cudaLaunchHostFunc(cs, on_tick_done, s->comp);
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&s->gexec, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        s->gexec = nullptr;
        return rc_of(e);
    }
    s->graph_groups = groups;
    return ESI_OK;
}

int group_of(const MapParams &mp, const DecayParams &dp, int W, int tile_h)
{
    const int th = tile_h == 4 ? 0 : tile_h == 8 ? 1 : 2;
    const int rd = mp.render_decay ? 1 : 0;
    const int dk = decay_kind_of(dp);
    const int vec = (W % 4 == 0) ? 1 : 0;
    return th * 12 + rd * 6 + dk * 2 + vec;
}

// Tiles of a stream at tile height th (4, 8 or 16); the state layout does not
// depend on it, so it may change between ticks.
void set_stream_tiles(Stream &st, int th)
{
    st.tile_h = th;
    st.th_log2 = th == 4 ? 2 : th == 8 ? 3 : 4;
    st.tiles_x = (st.W + kTileW - 1) / kTileW;
    st.n_tiles = st.tiles_x * ((st.H + th - 1) / th);
    st.group = group_of(st.mp, st.dp, st.W, th);
}

}  // namespace

// ------------------------------------------------------------------ C ABI
extern "C" {

int esi_server_create(size_t state_budget_bytes, const esi_server_opts *opts, void *cuda_stream,
                      esi_server **out)
{
    if (!out) return ESI_EINVAL;
    *out = nullptr;
    esi_server_opts o{};
    if (opts) o = *opts;
    if (!o.frame_period_us) o.frame_period_us = 10000;
    if (!o.max_events_per_tick) o.max_events_per_tick = 1 << 22;
    if (!o.max_streams) o.max_streams = 256;
    if (!o.frame_slots) o.frame_slots = 4;
    if (!o.tile_h) o.tile_h = 8;
    if (!o.max_stream_pixels) o.max_stream_pixels = 1280 * 720;
    if (!o.scan_chain) o.scan_chain = kScanChainDefault;
    if (!opts) o.use_graph = 1;
    if (o.frame_period_us < 1 || o.max_events_per_tick < kChunk || o.max_streams < 1 ||
        o.max_streams > 4096 || o.frame_slots < 2 || o.frame_slots > 64 ||
        (o.tile_h != 4 && o.tile_h != 8 && o.tile_h != 16) ||
        o.max_stream_pixels < 1 || o.scan_chain < 1 || o.scan_chain > kScanNever ||
        state_budget_bytes == 0)
        return ESI_EINVAL;
    esi_server *s = new (std::nothrow) esi_server();
    if (!s) return ESI_ENOMEM;
    s->opts = o;
    s->budget = state_budget_bytes;
    s->tile_h = o.tile_h;
    s->streams.resize((size_t)o.max_streams);
    // capacities: the largest stream allowed, at the smallest tile height (4
    // rows), bounds the tiles per stream
    constexpr int kMinTileH = 4;
    s->max_tiles = 0;
    {
        const long long maxp = o.max_stream_pixels;
        // tiles of a 128-wide layout cover at most ceil(P / 128) + rows; bound generously
        long long t = (maxp + (long long)kTileW * kMinTileH - 1) / ((long long)kTileW * kMinTileH) +
                      (long long)std::sqrt((double)maxp) + 2;
        s->max_tiles = (int)std::min<long long>(t, 16384);
    }
    s->cap_jobs = o.max_streams;
    s->cap_events = o.max_events_per_tick;
    s->cap_chunks = (int)((s->cap_events + kChunk - 1) / kChunk) + o.max_streams;
    s->cap_frames = o.max_streams * (o.frame_slots - 1);
    {
        // items: every tile of every stream; bounded by the pixels the budget can hold
        const long long px_budget = (long long)(state_budget_bytes / 12);
        const long long items = px_budget / ((long long)kTileW * kMinTileH) +
                                (long long)o.max_streams * (long long)(std::sqrt((double)o.max_stream_pixels) + 2);
        s->cap_items = (int)std::min<long long>(items, 1 << 22);
    }
    // staging / device table layout
    size_t off = align_up(sizeof(TickDir), 256);
    s->off_binjob = off;
    off = align_up(off + sizeof(BinJob) * (size_t)s->cap_jobs, 256);
    s->off_chunkjob = off;
    off = align_up(off + sizeof(int) * (size_t)s->cap_chunks, 256);
    s->off_tilejob = off;
    off = align_up(off + sizeof(TileArgs) * (size_t)s->cap_jobs, 256);
    s->off_win = off;
    off = align_up(off + sizeof(WinInfo) * (size_t)s->cap_frames, 256);
    s->off_fout = off;
    off = align_up(off + sizeof(void *) * (size_t)s->cap_frames, 256);
    s->off_items = off;
    off = align_up(off + sizeof(int2) * (size_t)s->cap_items, 256);
    s->off_events = off;
    off = align_up(off + sizeof(esi_event) * (size_t)s->cap_events, 256);
    s->tab_bytes = off;
    s->hrow_cap = (size_t)s->cap_chunks * (size_t)s->max_tiles;
    s->bin_mask = bin_mask_fits(kChunk, s->max_tiles);

    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = set_kernel_attributes();
    if (e == cudaSuccess) {
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
        s->tile_grid = std::max(1, sms) * 2;
        s->bin_grid = std::min(s->cap_chunks,
                               std::max(1, sms) * bin_tab_blocks_per_sm(kChunk, s->max_tiles, s->bin_mask));
    }
    if (e == cudaSuccess) {
        if (cuda_stream) {
            s->stream = (cudaStream_t)cuda_stream;
        } else {
            e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
            s->own_stream = e == cudaSuccess;
        }
    }
    if (e == cudaSuccess) e = cudaMalloc((void **)&s->arena_base, state_budget_bytes);
    if (e == cudaSuccess) e = cudaMalloc((void **)&s->dtab, s->tab_bytes);
    if (e == cudaSuccess) e = cudaMalloc((void **)&s->rec, (size_t)s->cap_chunks * kChunk * 8);
    if (e == cudaSuccess) e = cudaMalloc((void **)&s->hrow, s->hrow_cap * 4);
    if (e == cudaSuccess) e = cudaMalloc((void **)&s->dstatus, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaMemsetAsync(s->dstatus, 0, sizeof(DevStatus), s->stream);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        e = cudaMallocHost((void **)&s->stage[b], s->tab_bytes);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->stage_ev[b], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) {
        s->comp = new (std::nothrow) Completion();
        if (!s->comp) e = cudaErrorMemoryAllocation;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        int rc = rc_of(e);
        esi_server_destroy(s);
        return rc;
    }
    s->arena.init(state_budget_bytes);
    *out = s;
    return ESI_OK;
}

void esi_server_destroy(esi_server *s)
{
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->comp) {
        while (s->comp->done.load(std::memory_order_acquire) < s->ticks_issued) {
        }
    }
    for (TickRec *t : s->inflight) {
        cudaEventDestroy(t->ev0);
        cudaEventDestroy(t->ev1);
        delete t;
    }
    for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
    for (Stream &st : s->streams)
        if (st.slots_host) cudaFreeHost(st.slots_host);
    if (s->gexec) cudaGraphExecDestroy(s->gexec);
    for (int b = 0; b < 2; ++b) {
        if (s->stage[b]) cudaFreeHost(s->stage[b]);
        if (s->stage_ev[b]) cudaEventDestroy(s->stage_ev[b]);
    }
    cudaFree(s->arena_base);
    cudaFree(s->dtab);
    cudaFree(s->rec);
    cudaFree(s->hrow);
    cudaFree(s->dstatus);
    delete s->comp;
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
}

int esi_stream_open(esi_server *s, int width, int height, const esi_params *params, int *stream_id)
{
    if (!s || !stream_id) return ESI_EINVAL;
    int rc = validate_params(width, height, params);
    if (rc) return rc;
    if ((long long)width * height > s->opts.max_stream_pixels) return ESI_ERANGE;
    int id = -1;
    for (int i = 0; i < (int)s->streams.size(); ++i)
        if (!s->streams[i].open) {
            id = i;
            break;
        }
    if (id < 0) {
        s->n_refused += 1;
        return ESI_EBUSY;
    }
    const long long P = (long long)width * height;
    const size_t sbytes = align_up((size_t)P * 4, 256) + (size_t)P * 8;
    const size_t off = s->arena.alloc(sbytes);
    if (off == SIZE_MAX) {
        s->n_refused += 1;
        return ESI_EBUSY;
    }
    Stream &st = s->streams[id];
    st = Stream();
    st.W = width;
    st.H = height;
    st.P = P;
    st.prm = *params;
    prepare_params(*params, &st.dp, &st.mp);
    set_stream_tiles(st, s->tile_h);
    if (st.n_tiles > s->max_tiles) {
        s->arena.release(off, sbytes);
        return ESI_ERANGE;
    }
    st.arena_off = off;
    st.arena_bytes = sbytes;
    st.S = reinterpret_cast<float *>(s->arena_base + off);
    st.T = reinterpret_cast<long long *>(s->arena_base + off + align_up((size_t)P * 4, 256));
    st.last_event_t = params->t_origin_us;
    st.push_floor = params->t_origin_us;
    st.next_frame_t = params->t_origin_us + s->opts.frame_period_us;
    st.slot_t.assign((size_t)s->opts.frame_slots, 0);
    st.slot_lat.assign((size_t)s->opts.frame_slots, 0.0);
    cudaError_t e = cudaHostAlloc((void **)&st.slots_host, (size_t)s->opts.frame_slots * (size_t)P,
                                  cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&st.slots_dev, st.slots_host, 0);
    // Alg. 2 initialisation: S = 0, T = t_origin
    if (e == cudaSuccess) e = cudaMemsetAsync(st.S, 0, (size_t)P * 4, s->stream);
    if (e == cudaSuccess) e = launch_fill_i64(st.T, P, params->t_origin_us, s->stream);
    if (e != cudaSuccess) {
        if (st.slots_host) cudaFreeHost(st.slots_host);
        st.slots_host = nullptr;
        s->arena.release(off, sbytes);
        return rc_of(e);
    }
    st.open = true;
    s->used += sbytes;
    s->n_open += 1;
    s->n_admitted += 1;
    *stream_id = id;
    return ESI_OK;
}

int esi_stream_push(esi_server *s, int id, const esi_event *ev, size_t n)
{
    if (!s || id < 0 || id >= (int)s->streams.size() || !s->streams[id].open || (n && !ev))
        return ESI_EINVAL;
    Stream &st = s->streams[id];
    if (n == 0) return ESI_OK;
    long long prev = std::max(st.last_event_t, st.push_floor);
    for (size_t i = 0; i < n; ++i) {
        if (ev[i].t_us < prev) return ESI_ETIMEORDER;
        prev = ev[i].t_us;
    }
    if (st.pend_head > 0 && st.pend_head * 2 > st.pend.size()) {
        st.pend.erase(st.pend.begin(), st.pend.begin() + (long)st.pend_head);
        st.pend_head = 0;
    }
    st.pend.insert(st.pend.end(), ev, ev + n);
    st.last_event_t = prev;
    st.last_push_ns = wall_ns();
    s->n_packets += 1;
    return ESI_OK;
}

int esi_stream_watermark(esi_server *s, int id, int64_t t_us)
{
    if (!s || id < 0 || id >= (int)s->streams.size() || !s->streams[id].open) return ESI_EINVAL;
    Stream &st = s->streams[id];
    if (st.watermark != LLONG_MAX && (long long)t_us < st.watermark) return ESI_ETIMEORDER;
    st.watermark = t_us;
    return ESI_OK;
}

int esi_stream_set_tile_h(esi_server *s, int id, int tile_h)
{
    if (!s || id < 0 || id >= (int)s->streams.size() || !s->streams[id].open) return ESI_EINVAL;
    if (tile_h != 4 && tile_h != 8 && tile_h != 16) return ESI_EINVAL;
    Stream &st = s->streams[id];
    Stream probe = st;
    set_stream_tiles(probe, tile_h);
    if (probe.n_tiles > s->max_tiles) return ESI_ERANGE;
    set_stream_tiles(st, tile_h);
    return ESI_OK;
}

int esi_stream_autotune(esi_server *s, int id, const esi_event *sample, size_t n, int flags,
                        int *tile_h)
{
    if (!s || id < 0 || id >= (int)s->streams.size() || !s->streams[id].open || !sample || !n)
        return ESI_EINVAL;
    Stream &st = s->streams[id];
    // frames at the server's frame period over the sample
    std::vector<int64_t> tf;
    const long long t_first = sample[0].t_us, t_last = sample[n - 1].t_us;
    for (long long t = t_first + s->opts.frame_period_us; t <= t_last; t += s->opts.frame_period_us)
        tf.push_back(t);
    if (tf.empty()) tf.push_back(t_last);
    std::vector<esi_tuning> cands;
    for (int th : {4, 8, 16}) {
        if (st.tiles_x * ((st.H + th - 1) / th) > s->max_tiles) continue;
        esi_tuning t{};
        t.tile_w = kTileW;
        t.tile_h = th;
        t.chunk_events = kChunk;
        t.batch_records = kBatch;
        t.max_batch_events = kMaxChunksPerStream * kChunk;
        cands.push_back(t);
    }
    // the key's flags field carries a marker bit for serving shapes
    const AutotuneKey key{st.W, st.H, autotune_bucket(n, tf.size()), st.mp.render_decay,
                          decay_kind_of(st.dp), 0x100};
    esi_tuning best{};
    int rc = autotune_shapes(key, st.prm, s->stream, sample, n, tf.data(), tf.size(), cands,
                             (flags & ESI_AUTOTUNE_FORCE) != 0, &best);
    if (rc) return rc;
    rc = esi_stream_set_tile_h(s, id, best.tile_h);
    if (!rc && tile_h) *tile_h = best.tile_h;
    return rc;
}

int esi_server_tick(esi_server *s, int64_t now_us)
{
    if (!s) return ESI_EINVAL;
    const long long call_ns = wall_ns();
    poll(s);
    const int b = s->stage_next;
    if (s->stage_busy[b]) {
        cudaError_t e = cudaEventSynchronize(s->stage_ev[b]);
        if (e != cudaSuccess) return rc_of(e);
        s->stage_busy[b] = false;
    }
    unsigned char *stg = s->stage[b];
    TickDir *dir = reinterpret_cast<TickDir *>(stg);
    std::memset(dir, 0, sizeof(TickDir));
    BinJob *bj = reinterpret_cast<BinJob *>(stg + s->off_binjob);
    int *cj = reinterpret_cast<int *>(stg + s->off_chunkjob);
    TileArgs *tj = reinterpret_cast<TileArgs *>(stg + s->off_tilejob);
    WinInfo *win = reinterpret_cast<WinInfo *>(stg + s->off_win);
    unsigned char **fout = reinterpret_cast<unsigned char **>(stg + s->off_fout);
    esi_event *evs = reinterpret_cast<esi_event *>(stg + s->off_events);

    TickRec *rec = new (std::nothrow) TickRec();
    if (!rec) return ESI_ENOMEM;
    rec->call_ns = call_ns;
    int n_jobs = 0, n_chunks = 0, n_frames = 0;
    long long n_items_total = 0;
    long long n_ev = 0;
    size_t hrow_off = 0;
    std::vector<std::pair<int, int>> job_stream;  // (job, stream)
    const int K = s->opts.frame_slots;
    const long long ev_cap_stream = (long long)kMaxChunksPerStream * kChunk;

    for (int id = 0; id < (int)s->streams.size(); ++id) {
        Stream &st = s->streams[id];
        if (!st.open) continue;
        // due frames (at most K - 1 per tick, and never more than K - 1 in flight)
        const unsigned long long in_flight = st.seq_issued - st.seq_done;
        int can = (int)std::max<long long>(0, (long long)(K - 1) - (long long)in_flight);
        std::vector<long long> fr;
        long long tf = st.next_frame_t;
        const long long upto = std::min((long long)now_us, st.watermark);
        while (tf <= upto && (int)fr.size() < can) {
            fr.push_back(tf);
            tf += s->opts.frame_period_us;
        }
        // every tick applies what has arrived, so a frame's tick only has the
        // newest events left to do
        const size_t avail = st.pend.size() - st.pend_head;
        if (fr.empty() && avail == 0) continue;
        // events: t <= now, or <= the last frame when frames wait for the next tick
        long long lim_t = upto;
        if (tf <= upto) lim_t = fr.empty() ? st.push_floor : fr.back();
        const esi_event *pb = st.pend.data() + st.pend_head;
        size_t take = (size_t)(std::upper_bound(pb, pb + avail, lim_t,
                                                [](long long v, const esi_event &e) { return v < e.t_us; }) -
                               pb);
        take = std::min(take, (size_t)ev_cap_stream);
        if (n_ev + (long long)take > s->cap_events) take = (size_t)std::max<long long>(0, s->cap_events - n_ev);
        if (take > 0 && take < avail) {
            // frames after an event left for later must wait too
            const long long t_left = pb[take].t_us;
            while (!fr.empty() && fr.back() >= t_left) fr.pop_back();
        }
        if (take > 0) {
            // record times are 32-bit offsets from the first event
            const long long lim = pb[0].t_us + 0xffffffffll;
            size_t ok = (size_t)(std::upper_bound(pb, pb + take, lim,
                                                  [](long long v, const esi_event &e) { return v < e.t_us; }) -
                                 pb);
            if (ok < take) {
                take = ok;
                const long long t_left = pb[take].t_us;
                while (!fr.empty() && fr.back() >= t_left) fr.pop_back();
            }
        }
        if (take == 0 && fr.empty()) continue;
        const int chunks = (int)((take + kChunk - 1) / kChunk);
        if (n_jobs >= s->cap_jobs || n_chunks + chunks > s->cap_chunks ||
            n_frames + (int)fr.size() > s->cap_frames ||
            hrow_off + (size_t)chunks * st.n_tiles > s->hrow_cap ||
            n_items_total + st.n_tiles > s->cap_items)
            break;  // the tick is full: the rest waits for the next one
        const int j = n_jobs++;
        const long long t_base = take ? pb[0].t_us : fr.front();
        std::memcpy(evs + n_ev, pb, take * sizeof(esi_event));
        // binning job
        BinJob &B = bj[j];
        B.args.ring = reinterpret_cast<const esi_event *>(s->dtab + s->off_events) + n_ev;
        B.args.ring_mask = ~0ull >> 1;
        B.args.first = 0;
        B.args.n = (int)take;
        B.args.chunk = kChunk;
        B.args.t_base = t_base;
        B.args.W = st.W;
        B.args.H = st.H;
        B.args.tiles_x = st.tiles_x;
        B.args.n_tiles = st.n_tiles;
        B.args.th_log2 = st.th_log2;
        B.args.tw_log2 = 7;
        B.args.tile_bits = index_bits(st.n_tiles);
        B.args.rec = s->rec + (size_t)n_chunks * kChunk;
        B.args.hrow = s->hrow + hrow_off;
        B.args.use_mask = s->bin_mask ? 1 : 0;
        B.args.status = s->dstatus;
        B.args.rec_idx = nullptr;
        B.args.ev_out = nullptr;
        B.first_chunk = n_chunks;
        for (int c = 0; c < chunks; ++c) cj[n_chunks + c] = j;
        // tile job
        TileArgs &A = tj[j];
        A.rec = s->rec + (size_t)n_chunks * kChunk;
        A.hrow = s->hrow + hrow_off;
        A.n_chunks = chunks;
        A.chunk = kChunk;
        A.n_tiles = st.n_tiles;
        A.t_base = t_base;
        A.S = st.S;
        A.T = st.T;
        A.W = st.W;
        A.H = st.H;
        A.tiles_x = st.tiles_x;
        A.dp = st.dp;
        A.mp = st.mp;
        A.win = reinterpret_cast<const WinInfo *>(s->dtab + s->off_win) + n_frames;
        A.w_begin = 0;
        A.w_end = (int)fr.size();
        A.frames = nullptr;
        A.frame_outs = reinterpret_cast<unsigned char *const *>(s->dtab + s->off_fout) + n_frames;
        A.P = st.P;
        A.batch = kBatch;
        A.status = s->dstatus;
        A.rec_idx = nullptr;
        A.ev_out = nullptr;
        A.scan_chain = s->opts.scan_chain;
        for (size_t w = 0; w < fr.size(); ++w) {
            const long long d = fr[w] - t_base;
            win[n_frames + w].lim = std::min(std::max(d, -1ll), 0xffffffffll);
            win[n_frames + w].tf_f = (float)d;
            win[n_frames + w].pad = 0;
            const unsigned long long seq = st.seq_issued + w;
            fout[n_frames + w] = st.slots_dev + (size_t)(seq % (unsigned long long)K) * (size_t)st.P;
            rec->frames.push_back({id, seq, fr[w], st.last_push_ns});
        }
        job_stream.push_back({j, id});
        st.seq_issued += fr.size();
        if (!fr.empty()) st.next_frame_t = fr.back() + s->opts.frame_period_us;
        st.pend_head += take;
        if (!fr.empty()) st.push_floor = std::max(st.push_floor, fr.back());
        n_ev += (long long)take;
        n_chunks += chunks;
        n_frames += (int)fr.size();
        hrow_off += (size_t)chunks * st.n_tiles;
        dir->n_items[st.group] += st.n_tiles;
        n_items_total += st.n_tiles;
    }
    if (n_jobs == 0) {
        delete rec;
        s->n_ticks += 1;
        return ESI_OK;
    }
    // work items, grouped by variant
    int2 *items = reinterpret_cast<int2 *>(stg + s->off_items);
    unsigned long long groups = 0;
    long long item_off = 0;
    for (int g = 0; g < kGroups; ++g) {
        if (!dir->n_items[g]) continue;
        if (item_off + dir->n_items[g] > s->cap_items) {
            delete rec;
            return ESI_ERANGE;
        }
        groups |= 1ull << g;
        dir->off_items[g] = (long long)s->off_items + item_off * (long long)sizeof(int2);
        int2 *it = items + item_off;
        for (auto &js : job_stream) {
            const Stream &st = s->streams[js.second];
            if (st.group != g) continue;
            for (int t = 0; t < st.n_tiles; ++t) *it++ = make_int2(js.first, t);
        }
        item_off += dir->n_items[g];
    }
    dir->n_chunks = n_chunks;
    dir->off_binjob = (long long)s->off_binjob;
    dir->off_chunkjob = (long long)s->off_chunkjob;
    dir->off_tilejob = (long long)s->off_tilejob;

    // tables and events to the device; tick kernels; completion stamp
    cudaError_t e = cudaMemcpyAsync(s->dtab, stg, s->off_items + (size_t)item_off * sizeof(int2),
                                    cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess && n_ev)
        e = cudaMemcpyAsync(s->dtab + s->off_events, stg + s->off_events,
                            (size_t)n_ev * sizeof(esi_event), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaEventRecord(s->stage_ev[b], s->stream);
    if (e != cudaSuccess) {
        delete rec;
        return rc_of(e);
    }
    s->stage_busy[b] = true;
    s->stage_next = 1 - b;
    rec->ev0 = take_event(s);
    rec->ev1 = take_event(s);
    rec->id = s->ticks_issued;
    e = cudaEventRecord(rec->ev0, s->stream);
    int ngroups = 0;
    for (int g = 0; g < kGroups; ++g) ngroups += (int)((groups >> g) & 1ull);
    if (e == cudaSuccess) {
        if (s->opts.use_graph) {
            if (!s->gexec || (groups & ~s->graph_groups)) {
                int rc = build_graph(s, groups | s->graph_groups);
                if (rc) {
                    delete rec;
                    return rc;
                }
            }
            e = cudaGraphLaunch(s->gexec, s->stream);
            int ng = 0;
            for (int g = 0; g < kGroups; ++g) ng += (int)((s->graph_groups >> g) & 1ull);
            s->launches_per_tick = 1 + ng;
        } else {
            e = launch_bin_batch_tab(s->dtab, s->bin_grid, kChunk, s->max_tiles, s->bin_mask, s->stream);
            for (int g = 0; g < kGroups && e == cudaSuccess; ++g)
                if (groups & (1ull << g)) e = launch_group(s, g, s->stream);
            if (e == cudaSuccess) e = cudaLaunchHostFunc(s->stream, on_tick_done, s->comp);
            s->launches_per_tick = 1 + ngroups;
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(rec->ev1, s->stream);
    if (e != cudaSuccess) {
        delete rec;
        return rc_of(e);
    }
    s->ticks_issued += 1;
    s->inflight.push_back(rec);
    s->n_ticks += 1;
    s->n_events += (unsigned long long)n_ev;
    s->host_tick.push_back((double)(wall_ns() - call_ns) * 1e-6);
    return ESI_OK;
}

int esi_stream_frame(esi_server *s, int id, uint8_t *out, int64_t *t_frame, double *latency_ms)
{
    if (!s || id < 0 || id >= (int)s->streams.size() || !s->streams[id].open || !out)
        return ESI_EINVAL;
    poll(s);
    Stream &st = s->streams[id];
    if (st.seq_done == 0) return ESI_ESTATE;
    const unsigned long long seq = st.seq_done - 1;
    const int slot = (int)(seq % (unsigned long long)s->opts.frame_slots);
    std::memcpy(out, st.slots_host + (size_t)slot * (size_t)st.P, (size_t)st.P);
    if (t_frame) *t_frame = st.slot_t[slot];
    if (latency_ms) *latency_ms = st.slot_lat[slot];
    return ESI_OK;
}

int esi_stream_frame_seq(esi_server *s, int id, uint64_t seq, uint8_t *out, int64_t *t_frame)
{
    if (!s || id < 0 || id >= (int)s->streams.size() || !s->streams[id].open || !out)
        return ESI_EINVAL;
    poll(s);
    Stream &st = s->streams[id];
    if (seq >= st.seq_done) return ESI_ESTATE;
    // slot seq % K is reused by frame seq + K once that one is handed to a tick
    const unsigned long long K = (unsigned long long)s->opts.frame_slots;
    if (st.seq_issued > seq + K) return ESI_ERANGE;
    const int slot = (int)(seq % K);
    std::memcpy(out, st.slots_host + (size_t)slot * (size_t)st.P, (size_t)st.P);
    if (t_frame) *t_frame = st.slot_t[slot];
    return ESI_OK;
}

int esi_stream_set_frame_sink(esi_server *s, int id, uint8_t *out, uint64_t max_frames,
                              int64_t *t_frames)
{
    if (!s || id < 0 || id >= (int)s->streams.size() || !s->streams[id].open) return ESI_EINVAL;
    if (max_frames && !out) return ESI_EINVAL;
    poll(s);
    Stream &st = s->streams[id];
    st.sink = max_frames ? out : nullptr;
    st.sink_n = max_frames;
    st.sink_t = max_frames ? reinterpret_cast<long long *>(t_frames) : nullptr;
    return ESI_OK;
}

int esi_stream_frames_done(esi_server *s, int id, uint64_t *n_done)
{
    if (!s || id < 0 || id >= (int)s->streams.size() || !s->streams[id].open || !n_done)
        return ESI_EINVAL;
    poll(s);
    *n_done = s->streams[id].seq_done;
    return ESI_OK;
}

int esi_stream_state(esi_server *s, int id, float *S, int64_t *T)
{
    if (!s || id < 0 || id >= (int)s->streams.size() || !s->streams[id].open || !S || !T)
        return ESI_EINVAL;
    int rc = wait_all(s);
    if (rc) return rc;
    Stream &st = s->streams[id];
    cudaError_t e = cudaMemcpy(S, st.S, (size_t)st.P * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(T, st.T, (size_t)st.P * 8, cudaMemcpyDeviceToHost);
    return rc_of(e);
}

int esi_stream_close(esi_server *s, int id)
{
    if (!s || id < 0 || id >= (int)s->streams.size() || !s->streams[id].open) return ESI_EINVAL;
    int rc = wait_all(s);
    if (rc) return rc;
    Stream &st = s->streams[id];
    s->arena.release(st.arena_off, st.arena_bytes);
    s->used -= st.arena_bytes;
    if (st.slots_host) cudaFreeHost(st.slots_host);
    st = Stream();
    s->n_open -= 1;
    return ESI_OK;
}

int esi_server_sync(esi_server *s)
{
    if (!s) return ESI_EINVAL;
    return wait_all(s);
}

int esi_server_get_stats(esi_server *s, esi_server_stats *out)
{
    if (!s || !out) return ESI_EINVAL;
    poll(s);
    std::memset(out, 0, sizeof(*out));
    out->ticks = s->n_ticks;
    out->frames = s->n_frames;
    out->events = s->n_events;
    out->packets = s->n_packets;
    out->frame_latency_p50_ms = percentile(s->frame_lat, 0.50);
    out->frame_latency_p99_ms = percentile(s->frame_lat, 0.99);
    out->packet_latency_p50_ms = percentile(s->pkt_lat, 0.50);
    out->packet_latency_p99_ms = percentile(s->pkt_lat, 0.99);
    out->gpu_ms_per_tick = s->gpu_n ? s->gpu_ms / (double)s->gpu_n : 0.0;
    out->state_bytes_used = s->used;
    out->state_budget_bytes = s->budget;
    out->streams_open = s->n_open;
    out->kernel_launches_per_tick = s->launches_per_tick;
    out->streams_admitted = s->n_admitted;
    out->streams_refused = s->n_refused;
    out->events_refused = s->n_events_refused;
    out->host_tick_p50_ms = percentile(s->host_tick, 0.50);
    out->host_tick_p99_ms = percentile(s->host_tick, 0.99);
    out->gpu_tick_p99_ms = percentile(s->gpu_tick, 0.99);
    return ESI_OK;
}

int esi_server_reset_stats(esi_server *s)
{
    if (!s) return ESI_EINVAL;
    poll(s);
    s->frame_lat.clear();
    s->pkt_lat.clear();
    s->host_tick.clear();
    s->gpu_tick.clear();
    s->n_ticks = s->n_frames = s->n_events = s->n_packets = 0;
    s->n_admitted = s->n_refused = s->n_events_refused = 0;
    s->gpu_ms = 0.0;
    s->gpu_n = 0;
    return ESI_OK;
}

// --------------------------------------------------------------- executors
namespace {

// Wall-clock pacing: wait until stream time t_us (microseconds since t0_ns).
void wait_until(long long t0_ns, long long t_us)
{
    const long long target = t0_ns + t_us * 1000;
    for (;;) {
        const long long now = wall_ns();
        if (now >= target) return;
        if (target - now > 200000) {
            struct timespec ts = {0, (long)(target - now - 100000)};
            nanosleep(&ts, nullptr);
        }
    }
}

bool frames_due(const Stream &st, long long now)
{
    return st.open && st.next_frame_t <= std::min(now, st.watermark);
}

// Issue every frame of the streams selected by `which` (-1: all) that is due
// at `now`: the last tick may have left some behind (a full tick, or the
// frames a stream may have in flight).  Bounded; waits for ticks in flight.
int drain_frames(esi_server *s, int which, long long now)
{
    for (int guard = 0; guard < 4096; ++guard) {
        bool due = false;
        for (int id = 0; id < (int)s->streams.size() && !due; ++id)
            if ((which < 0 || id == which) && frames_due(s->streams[id], now)) due = true;
        if (!due) return ESI_OK;
        if (!s->inflight.empty()) {
            cudaError_t e = cudaEventSynchronize(s->inflight.front()->ev1);
            if (e != cudaSuccess) return rc_of(e);
        }
        int rc = esi_server_tick(s, now);
        if (rc) return rc;
    }
    return ESI_ERANGE;
}

}  // namespace

int esi_server_run(esi_server *s, const esi_packet *pk, size_t n, int64_t tick_us, int64_t t_end_us,
                   int realtime)
{
    if (!s || (n && !pk) || tick_us < 1 || t_end_us < 0) return ESI_EINVAL;
    for (size_t i = 1; i < n; ++i)
        if (pk[i].arrival_us < pk[i - 1].arrival_us) return ESI_EINVAL;
    for (size_t i = 0; i < n; ++i)
        if (pk[i].stream < 0 || pk[i].stream >= kMaxSlots || pk[i].kind < ESI_PACKET_EVENTS ||
            pk[i].kind > ESI_PACKET_CLOSE || (pk[i].kind == ESI_PACKET_OPEN && !pk[i].ev))
            return ESI_EINVAL;
    // slot -> server stream id; a slot no OPEN packet has bound names a server id
    constexpr int kUnbound = INT_MIN;
    std::vector<int> slot_id;
    std::vector<esi_stream_spec *> slot_spec;
    auto sid_of = [&](int slot) {
        return (size_t)slot < slot_id.size() && slot_id[slot] != kUnbound ? slot_id[slot] : slot;
    };
    auto bind = [&](int slot, int id, esi_stream_spec *spec) {
        if ((size_t)slot >= slot_id.size()) {
            slot_id.resize((size_t)slot + 1, kUnbound);
            slot_spec.resize((size_t)slot + 1, nullptr);
        }
        slot_id[slot] = id;
        if (spec) slot_spec[slot] = spec;
        if (slot_spec[slot]) slot_spec[slot]->stream_id = id;
    };
    const long long t0 = wall_ns();
    const long long min_gap = std::max<long long>(1, tick_us / 5);
    size_t i = 0;
    long long next_tick = tick_us, last_tick = LLONG_MIN / 2;
    for (;;) {
        long long now;
        if (realtime) {
            long long next_evt = next_tick;
            if (i < n) next_evt = std::min<long long>(next_evt, pk[i].arrival_us);
            wait_until(t0, next_evt);
            now = (wall_ns() - t0) / 1000;
        } else {
            now = next_tick;
        }
        for (; i < n && pk[i].arrival_us <= now; ++i) {
            const esi_packet &q = pk[i];
            int rc = ESI_OK;
            if (q.kind == ESI_PACKET_OPEN) {
                // the spec is the caller's, writable: the packet carries it as ev
                esi_stream_spec *sp = reinterpret_cast<esi_stream_spec *>(const_cast<esi_event *>(q.ev));
                int id = -1;
                rc = esi_stream_open(s, sp->width, sp->height, &sp->params, &id);
                if (rc == ESI_EBUSY) {  // refused admission: its packets are dropped
                    bind(q.stream, -1, sp);
                    continue;
                }
                if (!rc && sp->tile_h) rc = esi_stream_set_tile_h(s, id, sp->tile_h);
                if (!rc && sp->frame_sink)
                    rc = esi_stream_set_frame_sink(s, id, sp->frame_sink, sp->sink_frames,
                                                   sp->sink_t_frames);
                if (!rc) bind(q.stream, id, sp);
            } else {
                const int id = sid_of(q.stream);
                if (id < 0) {
                    if (q.kind == ESI_PACKET_EVENTS) s->n_events_refused += q.n;
                    continue;
                }
                if (q.kind == ESI_PACKET_CLOSE) {
                    // the stream's frames up to its last packet come first
                    rc = drain_frames(s, id, std::min<long long>(now, t_end_us));
                    if (!rc) rc = esi_stream_close(s, id);
                    bind(q.stream, -1, nullptr);
                } else {
                    rc = esi_stream_push(s, id, q.ev, (size_t)q.n);
                    if (!rc) rc = esi_stream_watermark(s, id, q.arrival_us);
                }
            }
            if (rc) return rc;
        }
        // tick at the tick period, and early when a packet has made a frame due
        bool due = false;
        if (realtime && now - last_tick >= min_gap)
            for (const Stream &st : s->streams)
                if (st.open && st.next_frame_t <= std::min<long long>(now, st.watermark)) {
                    due = true;
                    break;
                }
        if (now >= next_tick || due) {
            int rc = esi_server_tick(s, std::min<long long>(now, t_end_us));
            if (rc) return rc;
            last_tick = now;
            while (next_tick <= now) next_tick += tick_us;
            if (now >= t_end_us) break;
        }
    }
    int rc = drain_frames(s, -1, t_end_us);
    if (rc) return rc;
    return wait_all(s);
}

int esi_plain_run(int n_streams, const int *widths, const int *heights, const esi_params *params,
                  const esi_packet *pk, size_t n, int64_t tick_us, int64_t t_end_us,
                  int64_t frame_period_us, int realtime, esi_server_stats *out)
{
    if (n_streams < 1 || !widths || !heights || !params || (n && !pk) || tick_us < 1 ||
        frame_period_us < 1 || !out)
        return ESI_EINVAL;
    for (size_t i = 0; i < n; ++i)
        if (pk[i].kind != ESI_PACKET_EVENTS || pk[i].stream < 0 || pk[i].stream >= n_streams)
            return ESI_EINVAL;
    struct PS {
        esi_handle *h = nullptr;
        std::vector<unsigned char> frame;
        long long next_frame = 0, watermark = LLONG_MAX, last_push_ns = 0;
    };
    std::vector<PS> ps((size_t)n_streams);
    int rc = ESI_OK;
    for (int k = 0; k < n_streams && !rc; ++k) {
        rc = esi_create(widths[k], heights[k], &params[k], nullptr, &ps[k].h);
        if (!rc) {
            ps[k].frame.resize((size_t)widths[k] * heights[k]);
            ps[k].next_frame = params[k].t_origin_us + frame_period_us;
        }
    }
    std::vector<double> flat, plat;
    unsigned long long ticks = 0, frames = 0, events = 0, packets = 0;
    const long long t0 = wall_ns();
    size_t i = 0;
    long long next_tick = tick_us;
    while (!rc) {
        long long now;
        if (realtime) {
            long long next_evt = next_tick;
            if (i < n) next_evt = std::min<long long>(next_evt, pk[i].arrival_us);
            wait_until(t0, next_evt);
            now = (wall_ns() - t0) / 1000;
        } else {
            now = next_tick;
        }
        for (; i < n && pk[i].arrival_us <= now && !rc; ++i) {
            PS &p = ps[(size_t)pk[i].stream];
            rc = esi_push_events(p.h, pk[i].ev, (size_t)pk[i].n, 0);
            p.watermark = pk[i].arrival_us;
            p.last_push_ns = wall_ns();
            events += pk[i].n;
            packets += 1;
        }
        if (rc || now < next_tick) continue;
        const long long call = wall_ns();
        const long long t_now = std::min<long long>(now, t_end_us);
        for (int k = 0; k < n_streams && !rc; ++k) {
            PS &p = ps[(size_t)k];
            const long long upto = std::min(t_now, p.watermark);
            while (p.next_frame <= upto && !rc) {
                rc = esi_render_frame(p.h, p.next_frame, p.frame.data(), 0);
                const long long ready = wall_ns();
                flat.push_back((double)(ready - call) * 1e-6);
                if (p.last_push_ns) plat.push_back((double)(ready - p.last_push_ns) * 1e-6);
                frames += 1;
                p.next_frame += frame_period_us;
            }
        }
        ticks += 1;
        while (next_tick <= now) next_tick += tick_us;
        if (now >= t_end_us) break;
    }
    for (PS &p : ps) esi_destroy(p.h);
    std::memset(out, 0, sizeof(*out));
    out->ticks = ticks;
    out->frames = frames;
    out->events = events;
    out->packets = packets;
    out->frame_latency_p50_ms = percentile(flat, 0.50);
    out->frame_latency_p99_ms = percentile(flat, 0.99);
    out->packet_latency_p50_ms = percentile(plat, 0.50);
    out->packet_latency_p99_ms = percentile(plat, 0.99);
    out->streams_open = n_streams;
    return rc;
}

}  // extern "C"
