// Batched serving of many sensors (esi_server_* in esi.h).
//
// Each stream's pushed events wait in a ring in pinned, mapped host memory
// (one copy, split over worker threads when large).  A tick takes, for every
// stream with work, its pending events up to the tick's time and its due
// frame times, writes per-stream descriptors (ring position, sizes, frames)
// into one pinned staging table, copies that table to the device, and runs
// one batched binning launch (which reads the events from the rings) and,
// after it, one batched tile launch per parameter variant (tile height x
// render mode x decay kind x row alignment) as parallel graph branches.  The kernels
// read their sizes and per-stream descriptors from the device table, so one
// captured CUDA graph serves every tick; frames are written straight into
// mapped host memory.  A host function queued after each tick stamps its
// completion.
#include <time.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstring>
#include <condition_variable>
#include <cstdio>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
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
        used_ = 0;
        free_.clear();
        if (size) free_[0] = size;
    }
    size_t used() const { return used_; }
    // offset of a block of n bytes, or SIZE_MAX when nothing fits
    size_t alloc(size_t n)
    {
        n = align_up(n, 256);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            const size_t off = it->first, len = it->second;
            free_.erase(it);
            if (len > n) free_[off + n] = len - n;
            used_ += n;
            return off;
        }
        return SIZE_MAX;
    }
    void release(size_t off, size_t n)
    {
        n = align_up(n, 256);
        used_ -= n;
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
    size_t size_ = 0, used_ = 0;
    std::map<size_t, size_t> free_;
};

// Worker threads that split a large copy with the calling thread.
class CopyPool {
  public:
    ~CopyPool() { stop(); }
    bool start(int workers)
    {
        try {
            for (int k = 0; k < workers; ++k) th_.emplace_back([this, k] { run(k); });
        } catch (...) {
            stop();
            return false;
        }
        return true;
    }
    void stop()
    {
        {
            std::lock_guard<std::mutex> g(m_);
            stop_ = true;
        }
        cv_.notify_all();
        for (std::thread &t : th_) t.join();
        th_.clear();
    }
    // bytes split into workers + 1 parts; the caller copies the last one
    void copy(void *dst, const void *src, size_t bytes)
    {
        const int parts = (int)th_.size() + 1;
        const size_t part = (bytes / (size_t)parts + 63) & ~(size_t)63;  // 64-byte multiples
        {
            std::lock_guard<std::mutex> g(m_);
            dst_ = static_cast<unsigned char *>(dst);
            src_ = static_cast<const unsigned char *>(src);
            bytes_ = bytes;
            part_ = part;
            pending_ = (int)th_.size();
            gen_ += 1;
        }
        cv_.notify_all();
        const size_t a = std::min(bytes, part * (size_t)(parts - 1));
        std::memcpy(static_cast<unsigned char *>(dst) + a, static_cast<const unsigned char *>(src) + a,
                    bytes - a);
        std::unique_lock<std::mutex> l(m_);
        done_cv_.wait(l, [this] { return pending_ == 0; });
    }
    int workers() const { return (int)th_.size(); }

  private:
    void run(int k)
    {
        unsigned long long seen = 0;
        for (;;) {
            unsigned char *d;
            const unsigned char *s;
            size_t a, b;
            {
                std::unique_lock<std::mutex> l(m_);
                cv_.wait(l, [&] { return stop_ || gen_ != seen; });
                if (stop_) return;
                seen = gen_;
                d = dst_;
                s = src_;
                a = std::min(bytes_, part_ * (size_t)k);
                b = std::min(bytes_, part_ * (size_t)(k + 1));
            }
            if (b > a) std::memcpy(d + a, s + a, b - a);
            {
                std::lock_guard<std::mutex> g(m_);
                pending_ -= 1;
            }
            done_cv_.notify_one();
        }
    }
    std::vector<std::thread> th_;
    std::mutex m_;
    std::condition_variable cv_, done_cv_;
    unsigned long long gen_ = 0;
    int pending_ = 0;
    bool stop_ = false;
    unsigned char *dst_ = nullptr;
    const unsigned char *src_ = nullptr;
    size_t bytes_ = 0, part_ = 0;
};

constexpr size_t kParallelCopyBytes = 1 << 20;  // smaller pushes copy on the caller's thread

constexpr int kGroups = kTickGroups;
constexpr int kChunk = 2048;
constexpr int kBatch = 2048;
constexpr int kMaxChunksPerStream = 64;
constexpr long long kDeferCap = 65536;  // AT_FRAMES: pending events applied without a frame
constexpr unsigned long long kRingInit = 16384;  // events of a new stream's ring
constexpr int kFusedMaxTiles = 256;  // the fused tick launch serves streams of at most this many tiles
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
    // pending events: a ring in the pinned host pool, read by the device
    // through its mapped address; absolute indices done <= head <= tail:
    // [head, tail) pending, [done, head) read by ticks still in flight
    esi_event *ring_h = nullptr;
    const esi_event *ring_d = nullptr;
    size_t ring_off = 0, ring_bytes = 0;
    unsigned long long ring_cap = 0;  // events, a power of two
    unsigned long long head = 0, tail = 0, done = 0;
    long long last_event_t = 0;
    long long push_floor = 0;
    long long next_frame_t = 0;
    long long watermark = LLONG_MAX;      // events complete up to here
    long long last_push_ns = 0;
    unsigned char *slots_host = nullptr;  // frame_slots * P bytes in the host pool, mapped
    unsigned char *slots_dev = nullptr;
    size_t slots_off = 0, slots_bytes = 0;
    unsigned long long gen = 0;           // which opening of this id (ticks name it)
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
    unsigned long long gen;
    unsigned long long seq;
    long long t_frame;
    long long ref_push_ns;
};

struct TickRec {
    unsigned long long id = 0;
    struct Use {
        int stream;
        unsigned long long gen, upto;  // the ring index it read up to
    };
    std::vector<Use> used;
    long long call_ns = 0, issued_ns = 0;
    std::vector<TickFrame> frames;
    cudaEvent_t evc = nullptr;             // before the copies
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // around the kernels
    long long n_events = 0;
    int n_streams = 0, n_items = 0;
    int stage = 0;
};

constexpr size_t kTraceCap = 65536;  // tick trace records kept

// The pending event at absolute ring index i.
inline const esi_event &ring_at(const Stream &st, unsigned long long i)
{
    return st.ring_h[i & (st.ring_cap - 1)];
}

// How many of the n pending events from the ring's head have t <= t_lim
// (times are non-decreasing).
size_t ring_count_upto(const Stream &st, size_t n, long long t_lim)
{
    size_t lo = 0, hi = n;
    while (lo < hi) {
        const size_t mid = lo + (hi - lo) / 2;
        if (ring_at(st, st.head + mid).t_us <= t_lim) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

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
           off_fout = 0, tab_bytes = 0;
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
    int graph_fused = -1;                 // the graph is the fused launch of variant rd * 3 + dk
    int fused_grid[6] = {0, 0, 0, 0, 0, 0};  // persistent grid per fused variant (0: not yet sized)
    size_t fused_smem = 0;                // its shared memory (0: not yet sized)
    size_t off_sync = 0;
    Completion *comp = nullptr;
    unsigned long long ticks_issued = 0;
    std::vector<TickRec *> inflight;
    std::vector<cudaEvent_t> ev_pool;

    // statistics since the last reset
    std::vector<double> frame_lat, pkt_lat, host_tick, gpu_tick;
    long long last_now = LLONG_MIN;  // the latest tick time
    long long t0_ns = 0;             // creation (trace times are relative to it)
    std::vector<esi_tick_trace> trace;  // ring of kTraceCap records
    size_t trace_n = 0;                  // records written since the reset
    cudaEvent_t prev_end = nullptr;      // the last traced tick's end
    std::string err;  // the last failure, for esi_server_last_error
    unsigned long long dropped = 0;  // events outside their sensor, as last read
    // pinned host pool of the streams' event rings, and rings replaced by
    // larger ones that ticks in flight may still read: freed once the tick
    // count reaches the tag
    unsigned char *hpool = nullptr;
    unsigned char *hpool_d = nullptr;
    Arena harena;
    struct Retired {
        unsigned long long tag;
        size_t off, bytes;
    };
    std::vector<Retired> retired;
    // closed streams whose ticks are still in flight: their frames are still
    // delivered (sinks), their memory is freed once the tick count reaches tag
    struct Zombie {
        unsigned long long tag;
        Stream st;
    };
    std::vector<Zombie> zombies;
    unsigned long long gen_next = 1;
    size_t hpool_peak = 0;
    unsigned long long ring_grows = 0;
    CopyPool copiers;
    unsigned long long n_ticks = 0, n_frames = 0, n_events = 0, n_packets = 0;
    unsigned long long n_admitted = 0, n_refused = 0, n_events_refused = 0;
    double gpu_ms = 0.0;
    unsigned long long gpu_n = 0;
    int launches_per_tick = 0;
};

namespace {

// rc_of, keeping what failed for esi_server_last_error
int cuda_note(esi_server *s, const char *where, cudaError_t e)
{
    if (e != cudaSuccess) s->err = std::string(where) + ": " + cudaGetErrorString(e);
    return rc_of(e);
}

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

// Return a closed stream's device state, ring and frame slots to their arenas.
void free_stream_memory(esi_server *s, Stream &st)
{
    if (st.arena_bytes) s->arena.release(st.arena_off, st.arena_bytes);
    if (st.ring_bytes) s->harena.release(st.ring_off, st.ring_bytes);
    if (st.slots_bytes) s->harena.release(st.slots_off, st.slots_bytes);
    st.arena_bytes = st.ring_bytes = st.slots_bytes = 0;
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
        } else {
            ms = -1.0f;
        }
        esi_tick_trace tr{};
        tr.call_ns = t->call_ns - s->t0_ns;
        tr.issued_ns = t->issued_ns - s->t0_ns;
        tr.ready_ns = ready - s->t0_ns;
        tr.kernels_ms = ms;
        if (cudaEventElapsedTime(&tr.copy_ms, t->evc, t->ev0) != cudaSuccess) tr.copy_ms = -1.0f;
        tr.gap_ms = -1.0f;
        if (s->prev_end && cudaEventElapsedTime(&tr.gap_ms, s->prev_end, t->evc) != cudaSuccess)
            tr.gap_ms = -1.0f;
        tr.frames = (int)t->frames.size();
        tr.events = t->n_events;
        tr.streams = t->n_streams;
        tr.items = t->n_items;
        if (s->trace.size() < kTraceCap) s->trace.push_back(tr);
        else s->trace[s->trace_n % kTraceCap] = tr;
        s->trace_n += 1;
        if (s->prev_end) s->ev_pool.push_back(s->prev_end);
        s->prev_end = t->ev1;
        s->ev_pool.push_back(t->evc);
        s->ev_pool.push_back(t->ev0);
        for (const auto &u : t->used) {
            Stream &st = s->streams[u.stream];
            if (st.open && st.gen == u.gen) st.done = std::max(st.done, u.upto);
        }
        for (const TickFrame &f : t->frames) {
            const double lat = (double)(ready - t->call_ns) * 1e-6;
            s->frame_lat.push_back(lat);
            if (f.ref_push_ns) s->pkt_lat.push_back((double)(ready - f.ref_push_ns) * 1e-6);
            s->n_frames += 1;
            Stream *sp = &s->streams[f.stream];
            if (!sp->open || sp->gen != f.gen) {  // closed since: its zombie, if any
                sp = nullptr;
                for (auto &z : s->zombies)
                    if (z.st.gen == f.gen) sp = &z.st;
                if (!sp) continue;
            }
            Stream &st = *sp;
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
    // rings replaced, and streams closed, while ticks that read them were in flight
    const unsigned long long finished = s->comp->done.load(std::memory_order_acquire);
    size_t w = 0;
    for (size_t i = 0; i < s->retired.size(); ++i) {
        if (s->retired[i].tag <= finished) s->harena.release(s->retired[i].off, s->retired[i].bytes);
        else s->retired[w++] = s->retired[i];
    }
    s->retired.resize(w);
    w = 0;
    for (size_t i = 0; i < s->zombies.size(); ++i) {
        if (s->zombies[i].tag <= finished) free_stream_memory(s, s->zombies[i].st);
        else if (w != i) s->zombies[w++] = std::move(s->zombies[i]);
        else ++w;
    }
    s->zombies.resize(w);
}

void move_ring(esi_server *s, Stream &st, size_t off, unsigned long long cap, unsigned long long tag);

// Room for n more events in stream id's ring: frees the slots of finished
// ticks, waits for ticks in flight that still read slots it needs, or moves
// the pending events into a larger ring (the old one is freed once the ticks
// in flight are done).  ESI_ENOMEM when the host pool is full.
int ring_reserve(esi_server *s, int id, size_t n)
{
    Stream &st = s->streams[id];
    auto fits = [&] { return st.tail - st.done + n <= st.ring_cap; };
    if (fits()) return ESI_OK;
    poll(s);
    if (fits()) return ESI_OK;
    if (st.tail - st.head + n <= st.ring_cap) {
        // the pending events fit: wait for the ticks reading older slots
        while (!fits() && !s->inflight.empty()) {
            cudaError_t e = cudaEventSynchronize(s->inflight.front()->ev1);
            if (e != cudaSuccess) return cuda_note(s, "waiting for a tick", e);
            const unsigned long long before = s->inflight.front()->id;
            poll(s);
            if (!s->inflight.empty() && s->inflight.front()->id == before) {
                // its completion stamp is still being written (bounded)
                const long long t_give_up = wall_ns() + 2000000000ll;
                while (s->comp->done.load(std::memory_order_acquire) <= before) {
                    if (wall_ns() > t_give_up) return ESI_ETIMEOUT;
                }
                poll(s);
            }
        }
        if (!fits()) st.done = st.head;  // no tick in flight reads this ring any more
        return ESI_OK;
    }
    const unsigned long long need = st.tail - st.head + n;
    unsigned long long cap = st.ring_cap;
    while (cap < need + need / 4) cap *= 2;
    const size_t bytes = (size_t)cap * sizeof(esi_event);
    const size_t off = s->harena.alloc(bytes);
    if (off == SIZE_MAX) {
        char m[200];
        std::snprintf(m, sizeof(m),
                      "host pool full: stream %d needs a ring of %llu events (%zu MB); %zu of %zu MB held",
                      id, cap, bytes >> 20, s->harena.used() >> 20, (size_t)s->opts.host_pool_bytes >> 20);
        s->err = m;
        return ESI_ENOMEM;
    }
    s->hpool_peak = std::max(s->hpool_peak, s->harena.used());
    s->ring_grows += 1;
    move_ring(s, st, off, cap, s->inflight.empty() ? 0 : s->ticks_issued);
    return ESI_OK;
}

// Move stream st's pending events into the ring of cap events at pool
// offset off; the old ring is freed now (tag 0) or once the tick count
// reaches tag.
void move_ring(esi_server *s, Stream &st, size_t off, unsigned long long cap, unsigned long long tag)
{
    esi_event *nh = reinterpret_cast<esi_event *>(s->hpool + off);
    for (unsigned long long i = st.head; i < st.tail; ++i) nh[i & (cap - 1)] = ring_at(st, i);
    if (tag == 0) s->harena.release(st.ring_off, st.ring_bytes);
    else s->retired.push_back({tag, st.ring_off, st.ring_bytes});
    st.ring_h = nh;
    st.ring_d = reinterpret_cast<const esi_event *>(s->hpool_d + off);
    st.ring_off = off;
    st.ring_bytes = (size_t)cap * sizeof(esi_event);
    st.ring_cap = cap;
    st.done = st.head;
}

// After a tick took events: a ring grown large for a burst (16 times the
// initial size or more) and now mostly empty goes back to a smaller one (the
// tick being built still reads the old one).  Rings of ordinary size are left
// alone, so steady traffic does not grow and shrink them tick after tick.
void shrink_ring(esi_server *s, Stream &st)
{
    const unsigned long long pending = st.tail - st.head;
    if (st.ring_cap < 16 * kRingInit || pending > st.ring_cap / 16) return;
    unsigned long long cap = 4 * kRingInit;
    while (cap < 4 * pending) cap *= 2;
    if (cap >= st.ring_cap) return;
    const size_t off = s->harena.alloc((size_t)cap * sizeof(esi_event));
    if (off == SIZE_MAX) return;
    move_ring(s, st, off, cap, s->ticks_issued + 1);
}

// Copy n events into a ring: large copies are split over the copy threads.
void copy_events(esi_server *s, esi_event *dst, const esi_event *src, size_t n)
{
    const size_t bytes = n * sizeof(esi_event);
    if (bytes >= kParallelCopyBytes && s->copiers.workers() > 0) s->copiers.copy(dst, src, bytes);
    else std::memcpy(dst, src, bytes);
}

int wait_all(esi_server *s)
{
    cudaError_t e = cudaStreamSynchronize(s->stream);
    // the host-function node may still be finishing its store (bounded: 2 s)
    const long long t_give_up = wall_ns() + 2000000000ll;
    while (e == cudaSuccess && s->comp->done.load(std::memory_order_acquire) < s->ticks_issued) {
        if (wall_ns() > t_give_up) return ESI_ETIMEOUT;
    }
    poll(s);
    if (e != cudaSuccess) return cuda_note(s, "waiting for ticks", e);
    // what the kernels detected (the stream is idle: the status is final)
    DevStatus st{};
    e = cudaMemcpy(&st, s->dstatus, sizeof(DevStatus), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_note(s, "reading the device status", e);
    s->dropped = st.dropped;
    if (st.err) {
        s->err = std::string("device: a bounded wait gave up in ") +
                 (st.err_where == kWhereTickWait ? "a tick's tile items (their stream's binning)"
                                                  : "the binning's chunk copy");
        return st.err;
    }
    return ESI_OK;
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

// The fused tick launch of variant fv = rd * 3 + dk (grid sized once).
cudaError_t launch_fused(esi_server *s, int fv, cudaStream_t cs)
{
    if (!s->fused_grid[fv]) {
        int sms = 0;
        cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
        if (e != cudaSuccess) return e;
        s->fused_grid[fv] = std::max(1, sms) * tick_fused_blocks_per_sm(fv / 3, fv % 3, s->fused_smem);
    }
    return launch_tick_fused(s->dtab, s->fused_grid[fv], fv / 3, fv % 3, s->fused_smem, cs);
}

// Capture the per-tick graph: the fused launch of variant fused (>= 0), or
// for the variant groups in `groups` binning, then the groups' tile
// launches as parallel branches (they touch disjoint streams), joined at the
// end.
int build_graph(esi_server *s, unsigned long long groups, int fused)
{
    if (s->gexec) {
        cudaGraphExecDestroy(s->gexec);
        s->gexec = nullptr;
    }
    if (fused >= 0) groups = 0;
    std::vector<int> gl;
    for (int gi = 0; gi < kGroups; ++gi)
        if (groups & (1ull << gi)) gl.push_back(gi);
    std::vector<cudaStream_t> br(std::max<size_t>(gl.size(), 1), nullptr);
    std::vector<cudaEvent_t> ev(gl.size() + 1, nullptr);
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; i < br.size() && e == cudaSuccess; ++i)
        e = cudaStreamCreateWithFlags(&br[i], cudaStreamNonBlocking);
    for (size_t i = 0; i < ev.size() && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    cudaStream_t cs = br[0];
    cudaGraph_t g = nullptr;
    bool capturing = false;
    if (e == cudaSuccess) {
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        capturing = e == cudaSuccess;
    }
    if (e == cudaSuccess && fused >= 0) e = launch_fused(s, fused, cs);
    if (e == cudaSuccess && fused < 0)
        e = launch_bin_batch_tab(s->dtab, s->bin_grid, kChunk, s->max_tiles, s->bin_mask, cs);
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], cs);  // fork after binning
    for (size_t i = 1; i < gl.size() && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(br[i], ev[0], 0);
    for (size_t i = 0; i < gl.size() && e == cudaSuccess; ++i) e = launch_group(s, gl[i], br[i]);
    for (size_t i = 1; i < gl.size() && e == cudaSuccess; ++i) {  // join
        e = cudaEventRecord(ev[i], br[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev[i], 0);
    }
    if (capturing) {
        cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&s->gexec, g, 0);
    if (g) cudaGraphDestroy(g);
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    for (cudaStream_t x : br)
        if (x) cudaStreamDestroy(x);
    if (e != cudaSuccess) {
        s->gexec = nullptr;
        return cuda_note(s, "tick graph", e);
    }
    s->graph_groups = groups;
    s->graph_fused = fused;
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
    if (!o.apply_mode) o.apply_mode = ESI_APPLY_EVERY_TICK;
    if (!o.host_pool_bytes) o.host_pool_bytes = 512ll << 20;
    if (!o.copy_threads) o.copy_threads = 4;
    if (!o.fuse_tick) o.fuse_tick = 1;
    if (!opts) o.use_graph = 1;
    if (o.frame_period_us < 1 || o.max_events_per_tick < kChunk || o.max_streams < 1 ||
        o.max_streams > 4096 || o.frame_slots < 2 || o.frame_slots > 64 ||
        (o.tile_h != 4 && o.tile_h != 8 && o.tile_h != 16) ||
        o.max_stream_pixels < 1 || o.scan_chain < 1 || o.scan_chain > kScanNever ||
        (o.apply_mode != ESI_APPLY_EVERY_TICK && o.apply_mode != ESI_APPLY_AT_FRAMES) ||
        o.copy_threads < 1 || o.copy_threads > 16 || o.fuse_tick < 1 || o.fuse_tick > 2 ||
        o._reserved != 0 ||
        o.host_pool_bytes < (long long)(kRingInit * sizeof(esi_event)) ||
        state_budget_bytes == 0)
        return ESI_EINVAL;
    esi_server *s = new (std::nothrow) esi_server();
    if (!s) return ESI_ENOMEM;
    s->opts = o;
    s->t0_ns = wall_ns();
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
    s->off_sync = off;
    off = align_up(off + sizeof(unsigned) * (size_t)(s->cap_jobs + 1), 256);
    s->off_items = off;
    off = align_up(off + sizeof(int2) * (size_t)s->cap_items, 256);
    s->tab_bytes = off;
    // each stream's run table starts on a 128-byte line of its own
    s->hrow_cap = (size_t)s->cap_chunks * (size_t)s->max_tiles + (size_t)s->cap_jobs * 32;
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
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&s->hpool, (size_t)o.host_pool_bytes, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&s->hpool_d, s->hpool, 0);
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
    s->harena.init((size_t)o.host_pool_bytes);
    if (o.copy_threads > 1 && !s->copiers.start(o.copy_threads - 1)) {
        esi_server_destroy(s);
        return ESI_ENOMEM;
    }
    *out = s;
    return ESI_OK;
}

void esi_server_destroy(esi_server *s)
{
    if (!s) return;
    cudaError_t e = cudaSuccess;
    if (s->stream) e = cudaStreamSynchronize(s->stream);
    bool comp_idle = true;
    if (s->comp) {
        const long long t_give_up = wall_ns() + 2000000000ll;
        while (e == cudaSuccess && s->comp->done.load(std::memory_order_acquire) < s->ticks_issued &&
               wall_ns() < t_give_up) {
        }
        comp_idle = e == cudaSuccess && s->comp->done.load(std::memory_order_acquire) >= s->ticks_issued;
    }
    for (TickRec *t : s->inflight) {
        cudaEventDestroy(t->evc);
        cudaEventDestroy(t->ev0);
        cudaEventDestroy(t->ev1);
        delete t;
    }
    if (s->prev_end) cudaEventDestroy(s->prev_end);
    for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
    if (s->gexec) cudaGraphExecDestroy(s->gexec);
    for (int b = 0; b < 2; ++b) {
        if (s->stage[b]) cudaFreeHost(s->stage[b]);
        if (s->stage_ev[b]) cudaEventDestroy(s->stage_ev[b]);
    }
    if (s->hpool) cudaFreeHost(s->hpool);
    cudaFree(s->arena_base);
    cudaFree(s->dtab);
    cudaFree(s->rec);
    cudaFree(s->hrow);
    cudaFree(s->dstatus);
    // a completion stamp that may still run keeps its target (leaked)
    if (comp_idle) delete s->comp;
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
    const size_t rbytes = kRingInit * sizeof(esi_event);
    const size_t fbytes = (size_t)s->opts.frame_slots * (size_t)P;
    // memory of closed streams whose ticks are in flight comes back once
    // they finish: wait for them before refusing
    auto fits = [&] {
        const size_t a = s->arena.alloc(sbytes);
        if (a == SIZE_MAX) return false;
        s->arena.release(a, sbytes);
        const size_t r = s->harena.alloc(rbytes), f = s->harena.alloc(fbytes);
        if (r != SIZE_MAX) s->harena.release(r, rbytes);
        if (f != SIZE_MAX) s->harena.release(f, fbytes);
        return r != SIZE_MAX && f != SIZE_MAX;
    };
    poll(s);
    if (!fits() && (!s->zombies.empty() || !s->retired.empty())) {
        rc = wait_all(s);
        if (rc) return rc;
    }
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
    // its event ring and frame slots come from the pinned host pool
    const size_t roff = s->harena.alloc(rbytes);
    const size_t foff = roff == SIZE_MAX ? SIZE_MAX : s->harena.alloc(fbytes);
    if (foff == SIZE_MAX) {  // no room for its events or frames: refused like a full budget
        s->arena.release(off, sbytes);
        if (roff != SIZE_MAX) s->harena.release(roff, rbytes);
        st = Stream();
        s->n_refused += 1;
        return ESI_EBUSY;
    }
    s->hpool_peak = std::max(s->hpool_peak, s->harena.used());
    st.ring_off = roff;
    st.ring_bytes = rbytes;
    st.ring_cap = kRingInit;
    st.ring_h = reinterpret_cast<esi_event *>(s->hpool + roff);
    st.ring_d = reinterpret_cast<const esi_event *>(s->hpool_d + roff);
    st.slots_off = foff;
    st.slots_bytes = fbytes;
    st.slots_host = s->hpool + foff;
    st.slots_dev = s->hpool_d + foff;
    std::memset(st.slots_host, 0, fbytes);
    // Alg. 2 initialisation: S = 0, T = t_origin
    cudaError_t e = cudaMemsetAsync(st.S, 0, (size_t)P * 4, s->stream);
    if (e == cudaSuccess) e = launch_fill_i64(st.T, P, params->t_origin_us, s->stream);
    if (e != cudaSuccess) {
        free_stream_memory(s, st);
        st = Stream();
        return cuda_note(s, "stream open", e);
    }
    st.gen = s->gen_next++;
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
    int rc = ring_reserve(s, id, n);
    if (rc) return rc;
    // copy into the ring (two pieces where it wraps)
    const unsigned long long mask = st.ring_cap - 1;
    const size_t i0 = (size_t)(st.tail & mask);
    const size_t n1 = std::min(n, (size_t)(st.ring_cap - i0));
    copy_events(s, st.ring_h + i0, ev, n1);
    if (n1 < n) copy_events(s, st.ring_h, ev + n1, n - n1);
    st.tail += n;
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

namespace {

constexpr int kFlushNone = -1;  // tick_impl: apply as apply_mode says
constexpr int kFlushAll = -2;   // tick_impl: apply every stream's events

// One tick (esi_server_tick).  flush: kFlushNone, kFlushAll or a stream id
// whose events are applied whatever apply_mode says.
int tick_impl(esi_server *s, long long now_us, int flush)
{
    const long long call_ns = wall_ns();
    s->last_now = std::max(s->last_now, now_us);
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
        // every tick applies what has arrived (EVERY_TICK), so a frame's tick
        // only has the newest events left to do; or the events wait for the
        // frame's tick (AT_FRAMES), unless so many are pending that the
        // frame's tick could not take them all
        const size_t avail = (size_t)(st.tail - st.head);
        if (fr.empty() && avail == 0) continue;
        if (fr.empty() && s->opts.apply_mode == ESI_APPLY_AT_FRAMES && avail < (size_t)kDeferCap &&
            flush != kFlushAll && flush != id)
            continue;
        // events: t <= now, or <= the last frame when frames wait for the next tick
        long long lim_t = upto;
        if (tf <= upto) lim_t = fr.empty() ? st.push_floor : fr.back();
        size_t take = ring_count_upto(st, avail, lim_t);
        take = std::min(take, (size_t)ev_cap_stream);
        if (n_ev + (long long)take > s->cap_events) take = (size_t)std::max<long long>(0, s->cap_events - n_ev);
        if (take > 0 && take < avail) {
            // frames after an event left for later must wait too
            const long long t_left = ring_at(st, st.head + take).t_us;
            while (!fr.empty() && fr.back() >= t_left) fr.pop_back();
        }
        if (take > 0) {
            // record times are 32-bit offsets from the first event
            const long long lim = ring_at(st, st.head).t_us + 0xffffffffll;
            const size_t ok = ring_count_upto(st, take, lim);
            if (ok < take) {
                take = ok;
                const long long t_left = ring_at(st, st.head + take).t_us;
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
        const long long t_base = take ? ring_at(st, st.head).t_us : fr.front();
        // binning job: the device reads the events from the stream's ring
        BinJob &B = bj[j];
        B.args.ring = st.ring_d;
        B.args.ring_mask = st.ring_cap - 1;
        B.args.first = st.head;
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
            rec->frames.push_back({id, st.gen, seq, fr[w], st.last_push_ns});
        }
        job_stream.push_back({j, id});
        st.seq_issued += fr.size();
        if (!fr.empty()) st.next_frame_t = fr.back() + s->opts.frame_period_us;
        st.head += take;
        if (take) {
            rec->used.push_back({id, st.gen, st.head});
            shrink_ring(s, st);
        }
        if (!fr.empty()) st.push_floor = std::max(st.push_floor, fr.back());
        n_ev += (long long)take;
        n_chunks += chunks;
        n_frames += (int)fr.size();
        hrow_off = (hrow_off + (size_t)chunks * st.n_tiles + 31) & ~(size_t)31;
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
    // one fused launch when every group of the tick has 8-row tiles and the
    // same render mode and decay kind (the two row alignments of one
    // variant are adjacent groups, so their items form one run), and no
    // stream has more than kFusedMaxTiles tiles: the binning's per-tile
    // counters then leave the fused blocks as many per SM as the separate
    // launches get (with 900-tile streams the fused launch was measured
    // slower than binning plus tile launches)
    int fused = -1;
    if (s->opts.fuse_tick == 1 && groups) {
        const int g0 = __builtin_ctzll(groups) & ~1;
        int maxt = 0;
        for (auto &js : job_stream) maxt = std::max(maxt, s->streams[js.second].n_tiles);
        if (group_tile_h(g0) == 8 && (groups & ~(3ull << g0)) == 0 && maxt <= kFusedMaxTiles) {
            fused = group_rd(g0) * 3 + group_dk(g0);
            const int gf = (groups >> g0) & 1ull ? g0 : g0 + 1;
            dir->fused_off_items = dir->off_items[gf];
            dir->fused_n_items = dir->n_items[g0] + dir->n_items[g0 + 1];
            if (!s->fused_smem) {
                s->fused_smem = tick_fused_smem_bytes(kChunk, std::min(kFusedMaxTiles, s->max_tiles),
                                                      s->bin_mask, kBatch, kMaxChunksPerStream);
                s->graph_fused = -1;
            }
        }
    }
    dir->off_sync = (long long)s->off_sync;
    std::memset(stg + s->off_sync, 0, sizeof(unsigned) * (size_t)(n_jobs + 1));

    // a tick that fails to queue returns its events to the pool
    auto drop = [&](int rc) {
        for (cudaEvent_t ev : {rec->evc, rec->ev0, rec->ev1})
            if (ev) s->ev_pool.push_back(ev);
        delete rec;
        return rc;
    };
    // the table to the device (the kernels read the events from the
    // streams' rings); tick kernels; completion stamp
    rec->evc = take_event(s);
    cudaError_t e = cudaEventRecord(rec->evc, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->dtab, stg, s->off_items + (size_t)item_off * sizeof(int2),
                            cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaEventRecord(s->stage_ev[b], s->stream);
    if (e != cudaSuccess) return drop(cuda_note(s, "tick", e));
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
            const bool stale = fused >= 0 ? s->graph_fused != fused
                                          : s->graph_fused >= 0 || (groups & ~s->graph_groups);
            if (!s->gexec || stale) {
                int rc = build_graph(s, fused >= 0 ? 0ull : groups | (s->graph_fused >= 0 ? 0ull : s->graph_groups),
                                     fused);
                if (rc) return drop(rc);
            }
            e = cudaGraphLaunch(s->gexec, s->stream);
            int ng = 0;
            for (int g = 0; g < kGroups; ++g) ng += (int)((s->graph_groups >> g) & 1ull);
            s->launches_per_tick = fused >= 0 ? 1 : 1 + ng;
        } else if (fused >= 0) {
            e = launch_fused(s, fused, s->stream);
            s->launches_per_tick = 1;
        } else {
            e = launch_bin_batch_tab(s->dtab, s->bin_grid, kChunk, s->max_tiles, s->bin_mask, s->stream);
            for (int g = 0; g < kGroups && e == cudaSuccess; ++g)
                if (groups & (1ull << g)) e = launch_group(s, g, s->stream);
            s->launches_per_tick = 1 + ngroups;
        }
    }
    // the kernels' end, then the completion stamp: when the stamp is in, the
    // event is complete too
    if (e == cudaSuccess) e = cudaEventRecord(rec->ev1, s->stream);
    if (e == cudaSuccess) e = cudaLaunchHostFunc(s->stream, on_tick_done, s->comp);
    if (e != cudaSuccess) return drop(cuda_note(s, "tick", e));
    s->ticks_issued += 1;
    rec->n_events = n_ev;
    rec->n_streams = n_jobs;
    rec->n_items = (int)item_off;
    rec->issued_ns = wall_ns();
    s->inflight.push_back(rec);
    s->n_ticks += 1;
    s->n_events += (unsigned long long)n_ev;
    s->host_tick.push_back((double)(rec->issued_ns - call_ns) * 1e-6);
    return ESI_OK;
}

// Apply the pending events of stream `which` (kFlushAll: every stream) up
// to the last tick's time, then wait for every queued tick.  Bounded: a tick
// may be full and leave events for the next one.
int flush_events(esi_server *s, int which)
{
    for (int guard = 0; guard < 4096; ++guard) {
        bool left = false;
        for (int id = 0; id < (int)s->streams.size() && !left; ++id) {
            const Stream &st = s->streams[id];
            if (!st.open || (which != kFlushAll && id != which) || st.head == st.tail) continue;
            const long long upto = std::min(s->last_now, st.watermark);
            left = ring_at(st, st.head).t_us <= upto;
        }
        if (!left) return wait_all(s);
        if (!s->inflight.empty()) {
            cudaError_t e = cudaEventSynchronize(s->inflight.front()->ev1);
            if (e != cudaSuccess) return rc_of(e);
        }
        int rc = tick_impl(s, s->last_now, which);
        if (rc) return rc;
    }
    return ESI_ERANGE;
}

}  // namespace

int esi_server_tick(esi_server *s, int64_t now_us)
{
    if (!s) return ESI_EINVAL;
    return tick_impl(s, now_us, kFlushNone);
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
    int rc = flush_events(s, id);
    if (rc) return rc;
    Stream &st = s->streams[id];
    cudaError_t e = cudaMemcpy(S, st.S, (size_t)st.P * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(T, st.T, (size_t)st.P * 8, cudaMemcpyDeviceToHost);
    return rc_of(e);
}

int esi_stream_close(esi_server *s, int id)
{
    if (!s || id < 0 || id >= (int)s->streams.size() || !s->streams[id].open) return ESI_EINVAL;
    poll(s);
    Stream &st = s->streams[id];
    s->used -= st.arena_bytes;
    st.open = false;
    if (s->inflight.empty()) {
        free_stream_memory(s, st);
    } else {
        // ticks in flight may still touch its state or deliver its frames:
        // it lives on until they finish, and the id is free meanwhile
        s->zombies.push_back({s->ticks_issued, std::move(st)});
    }
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
    out->host_pool_bytes = (uint64_t)s->opts.host_pool_bytes;
    out->host_pool_used_bytes = s->harena.used();
    out->host_pool_peak_bytes = s->hpool_peak;
    out->ring_grows = s->ring_grows;
    out->events_dropped = s->dropped;
    return ESI_OK;
}

int esi_server_trace(esi_server *s, esi_tick_trace *out, size_t cap, size_t *n)
{
    if (!s || !n || (cap && !out)) return ESI_EINVAL;
    poll(s);
    const size_t have = s->trace.size();
    const size_t k = std::min(cap, have);
    // oldest first: once the ring wrapped, its oldest record sits at trace_n % kTraceCap
    const size_t first = have < kTraceCap ? 0 : s->trace_n % kTraceCap;
    for (size_t i = 0; i < k; ++i) out[i] = s->trace[(first + (have - k) + i) % have];
    *n = cap ? k : have;
    return ESI_OK;
}

const char *esi_server_last_error(esi_server *s)
{
    return s ? s->err.c_str() : "";
}

int esi_server_reset_stats(esi_server *s)
{
    if (!s) return ESI_EINVAL;
    poll(s);
    s->frame_lat.clear();
    s->pkt_lat.clear();
    s->host_tick.clear();
    s->gpu_tick.clear();
    s->trace.clear();
    s->trace_n = 0;
    s->n_ticks = s->n_frames = s->n_events = s->n_packets = 0;
    s->n_admitted = s->n_refused = s->n_events_refused = 0;
    s->gpu_ms = 0.0;
    s->gpu_n = 0;
    s->hpool_peak = s->harena.used();
    s->ring_grows = 0;
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
    s->err.clear();
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
        // a packet that makes its stream's frame due is rendered before the
        // packets queued behind it are taken (the watermarks of their
        // streams keep their events and frames out of that tick)
        bool early = false;
        for (; i < n && pk[i].arrival_us <= now && !early; ++i) {
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
                    early = !rc && realtime && now < t_end_us && now - last_tick >= min_gap &&
                            frames_due(s->streams[id], now);
                }
            }
            if (rc) {
                char m[160];
                std::snprintf(m, sizeof(m), "packet %zu (slot %d, kind %d, %llu events, arrival %lld us, now %lld us): ",
                              i, q.stream, q.kind, (unsigned long long)q.n, (long long)q.arrival_us, now);
                s->err = m + (s->err.empty() ? std::string(esi_strerror(rc)) : s->err);
                return rc;
            }
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
