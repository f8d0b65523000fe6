// Host side of the ESI C ABI (esi.h): handle life cycle, the pending-event
// ring, render planning (sub-batches, frame ranges) and the kernel launches.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "esi_api_impl.h"

using namespace esi;

namespace esi {

int cuda_fail(esi_handle *h, cudaError_t e)
{
    if (e == cudaSuccess) return ESI_OK;
    if (h) h->cuda_msg = cudaGetErrorString(e);
    return (e == cudaErrorMemoryAllocation) ? ESI_ENOMEM : ESI_ECUDA;
}

long long decay_cutoff(double k_per_s)
{
    if (!(k_per_s > 0.0)) return LLONG_MAX;
    const double kus = k_per_s * 1e-6;
    const double x = 1.0 / kus;
    if (!(x < 9.0e18)) return LLONG_MAX;
    long long c = (long long)std::floor(x) - 2;
    if (c < 0) c = 0;
    // smallest dt with 1 - kus * dt <= 0, evaluated in double as Eq. 4 is
    while (!(1.0 - kus * (double)c <= 0.0)) ++c;
    while (c > 0 && 1.0 - kus * (double)(c - 1) <= 0.0) --c;
    return c;
}

// Smallest dt with k dt >= 110 (exp(-110) is below FP32's smallest
// subnormal): Eq. 3's exponential decay is 0 from there on.
long long exp_cutoff(double k_per_s)
{
    if (!(k_per_s > 0.0)) return LLONG_MAX;
    const double x = std::ceil(110.0 / (k_per_s * 1e-6));
    return x < 9.0e18 ? (long long)x : LLONG_MAX;
}

int validate_params(int W, int H, const esi_params *p)
{
    if (!p) return ESI_EINVAL;
    if (W < 1 || H < 1 || W > 65535 || H > 65535) return ESI_EINVAL;
    if (!std::isfinite(p->C) || !(p->C > 0.0)) return ESI_EINVAL;
    if (!std::isfinite(p->k_per_s) || p->k_per_s < 0.0 || p->k_per_s > 1e12) return ESI_EINVAL;
    if (p->method < ESI_METHOD_ALG2 || p->method > ESI_METHOD_EQ3_EXP) return ESI_EINVAL;
    if (p->method != ESI_METHOD_EQ3_EXP && (!std::isfinite(p->b) || !(p->b > 0.0))) return ESI_EINVAL;
    if (!std::isfinite(p->s_min) || !std::isfinite(p->s_max)) return ESI_EINVAL;
    if (!((float)p->s_min < (float)p->s_max)) return ESI_EINVAL;
    if (!std::isfinite(p->s_max - p->s_min)) return ESI_EINVAL;
    if (p->render_decay != 0 && p->render_decay != 1) return ESI_EINVAL;
    return ESI_OK;
}

void prepare_params(const esi_params &p, DecayParams *dp, MapParams *mp)
{
    const double kus = p.k_per_s * 1e-6;
    dp->k_hi = (float)kus;
    dp->k_lo = (float)(kus - (double)dp->k_hi);
    dp->b = (float)p.b;
    dp->cutoff = decay_cutoff(p.k_per_s);
    if (p.k_per_s == 0.0) dp->b_mode = 4;
    else if (p.method == ESI_METHOD_EQ3_EXP) {
        dp->b_mode = kBModeExp;
        dp->b = 1.0f;
        dp->cutoff = exp_cutoff(p.k_per_s);
    }
    else if (p.b == 1.0) dp->b_mode = 1;
    else if (p.b == 2.0) dp->b_mode = 2;
    else if (p.b == 3.0) dp->b_mode = 3;
    else dp->b_mode = 0;
    mp->C = (float)p.C;
    // only Alg. 2 clamps the state; the map of Eq. 14 saturates for all
    mp->s_min = p.method == ESI_METHOD_ALG2 ? (float)p.s_min : -INFINITY;
    mp->s_max = p.method == ESI_METHOD_ALG2 ? (float)p.s_max : INFINITY;
    const double sc = 255.0 / (p.s_max - p.s_min);
    mp->scale = (float)sc;
    mp->offs = (float)(-p.s_min * sc);
    mp->render_decay = p.render_decay;
}

int validate_tuning(const esi_tuning &t)
{
    auto pow2 = [](int v) { return v > 0 && (v & (v - 1)) == 0; };
    if (t.tile_w == 128 || t.tile_w == 64) {
        if (t.tile_h != 4 && t.tile_h != 8 && t.tile_h != 16) return ESI_EINVAL;
    } else if (t.tile_w == 32) {
        if (t.tile_h != 16 && t.tile_h != 32) return ESI_EINVAL;
    } else {
        return ESI_EINVAL;
    }
    if (!pow2(t.chunk_events) || t.chunk_events < 512 || t.chunk_events > 8192) return ESI_EINVAL;
    if (!pow2(t.batch_records) || t.batch_records < 1024 || t.batch_records > 8192) return ESI_EINVAL;
    if (t.max_batch_events < t.chunk_events) return ESI_EINVAL;
    if (t.scan_chain < 1 || t.scan_chain > kScanNever) return ESI_EINVAL;
    if (t.split_rows < 1 || t.split_rows > 3) return ESI_EINVAL;
    return ESI_OK;
}

esi_tuning default_tuning(int W, int H)
{
    esi_tuning t;
    // small sensors: 64-pixel rows give twice the row walks (346x260: 198
    // tiles instead of 99 on 152 SMs); larger ones keep 128-pixel rows
    t.tile_w = (long long)W * H < 160000 ? 64 : 128;
    t.tile_h = 8;
    // large sensors: fewer, longer runs per tile and smaller sort batches
    // (1280x720: the autotuner's choice, 22.0 -> 25.0 G events/s)
    const bool large = (long long)W * H >= 600000;
    t.chunk_events = large ? 4096 : 2048;
    t.batch_records = large ? 2048 : 4096;
    t.max_batch_events = 1 << 22;
    t.scan_chain = kScanChainDefault;
    // one warp per row, batch by batch: the split-row kernel is measured
    // slower on the synthetic workloads (it executes about half as many
    // instructions again as the batch walk per record)
    t.split_rows = 2;
    return t;
}

}  // namespace esi

// ------------------------------------------------------------ handle helpers
static int apply_tuning(esi_handle *h, const esi_tuning &t)
{
    h->tun = t;
    h->tiles_x = (h->W + t.tile_w - 1) / t.tile_w;
    h->tiles_y = (h->H + t.tile_h - 1) / t.tile_h;
    h->n_tiles = h->tiles_x * h->tiles_y;
    int th_log2 = 0;
    while ((1 << th_log2) < t.tile_h) ++th_log2;
    h->th_log2 = th_log2;
    h->tw_log2 = t.tile_w == 32 ? 5 : t.tile_w == 64 ? 6 : 7;
    // the binning kernel keeps per-warp counters for every tile in shared memory
    if (bin_smem_bytes(t.chunk_events, h->n_tiles, false) + 1024 > (size_t)kMaxSmemPerBlock) return ESI_ERANGE;
    const int max_chunks = (t.max_batch_events + t.chunk_events - 1) / t.chunk_events;
    if (tile_smem_bytes(t.tile_h, t.batch_records, max_chunks) + tile_static_smem_bytes(t.tile_h, t.tile_w) >
        (size_t)kMaxSmemPerBlock)
        return ESI_ERANGE;
    // the split-row kernel keeps more per row and per batch in shared memory
    h->split = t.tile_w == 128 && t.split_rows != 2 &&
               tile_smem_bytes(t.tile_h, t.batch_records, max_chunks) +
                       tile_split_static_smem_bytes(t.tile_h) <= (size_t)kMaxSmemPerBlock;
    return ESI_OK;
}

int esi::sync_all(esi_handle *h)
{
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess && h->bin_stream) e = cudaStreamSynchronize(h->bin_stream);
    if (e == cudaSuccess && h->tile_stream) e = cudaStreamSynchronize(h->tile_stream);
    return cuda_fail(h, e);
}

template <class T>
static int ensure_pinned(esi_handle *h, T **p, size_t *cap, size_t need)
{
    if (need <= *cap) return ESI_OK;
    size_t nc = std::max(need, *cap * 2);
    if (*p) {
        int rc = sync_all(h);
        if (rc) return rc;
        cudaFreeHost(*p);
        *p = nullptr;
        *cap = 0;
    }
    cudaError_t e = cudaMallocHost((void **)p, nc * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(h, e);
    *cap = nc;
    return ESI_OK;
}

// Grow the pending ring so that it holds `need` events; pending events keep
// their absolute indices (position = index & (cap - 1)).
static int ensure_ring(esi_handle *h, unsigned long long need)
{
    if (need <= h->cap) return ESI_OK;
    unsigned long long nc = h->cap ? h->cap : (1ull << 20);
    while (nc < need) nc <<= 1;
    esi_event *nr = nullptr;
    cudaError_t e = cudaMalloc((void **)&nr, nc * sizeof(esi_event));
    if (e != cudaSuccess) return cuda_fail(h, e);
    // the full time mirror (8 B per slot) exists only once a small host push
    // has used it (esi_push_events allocates it then)
    long long *nm = nullptr, *ns = nullptr;
    if (h->tmirror) e = cudaMallocHost((void **)&nm, nc * sizeof(long long));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&ns, nc / kSparse * sizeof(long long));
    if (e != cudaSuccess) {
        cudaFree(nr);
        cudaFreeHost(nm);
        return cuda_fail(h, e);
    }
    const unsigned long long om = h->cap ? h->cap - 1 : 0, nmk = nc - 1;
    for (unsigned long long a = h->head; a < h->tail;) {
        const unsigned long long po = a & om, pn = a & nmk;
        const unsigned long long len = std::min({h->tail - a, h->cap - po, nc - pn});
        e = cudaMemcpyAsync(nr + pn, h->ring + po, len * sizeof(esi_event),
                            cudaMemcpyDeviceToDevice, h->stream);
        if (e != cudaSuccess) {
            cudaFree(nr);
            cudaFreeHost(nm);
            cudaFreeHost(ns);
            return cuda_fail(h, e);
        }
        if (nm) std::memcpy(&nm[pn], &h->tmirror[po], len * sizeof(long long));
        a += len;
    }
    // the sparse times of the pending events (and of the block holding head)
    const unsigned long long g_from = h->head / kSparse * kSparse;
    if (h->cap)
        for (unsigned long long g = std::max(g_from, h->sparse_from); g < h->tail; g += kSparse)
            ns[(g / kSparse) & (nc / kSparse - 1)] = h->tsparse[(g / kSparse) & (h->cap / kSparse - 1)];
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        cudaFree(nr);
        cudaFreeHost(nm);
        cudaFreeHost(ns);
        return cuda_fail(h, e);
    }
    if (h->ring) cudaFree(h->ring);
    if (h->tmirror) cudaFreeHost(h->tmirror);
    if (h->tsparse) cudaFreeHost(h->tsparse);
    if (h->ring) h->ring_grows += 1;
    h->ring = nr;
    h->cap = nc;
    h->tmirror = nm;
    h->tsparse = ns;
    h->sparse_from = std::max(g_from, h->sparse_from);
    return ESI_OK;
}

// Checks that ev[0..n) is non-decreasing in time and not earlier than prev,
// and writes the times into the host mirrors at ring positions tail .. tail+n
// (pushes of at most kHostCheckMax events).
static bool check_and_mirror(esi_handle *h, const esi_event *ev, size_t n, long long prev)
{
    const unsigned long long mask = h->cap - 1, tail = h->tail;
    long long *mir = h->tmirror;
    bool ok = true;
    long long last = prev;
    for (size_t i = 0; i < n; ++i) {
        const long long t = ev[i].t_us;
        ok &= t >= last;
        last = t;
        mir[(tail + i) & mask] = t;
    }
    const unsigned long long smask = h->cap / kSparse - 1;
    for (unsigned long long g = (tail + kSparse - 1) / kSparse * kSparse; g < tail + n; g += kSparse)
        h->tsparse[(g / kSparse) & smask] = ev[g - tail].t_us;
    return ok;
}

// ------------------------------------------------ times for planning
// Is the sparse time of absolute index g (a multiple of kSparse) held?
static bool sparse_ok(const esi_handle *h, unsigned long long g)
{
    return g >= h->sparse_from && g < h->tail && g + h->cap >= h->tail;
}

static long long sparse_t(const esi_handle *h, unsigned long long g)
{
    return h->tsparse[(g / kSparse) & (h->cap / kSparse - 1)];
}

// Exact times of pending indices [a0, a1) (at most 2 kSparse of them) into
// out: from the mirror when host pushes checked all of them, otherwise read
// back from the ring (a short copy on the auxiliary stream).
static int block_times(esi_handle *h, unsigned long long a0, unsigned long long a1, long long *out)
{
    if (a1 <= a0) return ESI_OK;
    bool exact = false;
    for (const auto &sp : h->exact_spans)
        if (sp.first <= a0 && a1 <= sp.second) exact = true;
    const unsigned long long mask = h->cap - 1;
    if (exact) {
        for (unsigned long long a = a0; a < a1; ++a) out[a - a0] = h->tmirror[a & mask];
        return ESI_OK;
    }
    cudaError_t e = cudaSuccess;
    for (unsigned long long a = a0; e == cudaSuccess && a < a1;) {
        const unsigned long long pos = a & mask;
        const unsigned long long len = std::min(a1 - a, h->cap - pos);
        e = cudaMemcpyAsync(h->hfetch + (a - a0), h->ring + pos, len * sizeof(esi_event),
                            cudaMemcpyDeviceToHost, h->aux_stream);
        a += len;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->aux_stream);
    if (e != cudaSuccess) return cuda_fail(h, e);
    for (unsigned long long a = a0; a < a1; ++a) out[a - a0] = h->hfetch[a - a0].t_us;
    return ESI_OK;
}

static int exact_t(esi_handle *h, unsigned long long a, long long *t)
{
    return block_times(h, a, a + 1, t);
}

// A time <= that of pending index a, no earlier than it by 2^31 us or more
// (the sparse time of its block, or the exact one).
static int lower_t(esi_handle *h, unsigned long long a, long long *t)
{
    const unsigned long long g = a / kSparse * kSparse, g2 = g + kSparse;
    if (g == a && sparse_ok(h, g)) {
        *t = sparse_t(h, g);
        return ESI_OK;
    }
    if (sparse_ok(h, g) && sparse_ok(h, g2) && sparse_t(h, g2) - sparse_t(h, g) < (1ll << 31)) {
        *t = sparse_t(h, g);
        return ESI_OK;
    }
    return exact_t(h, a, t);
}

// First absolute index in [lo, hi) (pending indices) whose time is > v
// (times non-decreasing): a search over the sparse times, then one block of
// at most kSparse - 1 exact times.
static int upper_bound_t(esi_handle *h, unsigned long long lo, unsigned long long hi, long long v,
                         unsigned long long *res)
{
    // no pending time exceeds the last pushed one: nothing to read back
    if (h->last_event_t <= v) {
        *res = hi;
        return ESI_OK;
    }
    unsigned long long blo = lo, bhi = hi;
    const unsigned long long G0 = (lo + kSparse - 1) / kSparse * kSparse;
    if (G0 < hi) {
        const unsigned long long nG = (hi - 1 - G0) / kSparse + 1;
        unsigned long long L = 0, R = nG;
        while (L < R) {
            const unsigned long long mid = L + (R - L) / 2;
            if (sparse_t(h, G0 + mid * kSparse) <= v) L = mid + 1; else R = mid;
        }
        // every index before G0 + L kSparse - ... : the answer lies in
        // (G0 + (L - 1) kSparse, G0 + L kSparse]
        blo = L == 0 ? lo : G0 + (L - 1) * kSparse + 1;
        bhi = L < nG ? G0 + L * kSparse : hi;
    }
    long long t[kSparse];
    int rc = block_times(h, blo, bhi, t);
    if (rc) return rc;
    unsigned long long a = blo;
    while (a < bhi && t[a - blo] <= v) ++a;
    *res = a;
    return ESI_OK;
}

int esi::read_status(esi_handle *h)
{
    cudaError_t e = cudaMemcpyAsync(h->hstatus, h->dstatus, sizeof(DevStatus),
                                    cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e);
    h->dropped = h->hstatus->dropped;
    if (h->hstatus->err) return h->hstatus->err;
    return ESI_OK;
}

static cudaEvent_t prof_event(esi_handle *h)
{
    if (!h->ev_pool.empty()) {
        cudaEvent_t e = h->ev_pool.back();
        h->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

int esi::prof_begin(esi_handle *h, cudaEvent_t *ev, cudaStream_t s)
{
    *ev = nullptr;
    if (!h->prof_on) return ESI_OK;
    *ev = prof_event(h);
    return cuda_fail(h, cudaEventRecord(*ev, s));
}

int esi::prof_end(esi_handle *h, int kind, cudaEvent_t start, cudaStream_t s)
{
    h->launches += 1;
    if (!h->prof_on || !start) return ESI_OK;
    cudaEvent_t stop = prof_event(h);
    cudaError_t e = cudaEventRecord(stop, s);
    h->prof_recs.push_back({kind, start, stop});
    return cuda_fail(h, e);
}

// ----------------------------------------------------------------- C ABI
extern "C" {

const char *esi_strerror(int code)
{
    switch (code) {
    case ESI_OK: return "ok";
    case ESI_EINVAL: return "invalid argument";
    case ESI_ENOMEM: return "out of memory";
    case ESI_EBUSY: return "busy: admission refused";
    case ESI_ETIMEORDER: return "time goes backwards";
    case ESI_ERANGE: return "value out of range for the layout";
    case ESI_ECUDA: return "CUDA runtime error";
    case ESI_ETIMEOUT: return "bounded device wait timed out";
    case ESI_ESTATE: return "call not valid in this state";
    default: return "unknown error";
    }
}

int esi_create(int width, int height, const esi_params *params, void *cuda_stream,
               esi_handle **out)
{
    if (!out) return ESI_EINVAL;
    *out = nullptr;
    int rc = validate_params(width, height, params);
    if (rc) return rc;
    esi_handle *h = new (std::nothrow) esi_handle();
    if (!h) return ESI_ENOMEM;
    h->W = width;
    h->H = height;
    h->P = (long long)width * height;
    h->prm = *params;
    prepare_params(*params, &h->dp, &h->mp);
    h->push_floor = params->t_origin_us;
    h->frame_floor = params->t_origin_us;
    h->last_event_t = params->t_origin_us;
    h->last_frame_t = params->t_origin_us;
    // the default shape, or for large sensors (too many tiles for the
    // binning's per-tile counters) taller tiles and smaller chunks
    rc = apply_tuning(h, default_tuning(width, height));
    for (int chunk : {2048, 1024, 512}) {
        if (rc != ESI_ERANGE) break;
        esi_tuning t = default_tuning(width, height);
        t.tile_w = 128;
        t.tile_h = 16;
        t.chunk_events = chunk;
        t.batch_records = 2048;
        rc = apply_tuning(h, t);
    }
    if (rc) {
        delete h;
        return rc;
    }
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = set_kernel_attributes();
    if (e == cudaSuccess) {
        if (cuda_stream) {
            h->stream = (cudaStream_t)cuda_stream;
        } else {
            e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
            h->own_stream = (e == cudaSuccess);
        }
    }
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->S, (size_t)h->P * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->T, (size_t)h->P * sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->dstatus, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&h->hstatus, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->hwin_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->bin_stream, cudaStreamNonBlocking);
    // block priorities: a push's short check (or unpack) kernels first, so a
    // push overlapping a render does not wait for the render's queued blocks;
    // then the tile kernel; the binning of the next sub-batch last
    int least = 0, greatest = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    const int tile_prio = greatest < least ? greatest + 1 : greatest;
    if (e == cudaSuccess)
        e = cudaStreamCreateWithPriority(&h->tile_stream, cudaStreamNonBlocking, tile_prio);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_tstart, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_tdone, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_start, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaStreamCreateWithPriority(&h->aux_stream, cudaStreamNonBlocking, greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->in_stream, cudaStreamNonBlocking);
    for (int r = 0; r < esi_handle::kSpans && e == cudaSuccess; ++r)
        e = cudaEventCreateWithFlags(&h->span[r].ev, cudaEventDisableTiming);
    for (int c = 0; c < 4 && e == cudaSuccess; ++c)
        e = cudaEventCreateWithFlags(&h->ev_chunk[c], cudaEventDisableTiming);
    for (int c = 0; c < 2 && e == cudaSuccess; ++c)
        e = cudaEventCreateWithFlags(&h->ev_unpk[c], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->dres, sizeof(PushResult));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&h->hres, sizeof(PushResult));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&h->hfetch, 2 * kSparse * sizeof(esi_event));
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        e = cudaEventCreateWithFlags(&h->ev_bin[b], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_tile[b], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        rc = cuda_fail(h, e);
        esi_destroy(h);
        return rc;
    }
    rc = esi::init_state(h);
    if (rc == ESI_OK) rc = ensure_ring(h, 1ull << 20);
    if (rc == ESI_OK) rc = cuda_fail(h, cudaStreamSynchronize(h->stream));
    if (rc) {
        esi_destroy(h);
        return rc;
    }
    *out = h;
    return ESI_OK;
}

void esi_destroy(esi_handle *h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->bin_stream) cudaStreamSynchronize(h->bin_stream);
    for (auto &r : h->prof_recs) {
        cudaEventDestroy(r.start);
        cudaEventDestroy(r.stop);
    }
    for (auto e : h->ev_pool) cudaEventDestroy(e);
    cudaFree(h->S);
    cudaFree(h->T);
    cudaFree(h->ring);
    for (int b = 0; b < 2; ++b) {
        cudaFree(h->rec[b]);
        cudaFree(h->hrow[b]);
        if (h->ev_bin[b]) cudaEventDestroy(h->ev_bin[b]);
        if (h->ev_tile[b]) cudaEventDestroy(h->ev_tile[b]);
    }
    if (h->ev_start) cudaEventDestroy(h->ev_start);
    if (h->bin_stream) cudaStreamDestroy(h->bin_stream);
    if (h->tile_stream) {
        cudaStreamSynchronize(h->tile_stream);
        cudaStreamDestroy(h->tile_stream);
    }
    if (h->ev_tstart) cudaEventDestroy(h->ev_tstart);
    if (h->ev_tdone) cudaEventDestroy(h->ev_tdone);
    cudaFree(h->dwin);
    cudaFree(h->dframes);
    cudaFree(h->diag);
    cudaFree(h->rec_idx[0]);
    cudaFree(h->rec_idx[1]);
    cudaFree(h->srt);
    cudaFree(h->srt_top);
    cudaFree(h->dstatus);
    cudaFreeHost(h->hstatus);
    cudaFreeHost(h->hwin);
    if (h->hwin_ev) cudaEventDestroy(h->hwin_ev);
    if (h->aux_stream) {
        cudaStreamSynchronize(h->aux_stream);
        cudaStreamDestroy(h->aux_stream);
    }
    if (h->in_stream) {
        cudaStreamSynchronize(h->in_stream);
        cudaStreamDestroy(h->in_stream);
    }
    for (int r = 0; r < esi_handle::kSpans; ++r)
        if (h->span[r].ev) cudaEventDestroy(h->span[r].ev);
    for (int c = 0; c < 4; ++c)
        if (h->ev_chunk[c]) cudaEventDestroy(h->ev_chunk[c]);
    for (int c = 0; c < 2; ++c)
        if (h->ev_unpk[c]) cudaEventDestroy(h->ev_unpk[c]);
    cudaFree(h->dsparse);
    cudaFree(h->pk_stage);
    cudaFree(h->dres);
    cudaFreeHost(h->hres);
    cudaFreeHost(h->hfetch);
    cudaFreeHost(h->tmirror);
    cudaFreeHost(h->tsparse);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
}

// Pushes below this many host events are checked on the host (lowest
// latency); larger ones and every device push are checked on the device.
static constexpr size_t kHostCheckMax = 1u << 16;
// events per chunk of a device-checked push
static constexpr unsigned long long kPushChunk = 1ull << 21;
// a host push that would overwrite ring slots a queued render still bins
// grows the ring (up to this many events) instead of waiting for it, so the
// next step's copy overlaps the current render
static constexpr unsigned long long kOverlapRingMax = 1ull << 28;

// One push of n >= 1 events: ev (16-byte events) or, when pk is set, packed
// words with times t_base + offset.  Packed host pushes reach here only above
// kHostCheckMax events (smaller ones are unpacked on the host first).
static int push_impl(esi_handle *h, const esi_event *ev, const unsigned long long *pk,
                     long long t_base, size_t n, int ev_on_device)
{
    const bool packed = pk != nullptr;
    const unsigned long long pending = h->tail - h->head;
    int rc = ensure_ring(h, pending + n);
    if (rc) return rc;
    if (!ev_on_device && !h->tmirror && h->tail + n > h->cap) {
        // the oldest render still binning slots this push would overwrite
        const unsigned long long o1 = h->tail + n - h->cap;
        unsigned long long a0 = ~0ull;
        for (int r = 0; r < esi_handle::kSpans; ++r) {
            const auto &sp = h->span[r];
            if (!sp.live || sp.a0 >= o1) continue;
            if (cudaEventQuery(sp.ev) == cudaErrorNotReady) {
                a0 = std::min(a0, sp.a0);
                // "not ready" is no failure: keep it out of the launch checks
                if (cudaPeekAtLastError() == cudaErrorNotReady) cudaGetLastError();
            }
        }
        if (a0 != ~0ull && h->tail - a0 + n <= kOverlapRingMax) {
            // room for twice that, so a deeper pipeline later needs no second
            // growth (each waits for the queued work)
            rc = ensure_ring(h, std::min(2 * (h->tail - a0 + n), kOverlapRingMax));
            if (rc) return rc;
        }
    }
    const unsigned long long mask = h->cap - 1;
    const long long prev = std::max(h->push_floor, h->last_event_t);
    const cudaMemcpyKind kind = ev_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    // device events keep the order of the handle's stream (they may come from
    // work queued on it); host events go on in_stream once the slots they
    // overwrite have been binned
    const cudaStream_t cs = ev_on_device ? h->stream : h->in_stream;
    cudaError_t e = cudaSuccess;
    if (!ev_on_device && h->tail + n > h->cap) {
        // the slots written held indices [o0, o1); wait for the newest render
        // that consumed one of them (renders bin in order, so older ones are
        // done by then).  Before the oldest tracked render: wait for that one.
        const unsigned long long o0 = h->tail - h->cap, o1 = h->tail + n - h->cap;
        int pick = -1;
        unsigned long long best = 0, oldest_a0 = ~0ull;
        int oldest = -1;
        for (int r = 0; r < esi_handle::kSpans; ++r) {
            const auto &sp = h->span[r];
            if (!sp.live) continue;
            if (sp.a0 < oldest_a0) {
                oldest_a0 = sp.a0;
                oldest = r;
            }
            if (sp.a0 < o1 && o0 < sp.a1 && sp.a1 > best) {
                best = sp.a1;
                pick = r;
            }
        }
        if (pick < 0 && oldest >= 0 && o0 < oldest_a0) pick = oldest;
        if (pick >= 0) {
            const cudaError_t q = cudaEventQuery(h->span[pick].ev);
            if (q == cudaErrorNotReady) {
                if (cudaPeekAtLastError() == cudaErrorNotReady) cudaGetLastError();
                e = cudaStreamWaitEvent(cs, h->span[pick].ev, 0);
                h->push_waits += 1;
            } else if (q != cudaSuccess) {
                e = q;
            }
        }
    }
    if (e != cudaSuccess) return cuda_fail(h, e);
    // events [i0, i1) of the push into their ring slots (split at the wrap)
    auto copy_in = [&](unsigned long long i0, unsigned long long i1) {
        for (unsigned long long i = i0; e == cudaSuccess && i < i1;) {
            const unsigned long long pos = (h->tail + i) & mask;
            const unsigned long long len = std::min(i1 - i, h->cap - pos);
            e = cudaMemcpyAsync(h->ring + pos, ev + i, len * sizeof(esi_event), kind, cs);
            i += len;
        }
    };
    if (!packed && !ev_on_device && n <= kHostCheckMax && !h->tmirror) {
        e = cudaMallocHost((void **)&h->tmirror, h->cap * sizeof(long long));
        if (e != cudaSuccess) {
            h->tmirror = nullptr;
            return cuda_fail(h, e);
        }
    }
    if (!packed && !ev_on_device && n <= kHostCheckMax) {
        // the copy starts first; the time-order check and the host mirror of
        // the times run meanwhile (a rejected batch leaves ring slots past
        // tail that nothing reads)
        copy_in(0, n);
        if (e != cudaSuccess) return cuda_fail(h, e);
        const bool ordered = check_and_mirror(h, ev, n, prev);
        // the caller may reuse its buffer as soon as this returns
        e = cudaStreamSynchronize(cs);
        if (e != cudaSuccess) return cuda_fail(h, e);
        if (!ordered) return ESI_ETIMEORDER;
        // every time of this push is in the mirror (adjacent spans merge)
        if (!h->exact_spans.empty() && h->exact_spans.back().second == h->tail)
            h->exact_spans.back().second = h->tail + n;
        else
            h->exact_spans.push_back({h->tail, h->tail + n});
        h->last_event_t = ev[n - 1].t_us;
    } else {
        // chunk by chunk: the copies follow one another on the push stream;
        // each chunk, once in, is checked on the device, and every
        // kSparse-th time kept and brought to the sparse mirror, on the aux
        // stream while the next chunks are copied in
        const unsigned long long g0 = (h->tail + kSparse - 1) / kSparse * kSparse;
        rc = ensure_device(h, &h->dsparse, &h->dsparse_cap, (size_t)(n / kSparse + 2));
        if (!rc && packed && !ev_on_device)
            rc = ensure_device(h, &h->pk_stage, &h->pk_stage_cap, (size_t)(2 * kPushChunk));
        if (rc) return rc;
        const unsigned long long smask = h->cap / kSparse - 1;
        e = cudaMemsetAsync(h->dres, 0, sizeof(PushResult), cs);
        int j = 0;
        for (unsigned long long c0 = 0; e == cudaSuccess && c0 < n; c0 += kPushChunk, ++j) {
            const unsigned long long c1 = std::min<unsigned long long>(n, c0 + kPushChunk);
            if (!packed) {
                copy_in(c0, c1);
                if (e == cudaSuccess) e = cudaEventRecord(h->ev_chunk[j & 3], cs);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(h->aux_stream, h->ev_chunk[j & 3], 0);
                if (e == cudaSuccess)
                    e = launch_push_check(h->ring, mask, h->tail, c0, (long long)(c1 - c0), n, prev,
                                          g0, h->dsparse, h->dres, h->aux_stream);
            } else {
                // host words go through staging buffer j & 1 (free once the
                // unpack of chunk j - 2 is done); device words are read where
                // they are, after the work queued on the handle's stream
                const unsigned long long *src = pk + c0;
                if (!ev_on_device) {
                    unsigned long long *st = h->pk_stage + (size_t)(j & 1) * kPushChunk;
                    if (j >= 2) e = cudaStreamWaitEvent(cs, h->ev_unpk[j & 1], 0);
                    if (e == cudaSuccess)
                        e = cudaMemcpyAsync(st, pk + c0, (c1 - c0) * sizeof(unsigned long long),
                                            cudaMemcpyHostToDevice, cs);
                    src = st;
                }
                if (e == cudaSuccess && (!ev_on_device || j == 0)) {
                    e = cudaEventRecord(h->ev_chunk[j & 3], cs);
                    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->aux_stream, h->ev_chunk[j & 3], 0);
                }
                if (e == cudaSuccess)
                    e = launch_push_unpack(src, h->ring, mask, h->tail, c0, (long long)(c1 - c0), n,
                                           t_base, prev, g0, h->dsparse, h->dres, h->aux_stream);
                if (e == cudaSuccess && !ev_on_device)
                    e = cudaEventRecord(h->ev_unpk[j & 1], h->aux_stream);
            }
            // sparse entries j of this chunk: indices g0 + j kSparse in [tail + c0, tail + c1)
            const unsigned long long ja = (std::max(g0, (h->tail + c0 + kSparse - 1) / kSparse * kSparse) - g0) / kSparse;
            const unsigned long long jb = (std::max(g0, (h->tail + c1 + kSparse - 1) / kSparse * kSparse) - g0) / kSparse;
            for (unsigned long long j = ja; e == cudaSuccess && j < jb;) {
                const unsigned long long pos = (g0 / kSparse + j) & smask;
                const unsigned long long len = std::min(jb - j, smask + 1 - pos);
                e = cudaMemcpyAsync(h->tsparse + pos, h->dsparse + j, len * sizeof(long long),
                                    cudaMemcpyDeviceToHost, h->aux_stream);
                j += len;
            }
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->hres, h->dres, sizeof(PushResult), cudaMemcpyDeviceToHost,
                                h->aux_stream);
        // the caller may reuse its buffer as soon as this returns
        if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->aux_stream);
        if (e != cudaSuccess) return cuda_fail(h, e);
        if (h->hres->bad) return ESI_ETIMEORDER;  // ring slots past tail are ignored
        h->last_event_t = h->hres->last;
    }
    if (ev_on_device) h->dev_push_pending = true;
    h->tail += n;
    h->pushed += n;
    return ESI_OK;
}

int esi_push_events(esi_handle *h, const esi_event *ev, size_t n, int ev_on_device)
{
    if (!h || (n && !ev) || (ev_on_device != 0 && ev_on_device != 1)) return ESI_EINVAL;
    if (n == 0) return ESI_OK;
    return push_impl(h, ev, nullptr, 0, n, ev_on_device);
}

int esi_push_packed(esi_handle *h, const uint64_t *pk, size_t n, int64_t t_base_us,
                    int pk_on_device)
{
    if (!h || (n && !pk) || (pk_on_device != 0 && pk_on_device != 1)) return ESI_EINVAL;
    if (t_base_us < -(1LL << 62) || t_base_us > (1LL << 62)) return ESI_EINVAL;
    if (pk_on_device && (reinterpret_cast<uintptr_t>(pk) & 7u)) return ESI_EINVAL;
    if (n == 0) return ESI_OK;
    if (!pk_on_device && n <= kHostCheckMax) {
        // small host pushes keep the host-checked path: unpack here
        try {
            h->pk_host.resize(n);
        } catch (...) {
            return ESI_ENOMEM;
        }
        for (size_t i = 0; i < n; ++i) {
            const uint64_t w = pk[i];
            esi_event &e = h->pk_host[i];
            e.t_us = (long long)t_base_us + (long long)(w >> kPackTShift);
            e.x = (uint16_t)(w & 0xffffu);
            e.y = (uint16_t)((w >> 16) & 0xffffu);
            e.p = ((w >> 32) & 1u) ? 1 : -1;
            e._pad[0] = e._pad[1] = e._pad[2] = 0;
        }
        return push_impl(h, h->pk_host.data(), nullptr, 0, n, 0);
    }
    return push_impl(h, nullptr, reinterpret_cast<const unsigned long long *>(pk),
                     (long long)t_base_us, n, pk_on_device);
}

int esi_render_frames(esi_handle *h, const int64_t *t_frames, size_t m, uint8_t *out,
                      int out_on_device)
{
    if (!h || !t_frames || m == 0 || !out || out_on_device < 0 || out_on_device > 2)
        return ESI_EINVAL;
    if (m > (size_t)INT_MAX) return ESI_EINVAL;
    if ((long long)t_frames[0] < h->frame_floor) return ESI_ETIMEORDER;
    for (size_t w = 1; w < m; ++w)
        if (t_frames[w] < t_frames[w - 1]) return ESI_ETIMEORDER;
    return esi::render_impl(h, t_frames, (int)m, out, out_on_device);
}

int esi_render_frame(esi_handle *h, int64_t t_frame_us, uint8_t *out, int out_on_device)
{
    return esi_render_frames(h, &t_frame_us, 1, out, out_on_device);
}

int esi_get_state(esi_handle *h, float *S, int64_t *T, int on_device)
{
    if (!h || !S || !T || (on_device != 0 && on_device != 1)) return ESI_EINVAL;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaError_t e = cudaMemcpyAsync(S, h->S, (size_t)h->P * sizeof(float), k, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(T, h->T, (size_t)h->P * sizeof(long long), k, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e);
    return esi::read_status(h);
}

int esi_set_state(esi_handle *h, const float *S, const int64_t *T, int on_device)
{
    if (!h || !S || !T || (on_device != 0 && on_device != 1)) return ESI_EINVAL;
    std::vector<long long> tmp;
    const long long *Th = reinterpret_cast<const long long *>(T);
    if (on_device) {
        try {
            tmp.resize((size_t)h->P);
        } catch (...) {
            return ESI_ENOMEM;
        }
        cudaError_t e = cudaMemcpyAsync(tmp.data(), T, (size_t)h->P * sizeof(long long),
                                        cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e);
        Th = tmp.data();
    }
    long long tmax = LLONG_MIN;
    for (long long i = 0; i < h->P; ++i) tmax = std::max(tmax, (long long)Th[i]);
    if (h->tail > h->head) {
        long long t0 = 0;
        int rc2 = exact_t(h, h->head, &t0);
        if (rc2) return rc2;
        if (t0 < tmax) return ESI_ETIMEORDER;
    }
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaError_t e = cudaMemcpyAsync(h->S, S, (size_t)h->P * sizeof(float), k, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->T, T, (size_t)h->P * sizeof(long long), k, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e);
    h->push_floor = std::max(h->push_floor, tmax);
    h->frame_floor = std::max(h->frame_floor, tmax);
    return ESI_OK;
}

int esi_synchronize(esi_handle *h)
{
    if (!h) return ESI_EINVAL;
    return esi::read_status(h);
}

int esi_get_stats(esi_handle *h, esi_stats *out)
{
    if (!h || !out) return ESI_EINVAL;
    int rc = esi::read_status(h);
    out->events_pushed = h->pushed;
    out->events_consumed = h->consumed;
    out->events_dropped = h->dropped;
    out->events_pending = h->tail - h->head;
    out->frames_rendered = h->frames;
    out->kernel_launches = h->launches;
    out->last_event_t_us = h->last_event_t;
    out->last_frame_t_us = h->last_frame_t;
    out->ring_capacity = h->cap;
    out->ring_grows = h->ring_grows;
    out->push_waits = h->push_waits;
    return rc;
}

int esi_set_tuning(esi_handle *h, const esi_tuning *t)
{
    if (!h || !t) return ESI_EINVAL;
    esi_tuning d = default_tuning(h->W, h->H);
    esi_tuning n = *t;
    if (!n.tile_w) n.tile_w = d.tile_w;
    if (!n.tile_h) n.tile_h = (n.tile_w == 32) ? 32 : d.tile_h;
    if (!n.chunk_events) n.chunk_events = d.chunk_events;
    if (!n.batch_records) n.batch_records = d.batch_records;
    if (!n.max_batch_events) n.max_batch_events = d.max_batch_events;
    if (!n.scan_chain) n.scan_chain = d.scan_chain;
    if (!n.split_rows) n.split_rows = d.split_rows;
    int rc = validate_tuning(n);
    if (rc) return rc;
    esi_tuning old = h->tun;
    rc = apply_tuning(h, n);
    if (rc) apply_tuning(h, old);
    return rc;
}

int esi_get_tuning(esi_handle *h, esi_tuning *out)
{
    if (!h || !out) return ESI_EINVAL;
    *out = h->tun;
    return ESI_OK;
}

int esi_profile_enable(esi_handle *h, int enable)
{
    if (!h) return ESI_EINVAL;
    h->prof_on = enable != 0;
    return ESI_OK;
}

int esi_profile_read(esi_handle *h, esi_kernel_time *out, int max)
{
    if (!h || max < 0 || (max > 0 && !out)) return ESI_EINVAL;
    int src = sync_all(h);
    if (src) return src;
    for (auto &r : h->prof_recs) {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, r.start, r.stop);
        if (r.kind >= 0 && r.kind < kNumKernelKinds) {
            h->prof_ms[r.kind] += ms;
            h->prof_n[r.kind] += 1;
        }
        h->ev_pool.push_back(r.start);
        h->ev_pool.push_back(r.stop);
    }
    h->prof_recs.clear();
    int n = 0;
    for (int k = 0; k < kNumKernelKinds; ++k) {
        if (!h->prof_n[k]) continue;
        if (n < max) {
            std::memset(out[n].name, 0, sizeof(out[n].name));
            std::strncpy(out[n].name, kKernelNames[k], sizeof(out[n].name) - 1);
            out[n].launches = h->prof_n[k];
            out[n].total_ms = h->prof_ms[k];
        }
        ++n;
    }
    return n;
}

int esi_profile_reset(esi_handle *h)
{
    if (!h) return ESI_EINVAL;
    int src = sync_all(h);
    for (auto &r : h->prof_recs) {
        h->ev_pool.push_back(r.start);
        h->ev_pool.push_back(r.stop);
    }
    h->prof_recs.clear();
    for (int k = 0; k < kNumKernelKinds; ++k) {
        h->prof_ms[k] = 0.0;
        h->prof_n[k] = 0;
    }
    return src;
}

}  // extern "C"

// --------------------------------------------------------------- rendering
int esi::init_state(esi_handle *h)
{
    // Alg. 2 initialisation: S = 0, T = t_origin
    cudaError_t e = cudaMemsetAsync(h->S, 0, (size_t)h->P * sizeof(float), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->dstatus, 0, sizeof(DevStatus), h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e);
    return fill_i64(h, h->T, h->P, h->prm.t_origin_us);
}

int esi::plan_subbatches(esi_handle *h, unsigned long long n_split, const int64_t *tf, int m,
                         std::vector<SubBatch> *plan_out)
{
    const unsigned long long maxb = (unsigned long long)h->tun.max_batch_events;
    std::vector<SubBatch> &plan = *plan_out;
    plan.clear();
    int rc = ESI_OK;
    {
        unsigned long long i = 0;
        int w = 0;
        for (;;) {
            SubBatch sb;
            sb.i0 = i;
            // a split at an index the sparse mirror holds keeps its time exact
            // without reading it back
            auto aligned = [&](unsigned long long j) {
                const unsigned long long g = (h->head + j) / kSparse * kSparse;
                return g > h->head + i ? g - h->head : j;
            };
            sb.i1 = std::min(n_split, i + maxb);
            if (sb.i1 < n_split) sb.i1 = aligned(sb.i1);
            sb.t_base = 0;
            if (sb.i1 > i) {
                // a base no later than the first event (record times are
                // 32-bit offsets from it)
                rc = lower_t(h, h->head + i, &sb.t_base);
                if (rc) return rc;
                const long long lim = sb.t_base + 0xffffffffll;
                unsigned long long cut = 0;
                rc = upper_bound_t(h, h->head + i, h->head + sb.i1, lim, &cut);
                if (rc) return rc;
                if (cut - h->head < sb.i1) sb.i1 = std::max(aligned(cut - h->head), i + 1);
            } else if (w < m) {
                sb.t_base = tf[w];
            }
            sb.w0 = w;
            sb.w1 = m;
            if (sb.i1 < n_split) {
                // frames before the next sub-batch's first time complete
                // here (exact: the launch emits them among its records)
                const unsigned long long a1 = h->head + sb.i1;
                long long tn = 0;
                if (a1 % kSparse == 0 && sparse_ok(h, a1)) {
                    tn = sparse_t(h, a1);
                } else {
                    rc = exact_t(h, a1, &tn);
                    if (rc) return rc;
                }
                sb.w1 = (int)(std::lower_bound(tf + w, tf + m, (int64_t)tn) - tf);
            }
            plan.push_back(sb);
            i = sb.i1;
            w = sb.w1;
            if (i >= n_split && w >= m) break;
        }
    }
    return ESI_OK;
}

int esi::render_impl(esi_handle *h, const int64_t *tf, int m, uint8_t *out, int out_on_device)
{
    const long long t_last = tf[m - 1];
    unsigned long long n_end = 0;
    int rc = upper_bound_t(h, h->head, h->tail, t_last, &n_end);
    if (rc) return rc;
    const unsigned long long n_split = n_end - h->head;
    const esi_tuning &tu = h->tun;
    const int chunk = tu.chunk_events;
    const unsigned long long maxb = (unsigned long long)tu.max_batch_events;

    // plan: sub-batches of at most max_batch_events whose record times fit in
    // 32 bits; each completes the frames that end before its successor starts
    std::vector<SubBatch> plan;
    rc = plan_subbatches(h, n_split, tf, m, &plan);
    if (rc) return rc;
    // the staging buffer may still feed the previous render's queued copy
    if (h->hwin_busy) {
        cudaError_t e0 = cudaEventSynchronize(h->hwin_ev);
        if (e0 != cudaSuccess) return cuda_fail(h, e0);
        h->hwin_busy = false;
    }
    rc = ensure_pinned(h, &h->hwin, &h->hwin_cap, (size_t)m);
    if (!rc) rc = ensure_device(h, &h->dwin, &h->dwin_cap, (size_t)m);
    if (rc) return rc;
    for (const SubBatch &sb : plan)
        for (int w = sb.w0; w < sb.w1; ++w) {
            const long long d = (long long)tf[w] - sb.t_base;
            h->hwin[w].lim = std::min(std::max(d, -1ll), 0xffffffffll);
            h->hwin[w].tf_f = (float)d;
            h->hwin[w].pad = 0;
        }
    cudaError_t e = cudaMemcpyAsync(h->dwin, h->hwin, (size_t)m * sizeof(WinInfo),
                                    cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(h->hwin_ev, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e);
    h->hwin_busy = true;
    // host output: pinned (page-locked, mapped) buffers are written by the
    // kernels directly; other host buffers through a device staging copy
    uint8_t *frames = out;
    bool staged_out = false;
    const bool host_out = out_on_device != 1;   // 0: host, waits; 2: host, returns at once
    if (host_out) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, out) == cudaSuccess && at.type == cudaMemoryTypeHost &&
            at.devicePointer) {
            frames = static_cast<uint8_t *>(at.devicePointer);
        } else {
            cudaGetLastError();
            rc = ensure_device(h, &h->dframes, &h->dframes_cap, (size_t)m * (size_t)h->P);
            if (rc) return rc;
            frames = h->dframes;
            staged_out = true;
        }
    }
    // both scratch halves fit the current shape: the halves alternate across
    // renders, so a one-sub-batch render may use either
    for (int b = 0; b < 2; ++b) {
        const size_t max_chunks = (size_t)((maxb + chunk - 1) / chunk);
        rc = ensure_device(h, &h->rec[b], &h->rec_cap[b], max_chunks * (size_t)chunk);
        if (!rc) rc = ensure_device(h, &h->hrow[b], &h->hrow_cap[b], max_chunks * (size_t)h->n_tiles);
        if (rc) return rc;
    }
    if (h->split) {
        // each tile's region has room for all its records in every row's part
        rc = ensure_device(h, &h->srt, &h->srt_cap, (size_t)maxb * (size_t)tu.tile_h);
        if (!rc) rc = ensure_device(h, &h->srt_top, &h->srt_top_cap, 1);
        if (rc) return rc;
    }
    // binning reads only the ring and its own scratch half: it may start
    // during the previous render's last tile kernel (the halves alternate
    // across renders), after device pushes queued on the handle's stream
    if (h->dev_push_pending) {
        e = cudaEventRecord(h->ev_start, h->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->bin_stream, h->ev_start, 0);
        if (e != cudaSuccess) return cuda_fail(h, e);
        h->dev_push_pending = false;
    }
    // a lane's pixels go out as one frame word when rows and the buffer allow
    const unsigned wb = h->tun.tile_w == 64 ? 2u : 4u;
    const bool vec = (h->W % (int)wb == 0) && (((uintptr_t)frames & (wb - 1u)) == 0);
    // the tile stream starts after everything queued on the handle's stream
    // (pushes of device events, the frame table, state writes)
    e = cudaEventRecord(h->ev_tstart, h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->tile_stream, h->ev_tstart, 0);
    if (e != cudaSuccess) return cuda_fail(h, e);
    for (const SubBatch &sb : plan) {
        const int nb = (int)(sb.i1 - sb.i0);
        const int n_chunks = (nb + chunk - 1) / chunk;
        const int buf = h->next_buf;
        h->next_buf ^= 1;
        if (nb > 0) {
            // the buffer's previous tile kernel must be done reading it
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
            cudaEvent_t ev;
            rc = prof_begin(h, &ev, h->bin_stream);
            if (!rc) rc = cuda_fail(h, launch_bin(ba, n_chunks, h->bin_stream));
            if (!rc) rc = prof_end(h, kKindBin, ev, h->bin_stream);
            if (!rc) rc = cuda_fail(h, cudaEventRecord(h->ev_bin[buf], h->bin_stream));

            if (!rc) rc = cuda_fail(h, cudaStreamWaitEvent(h->tile_stream, h->ev_bin[buf], 0));
            if (rc) return rc;
        }
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
        ta.w_begin = sb.w0;
        ta.w_end = sb.w1;
        ta.frames = frames;
        ta.frame_outs = nullptr;
        ta.P = h->P;
        ta.batch = tu.batch_records;
        ta.status = h->dstatus;
        ta.scan_chain = tu.scan_chain;
        if (h->split) {
            // the split-row kernel hands every tile a region of the scratch
            ta.srt = h->srt;
            ta.srt_cap = h->srt_cap;
            ta.srt_top = h->srt_top;
            ta.max_splits = tu.split_rows == 1 ? kTileW : 0;
            e = cudaMemsetAsync(h->srt_top, 0, sizeof(unsigned long long), h->tile_stream);
            if (e != cudaSuccess) return cuda_fail(h, e);
        }
        cudaEvent_t ev;
        rc = prof_begin(h, &ev, h->tile_stream);
        if (!rc) rc = cuda_fail(h, h->split ? launch_tile_split(ta, tu.tile_h, vec, h->tile_stream)
                                            : launch_tile(ta, tu.tile_h, tu.tile_w, vec, h->tile_stream));
        if (!rc) rc = prof_end(h, kKindTile, ev, h->tile_stream);
        if (!rc) rc = cuda_fail(h, cudaEventRecord(h->ev_tile[buf], h->tile_stream));
        if (rc) return rc;
        h->tile_pending[buf] = true;
    }
    if (n_split > 0) {
        // the binning launches of this render read ring indices [head, head + n_split)
        auto &sp = h->span[h->span_next];
        e = cudaEventRecord(sp.ev, h->bin_stream);
        if (e != cudaSuccess) return cuda_fail(h, e);
        sp.a0 = h->head;
        sp.a1 = h->head + n_split;
        sp.live = true;
        h->span_next = (h->span_next + 1) % esi_handle::kSpans;
    }
    h->head += n_split;
    h->consumed += n_split;
    while (!h->exact_spans.empty() && h->exact_spans.front().second <= h->head)
        h->exact_spans.erase(h->exact_spans.begin());
    h->frames += (unsigned long long)m;
    h->last_frame_t = t_last;
    h->frame_floor = std::max(h->frame_floor, (long long)t_last);
    h->push_floor = std::max(h->push_floor, (long long)t_last);
    // the handle's stream continues after the render's tile kernels
    e = cudaEventRecord(h->ev_tdone, h->tile_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->ev_tdone, 0);
    if (e != cudaSuccess) return cuda_fail(h, e);
    if (host_out) {
        if (staged_out) {
            e = cudaMemcpyAsync(out, frames, (size_t)m * (size_t)h->P, cudaMemcpyDeviceToHost, h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e);
        }
        if (out_on_device == 0) return read_status(h);
    }
    return ESI_OK;
}

int esi::fill_i64(esi_handle *h, long long *dst, long long n, long long value)
{
    cudaEvent_t ev;
    int rc = prof_begin(h, &ev, h->stream);
    if (!rc) rc = cuda_fail(h, launch_fill_i64(dst, n, value, h->stream));
    if (!rc) rc = prof_end(h, kKindFill, ev, h->stream);
    return rc;
}
