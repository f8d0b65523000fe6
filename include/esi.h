/*
 * esi.h -- C ABI of the GB300 (sm_103a) implementation of Event-based Single
 * Integration (ESI), arXiv 2508.02238.
 *
 * The method (Sec. III): an event camera emits events e = {x, y, t, p}
 * (Sec. III-A).  Every event updates its pixel's accumulation S and
 * last-decay time T (Alg. 2): S += p C; dt = t - T; S *= d(dt); T = t;
 * S = min(max(S, S_min), S_max), with the decay d(t) = max{(1 - k t)^b, 0}
 * of Eq. 4 (read as max(1 - k t, 0)^b) and the clamp of Eq. 13.  A frame maps
 * S linearly to 8 bits (Eq. 14).  S and T are the whole state (Sec. III-B).
 *
 * Conventions for every call:
 *   - Return 0 (ESI_OK) or a negative ESI_E* code; esi_strerror() names it.
 *   - Pointers are plain host or device pointers as the *_on_device flag
 *     says; the caller owns every buffer it passes.  No call keeps a pointer
 *     the caller passed after it returns, with one exception: a render with
 *     out_on_device = 2 writes its host buffer until the next call that
 *     waits (esi_synchronize).
 *   - Time is int64 microseconds.  k is given per second.
 *   - A handle (and a server) is not thread-safe: drive it from one thread.
 *   - Device work runs on the CUDA stream given at creation (NULL = a stream
 *     the library creates).  Calls that write host memory wait for their
 *     own work (a render with out_on_device = 2 excepted); calls that only
 *     write device memory return once the work is queued, and errors found
 *     by the device are reported by the next call that waits
 *     (esi_synchronize, esi_get_state, a render with out_on_device = 0).
 */
#ifndef ESI_H
#define ESI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- errors */
#define ESI_OK 0
#define ESI_EINVAL (-1)      /* bad argument: params, sizes, pointers, ids    */
#define ESI_ENOMEM (-2)      /* device or host allocation failed             */
#define ESI_EBUSY (-3)       /* admission refused: state budget exhausted    */
#define ESI_ETIMEORDER (-4)  /* event or frame time goes backwards           */
#define ESI_ERANGE (-5)      /* a value is outside what the layout can hold  */
#define ESI_ECUDA (-6)       /* a CUDA runtime call failed                   */
#define ESI_ETIMEOUT (-7)    /* a bounded device-side wait gave up           */
#define ESI_ESTATE (-8)      /* call not valid in the current state          */

/* ----------------------------------------------------------------- types */

/*
 * One event (Sec. III-A): pixel (x, y), time t_us, polarity p.  p > 0 counts
 * as +1 and anything else as -1 (the paper's p in {+1, -1}; DAVIS 0/1 also
 * works).  16 bytes, little endian, no padding between fields.
 */
typedef struct {
    int64_t t_us;
    uint16_t x;
    uint16_t y;
    int8_t p;
    uint8_t _pad[3];
} esi_event;

/*
 * Method parameters.  C: contrast step per event (Alg. 2), > 0.  k_per_s,
 * b: decay of Eq. 4, 0 <= k <= 1e12 (k = 0 gives the plain integration of
 * Eq. 2), b > 0.  s_min < s_max: clamp bounds of Eq. 13, also the ends of
 * the linear map of Eq. 14; both finite.  t_origin_us: initial T of every
 * pixel (Alg. 2 uses 0).  render_decay: 0 maps S as stored (Alg. 2); 1 maps
 * the decay view S d(t_frame - T), which is not written back.
 * method: which per-event update runs (Sec. III-B, III-C):
 *   ESI_METHOD_ALG2     Alg. 2: S += p C; S *= d(t - T); T = t; clamp to
 *                       [s_min, s_max] (Eq. 13).  The default (0).
 *   ESI_METHOD_ALG1     Alg. 1: the same without the clamp.
 *   ESI_METHOD_EQ3_EXP  Eq. 3 with d(t) = exp(-k t): S = S d(t - T) + p C;
 *                       T = t, no clamp.  S is Eq. 3's sum
 *                       C sum_{t_i <= T} p_i exp(-k (T - t_i)); b is unused.
 * Without a clamp the state is unbounded; the map of Eq. 14 saturates every
 * method's frame to [0, 255].
 */
#define ESI_METHOD_ALG2 0
#define ESI_METHOD_ALG1 1
#define ESI_METHOD_EQ3_EXP 2
typedef struct {
    double C;
    double k_per_s;
    double b;
    double s_min;
    double s_max;
    int64_t t_origin_us;
    int32_t render_decay;
    int32_t method;       /* ESI_METHOD_* */
} esi_params;

/* Counters of one handle (or one server stream). */
typedef struct {
    uint64_t events_pushed;    /* accepted by esi_push_events               */
    uint64_t events_consumed;  /* taken by renders (applied or dropped)     */
    uint64_t events_dropped;   /* x >= W or y >= H: never applied           */
    uint64_t events_pending;   /* pushed, t later than every rendered frame */
    uint64_t frames_rendered;
    uint64_t kernel_launches;  /* device kernels this handle has launched   */
    int64_t last_event_t_us;
    int64_t last_frame_t_us;
    uint64_t ring_capacity;    /* events the device ring holds now          */
    uint64_t ring_grows;       /* times it moved into a larger one          */
    uint64_t push_waits;       /* host pushes queued behind a render still binning */
} esi_stats;

/*
 * Launch-shape knobs (all 0 = library default).  tile_w: pixels per tile
 * row, 128 (four per thread), 64 (two per thread) or 32 (one per thread):
 * narrower rows give more independent row walks.  tile_h: rows per tile, 4,
 * 8 or 16 with tile_w = 128 or 64, 16 or 32 with tile_w = 32.  chunk_events: events per binning block
 * (power of two, 512..8192).  batch_records: records a tile sorts in shared
 * memory at once (power of two, 1024..8192).  max_batch_events: events per
 * binning pass of a render (>= chunk_events).  scan_chain: the tile kernel
 * applies a row's due events 32 at a time; a group in which one pixel has at
 * least scan_chain events (1..32) is composed as a segmented scan of the
 * events' clamped-affine maps (Alg. 2's update with the clamp of Eq. 13 is
 * such a map, and they compose associatively) in log2 steps instead of event
 * by event; its rounding then differs from the event-by-event loop by a few
 * units in the last place.  33 turns the scan off: every group runs event
 * by event in arrival order, and results are bit-identical across every
 * launch shape.  Default 8.  split_rows (128-pixel rows only): 1 = a tile's
 * rows are sorted as a whole and divided among its warps by work, a busy row
 * split at record boundaries, the state at each split obtained by composing
 * the events before it (the same clamped-affine maps); rounding then differs
 * from the event-by-event loop by a few units in the last place at split
 * rows.  2 = one warp per row, walking the tile's records batch by batch.
 * 3 = rows sorted as a whole, one warp per row, no split (results as with
 * 2).  Default 2: on the synthetic workloads of this library the split-row
 * kernel runs about 1.4 times longer than the batch walk.
 */
typedef struct {
    int32_t tile_h;
    int32_t chunk_events;
    int32_t batch_records;
    int32_t max_batch_events;
    int32_t tile_w;
    int32_t scan_chain;
    int32_t split_rows;
} esi_tuning;

/* Per-kernel device time collected while profiling is on. */
typedef struct {
    char name[32];
    uint64_t launches;
    double total_ms;
} esi_kernel_time;

typedef struct esi_handle esi_handle;

/* ------------------------------------------------------- one sensor path */

/*
 * Create the state of one width x height sensor (Alg. 2 initialisation:
 * S = 0, T = t_origin for every pixel) on the current CUDA device.
 * width, height in [1, 65535].  cuda_stream: a cudaStream_t or NULL.
 * Errors: ESI_EINVAL for bad sizes or parameters (checked before any CUDA
 * call), ESI_ERANGE for sensors with more tiles than the binning can count
 * in shared memory (above about 10,000 tiles of 128 x 16 pixels, some
 * 20 M pixels), ESI_ENOMEM, ESI_ECUDA.
 */
int esi_create(int width, int height, const esi_params *params,
               void *cuda_stream, esi_handle **out);

/*
 * Queue n events (Sec. III-A) for the next renders.  Times must be
 * non-decreasing within the batch and not earlier than the last event
 * pushed before, nor than t_origin or the last frame time; otherwise the
 * whole batch is rejected with ESI_ETIMEORDER and nothing is queued.
 * Events with x >= W or y >= H are accepted but dropped (counted, never
 * applied).  ev_on_device = 0: host buffer, copied before the call
 * returns; the copy may run while earlier renders are still on the device
 * (it waits only for renders that read the ring slots it overwrites).
 * ev_on_device = 1: device buffer, copied on the handle's stream after the
 * work queued on it; the call waits for that copy.  Pushes of more than
 * 65,536 events and all device pushes are checked for time order on the
 * device, smaller host pushes on the host.  n = 0 is a no-op.
 */
int esi_push_events(esi_handle *h, const esi_event *ev, size_t n, int ev_on_device);

/*
 * Packed events: one little-endian uint64 per event, half the bytes of
 * esi_event on the host link.  The paper has no counterpart (it gives no
 * encoding); the events it carries are those of Sec. III-A.
 *   bits  0..15  x
 *   bits 16..31  y
 *   bit  32      polarity: 1 = +1, 0 = -1
 *   bits 33..63  t_us - t_base_us, 0 .. 2^31 - 1 (about 35 minutes)
 * ESI_PACK_EVENT builds one word; dt_us must be in that range.
 */
#define ESI_PACK_T_SHIFT 33
#define ESI_PACK_EVENT(x, y, on, dt_us)                                           \
    ((uint64_t)(uint16_t)(x) | ((uint64_t)(uint16_t)(y) << 16) |                 \
     ((uint64_t)((on) ? 1 : 0) << 32) | ((uint64_t)(dt_us) << ESI_PACK_T_SHIFT))

/*
 * esi_push_events for n packed events: event i is
 * {t_base_us + (pk[i] >> 33), x, y, +1 or -1} as laid out above, and every
 * rule, error and return point of esi_push_events applies to those events
 * (host pushes of at most 65,536 events are unpacked and checked on the
 * host; larger ones and device pushes are unpacked into the device ring and
 * checked there, chunk by chunk, the copy of the next chunk overlapping).
 * pk: pk_on_device = 0 host array (page-locked for the fastest copy),
 * 1 device array (8-byte aligned, read after the work queued on the
 * handle's stream); the caller keeps ownership and may reuse it once the
 * call returns.  ESI_EINVAL as esi_push_events, and also for a device pk
 * that is not 8-byte aligned or t_base_us outside [-2^62, 2^62].
 */
int esi_push_packed(esi_handle *h, const uint64_t *pk, size_t n, int64_t t_base_us,
                    int pk_on_device);

/*
 * Apply every queued event with t <= t_frame_us in push order (Alg. 2
 * loop; a frame at t shows the events t_n <= t, the condition under Eq. 5)
 * and write the Eq. 14 frame, W * H bytes row-major (y * W + x), to out.
 * Later events stay queued.  t_frame_us must not be earlier than the
 * previous frame or t_origin (ESI_ETIMEORDER).  out_on_device: 1 = device
 * buffer (the call returns once the work is queued); 0 = host buffer, the
 * call waits for the frame; 2 = host buffer, the call returns once the work
 * is queued and the frame is complete after esi_synchronize (or any call
 * that waits).  A page-locked host buffer is written by the kernels
 * directly; another one through a device copy.
 */
int esi_render_frame(esi_handle *h, int64_t t_frame_us, uint8_t *out, int out_on_device);

/*
 * m frames at non-decreasing times t_frames[0..m-1] (a host array): frame w
 * shows every queued event with t <= t_frames[w], exactly as m calls of
 * esi_render_frame would, in one pass over the events.  out holds m * W * H
 * bytes, frame w at offset w * W * H.
 */
int esi_render_frames(esi_handle *h, const int64_t *t_frames, size_t m,
                      uint8_t *out, int out_on_device);

/*
 * Checkpoint: copy S (float32, W * H) and T (int64 us, W * H) out.  Waits
 * for queued work and reports device-side errors.  Queued events are not
 * part of S, T (they stay queued).
 */
int esi_get_state(esi_handle *h, float *S, int64_t *T, int on_device);

/*
 * Resume: replace S and T.  Every T must be <= the earliest queued event and
 * later pushes must not be earlier than max(T) (ESI_ETIMEORDER otherwise).
 */
int esi_set_state(esi_handle *h, const float *S, const int64_t *T, int on_device);

/* Wait for the handle's queued device work; returns a device-side error. */
int esi_synchronize(esi_handle *h);

/*
 * Continuous-time output (Alg. 2 per event; Alg. 1 or Eq. 3 by the method):
 * applies every queued event to the state, as a render at the last queued
 * time would, and writes out[i] = S of the i-th queued event's pixel (push
 * order) right after that event is applied: float32, one value per event,
 * NaN for an event outside the sensor.  *n_out receives the number of events
 * (events_pending before the call; 0 leaves out untouched).  out holds cap
 * floats (ESI_ERANGE if cap < events_pending).  No frame is rendered; later
 * frames must not be earlier than the last applied event.  The state
 * afterwards is bit-identical to the one such a render leaves.  Waits for
 * the result; reports device-side errors.
 */
int esi_event_states(esi_handle *h, float *out, size_t cap, int out_on_device, size_t *n_out);

/*
 * Noise-accumulation map of Fig. 4 (Sec. III-B): out[y * W + x] =
 * ln(1 + |S(x, y)|) of the current state, float32, W * H, row-major.  The
 * figure draws it for the plain integration of Eq. 2 in event units
 * (method ESI_METHOD_ALG1, k = 0, C = 1); there, with a 15 % contrast
 * threshold, 1.8 means a doubled and 2.2 a tripled intensity.  Queued
 * events are not part of S.  Waits for the result; reports device-side
 * errors.
 */
int esi_noise_map(esi_handle *h, float *out, int out_on_device);

/*
 * Per-pixel event counts of the handle's sensor (Sec. III-B's event-trigger
 * rate, times the window): counts[y * W + x] = the number of the n events
 * at (x, y), uint32, W * H, overwritten.  Events with x >= W or y >= H are
 * not counted; the events need not be in time order and are not queued.
 * Host buffers are staged through device memory the handle keeps.  Waits
 * for the result.  Errors: ESI_EINVAL, ESI_ERANGE (n > 2^40), ESI_ENOMEM,
 * ESI_ECUDA.
 */
int esi_count_events(esi_handle *h, const esi_event *events, size_t n, int events_on_device,
                     uint32_t *counts, int counts_on_device);

/*
 * Inspection of the render's first sorting level.  Alg. 2 applies events in
 * stream order; on the GPU a render first reorders them by pixel, which is
 * legal because a pixel's state depends only on its own events in time order
 * (Eq. 5, Sec. III-B), and the sort must be stable to keep that order.  This
 * call runs the render's binning kernel alone: events first .. first + n - 1
 * of a device ring of ring_capacity events (a power of two, index i at
 * ring[i % ring_capacity], 16-byte aligned; n <= ring_capacity) are cut into
 * chunks of shape->chunk_events consecutive events, and each chunk's records
 * are stably sorted by pixel tile (shape->tile_w x shape->tile_h pixels;
 * zeros take 128 x 8 and 2048-event chunks).  Output, device buffers owned by
 * the caller:
 *   records  ceil(n / chunk) * chunk uint64; chunk c's records start at
 *            c * chunk: record = (t - t_base) mod 2^32 in the low 32 bits,
 *            ((row_in_tile * tile_w + x_in_tile) << 1 | (p > 0)) in the high
 *            32 bits; events outside the sensor are left out, so the chunk's
 *            valid records are its first (events - dropped) slots.
 *   runs     [tile][chunk] uint32, tiles row-major over the sensor (tile
 *            index (y / tile_h) * ceil(W / tile_w) + x / tile_w): the tile's
 *            records in the chunk start at (runs >> 16) and number
 *            (runs & 0xffff).
 * *dropped (may be NULL) receives the count of events outside the sensor.
 * Waits for the result.  Errors: ESI_EINVAL (sizes, shape, pointers),
 * ESI_ERANGE (more tiles than the binning holds), ESI_ENOMEM, ESI_ECUDA,
 * ESI_ETIMEOUT (a bounded device wait gave up).
 */
int esi_bin_events(int width, int height, const esi_tuning *shape, const esi_event *ring,
                   uint64_t ring_capacity, uint64_t first, size_t n, int64_t t_base,
                   uint64_t *records, uint32_t *runs, uint64_t *dropped, void *cuda_stream);

/* Counters; waits for queued work so that the drop count is exact. */
int esi_get_stats(esi_handle *h, esi_stats *out);

/* Launch-shape knobs; ESI_EINVAL for values outside the documented sets. */
int esi_set_tuning(esi_handle *h, const esi_tuning *t);
int esi_get_tuning(esi_handle *h, esi_tuning *out);

#define ESI_AUTOTUNE_FORCE 1      /* measure even when a cached choice exists  */
#define ESI_AUTOTUNE_WIDE_ONLY 2  /* only 128-pixel tile rows (serving tiles)  */

/*
 * Choose the launch shape for this sensor: run a host sample of n events and
 * m frame times (time-ordered, not before t_origin) through a scratch handle
 * of the same sensor and parameters once per candidate shape (tile width and
 * height, chunk_events, batch_records, max_batch_events), time each render
 * with CUDA events, apply the fastest to h and write it to *chosen.  The
 * choice is cached per (W, H, events-per-frame bucket, render mode, decay
 * kind, flags) for the life of the process; a cached choice is applied
 * without measuring unless flags has ESI_AUTOTUNE_FORCE.  h's state and
 * queued events are untouched.
 */
int esi_autotune(esi_handle *h, const esi_event *sample, size_t n, const int64_t *t_frames,
                 size_t m, int flags, esi_tuning *chosen);

/*
 * Device-time profiling of the handle's kernels (CUDA events around each
 * launch on the handle's stream).  esi_profile_read waits, writes up to
 * max entries and returns how many kernels it knows (>= 0).
 */
int esi_profile_enable(esi_handle *h, int enable);
int esi_profile_read(esi_handle *h, esi_kernel_time *out, int max);
int esi_profile_reset(esi_handle *h);

/* Free everything the handle owns.  NULL is a no-op. */
void esi_destroy(esi_handle *h);

/* Static text for an ESI_* code. */
const char *esi_strerror(int code);

/* ------------------------------------------------------------ serving */

/*
 * Batched serving of many sensors.  The paper runs one camera (Sec. IV-C);
 * this interface is the library's own: every stream is the single-sensor path
 * above (same parameters, same per-pixel semantics, same results), and one
 * tick processes all streams together in one binning launch and one tile
 * launch per parameter variant, replayed as a CUDA graph.
 *
 * Time: streams share the caller's clock now_us (int64 us).  Stream frames
 * fall at t_origin + k * frame_period_us, k >= 1.  The caller pushes each
 * stream's events as its packets arrive; esi_server_tick(now_us) promises
 * that every event with t <= now_us has been pushed.  The tick applies
 * pushed events with t <= now_us (every stream's, or only those of streams
 * with a frame due: esi_server_opts.apply_mode), renders every frame with
 * t_frame <= now_us (at most frame_slots - 1 per stream per tick; the rest
 * follow in the next ticks) and returns once the work is queued.  Frames land
 * in host memory the GPU writes directly; esi_stream_frame returns the newest
 * finished one.
 *
 * Admission: each stream's device state (12 bytes per pixel) comes from an
 * arena of state_budget_bytes reserved at creation; esi_stream_open returns
 * ESI_EBUSY when it does not fit (nor its event ring and frame slots in the
 * pinned host pool), and esi_stream_close returns the space, so a later open
 * can succeed.  Streams may open and close between ticks; work of
 * successive ticks overlaps on the device (two host staging buffers).
 */
typedef struct {
    int64_t frame_period_us;      /* default 10000 (100 frames/s)            */
    int64_t max_events_per_tick;  /* default 4194304                         */
    int32_t max_streams;          /* default 256                             */
    int32_t frame_slots;          /* finished frames kept per stream, >= 2; default 4 */
    int32_t use_graph;            /* 1 (default): replay a captured graph    */
    int32_t tile_h;               /* rows per 128-pixel tile of new streams: 0 = 8, or 4, 16 */
    int32_t max_stream_pixels;    /* largest W * H accepted; default 1280*720 */
    int32_t scan_chain;           /* as esi_tuning.scan_chain; 0 = default (8) */
    int32_t apply_mode;           /* when a stream's events are applied: 0 = default
                                   * (ESI_APPLY_EVERY_TICK), ESI_APPLY_EVERY_TICK or
                                   * ESI_APPLY_AT_FRAMES */
    int32_t copy_threads;         /* host threads that copy a large push into its
                                   * ring, the caller's included: 0 = default (4),
                                   * 1 .. 16                                   */
    int32_t fuse_tick;            /* 0 = default (1); 1: a tick whose streams all
                                   * use 8-row tiles, have at most 256 tiles of
                                   * 128 x 8 pixels each (about 260 k pixels) and
                                   * share render mode and decay kind runs as one
                                   * persistent launch (binning and tiles); 2:
                                   * always one binning launch and one tile
                                   * launch per variant                          */
    int32_t _reserved;
    int64_t host_pool_bytes;      /* pinned, mapped host memory holding the
                                   * streams' pending events (a ring per stream,
                                   * grown on demand) and frame slots
                                   * (frame_slots x W x H each); 0 = default
                                   * (512 MB)                                  */
} esi_server_opts;

/* esi_server_opts.apply_mode.  EVERY_TICK: each tick applies every stream's
 * pushed events up to the tick's time, so a frame's tick has only the newest
 * events left; each tick then reads and writes the state of every tile that
 * received an event.  AT_FRAMES: a stream's events wait on the host until the
 * tick that renders its next frame (or until 65536 events are pending), so
 * each tile's state is read and written about once per frame.  Both give the
 * same results; EVERY_TICK keeps frame ticks short (lower p99 latency),
 * AT_FRAMES does less device work per event. */
#define ESI_APPLY_EVERY_TICK 1
#define ESI_APPLY_AT_FRAMES 2

/* Latencies in milliseconds over the frames finished since the last reset:
 * frame latency = frame ready - the tick call that rendered it;
 * packet-to-frame latency = frame ready - the push of the stream's newest
 * packet at that tick (the packet that made the frame renderable). */
typedef struct {
    uint64_t ticks;
    uint64_t frames;
    uint64_t events;
    uint64_t packets;
    double frame_latency_p50_ms;
    double frame_latency_p99_ms;
    double packet_latency_p50_ms;
    double packet_latency_p99_ms;
    double gpu_ms_per_tick;       /* mean device time of a tick's kernels   */
    uint64_t state_bytes_used;
    uint64_t state_budget_bytes;
    int32_t streams_open;
    int32_t kernel_launches_per_tick;
    uint64_t streams_admitted;    /* esi_stream_open calls that succeeded     */
    uint64_t streams_refused;     /* ESI_EBUSY answers (admission refused)    */
    uint64_t events_refused;      /* executor events of refused streams      */
    double host_tick_p50_ms;      /* host time of a tick call with work: packing */
    double host_tick_p99_ms;      /*   the events and tables, queueing the work  */
    double gpu_tick_p99_ms;       /* device time of a tick's kernels, 99th pct  */
    uint64_t host_pool_bytes;     /* pinned host pool of the event rings        */
    uint64_t host_pool_used_bytes;  /* held by rings now (retired ones included) */
    uint64_t host_pool_peak_bytes;  /* the most held since the last reset        */
    uint64_t ring_grows;          /* rings moved into larger ones              */
    uint64_t events_dropped;      /* x >= W or y >= H: never applied (as of the
                                   * last esi_server_sync or state read)      */
} esi_server_stats;

typedef struct esi_server esi_server;

/* opts may be NULL (defaults); cuda_stream as in esi_create. */
int esi_server_create(size_t state_budget_bytes, const esi_server_opts *opts,
                      void *cuda_stream, esi_server **out);

/* Open a width x height stream (params as in esi_create); ESI_EBUSY when
 * its state does not fit the budget or max_streams streams are open. */
int esi_stream_open(esi_server *srv, int width, int height, const esi_params *params,
                    int *stream_id);

/* Queue one packet of n host events (time-ordered, not earlier than the
 * stream's last event or last frame); copied before the call returns. */
int esi_stream_push(esi_server *srv, int stream_id, const esi_event *ev, size_t n);

/* Declare that every event of the stream with t <= t_us has been pushed (the
 * end time of the packet just pushed).  Once a stream has a watermark, its
 * frames become due at t_frame <= min(now_us, watermark) and a tick applies
 * its events up to that time; without one, now_us alone decides. */
int esi_stream_watermark(esi_server *srv, int stream_id, int64_t t_us);

/* Process every stream up to now_us (see above). */
int esi_server_tick(esi_server *srv, int64_t now_us);

/* Copy the newest finished frame (W * H bytes) of a stream into the host
 * buffer out; ESI_ESTATE if none has finished yet.  t_frame, latency_ms
 * (frame latency as in esi_server_stats) may be NULL. */
int esi_stream_frame(esi_server *srv, int stream_id, uint8_t *out, int64_t *t_frame,
                     double *latency_ms);

/* Frames by number, for callers that read less often than frames finish:
 * frame seq (0, 1, ... in frame-time order) of a stream is held until frame
 * seq + frame_slots is handed to a tick.  esi_stream_frames_done writes the
 * number of the stream's finished frames; esi_stream_frame_seq copies frame
 * seq (W * H bytes) into the host buffer out and its time into *t_frame (may
 * be NULL): ESI_ESTATE if it has not finished, ESI_ERANGE if its slot has
 * been reused. */
int esi_stream_frames_done(esi_server *srv, int stream_id, uint64_t *n_done);
/* Keep every frame: from now on, each finished frame seq < max_frames of the
 * stream is also copied by the host, when its tick is seen finished, to
 * out + seq * W * H (a host buffer of max_frames * W * H bytes), and its time
 * to t_frames[seq] (may be NULL).  max_frames = 0 removes the sink.  The
 * buffers must stay valid until the stream closes or the sink is removed. */
int esi_stream_set_frame_sink(esi_server *srv, int stream_id, uint8_t *out,
                              uint64_t max_frames, int64_t *t_frames);
int esi_stream_frame_seq(esi_server *srv, int stream_id, uint64_t seq, uint8_t *out,
                         int64_t *t_frame);

/* Tile height (4, 8 or 16 rows of 128 pixels) of one stream's work items
 * from the next tick on; the state layout does not depend on it.  ESI_ERANGE
 * when the stream would have more tiles than the server's tables hold. */
int esi_stream_set_tile_h(esi_server *srv, int stream_id, int tile_h);

/* Autotune one stream's tile height: time a host sample of its events (n,
 * time-ordered, any time range) rendered at the server's frame period for
 * each tile height on a scratch sensor of the same size and parameters (as
 * esi_autotune), then apply the fastest (esi_stream_set_tile_h) and write it
 * to *tile_h (may be NULL).  Choices are cached per (W, H, events-per-frame
 * bucket, render mode, decay kind) for the process; ESI_AUTOTUNE_FORCE
 * measures again.  The stream's state and pending events are untouched. */
int esi_stream_autotune(esi_server *srv, int stream_id, const esi_event *sample, size_t n,
                        int flags, int *tile_h);

/* Copy a stream's state (as esi_get_state with host buffers) after every
 * pushed event with t <= the latest tick's time has been applied (events the
 * apply mode held back are applied first); waits. */
int esi_stream_state(esi_server *srv, int stream_id, float *S, int64_t *T);

/* Close a stream.  Returns at once: the id may be reused by the next open;
 * ticks already queued still finish its work and deliver its frames to its
 * frame sink, and its state, ring and frame slots go back to the budget and
 * the host pool when they are done (esi_stream_open waits for them when it
 * needs that memory). */
int esi_stream_close(esi_server *srv, int stream_id);

/* Wait for all queued ticks.  Returns a failure the device detected in them
 * (ESI_ETIMEOUT: a bounded wait in a kernel gave up; esi_server_last_error
 * says which), once and for every later call. */
int esi_server_sync(esi_server *srv);

int esi_server_get_stats(esi_server *srv, esi_server_stats *out);

/* What the server's last failed call ran into (a CUDA error, the host pool
 * being full, the executor's packet), or "" when no call has failed.  The
 * string stays valid until the next call on the server. */
const char *esi_server_last_error(esi_server *srv);

/* One finished tick that had work, as the server saw it.  Host times are in
 * nanoseconds since the server's creation (steady clock); device times come
 * from CUDA events on the server's stream. */
typedef struct {
    int64_t call_ns;      /* esi_server_tick called                               */
    int64_t issued_ns;    /* its copies and kernels queued (the call returns)     */
    int64_t ready_ns;     /* its completion stamp: its frames readable (may come
                           * before issued_ns: a small tick can finish on the
                           * device before its call returns)                    */
    float copy_ms;        /* device: the tick's table copy                         */
    float kernels_ms;     /* device: the tick's kernels                           */
    float gap_ms;         /* device: from the previous traced tick's end to this
                           * tick's start; near 0 when it queued behind it; -1 for
                           * the first                                              */
    int32_t frames;       /* frames it rendered                                    */
    int64_t events;       /* events it applied                                     */
    int32_t streams;      /* streams with work                                     */
    int32_t items;        /* (stream, tile) work items                             */
} esi_tick_trace;

/* Copy the trace of the last finished ticks (at most 65536 are kept, since
 * the last esi_server_reset_stats), oldest first: up to cap records into out,
 * the number copied into *n.  out may be NULL with cap 0 to ask for *n. */
int esi_server_trace(esi_server *srv, esi_tick_trace *out, size_t cap, size_t *n);
int esi_server_reset_stats(esi_server *srv);
void esi_server_destroy(esi_server *srv);

/* One packet of a stream for the executors below. */
#define ESI_PACKET_EVENTS 0  /* n events at ev                                      */
#define ESI_PACKET_OPEN 1    /* esi_server_run: the stream joins; ev points to an
                                esi_stream_spec                                    */
#define ESI_PACKET_CLOSE 2   /* esi_server_run: the stream leaves                  */
typedef struct {
    int32_t stream;       /* esi_server_run: the caller's stream slot (below);
                             esi_plain_run: stream index                       */
    int32_t kind;         /* ESI_PACKET_*; esi_plain_run takes only EVENTS     */
    int64_t arrival_us;   /* arrival time; the stream is complete up to it    */
    const esi_event *ev;  /* the packet's host events                          */
    uint64_t n;
} esi_packet;

/* A stream that joins during esi_server_run (ESI_PACKET_OPEN); caller-owned,
 * valid for the call.  The executor writes stream_id. */
typedef struct {
    int32_t width, height;
    int32_t tile_h;       /* 0: the server's default; else 4, 8 or 16         */
    int32_t stream_id;    /* out: the server stream id while it is open, -1
                             once refused admission or closed               */
    esi_params params;    /* frames at params.t_origin_us + k * frame period   */
    uint8_t *frame_sink;  /* NULL, or a frame sink as esi_stream_set_frame_sink */
    uint64_t sink_frames;
    int64_t *sink_t_frames;
} esi_stream_spec;

/*
 * Serving executor: feeds packets (sorted by arrival_us) to the server as
 * they arrive (esi_stream_push, then esi_stream_watermark(arrival_us)) and
 * ticks every tick_us of stream time until t_end_us, then waits for the
 * device.  realtime = 1 paces stream time with the wall clock (stream time 0
 * = the call), so latencies are those of live serving: a packet that makes
 * its stream's frame due is followed by a tick at once (at most one every
 * tick_us / 5), before the packets queued behind it are taken; realtime = 0
 * advances tick by tick as fast as host and device allow (throughput).
 *
 * Streams join and leave on the packets' schedule.  An OPEN packet opens a
 * stream (esi_stream_open, then its tile height) and binds the packet's slot
 * to it; when admission is refused (ESI_EBUSY) the slot's later packets are
 * dropped and counted (streams_refused, events_refused).  A CLOSE packet
 * renders the slot's frames that are due (up to its last packet), then closes
 * the stream (esi_stream_close); its events
 * after its last frame are discarded.  After the last tick the executor ticks
 * again at t_end_us until every due frame is issued, then waits.
 * A slot that no OPEN packet of this call has bound names a server stream id
 * directly (streams opened before the call).  Slots are in [0, 2^20).  Other
 * errors end the call.
 */
int esi_server_run(esi_server *srv, const esi_packet *packets, size_t n_packets,
                   int64_t tick_us, int64_t t_end_us, int realtime);

/*
 * The same workload without batching, for comparison: one esi_handle per
 * stream; at every tick each stream renders its due frames with its own
 * esi_render_frame calls (host output, no graph).  Fills out's counters and
 * latencies with the definitions of esi_server_stats.
 */
int esi_plain_run(int n_streams, const int *widths, const int *heights,
                  const esi_params *params, const esi_packet *packets, size_t n_packets,
                  int64_t tick_us, int64_t t_end_us, int64_t frame_period_us, int realtime,
                  esi_server_stats *out);

/* ---------------------------------------------- allocation-free render */

/*
 * The paper has no counterpart to this call; it is an interface of this
 * library.  It renders like esi_render_frames but allocates no memory at all,
 * for callers that cannot allocate device memory: applications that reserve
 * the GPU's memory up front in their own pool and forbid any other
 * allocation, plugins that must not go around their host framework's
 * allocator, and real-time loops in which cudaMalloc / cudaFree, which may
 * synchronise the whole device, would stall other work.
 *
 * The scratch it needs (binned records, run table, per-frame constants,
 * status) lives in one fixed device array of about 12.2 MB that every GPU
 * which loads this library holds until the process exits.  The first call on
 * each device sets that device up (it looks up the array's device address and
 * the kernels' shared-memory limits, with that device current); make that
 * first call before any stream capture.  All calls share the array, so calls
 * that overlap on the GPU (other streams, other host threads) race and must
 * be serialised by the caller.  Each call synchronises the stream it is
 * given (it reads the device-side checks back) before it returns.
 *
 * Inputs and outputs, all owned by the caller:
 *   events    device array of n events, 16-byte aligned (ESI_EINVAL
 *             otherwise: the events are staged by 16-byte bulk copies),
 *             non-decreasing in time (ESI_ETIMEORDER), none later than
 *             t_frames[m-1] (ESI_EINVAL) or earlier than its pixel's T
 *             (ESI_ETIMEORDER); out-of-range pixels are skipped.  n may be 0.
 *             An input error is found before any state changes: S, T and
 *             frames are then left as they were.
 *   t_frames  host array of m non-decreasing frame times.
 *   S, T      device arrays of W * H float32 / int64 with their natural
 *             alignment (ESI_EINVAL otherwise): the state, read and updated
 *             in place (start from S = 0, T = t_origin).  When S and T are
 *             16-byte aligned and W % 4 == 0 (and frames 4-byte aligned) the
 *             kernels move four pixels per access; otherwise one at a time.
 *   frames    device array of m * W * H bytes, frame w at offset w * W * H.
 * Limits (ESI_ERANGE beyond them): n <= 1048576 events, m <= 4096 frames,
 * ceil(W / 128) * ceil(H / 8) <= 2048 pixel tiles, and the last event at
 * most 2^32 - 1 us after the first.  params as for esi_create; render_decay
 * is honoured.
 */
int esi_render_frames_noalloc(int width, int height, const esi_params *params,
                              const esi_event *events, size_t n,
                              const int64_t *t_frames, size_t m, float *S,
                              int64_t *T, uint8_t *frames, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* ESI_H */
