// esi_render_frames_noalloc: the render path with its scratch in a fixed
// device array, for callers that must not allocate device memory.
//
// The scratch is one file-scope __device__ array (kScratchBytes, about 12 MB)
// that every device which loads this library holds until the process exits.
// Host code may not use the array's name as a device address (in host code
// it names a host-side stand-in), so the first call on each device looks the
// address up with cudaGetSymbolAddress, with that device current, and keeps
// it.  Every call shares the array and finds the previous call's contents in
// it; the status words are cleared at the start of each call, and everything
// else a call reads is written by that call first.
#include <algorithm>
#include <climits>
#include <cstring>
#include <mutex>

#include "esi_api_impl.h"
#include "esi_internal.h"

namespace esi {
namespace {

constexpr int kNaChunk = 2048;          // events per binning block
constexpr int kNaTileH = 8;             // rows per tile
constexpr int kNaBatch = 4096;          // records per shared-memory batch
constexpr long long kNaMaxEvents = 1ll << 20;
constexpr int kNaMaxChunks = (int)(kNaMaxEvents / kNaChunk);
constexpr int kNaMaxTiles = 2048;
constexpr int kNaMaxFrames = 4096;

constexpr size_t kOffRec = 0;
constexpr size_t kOffHrow = kOffRec + (size_t)kNaMaxEvents * 8;
constexpr size_t kOffWin = kOffHrow + (size_t)kNaMaxChunks * kNaMaxTiles * 4;
constexpr size_t kOffTf = kOffWin + (size_t)kNaMaxFrames * sizeof(WinInfo);
constexpr size_t kOffStatus = kOffTf + (size_t)kNaMaxFrames * 8;
constexpr size_t kScratchBytes = kOffStatus + 256;

constexpr int kMaxDevices = 64;

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

std::mutex g_setup_mu;
unsigned char *g_scratch_dev[kMaxDevices] = {};

// Once per device, with that device current: the scratch array's device
// address and the kernels' shared-memory limits.
int setup_device(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= kMaxDevices) return ESI_ERANGE;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return ESI_ECUDA;
        e = set_kernel_attributes();
        if (e != cudaSuccess) return ESI_ECUDA;
        g_scratch_dev[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_dev[dev];
    return ESI_OK;
}

// Events must be in time order, inside the sensor's reach of time: not before
// their pixel's T, not after the last frame.
__global__ void esi_noalloc_check_kernel(const esi_event *ev, long long n, const long long *T,
                                         int W, int H, long long t_last, DevStatus *st)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long t = ev[i].t_us;
        if (i > 0 && t < ev[i - 1].t_us) atomicCAS(&st->err, 0, ESI_ETIMEORDER);
        if (t > t_last) atomicCAS(&st->err, 0, ESI_EINVAL);
        const int x = ev[i].x, y = ev[i].y;
        if (x < W && y < H && t < T[(long long)y * W + x]) atomicCAS(&st->err, 0, ESI_ETIMEORDER);
    }
}

// Per-frame constants relative to the first event's time (as the handle path
// computes them on the host).
__global__ void esi_noalloc_win_kernel(const long long *tf, int m, long long t_base, WinInfo *win)
{
    for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < m; w += gridDim.x * blockDim.x) {
        const long long d = tf[w] - t_base;
        win[w].lim = d < -1 ? -1 : (d > 0xffffffffll ? 0xffffffffll : d);
        win[w].tf_f = __ll2float_rn(d);
        win[w].pad = 0;
    }
}

int cuda_rc(cudaError_t e)
{
    if (e == cudaSuccess) return ESI_OK;
    return ESI_ECUDA;
}

}  // namespace
}  // namespace esi

using namespace esi;

extern "C" int esi_render_frames_noalloc(int width, int height, const esi_params *params,
                                         const esi_event *events, size_t n,
                                         const int64_t *t_frames, size_t m, float *S,
                                         int64_t *T, uint8_t *frames, void *cuda_stream)
{
    int rc = validate_params(width, height, params);
    if (rc) return rc;
    if ((n && !events) || !t_frames || m == 0 || !S || !T || !frames) return ESI_EINVAL;
    // the binning stages events with 16-byte bulk copies (TMA), whose global
    // source must be 16-byte aligned; S and T need their natural alignment
    if (n && (reinterpret_cast<uintptr_t>(events) & 15u)) return ESI_EINVAL;
    if ((reinterpret_cast<uintptr_t>(S) & 3u) || (reinterpret_cast<uintptr_t>(T) & 7u))
        return ESI_EINVAL;
    if (n > (size_t)kNaMaxEvents || m > (size_t)kNaMaxFrames) return ESI_ERANGE;
    const int tiles_x = (width + kTileW - 1) / kTileW;
    const int n_tiles = tiles_x * ((height + kNaTileH - 1) / kNaTileH);
    if (n_tiles > kNaMaxTiles) return ESI_ERANGE;
    for (size_t w = 1; w < m; ++w)
        if (t_frames[w] < t_frames[w - 1]) return ESI_ETIMEORDER;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ESI_ECUDA;
    unsigned char *scratch = nullptr;
    rc = setup_device(dev, &scratch);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    unsigned long long *rec = reinterpret_cast<unsigned long long *>(scratch + kOffRec);
    unsigned *hrow = reinterpret_cast<unsigned *>(scratch + kOffHrow);
    WinInfo *win = reinterpret_cast<WinInfo *>(scratch + kOffWin);
    long long *tf = reinterpret_cast<long long *>(scratch + kOffTf);
    DevStatus *st = reinterpret_cast<DevStatus *>(scratch + kOffStatus);

    DecayParams dp;
    MapParams mp;
    prepare_params(*params, &dp, &mp);
    const long long t_last_frame = t_frames[m - 1];

    long long t_ends[2] = {0, 0};
    if (n) {
        rc = cuda_rc(cudaMemcpyAsync(&t_ends[0], &events[0].t_us, 8, cudaMemcpyDeviceToHost, s));
        if (!rc) rc = cuda_rc(cudaMemcpyAsync(&t_ends[1], &events[n - 1].t_us, 8,
                                              cudaMemcpyDeviceToHost, s));
        if (!rc) rc = cuda_rc(cudaStreamSynchronize(s));
        if (rc) return rc;
        if (t_ends[1] - t_ends[0] > 0xffffffffll) return ESI_ERANGE;
    }
    const long long t_base = n ? t_ends[0] : t_frames[0];

    // status starts at zero on every call; inputs are checked before any state changes
    rc = cuda_rc(cudaMemsetAsync(st, 0, sizeof(DevStatus), s));
    if (!rc && n) {
        const long long blocks = std::min<long long>(((long long)n + 255) / 256, 152LL * 8);
        esi_noalloc_check_kernel<<<(unsigned)blocks, 256, 0, s>>>(
            events, (long long)n, reinterpret_cast<const long long *>(T), width, height,
            t_last_frame, st);
        rc = cuda_rc(cudaGetLastError());
    }
    if (rc) return rc;
    DevStatus hs;
    rc = cuda_rc(cudaMemcpyAsync(&hs, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    if (!rc) rc = cuda_rc(cudaStreamSynchronize(s));
    if (rc) return rc;
    if (hs.err) return hs.err;

    rc = cuda_rc(cudaMemcpyAsync(tf, t_frames, m * sizeof(long long), cudaMemcpyHostToDevice, s));
    if (rc) return rc;
    esi_noalloc_win_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(tf, (int)m, t_base, win);
    rc = cuda_rc(cudaGetLastError());
    if (rc) return rc;

    const int n_chunks = (int)((n + kNaChunk - 1) / kNaChunk);
    if (n) {
        BinArgs ba;
        ba.ring = events;
        ba.ring_mask = ~0ull >> 1;   // one contiguous buffer: never wraps
        ba.first = 0;
        ba.n = (int)n;
        ba.chunk = kNaChunk;
        ba.t_base = t_base;
        ba.W = width;
        ba.H = height;
        ba.tiles_x = tiles_x;
        ba.n_tiles = n_tiles;
        ba.th_log2 = 3;
        ba.tw_log2 = 7;
        ba.tile_bits = index_bits(n_tiles);
        ba.rec = rec;
        ba.hrow = hrow;
        ba.use_mask = 0;
        ba.status = st;
        rc = cuda_rc(launch_bin(ba, n_chunks, s));
        if (rc) return rc;
    }
    TileArgs ta;
    ta.rec = rec;
    ta.hrow = hrow;
    ta.n_chunks = n_chunks;
    ta.chunk = kNaChunk;
    ta.n_tiles = n_tiles;
    ta.t_base = t_base;
    ta.S = S;
    ta.T = reinterpret_cast<long long *>(T);
    ta.W = width;
    ta.H = height;
    ta.tiles_x = tiles_x;
    ta.dp = dp;
    ta.mp = mp;
    ta.win = win;
    ta.w_begin = 0;
    ta.w_end = (int)m;
    ta.frames = frames;
    ta.frame_outs = nullptr;
    ta.P = (long long)width * height;
    ta.batch = kNaBatch;
    ta.status = st;
    ta.scan_chain = kScanChainDefault;
    // the vector tile path moves a lane's four pixels as one float4 of S, two
    // 16-byte words of T and one 32-bit frame word: it needs S and T 16-byte
    // aligned and frames 4-byte aligned; otherwise the scalar path runs
    const bool vec = (width % 4 == 0) && ((reinterpret_cast<uintptr_t>(frames) & 3u) == 0) &&
                     (((reinterpret_cast<uintptr_t>(S) | reinterpret_cast<uintptr_t>(T)) & 15u) == 0);
    rc = cuda_rc(launch_tile(ta, kNaTileH, kTileW, vec, s));
    if (rc) return rc;
    rc = cuda_rc(cudaMemcpyAsync(&hs, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    if (!rc) rc = cuda_rc(cudaStreamSynchronize(s));
    if (rc) return rc;
    return hs.err;
}
