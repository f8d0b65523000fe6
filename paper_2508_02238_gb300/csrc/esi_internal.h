// Internal types shared by the ESI host code and its sm_103a kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "esi.h"

namespace esi {

constexpr int kTileW = 128;  // a tile row is one warp: lane l owns x = 4l .. 4l + 3
// Shortest same-pixel chain in a group of 32 records that the tile kernel
// composes with the segmented scan: the default, and the value that turns
// the scan off (a group holds at most 32 records).
constexpr int kScanChainDefault = 8;
constexpr int kScanNever = 33;
constexpr int kMaxSmemPerBlock = 227 * 1024;

// Decay of Eq. 4, d(dt) = max(1 - k dt, 0)^b, prepared for the device.
//   k_hi + k_lo is k per microsecond (k * 1e-6 in double) split into floats so
//   that 1 - k dt can be formed without cancellation error near the cutoff.
//   cutoff is the smallest integer dt with 1 - k dt <= 0 evaluated in double
//   (so the device takes the d = 0 decision in the same precision as the
//   definition); INT64_MAX when k = 0.
// b_mode of Eq. 3 read with d(t) = exp(-k t): S <- S d(dt) + p C.
constexpr int kBModeExp = 5;

struct DecayParams {
    float k_hi;
    float k_lo;
    float b;
    int b_mode;         // 0: powf; 1, 2, 3: integer b; 4: k == 0 (d = 1);
                        // 5: exp(-k t) with Eq. 3's order (kBModeExp)
    long long cutoff;   // d = 0 for dt >= cutoff
};

// Clamp of Eq. 13 and linear map of Eq. 14: B = rint(v * scale + offs).
struct MapParams {
    float C;
    float s_min;        // per-event clamp of Eq. 13 (-inf / +inf for the
    float s_max;        // methods without one: Alg. 1, Eq. 3)
    float scale;        // 255 / (s_max - s_min)
    float offs;         // -s_min * scale
    int render_decay;
};

// Device-side status, read back at synchronising calls.
struct DevStatus {
    unsigned long long dropped;   // events with x >= W or y >= H
    int err;                      // ESI_* code of a device-detected failure
    int err_where;                // which kernel / wait gave up (kWhere*)
};
constexpr int kWhereBinCopy = 1;   // the binning's bulk copy of its chunk
constexpr int kWhereTickWait = 2;  // a fused tick's tile item waiting for its stream's binning

// The binning finds same-tile lanes of a warp through kBinMaskSlots mask
// words per warp in shared memory, indexed by tile mod kBinMaskSlots, and one
// ballot per higher tile-index bit (or, without the words, one ballot per
// tile-index bit).
constexpr int kBinMaskSlotBits = 8;
constexpr int kBinMaskSlots = 1 << kBinMaskSlotBits;

// Result of a device-checked push: an order violation anywhere, and the time
// of the push's last event.
struct PushResult {
    int bad;
    int pad;
    long long last;
};

// Host pushes keep the time of every kSparse-th absolute ring index for
// planning (device-checked ones keep only those).
constexpr unsigned kSparse = 32;

// Packed events: time offset in the top 31 bits of the word (esi.h).
constexpr int kPackTShift = 33;

// Arguments of the binning kernel (one block per chunk of events).
struct BinArgs {
    const esi_event *ring;        // pending-event ring
    unsigned long long ring_mask; // capacity - 1 (capacity is a power of two)
    unsigned long long first;     // ring position of the sub-batch's first event
    int n;                        // events in the sub-batch
    int chunk;                    // events per block (power of two)
    long long t_base;             // record times are t - t_base (< 2^32)
    int W, H, tiles_x, n_tiles;
    int th_log2;                  // log2 of rows per tile
    int tw_log2;                  // log2 of pixels per tile row (5, 6 or 7)
    int tile_bits;                // bits of a tile index (n_tiles <= 2^tile_bits)
    unsigned long long *rec;      // out: records, block c at rec + c * chunk
    unsigned int *hrow;           // out: [tile][chunk] (start << 16 | count)
    int use_mask;                 // same-tile lanes by shared mask words
    DevStatus *status;
    // per-event output (esi_event_states; both set, or both null for renders):
    unsigned *rec_idx = nullptr;  // out: beside each record, its event's index in the sub-batch
    float *ev_out = nullptr;      // out: NaN at the index of every event outside the sensor
};

// Per-frame constants of one tile-kernel launch, relative to its t_base:
// lim = clamp(t_frame - t_base, -1, 2^32 - 1) decides which records are due
// (record offsets are < 2^32); tf_f = t_frame - t_base in FP32 feeds the
// render-time decay view.
struct WinInfo {
    long long lim;
    float tf_f;
    int pad;
};

// Arguments of the tile kernel (one block per 128 x TH pixel tile).
struct TileArgs {
    const unsigned long long *rec;
    const unsigned int *hrow;
    int n_chunks;
    int chunk;
    int n_tiles;
    long long t_base;
    float *S;
    long long *T;
    int W, H, tiles_x;
    DecayParams dp;
    MapParams mp;
    const WinInfo *win;           // per-frame constants (device), indexed by frame
    int w_begin, w_end;           // frames this launch completes
    unsigned char *frames;        // frame w at frames + w * P ...
    unsigned char *const *frame_outs;  // ... or at frame_outs[w] when this is set
    long long P;
    int batch;                    // records sorted per shared-memory batch
    DevStatus *status;
    // per-event output (esi_event_states' instantiations only; null otherwise)
    const unsigned *rec_idx = nullptr;  // event index (in the sub-batch) beside each record
    float *ev_out = nullptr;            // S right after each event, at its index
    // a group whose longest same-pixel chain has at least this many records
    // is composed by the segmented scan; shorter ones event by event
    // (kScanNever: always event by event, bit-identical across launch shapes)
    int scan_chain = kScanNever;
    // split-row tile kernel (esi_tile_split.cuh): scratch for every tile's
    // row-sorted records (srt_cap records; srt_top, zeroed before each
    // launch, hands out the tiles' regions) and the most splits of a round
    // (0: rows are walked whole, one warp each)
    unsigned long long *srt = nullptr;
    unsigned long long srt_cap = 0;
    unsigned long long *srt_top = nullptr;
    int max_splits = 0;
};

// One stream segment of a batched binning launch: the chunks
// first_chunk .. first_chunk + ceil(args.n / args.chunk) - 1 of the tick.
struct BinJob {
    BinArgs args;
    int first_chunk;
    int pad;
};

// Directory at the start of a serving tick's device table: the batched
// kernels find their sizes and descriptor arrays through it.
// tile height (3) x render mode (2) x decay kind (3) x row alignment (2)
constexpr int kTickGroups = 36;
struct TickDir {
    int n_chunks;
    int n_items[kTickGroups];
    int fused_n_items;            // work items of the fused tick launch
    int pad[2];
    long long off_binjob;
    long long off_chunkjob;
    long long off_tilejob;
    long long off_items[kTickGroups];
    long long fused_off_items;    // its items (a run of the groups' item lists)
    long long off_sync;           // u32 [0]: work counter; [1 + job]: the job's chunks binned
};

// Record layout (8 bytes): low 32 bits t - t_base; high 32 bits
// (pixel-in-tile << 1) | (p > 0), pixel-in-tile = row * tile width + x.
__host__ __device__ inline unsigned long long make_record(unsigned int toff,
                                                          unsigned int pit,
                                                          unsigned int pos)
{
    return (unsigned long long)toff | ((unsigned long long)((pit << 1) | pos) << 32);
}

// Bits needed to hold indices 0 .. n-1 (at least 1).
inline int index_bits(int n)
{
    int b = 1;
    while ((1 << b) < n) ++b;
    return b;
}

// Launchers (esi_kernels.cu).
size_t bin_smem_bytes(int chunk, int n_tiles, bool mask);
bool bin_mask_fits(int chunk, int n_tiles);
size_t tile_smem_bytes(int tile_h, int batch, int n_chunks);
// The same for the per-event-output instantiations (index arrays added).
size_t tile_smem_bytes_ev(int tile_h, int batch, int n_chunks);
size_t tile_static_smem_bytes(int tile_h, int tile_w);
cudaError_t launch_bin(const BinArgs &a, int n_chunks, cudaStream_t s);
cudaError_t launch_tile(const TileArgs &a, int tile_h, int tile_w, bool vec, cudaStream_t s);
// Tile kernel that writes S after every event (a.rec_idx, a.ev_out) and
// renders no frame (a.w_begin == a.w_end).
cudaError_t launch_tile_ev(const TileArgs &a, int tile_h, int tile_w, cudaStream_t s);
cudaError_t launch_tile_w128(const TileArgs &a, int tile_h, bool vec, cudaStream_t s);
// Split-row tile kernel (128-pixel rows; a.srt, a.srt_top set).
cudaError_t launch_tile_split(const TileArgs &a, int tile_h, bool vec, cudaStream_t s);
size_t tile_split_static_smem_bytes(int tile_h);
cudaError_t set_tile_split_attributes();
cudaError_t launch_tile_w32(const TileArgs &a, int tile_h, cudaStream_t s);
cudaError_t launch_tile_w64(const TileArgs &a, int tile_h, bool vec, cudaStream_t s);
cudaError_t launch_tile_ev_w128(const TileArgs &a, int tile_h, cudaStream_t s);
cudaError_t launch_tile_ev_w64(const TileArgs &a, int tile_h, cudaStream_t s);
cudaError_t launch_tile_ev_w32(const TileArgs &a, int tile_h, cudaStream_t s);
cudaError_t launch_tile_tab_w128(const unsigned char *tab, int group, int grid, int tile_h, int rd,
                                 int dk, bool vec, int batch, int max_chunks, cudaStream_t s);
cudaError_t set_tile_attributes_w128();
cudaError_t set_tile_attributes_w32();
cudaError_t set_tile_attributes_w64();
cudaError_t launch_bin_batch_tab(const unsigned char *tab, int grid, int chunk, int max_tiles,
                                 bool mask, cudaStream_t s);
// One launch for a whole serving tick whose streams all use 8-row tiles and
// share render mode rd and decay kind dk: a persistent grid takes the tick's
// binning chunks, then its tile items, from one counter; a tile item waits
// (bounded) until its stream's chunks are binned.
cudaError_t launch_tick_fused(const unsigned char *tab, int grid, int rd, int dk, size_t smem,
                              cudaStream_t s);
size_t tick_fused_smem_bytes(int chunk, int max_tiles, bool mask, int batch, int max_chunks);
int tick_fused_blocks_per_sm(int rd, int dk, size_t smem);
// Resident blocks per SM of the batched binning kernel (its persistent grid).
int bin_tab_blocks_per_sm(int chunk, int max_tiles, bool mask);
cudaError_t launch_tile_batch_tab(const unsigned char *tab, int group, int grid, int tile_h, int rd,
                                  int dk, bool vec, int batch, int max_chunks, cudaStream_t s);
int decay_kind_of(const DecayParams &dp);
cudaError_t set_kernel_attributes();

}  // namespace esi
