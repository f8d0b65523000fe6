// sm_103a kernels of the ESI hot path.
//
//   esi_bin_kernel   one block per chunk of consecutive events: bulk-copies
//                    the chunk into shared memory (TMA), validates x < W,
//                    y < H, and writes the chunk's events as 8-byte records
//                    stably sorted by pixel tile, plus the chunk's column of
//                    the tile-major (start, count) run table.  Events of one
//                    tile stay in arrival (= time) order: ranks come from
//                    same-tile peer masks (one ballot per tile-index bit)
//                    over warp slices that are themselves in order.
//   esi_tile_kernel  one block per tile, one warp per tile row (esi_tile.cuh):
//                    gathers the tile's runs from every chunk in chunk order
//                    (so arrival order is kept), stable-sorts each batch by
//                    row in shared memory, and walks each row frame by frame:
//                    the due records 32 at a time through Alg. 2, then the
//                    Eq. 14 codes of the row's pixels at the frame.
//   esi_push_check_kernel  time-order check of a large push on the device.
//   esi_push_unpack_kernel the same for packed 8-byte events, which it
//                          widens into the ring's 16-byte slots.
//
// Per-pixel independence (each pixel's state depends only on its own
// time-ordered events, Eq. 5 and Alg. 2) is what makes the reorder legal.
#include <algorithm>
#include <cstdint>

#include "esi_device.cuh"
#include "esi_internal.h"
#include "esi_tile.cuh"

namespace esi {

constexpr int kBinThreads = 256;
constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // 1 s

static __host__ __device__ inline int round_up(int v, int m) { return (v + m - 1) / m * m; }

// Shared-memory layout of the binning kernel.  The staged events' 16-byte
// slots are reused: once phase 1 has read event k, slot k's first half holds
// its record, and phase 3 sorts the records into the slots' second halves.
static __host__ __device__ inline size_t bin_layout(int chunk, int n_tiles, bool mask,
                                                    size_t *off_tstart, size_t *off_cnt)
{
    constexpr int NW = kBinThreads / 32;
    size_t o = 0;
    o += (size_t)chunk * 16;                       // staged events, then records
    *off_tstart = o;
    o += (size_t)round_up(n_tiles + 1, 4) * 4;     // tile starts (+ total)
    *off_cnt = o;
    o += (size_t)NW * round_up(n_tiles, 8) * 2;    // per-warp tile counters
    o += (size_t)chunk * 2;                        // event: offset within its warp's tile run
    o += (size_t)chunk * 2;                        // event: tile (0xffff = dropped)
    if (mask)
        o += (size_t)NW * kBinMaskSlots * 4;       // per-warp lane masks (kept zero)
    return o;
}

// Shared memory for chunks of `chunk` events over at most n_tiles tiles.
size_t bin_smem_bytes(int chunk, int n_tiles, bool mask)
{
    size_t a, b;
    return bin_layout(chunk, n_tiles, mask, &a, &b);
}

// Whether chunks over up to n_tiles tiles can take the mask-word layout.
bool bin_mask_fits(int chunk, int n_tiles)
{
    return bin_smem_bytes(chunk, n_tiles, true) + 1024 <= (size_t)kMaxSmemPerBlock;
}

// One chunk of events: block-level body shared by the single-sensor and the
// batched binning kernels.  cidx is the chunk's index within a.n's events.
// EV: also write each record's event index (a.rec_idx) and NaN for events
// outside the sensor (a.ev_out), for esi_event_states.  PLAIN: the block
// reads the chunk with 16-byte loads instead of a bulk copy (the serving
// tick's events stay in mapped host memory).
template <bool EV = false, bool PLAIN = false>
__device__ __forceinline__ void bin_chunk(const BinArgs &a, int cidx)
{
    constexpr int NT = kBinThreads, NW = NT / 32;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bar;
    __shared__ unsigned scan_tmp[NW + 1];
    __shared__ unsigned s_drop;

    const int chunk = a.chunk, n_tiles = a.n_tiles;
    const int ntp = round_up(n_tiles, 8);
    const bool use_mask = a.use_mask != 0;
    size_t off_tstart, off_cnt;
    bin_layout(chunk, n_tiles, use_mask, &off_tstart, &off_cnt);
    int4 *sev = reinterpret_cast<int4 *>(smem);
    // slot k: record of event k (first half), sorted record k (second half)
    unsigned long long *srec = reinterpret_cast<unsigned long long *>(smem);
    unsigned *tstart = reinterpret_cast<unsigned *>(smem + off_tstart);
    unsigned short *cnt = reinterpret_cast<unsigned short *>(smem + off_cnt);
    unsigned short *loff = cnt + NW * ntp;
    unsigned short *ltile = loff + chunk;
    unsigned *tmask = reinterpret_cast<unsigned *>(ltile + chunk);   // [NW][kBinMaskSlots]

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long c0 = (long long)cidx * chunk;
    const int nc = (int)min((long long)chunk, (long long)a.n - c0);

    if (tid == 0) {
        if (!PLAIN) mbar_init(&bar, 1);
        s_drop = 0;
    }
    __syncthreads();
    if (PLAIN) {
        const int4 *src = reinterpret_cast<const int4 *>(a.ring);
        const unsigned long long f0 = a.first + (unsigned long long)c0;
#pragma unroll 4
        for (int i = tid; i < nc; i += NT) sev[i] = src[(f0 + (unsigned long long)i) & a.ring_mask];
    }
    if (!PLAIN && tid == 0) {
        // the chunk's ring range may wrap around the end of the ring
        const unsigned long long cap = a.ring_mask + 1ull;
        const unsigned long long r0 = (a.first + (unsigned long long)c0) & a.ring_mask;
        const int n1 = (int)min((unsigned long long)nc, cap - r0);
        mbar_expect_tx(&bar, (unsigned)nc * 16u);
        bulk_g2s_stream(sev, a.ring + r0, (unsigned)n1 * 16u, &bar);
        if (n1 < nc) bulk_g2s_stream(sev + n1, a.ring, (unsigned)(nc - n1) * 16u, &bar);
    }
    __shared__ int s_copy_ok;
    // counters (NW * ntp u16, a multiple of 8, 16-byte aligned) and mask
    // words to zero, 16 bytes at a time
    for (int i = tid; i < NW * ntp / 8; i += NT) reinterpret_cast<uint4 *>(cnt)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (use_mask)
        for (int i = tid; i < NW * kBinMaskSlots / 4; i += NT)
            reinterpret_cast<uint4 *>(tmask)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (PLAIN && tid == 0) s_copy_ok = 1;
    if (!PLAIN && tid == 0) {
        // one thread waits for the copy; the others sleep at the barrier
        int ok = mbar_wait_bounded(&bar, 0, kWaitLimitNs) ? 1 : 0;
        if (!ok) {
            // never read a partial chunk: report, give the copy one more
            // bounded wait so it does not land in reassigned shared memory
            set_error(a.status, ESI_ETIMEOUT, kWhereBinCopy);
            mbar_wait_bounded(&bar, 0, kWaitLimitNs);
        }
        s_copy_ok = ok;
    }
    __syncthreads();
    if (!s_copy_ok) return;

    const int W = a.W, H = a.H, tiles_x = a.tiles_x, thl = a.th_log2, tbits = a.tile_bits;
    const int twl = a.tw_log2;
    const int per = chunk / NW;
    const int s0 = warp * per;
    const int s1 = min(s0 + per, nc);

    // phase 1: in arrival order, each warp ranks its slice's events within
    // their tile (peers by mask words and ballots), keeping the offset inside
    // its own run, and turns each event into its record in place
    const int th_mask = (1 << thl) - 1;
    unsigned drop = 0;
    for (int base = s0; base < s1; base += 32) {
        const int k = base + lane;
        int tile = -1;
        if (k < s1) {
            const int4 e = sev[k];
            const int x = e.z & 0xffff, y = (int)((unsigned)e.z >> 16);
            if (x < W && y < H) {
                tile = (y >> thl) * tiles_x + (x >> twl);
                const long long t = ((long long)(unsigned)e.y << 32) | (unsigned)e.x;
                const unsigned pit = ((unsigned)(y & th_mask) << twl) | (unsigned)(x & ((1 << twl) - 1));
                const bool pos = (signed char)(e.w & 0xff) > 0;
                srec[2 * k] = make_record((unsigned)(t - a.t_base), pit, pos ? 1u : 0u);
            } else {
                ++drop;
                if constexpr (EV) a.ev_out[c0 + k] = __int_as_float(0x7fc00000);
            }
        }
        const bool valid = tile >= 0;
        unsigned peers;
        if (use_mask) {
            // each lane sets its bit in its tile's mask word (slot tile mod
            // kBinMaskSlots), reads the word and clears it once every lane
            // has read; lanes whose tiles share the slot are told apart by
            // one ballot per higher tile-index bit
            unsigned *mw = tmask + warp * kBinMaskSlots + (valid ? (tile & (kBinMaskSlots - 1)) : 0);
            if (valid) atomicOr(mw, 1u << lane);
            __syncwarp();
            peers = valid ? *mw : 0u;
            __syncwarp();
            if (valid) *mw = 0u;
            for (int b = kBinMaskSlotBits; b < tbits; ++b) {
                const bool bit = (tile >> b) & 1;
                const unsigned v = __ballot_sync(kFull, bit);
                peers &= bit ? v : ~v;
            }
        } else {
            peers = warp_peers((unsigned)tile, tbits, valid);
        }
        const unsigned rank = __popc(peers & lanemask_lt());
        const unsigned pre = valid ? cnt[warp * ntp + tile] : 0u;
        __syncwarp();
        if (valid && rank == 0) cnt[warp * ntp + tile] = (unsigned short)(pre + __popc(peers));
        if (k < s1) {
            loff[k] = (unsigned short)(pre + rank);
            ltile[k] = valid ? (unsigned short)tile : (unsigned short)0xffff;
        }
        __syncwarp();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) drop += __shfl_xor_sync(kFull, drop, o);
    if (lane == 0 && drop) atomicAdd(&s_drop, drop);
    __syncthreads();

    // phase 2: warp offsets within each tile, tile starts within the chunk;
    // two tiles per 32-bit word of counters (counts stay below 2^16)
    for (int j2 = tid; j2 < ntp / 2; j2 += NT) {
        unsigned run_lo = 0, run_hi = 0;
        for (int w = 0; w < NW; ++w) {
            unsigned *p2 = reinterpret_cast<unsigned *>(cnt + w * ntp) + j2;
            const unsigned v = *p2;
            *p2 = run_lo | (run_hi << 16);
            run_lo += v & 0xffffu;
            run_hi += v >> 16;
        }
        const int j = 2 * j2;
        if (j < n_tiles) tstart[j] = run_lo;
        if (j + 1 < n_tiles) tstart[j + 1] = run_hi;
    }
    __syncthreads();
    const unsigned total = block_exclusive_scan<NT>(tstart, n_tiles, scan_tmp);
    if (tid == 0) tstart[n_tiles] = total;
    __syncthreads();
    // tile-major run table: a tile reads its runs of every chunk contiguously
    const size_t n_chunks_all = ((size_t)a.n + a.chunk - 1) / a.chunk;
    for (int j = tid; j < n_tiles; j += NT)
        a.hrow[(size_t)j * n_chunks_all + cidx] = (tstart[j] << 16) | (tstart[j + 1] - tstart[j]);

    // phase 3: every record to its stable place in tile order (the second
    // halves of the slots); each warp scatters the slice it ranked
    const int w = warp;
    for (int k = warp * per + lane; k < min(nc, (warp + 1) * per); k += 32) {
        const unsigned tile = ltile[k];
        if (tile == 0xffffu) continue;
        const unsigned q = tstart[tile] + cnt[w * ntp + tile] + loff[k];
        srec[2 * q + 1] = srec[2 * k];
        if constexpr (EV) a.rec_idx[c0 + q] = (unsigned)(c0 + k);
    }
    __syncthreads();

    // phase 4: the chunk's records, tile-sorted, to global memory
    unsigned long long *dst = a.rec + c0;
    for (unsigned i = tid; i < total; i += NT) dst[i] = srec[2 * i + 1];
    if (tid == 0 && s_drop) atomicAdd(&a.status->dropped, (unsigned long long)s_drop);
}

__global__ void __launch_bounds__(kBinThreads) esi_bin_kernel(BinArgs a) { bin_chunk(a, blockIdx.x); }

__global__ void __launch_bounds__(kBinThreads) esi_bin_ev_kernel(BinArgs a) { bin_chunk<true>(a, blockIdx.x); }

// Batched binning of a serving tick: a persistent grid walks the tick's
// chunks; the tick directory names the stream segment (job) each chunk
// belongs to.
__global__ void __launch_bounds__(kBinThreads) esi_bin_tab_kernel(const unsigned char *tab)
{
    const TickDir *d = reinterpret_cast<const TickDir *>(tab);
    const int n = d->n_chunks;
    const BinJob *jobs = reinterpret_cast<const BinJob *>(tab + d->off_binjob);
    const int *cj = reinterpret_cast<const int *>(tab + d->off_chunkjob);
    for (int c = blockIdx.x; c < n; c += gridDim.x) {
        const BinJob &j = jobs[cj[c]];
        bin_chunk<false, true>(j.args, c - j.first_chunk);
        __syncthreads();  // shared memory (and the copy barrier) serve the next chunk
    }
}

// Until the counter reaches need (bounded by limit_ns): the acquire load
// orders the reads that follow after the writes released before each add.
__device__ __forceinline__ bool wait_count(const unsigned *p, unsigned need, unsigned long long limit_ns)
{
    const unsigned long long t0 = global_ns();
    for (;;) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
        if (v >= need) return true;
        if (global_ns() - t0 > limit_ns) return false;
        __nanosleep(128);
    }
}

// A whole serving tick in one launch (streams with 8-row tiles, one render
// mode and decay kind; the row alignment is read per stream).  The blocks
// take the tick's binning chunks from a counter in the tick table until none
// is left, then walk the tile items grid-stride; a block reaches the items
// only after every chunk has been taken by a running block, so its wait for
// a stream's chunks always ends.
template <int RD, int DK>
__global__ void __launch_bounds__(kBinThreads) esi_tick_fused_kernel(const unsigned char *tab)
{
    static_assert(kBinThreads == 8 * 32, "one warp per row of an 8-row tile");
    const TickDir *d = reinterpret_cast<const TickDir *>(tab);
    const BinJob *bjobs = reinterpret_cast<const BinJob *>(tab + d->off_binjob);
    const int *cj = reinterpret_cast<const int *>(tab + d->off_chunkjob);
    const TileArgs *tjobs = reinterpret_cast<const TileArgs *>(tab + d->off_tilejob);
    const int2 *items = reinterpret_cast<const int2 *>(tab + d->fused_off_items);
    unsigned *sync = reinterpret_cast<unsigned *>(const_cast<unsigned char *>(tab) + d->off_sync);
    const int n_chunks = d->n_chunks, n_items = d->fused_n_items;
    __shared__ int s_w, s_ok;
    for (;;) {
        if (threadIdx.x == 0) s_w = (int)atomicAdd(&sync[0], 1u);
        __syncthreads();
        const int w = s_w;
        if (w >= n_chunks) break;
        const int j = cj[w];
        bin_chunk<false, true>(bjobs[j].args, w - bjobs[j].first_chunk);
        __syncthreads();  // every record and run entry of the chunk is written; s_w is read
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(&sync[1 + j], 1u);
        }
    }
    for (int i = blockIdx.x; i < n_items; i += gridDim.x) {
        const int2 it = items[i];
        if (threadIdx.x == 0) {
            const BinArgs &ba = bjobs[it.x].args;
            const unsigned need = (unsigned)((ba.n + ba.chunk - 1) / ba.chunk);
            s_ok = wait_count(&sync[1 + it.x], need, kWaitLimitNs) ? 1 : 0;
            if (!s_ok) set_error(ba.status, ESI_ETIMEOUT, kWhereTickWait);
            __threadfence();
        }
        __syncthreads();
        if (s_ok) tile_body<8, 4, RD, DK, false, false, true>(tjobs[it.x], it.y);
        __syncthreads();  // shared memory serves the next item; s_ok is rewritten
    }
}

size_t tick_fused_smem_bytes(int chunk, int max_tiles, bool mask, int batch, int max_chunks)
{
    const size_t b = bin_smem_bytes(chunk, max_tiles, mask);
    const size_t t = tile_smem_bytes(8, batch, max_chunks);
    return b > t ? b : t;
}

#define ESI_TICK_FUSED_VARIANTS X(0, kDecayGeneral) X(0, kDecaySquare) X(0, kDecayNone) \
    X(1, kDecayGeneral) X(1, kDecaySquare) X(1, kDecayNone)

int tick_fused_blocks_per_sm(int rd, int dk, size_t smem)
{
    int nb = 0;
    cudaError_t e = cudaErrorInvalidValue;
#define X(RD, DK) \
    if (rd == RD && dk == DK) \
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, esi_tick_fused_kernel<RD, DK>, kBinThreads, smem);
    ESI_TICK_FUSED_VARIANTS
#undef X
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

cudaError_t launch_tick_fused(const unsigned char *tab, int grid, int rd, int dk, size_t smem,
                              cudaStream_t s)
{
#define X(RD, DK)                                                                        \
    if (rd == RD && dk == DK) {                                                          \
        esi_tick_fused_kernel<RD, DK><<<grid, kBinThreads, smem, s>>>(tab);              \
        return cudaGetLastError();                                                       \
    }
    ESI_TICK_FUSED_VARIANTS
#undef X
    return cudaErrorInvalidValue;
}

// Dynamic shared memory a kernel may ask for: the 227 KB per block minus its
// static part.
cudaError_t allow_dynamic_smem_impl(const void *kernel)
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    const int max_dyn = kMaxSmemPerBlock - (int)fa.sharedSizeBytes;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn);
}

size_t tile_smem_bytes(int tile_h, int batch, int n_chunks)
{
    size_t a, b, c, d;
    return tile_layout(batch, n_chunks, tile_h, &a, &b, &c, &d);
}


size_t tile_smem_bytes_ev(int tile_h, int batch, int n_chunks)
{
    size_t a, b;
    return tile_layout_ev(batch, n_chunks, tile_h, &a, &b);
}

size_t tile_static_smem_bytes(int tile_h, int tile_w)
{
    // pixel state (S, F, O and a peer mask per pixel), staged frames and the
    // sort scratch
    return (size_t)tile_h * tile_w * 20 + (size_t)kStageFrames * sizeof(WinInfo) +
           (size_t)tile_h * tile_h * 2 + 1024;
}

int decay_kind_of(const DecayParams &dp)
{
    if (dp.b_mode == 4) return kDecayNone;
    if (dp.b_mode == 2) return kDecaySquare;
    return kDecayGeneral;
}

cudaError_t set_kernel_attributes()
{
    cudaError_t e = allow_dynamic_smem_impl((const void *)esi_bin_kernel);
    if (e == cudaSuccess) e = allow_dynamic_smem_impl((const void *)esi_bin_ev_kernel);
    if (e == cudaSuccess) e = allow_dynamic_smem_impl((const void *)esi_bin_tab_kernel);
#define X(RD, DK) \
    if (e == cudaSuccess) e = allow_dynamic_smem_impl((const void *)esi_tick_fused_kernel<RD, DK>);
    ESI_TICK_FUSED_VARIANTS
#undef X
    if (e == cudaSuccess) e = set_tile_attributes_w128();
    if (e == cudaSuccess) e = set_tile_attributes_w32();
    if (e == cudaSuccess) e = set_tile_attributes_w64();
    if (e == cudaSuccess) e = set_tile_split_attributes();
    return e;
}

cudaError_t launch_bin(const BinArgs &a, int n_chunks, cudaStream_t s)
{
    const size_t smem = bin_smem_bytes(a.chunk, a.n_tiles, a.use_mask != 0);
    if (a.rec_idx)
        esi_bin_ev_kernel<<<n_chunks, kBinThreads, smem, s>>>(a);
    else
        esi_bin_kernel<<<n_chunks, kBinThreads, smem, s>>>(a);
    return cudaGetLastError();
}

int bin_tab_blocks_per_sm(int chunk, int max_tiles, bool mask)
{
    int nb = 0;
    const size_t smem = bin_smem_bytes(chunk, max_tiles, mask);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, esi_bin_tab_kernel, kBinThreads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

cudaError_t launch_bin_batch_tab(const unsigned char *tab, int grid, int chunk, int max_tiles,
                                 bool mask, cudaStream_t s)
{
    const size_t smem = bin_smem_bytes(chunk, max_tiles, mask);
    esi_bin_tab_kernel<<<grid, kBinThreads, smem, s>>>(tab);
    return cudaGetLastError();
}

cudaError_t launch_tile(const TileArgs &a, int tile_h, int tile_w, bool vec, cudaStream_t s)
{
    if (tile_w == 32) return launch_tile_w32(a, tile_h, s);
    if (tile_w == 64) return launch_tile_w64(a, tile_h, vec, s);
    return launch_tile_w128(a, tile_h, vec, s);
}

cudaError_t launch_tile_ev(const TileArgs &a, int tile_h, int tile_w, cudaStream_t s)
{
    if (tile_w == 32) return launch_tile_ev_w32(a, tile_h, s);
    if (tile_w == 64) return launch_tile_ev_w64(a, tile_h, s);
    return launch_tile_ev_w128(a, tile_h, s);
}

cudaError_t launch_tile_batch_tab(const unsigned char *tab, int group, int grid, int tile_h, int rd,
                                  int dk, bool vec, int batch, int max_chunks, cudaStream_t s)
{
    return launch_tile_tab_w128(tab, group, grid, tile_h, rd, dk, vec, batch, max_chunks, s);
}

}  // namespace esi

namespace esi {

__global__ void esi_fill_i64_kernel(long long *dst, long long n, long long value)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = value;
}

__global__ void esi_push_check_kernel(const esi_event *ring, unsigned long long mask,
                                      unsigned long long a0, unsigned long long first, long long cnt,
                                      unsigned long long n, long long prev, unsigned long long g0,
                                      long long *sparse, PushResult *res)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < cnt;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long k = first + (unsigned long long)i;
        const unsigned long long g = a0 + k;
        const long long t = ring[g & mask].t_us;
        const long long tp = k ? ring[(g - 1) & mask].t_us : prev;
        if (t < tp) res->bad = 1;
        if (g % kSparse == 0) sparse[(g - g0) / kSparse] = t;
        if (k == n - 1) res->last = t;
    }
}

cudaError_t launch_push_check(const esi_event *ring, unsigned long long mask, unsigned long long a0,
                              unsigned long long first, long long cnt, unsigned long long n,
                              long long prev, unsigned long long g0, long long *sparse,
                              PushResult *res, cudaStream_t s)
{
    if (cnt <= 0) return cudaSuccess;
    const long long blocks = std::min<long long>((cnt + 255) / 256, 152LL * 8);
    esi_push_check_kernel<<<(unsigned)blocks, 256, 0, s>>>(ring, mask, a0, first, cnt, n, prev, g0,
                                                           sparse, res);
    return cudaGetLastError();
}

// The same checks for packed words: word i of src becomes ring slot a0 +
// first + i (one 16-byte store), its time compared with word i - 1's (the
// ring slot before it, written by the previous launch, at i = 0).
__global__ void esi_push_unpack_kernel(const unsigned long long *src, esi_event *ring,
                                       unsigned long long mask, unsigned long long a0,
                                       unsigned long long first, long long cnt,
                                       unsigned long long n, long long t_base, long long prev,
                                       unsigned long long g0, long long *sparse, PushResult *res)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < cnt;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long k = first + (unsigned long long)i;
        const unsigned long long g = a0 + k;
        const unsigned long long w = src[i];
        const long long t = t_base + (long long)(w >> kPackTShift);
        // x, y as they are; polarity byte 1 or -1 (0xff); padding 0
        const unsigned long long xyp =
            (w & 0xffffffffull) | ((w >> 32) & 1ull ? 0x01ull : 0xffull) << 32;
        *reinterpret_cast<longlong2 *>(ring + (g & mask)) = make_longlong2(t, (long long)xyp);
        const long long tp = i ? t_base + (long long)(src[i - 1] >> kPackTShift)
                               : (k ? ring[(g - 1) & mask].t_us : prev);
        if (t < tp) res->bad = 1;
        if (g % kSparse == 0) sparse[(g - g0) / kSparse] = t;
        if (k == n - 1) res->last = t;
    }
}

cudaError_t launch_push_unpack(const unsigned long long *src, esi_event *ring,
                               unsigned long long mask, unsigned long long a0,
                               unsigned long long first, long long cnt, unsigned long long n,
                               long long t_base, long long prev, unsigned long long g0,
                               long long *sparse, PushResult *res, cudaStream_t s)
{
    if (cnt <= 0) return cudaSuccess;
    const long long blocks = std::min<long long>((cnt + 255) / 256, 152LL * 8);
    esi_push_unpack_kernel<<<(unsigned)blocks, 256, 0, s>>>(src, ring, mask, a0, first, cnt, n,
                                                            t_base, prev, g0, sparse, res);
    return cudaGetLastError();
}

cudaError_t launch_fill_i64(long long *dst, long long n, long long value, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const long long blocks = std::min<long long>((n + 255) / 256, 152LL * 8);
    esi_fill_i64_kernel<<<(unsigned)blocks, 256, 0, s>>>(dst, n, value);
    return cudaGetLastError();
}

}  // namespace esi
