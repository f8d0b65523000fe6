// sm_103a kernels of the ESI hot path.
//
//   esi_bin_kernel   one block per chunk of consecutive events: bulk-copies
//                    the chunk into shared memory (TMA), validates x < W,
//                    y < H, and writes the chunk's events as 8-byte records
//                    stably sorted by pixel tile, plus the chunk's per-tile
//                    (start, count) row.  Events of one tile stay in arrival
//                    (= time) order: ranks come from warp match_any over warp
//                    slices that are themselves in order.
//   esi_tile_kernel  one block per 128 x TH pixel tile (one warp per row, four
//                    pixels per lane): gathers the tile's runs from every
//                    chunk in chunk order (so arrival order is kept),
//                    stable-sorts each batch by row and then by lane in shared
//                    memory, and lets every lane walk its own pixels' events
//                    through Alg. 2, emitting the Eq. 14 codes of its four
//                    pixels (one 32-bit store) at every frame time.
//
// Per-pixel independence (each pixel's state depends only on its own
// time-ordered events, Eq. 5 and Alg. 2) is what makes the reorder legal.
#include <algorithm>
#include <cstdint>

#include "esi_device.cuh"
#include "esi_internal.h"

namespace esi {

constexpr int kBinThreads = 256;
constexpr int kStageFrames = 256;   // per-frame constants a tile block keeps in shared memory
constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // 1 s
constexpr int kWhereBinCopy = 1;

static __host__ __device__ inline int round_up(int v, int m) { return (v + m - 1) / m * m; }

// Shared-memory layout of the binning kernel.
static __host__ __device__ inline size_t bin_layout(int chunk, int n_tiles, size_t *off_sort,
                                                    size_t *off_tstart, size_t *off_cnt)
{
    constexpr int NW = kBinThreads / 32;
    size_t o = 0;
    o += (size_t)chunk * 16;                       // staged events
    *off_sort = o;
    o += (size_t)chunk * 8;                        // sorted records
    *off_tstart = o;
    o += (size_t)round_up(n_tiles + 1, 4) * 4;     // tile starts (+ total)
    *off_cnt = o;
    o += (size_t)NW * round_up(n_tiles, 8) * 2;    // per-warp tile counters
    o += (size_t)chunk * 2;                        // event: offset within its warp's tile run
    o += (size_t)chunk * 2;                        // event: tile (0xffff = dropped)
    return o;
}

size_t bin_smem_bytes(int chunk, int n_tiles)
{
    size_t a, b, c;
    return bin_layout(chunk, n_tiles, &a, &b, &c);
}

// One chunk of events: block-level body shared by the single-sensor and the
// batched binning kernels.  cidx is the chunk's index within a.n's events.
__device__ __forceinline__ void bin_chunk(const BinArgs &a, int cidx)
{
    constexpr int NT = kBinThreads, NW = NT / 32;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bar;
    __shared__ unsigned scan_tmp[NW + 1];
    __shared__ unsigned s_drop;

    const int chunk = a.chunk, n_tiles = a.n_tiles;
    const int ntp = round_up(n_tiles, 8);
    size_t off_sort, off_tstart, off_cnt;
    bin_layout(chunk, n_tiles, &off_sort, &off_tstart, &off_cnt);
    int4 *sev = reinterpret_cast<int4 *>(smem);
    unsigned long long *ssort = reinterpret_cast<unsigned long long *>(smem + off_sort);
    unsigned *tstart = reinterpret_cast<unsigned *>(smem + off_tstart);
    unsigned short *cnt = reinterpret_cast<unsigned short *>(smem + off_cnt);
    unsigned short *loff = cnt + NW * ntp;
    unsigned short *ltile = loff + chunk;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long c0 = (long long)cidx * chunk;
    const int nc = (int)min((long long)chunk, (long long)a.n - c0);

    if (tid == 0) {
        mbar_init(&bar, 1);
        s_drop = 0;
    }
    __syncthreads();
    if (tid == 0) {
        // the chunk's ring range may wrap around the end of the ring
        const unsigned long long cap = a.ring_mask + 1ull;
        const unsigned long long r0 = (a.first + (unsigned long long)c0) & a.ring_mask;
        const int n1 = (int)min((unsigned long long)nc, cap - r0);
        mbar_expect_tx(&bar, (unsigned)nc * 16u);
        bulk_g2s(sev, a.ring + r0, (unsigned)n1 * 16u, &bar);
        if (n1 < nc) bulk_g2s(sev + n1, a.ring, (unsigned)(nc - n1) * 16u, &bar);
    }
    __shared__ int s_copy_ok;
    for (int i = tid; i < NW * ntp; i += NT) cnt[i] = 0;
    if (tid == 0) {
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
    const int per = chunk / NW;
    const int s0 = warp * per;
    const int s1 = min(s0 + per, nc);

    // phase 1: in arrival order, each warp ranks its slice's events within
    // their tile (peers by ballot), keeping the offset inside its own run
    unsigned drop = 0;
    for (int base = s0; base < s1; base += 32) {
        const int k = base + lane;
        int tile = -1;
        if (k < s1) {
            const int4 e = sev[k];
            const int x = e.z & 0xffff, y = (int)((unsigned)e.z >> 16);
            if (x < W && y < H)
                tile = (y >> thl) * tiles_x + (x >> 7);
            else
                ++drop;
        }
        const bool valid = tile >= 0;
        const unsigned peers = warp_peers((unsigned)tile, tbits, valid);
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

    // phase 2: warp offsets within each tile, tile starts within the chunk
    for (int j = tid; j < n_tiles; j += NT) {
        unsigned run = 0;
        for (int w = 0; w < NW; ++w) {
            const unsigned v = cnt[w * ntp + j];
            cnt[w * ntp + j] = (unsigned short)run;
            run += v;
        }
        tstart[j] = run;
    }
    __syncthreads();
    const unsigned total = block_exclusive_scan<NT>(tstart, n_tiles, scan_tmp);
    if (tid == 0) tstart[n_tiles] = total;
    __syncthreads();
    unsigned *hrow = a.hrow + (size_t)cidx * n_tiles;
    for (int j = tid; j < n_tiles; j += NT)
        hrow[j] = (tstart[j] << 16) | (tstart[j + 1] - tstart[j]);

    // phase 3: scatter every event to its stable place in tile order
    const int th_mask = (1 << thl) - 1;
    for (int k = tid; k < nc; k += NT) {
        const unsigned tile = ltile[k];
        if (tile == 0xffffu) continue;
        const int4 e = sev[k];
        const int x = e.z & 0xffff, y = (int)((unsigned)e.z >> 16);
        const long long t = ((long long)(unsigned)e.y << 32) | (unsigned)e.x;
        const unsigned pit = ((unsigned)(y & th_mask) << 7) | (unsigned)(x & 127);
        const bool pos = (signed char)(e.w & 0xff) > 0;
        const int w = k / per;
        ssort[tstart[tile] + cnt[w * ntp + tile] + loff[k]] =
            make_record((unsigned)(t - a.t_base), pit, pos ? 1u : 0u);
    }
    __syncthreads();

    // phase 4: the chunk's records, tile-sorted, to global memory
    unsigned long long *dst = a.rec + c0;
    for (unsigned i = tid; i < total; i += NT) dst[i] = ssort[i];
    if (tid == 0 && s_drop) atomicAdd(&a.status->dropped, (unsigned long long)s_drop);
}

__global__ void __launch_bounds__(kBinThreads) esi_bin_kernel(BinArgs a) { bin_chunk(a, blockIdx.x); }

// Batched binning of a serving tick: block c bins chunk c of the tick; the
// tick directory names the stream segment (job) each chunk belongs to.  The
// grid is sized for the capacity; blocks past the tick's chunks return.
__global__ void __launch_bounds__(kBinThreads) esi_bin_tab_kernel(const unsigned char *tab)
{
    const TickDir *d = reinterpret_cast<const TickDir *>(tab);
    const int c = blockIdx.x;
    if (c >= d->n_chunks) return;
    const BinJob *jobs = reinterpret_cast<const BinJob *>(tab + d->off_binjob);
    const int *cj = reinterpret_cast<const int *>(tab + d->off_chunkjob);
    const BinJob &j = jobs[cj[c]];
    bin_chunk(j.args, c - j.first_chunk);
}

// Shared-memory layout of the tile kernel (dynamic part).
static __host__ __device__ inline size_t tile_layout(int batch, int n_chunks, size_t *off_b,
                                                     size_t *off_runpre, size_t *off_runoff,
                                                     size_t *off_lpos)
{
    size_t o = (size_t)(batch + 2) * 8;   // batch + the next batch's first record
    *off_b = o;
    o += (size_t)batch * 8;
    *off_runpre = o;
    o += (size_t)round_up(n_chunks + 1, 4) * 4;
    *off_runoff = o;
    o += (size_t)round_up(n_chunks, 4) * 4;
    *off_lpos = o;                   // record: offset inside its warp's row run
    o += (size_t)round_up(batch, 8) * 2;
    return o;
}

size_t tile_smem_bytes(int tile_h, int batch, int n_chunks)
{
    (void)tile_h;
    size_t a, b, c, d;
    return tile_layout(batch, n_chunks, &a, &b, &c, &d);
}

// Largest c in [0, n) with pre[c] <= g (pre[0] = 0 <= g < pre[n]).
__device__ __forceinline__ int run_of(const unsigned *pre, int n, unsigned g)
{
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] <= g) lo = mid; else hi = mid;
    }
    return lo;
}

// One block per 128 x TH tile; warp w owns tile row w, lane l owns the four
// pixels x = 4l .. 4l + 3 of that row for loads, stores and frame codes.
// Events are applied event-parallel: a row's records are in time order, so at
// each frame the due records go 32 at a time, one per lane; lanes holding the
// same pixel (match_any) apply theirs in arrival order, rank by rank, to the
// pixel state kept in shared memory.  RD: render_decay; DK: decay kind; VEC:
// rows start 4-byte aligned (W % 4 == 0), so a lane's four pixels move as one
// float4 / two longlong2 / one 32-bit frame word.
template <int TH, int RD, int DK, bool VEC>
__device__ __forceinline__ void tile_body(const TileArgs &a, int tile)
{
    constexpr int NT = TH * 32;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ unsigned short rcnt[TH][TH];   // [warp][row] counts, then offsets
    constexpr int RB = (TH == 4) ? 2 : (TH == 8) ? 3 : (TH == 16) ? 4 : 5;  // bits of a row index
    __shared__ unsigned rowstart[TH + 1];
    __shared__ unsigned scan_tmp[NT / 32 + 1];
    __shared__ long long s_tnext;
    __shared__ WinInfo swin[kStageFrames];              // this launch's frames, if they fit
    __shared__ __align__(16) float sS[TH][kTileW];      // S of the tile's pixels
    __shared__ __align__(16) float sF[TH][kTileW];      // (float)(T - t_base)
    __shared__ __align__(16) long long sO[TH][kTileW];  // T - t_base

    const int R = a.batch, n_chunks = a.n_chunks;
    size_t off_b, off_runpre, off_runoff, off_lpos;
    tile_layout(R, n_chunks, &off_b, &off_runpre, &off_runoff, &off_lpos);
    unsigned long long *A = reinterpret_cast<unsigned long long *>(smem);
    unsigned long long *B = reinterpret_cast<unsigned long long *>(smem + off_b);
    unsigned *runpre = reinterpret_cast<unsigned *>(smem + off_runpre);
    unsigned *runoff = reinterpret_cast<unsigned *>(smem + off_runoff);
    unsigned short *lpos = reinterpret_cast<unsigned short *>(smem + off_lpos);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int x0 = (tile % a.tiles_x) * kTileW + 4 * lane;
    const int y = (tile / a.tiles_x) * TH + warp;
    const int nval = (y < a.H) ? max(0, min(4, a.W - x0)) : 0;
    const long long pix0 = (long long)y * a.W + x0;
    const long long tb = a.t_base;
    const DecayParams dp = a.dp;
    const MapParams mp = a.mp;
    float *rS = sS[warp];
    float *rF = sF[warp];
    long long *rO = sO[warp];

    // this tile's run in every chunk, in chunk (= arrival) order
    for (int c = tid; c < n_chunks; c += NT) {
        const unsigned h = a.hrow[(size_t)c * a.n_tiles + tile];
        runpre[c] = h & 0xffffu;
        runoff[c] = h >> 16;
    }
    // the launch's per-frame constants, staged in shared memory when they fit
    const int nwin = a.w_end - a.w_begin;
    const bool staged = nwin <= kStageFrames;
    if (staged)
        for (int i = tid; i < nwin; i += NT) swin[i] = a.win[a.w_begin + i];
    __syncthreads();
    const unsigned total = block_exclusive_scan<NT>(runpre, n_chunks, scan_tmp);
    if (tid == 0) runpre[n_chunks] = total;
    __syncthreads();
    // a tile with no record and no frame in this launch keeps its state as is
    if (total == 0 && a.w_end == a.w_begin) return;

    {
        float s4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        long long o4[4] = {0, 0, 0, 0};
        if (VEC && nval == 4) {
            const float4 v = *reinterpret_cast<const float4 *>(a.S + pix0);
            const longlong2 t01 = *reinterpret_cast<const longlong2 *>(a.T + pix0);
            const longlong2 t23 = *reinterpret_cast<const longlong2 *>(a.T + pix0 + 2);
            s4[0] = v.x; s4[1] = v.y; s4[2] = v.z; s4[3] = v.w;
            o4[0] = t01.x - tb; o4[1] = t01.y - tb; o4[2] = t23.x - tb; o4[3] = t23.y - tb;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (q < nval) {
                    s4[q] = a.S[pix0 + q];
                    o4[q] = a.T[pix0 + q] - tb;
                }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            rS[4 * lane + q] = s4[q];
            rO[4 * lane + q] = o4[q];
            rF[4 * lane + q] = RD ? __ll2float_rn(o4[q]) : 0.0f;
        }
    }


    // Alg. 2 for a group of due records (one per valid lane, time order):
    // S += p C; dt = t - T; S *= d(dt); T = t; clamp (Eq. 13)
    auto apply_group = [&](unsigned long long r, bool valid) {
        const int x = (int)((r >> 33) & 127u);
        const unsigned peers = warp_peers_n<7>((unsigned)x, valid);
        const unsigned rank = __popc(peers & lanemask_lt());
        const unsigned maxr = __reduce_max_sync(kFull, valid ? rank : 0u);
        for (unsigned k = 0; k <= maxr; ++k) {
            if (valid && rank == k) {
                const unsigned toff = (unsigned)r;
                float s = rS[x] + (((r >> 32) & 1u) ? mp.C : -mp.C);
                s = s * decay_state_k<DK>((long long)toff - rO[x], dp);
                rS[x] = fminf(fmaxf(s, mp.s_min), mp.s_max);
                rO[x] = (long long)toff;
                if (RD) rF[x] = __uint2float_rn(toff);
            }
            __syncwarp();
        }
    };

    int wi = a.w_begin;
    for (unsigned b0 = 0;; b0 += (unsigned)R) {
        const int nb = (int)min((unsigned)R, total - min(total, b0));
        const bool last = b0 + (unsigned)R >= total;

        // gather the batch (records b0 .. b0 + nb of this tile, arrival
        // order, plus the next batch's first record): one thread per run,
        // asynchronous copies, so every record of the batch is in flight
        const unsigned next = last ? 0u : 1u;
        if (nb > 0) {
            const unsigned bend = b0 + (unsigned)nb + next;
            const int cfirst = run_of(runpre, n_chunks, b0);
            const int clast = run_of(runpre, n_chunks, bend - 1u);
            for (int c = cfirst + tid; c <= clast; c += NT) {
                const unsigned rs = max(runpre[c], b0), re = min(runpre[c + 1], bend);
                const unsigned long long *src =
                    a.rec + (size_t)c * a.chunk + runoff[c] + (rs - runpre[c]);
                for (unsigned i = 0; i + rs < re; ++i) cp_async8(&A[rs - b0 + i], src + i);
            }
        }
        cp_async_wait_all();
        __syncthreads();
        if (tid == 0) s_tnext = last ? 0x7fffffffffffffffll : (long long)(unsigned)A[nb];
        for (int i = tid; i < TH * TH; i += NT) (&rcnt[0][0])[i] = 0;
        __syncthreads();

        // stable counting sort of the batch by row (A -> B): each row's
        // records stay in arrival (= time) order
        const int sl = (nb + TH - 1) / TH;
        const int s0 = min(warp * sl, nb), s1 = min(s0 + sl, nb);
        for (int base = s0; base < s1; base += 32) {
            const int k = base + lane;
            const bool valid = k < s1;
            const int row = valid ? (int)(A[k] >> 40) : 0;
            const unsigned peers = warp_peers_n<RB>((unsigned)row, valid);
            const unsigned rank = __popc(peers & lanemask_lt());
            const unsigned pre = valid ? rcnt[warp][row] : 0u;
            __syncwarp();
            if (valid && rank == 0) rcnt[warp][row] = (unsigned short)(pre + __popc(peers));
            if (valid) lpos[k] = (unsigned short)(pre + rank);
            __syncwarp();
        }
        __syncthreads();
        {
            const int row = tid / TH, w = tid % TH;
            const unsigned v = (tid < TH * TH) ? rcnt[w][row] : 0u;
            unsigned tot;
            const unsigned ex = block_exclusive_scan1<NT>(v, scan_tmp, &tot);
            if (tid < TH * TH) {
                rcnt[w][row] = (unsigned short)ex;
                if (w == 0) rowstart[row] = ex;
            }
            if (tid == 0) rowstart[TH] = (unsigned)nb;
        }
        __syncthreads();
        for (int k = tid; k < nb; k += NT) {
            const unsigned long long r = A[k];
            const int row = (int)(r >> 40);
            B[rcnt[k / max(sl, 1)][row] + lpos[k]] = r;
        }
        __syncthreads();

        // walk this warp's row, frame by frame
        int cur = (int)rowstart[warp];
        const int re = (int)rowstart[warp + 1];
        const long long tnext = s_tnext;
        while (wi < a.w_end) {
            const WinInfo wv = staged ? swin[wi - a.w_begin] : a.win[wi];
            if (wv.lim >= tnext) break;  // later records of this tile may be due
            for (;;) {
                const int k = cur + lane;
                unsigned long long r = 0;
                bool valid = false;
                if (k < re) {
                    r = B[k];
                    valid = (long long)(unsigned)r <= wv.lim;
                }
                const unsigned vm = __ballot_sync(kFull, valid);
                if (vm == 0u) break;
                apply_group(r, valid);
                const int nv = __popc(vm);
                cur += nv;
                if (nv < 32) break;
            }
            // Eq. 14 codes of the lane's four pixels at this frame
            const float4 s4 = *reinterpret_cast<const float4 *>(rS + 4 * lane);
            float v[4] = {s4.x, s4.y, s4.z, s4.w};
            if (RD) {
                const float4 f4 = *reinterpret_cast<const float4 *>(rF + 4 * lane);
                v[0] *= decay_view_k<DK>(wv.tf_f - f4.x, dp);
                v[1] *= decay_view_k<DK>(wv.tf_f - f4.y, dp);
                v[2] *= decay_view_k<DK>(wv.tf_f - f4.z, dp);
                v[3] *= decay_view_k<DK>(wv.tf_f - f4.w, dp);
            }
            unsigned code[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) code[q] = quantize_u8(fmaf(v[q], mp.scale, mp.offs));
            unsigned char *fr =
                (a.frame_outs ? a.frame_outs[wi] : a.frames + (long long)wi * a.P) + pix0;
            if (VEC) {
                if (nval == 4)
                    *reinterpret_cast<unsigned *>(fr) =
                        code[0] | (code[1] << 8) | (code[2] << 16) | (code[3] << 24);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (q < nval) fr[q] = (unsigned char)code[q];
            }
            ++wi;
        }
        // the rest of this batch's row precedes the next batch's records
        for (; cur < re; cur += 32) {
            const int k = cur + lane;
            const bool valid = k < re;
            apply_group(valid ? B[k] : 0ull, valid);
        }
        if (last) break;
        __syncthreads();  // A, B, rcnt are rewritten by the next batch
    }

    __syncwarp();
    if (VEC && nval == 4) {
        const float4 s4 = *reinterpret_cast<const float4 *>(rS + 4 * lane);
        *reinterpret_cast<float4 *>(a.S + pix0) = s4;
        *reinterpret_cast<longlong2 *>(a.T + pix0) =
            make_longlong2(rO[4 * lane] + tb, rO[4 * lane + 1] + tb);
        *reinterpret_cast<longlong2 *>(a.T + pix0 + 2) =
            make_longlong2(rO[4 * lane + 2] + tb, rO[4 * lane + 3] + tb);
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (q < nval) {
                a.S[pix0 + q] = rS[4 * lane + q];
                a.T[pix0 + q] = rO[4 * lane + q] + tb;
            }
    }
}

#define ESI_TILE_BOUNDS(TH) __launch_bounds__(TH * 32, (TH * 32 >= 1024) ? 1 : 1024 / (TH * 32))

template <int TH, int RD, int DK, bool VEC>
__global__ void ESI_TILE_BOUNDS(TH) esi_tile_kernel(TileArgs a)
{
    tile_body<TH, RD, DK, VEC>(a, blockIdx.x);
}

// Batched tiles of a serving tick: a persistent grid walks the work items
// (stream job, tile) of one parameter variant group.
template <int TH, int RD, int DK, bool VEC>
__global__ void ESI_TILE_BOUNDS(TH) esi_tile_tab_kernel(const unsigned char *tab, int group)
{
    const TickDir *d = reinterpret_cast<const TickDir *>(tab);
    const int n = d->n_items[group];
    const int2 *items = reinterpret_cast<const int2 *>(tab + d->off_items[group]);
    const TileArgs *jobs = reinterpret_cast<const TileArgs *>(tab + d->off_tilejob);
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const int2 it = items[i];
        tile_body<TH, RD, DK, VEC>(jobs[it.x], it.y);
        __syncthreads();  // shared memory is reused by the next item
    }
}

#define ESI_TILE_VARIANTS(TH)                                                     \
    X(TH, 0, kDecayGeneral, false) X(TH, 0, kDecayGeneral, true)                  \
    X(TH, 0, kDecaySquare, false) X(TH, 0, kDecaySquare, true)                    \
    X(TH, 0, kDecayNone, false) X(TH, 0, kDecayNone, true)                        \
    X(TH, 1, kDecayGeneral, false) X(TH, 1, kDecayGeneral, true)                  \
    X(TH, 1, kDecaySquare, false) X(TH, 1, kDecaySquare, true)                    \
    X(TH, 1, kDecayNone, false) X(TH, 1, kDecayNone, true)

static int decay_kind(const DecayParams &dp)
{
    if (dp.b_mode == 4) return kDecayNone;
    if (dp.b_mode == 2) return kDecaySquare;
    return kDecayGeneral;
}

// Dynamic shared memory a kernel may ask for: the 227 KB per block minus its
// static part.
template <class K>
static cudaError_t allow_dynamic_smem(K kernel)
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    const int max_dyn = kMaxSmemPerBlock - (int)fa.sharedSizeBytes;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn);
}

size_t tile_static_smem_bytes(int tile_h)
{
    // pixel state (S, F, O per pixel), staged frames and the sort scratch
    return (size_t)tile_h * kTileW * 16 + (size_t)kStageFrames * sizeof(WinInfo) +
           (size_t)tile_h * tile_h * 2 + 1024;
}

cudaError_t set_kernel_attributes()
{
    cudaError_t e = allow_dynamic_smem(esi_bin_kernel);
    if (e == cudaSuccess) e = allow_dynamic_smem(esi_bin_tab_kernel);
    if (e != cudaSuccess) return e;
#define X(TH, RD, DK, V)                                                                    \
    e = allow_dynamic_smem(esi_tile_kernel<TH, RD, DK, V>);                                 \
    if (e == cudaSuccess) e = allow_dynamic_smem(esi_tile_tab_kernel<TH, RD, DK, V>);       \
    if (e != cudaSuccess) return e;
    ESI_TILE_VARIANTS(4)
    ESI_TILE_VARIANTS(8)
    ESI_TILE_VARIANTS(16)
    ESI_TILE_VARIANTS(32)
#undef X
    return cudaSuccess;
}

cudaError_t launch_bin(const BinArgs &a, int n_chunks, cudaStream_t s)
{
    const size_t smem = bin_smem_bytes(a.chunk, a.n_tiles);
    esi_bin_kernel<<<n_chunks, kBinThreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_bin_batch_tab(const unsigned char *tab, int grid, int chunk, int max_tiles,
                                 cudaStream_t s)
{
    const size_t smem = bin_smem_bytes(chunk, max_tiles);
    esi_bin_tab_kernel<<<grid, kBinThreads, smem, s>>>(tab);
    return cudaGetLastError();
}

cudaError_t launch_tile_batch_tab(const unsigned char *tab, int group, int grid, int tile_h, int rd,
                                  int dk, bool vec, int batch, int max_chunks, cudaStream_t s)
{
    const size_t smem = tile_smem_bytes(tile_h, batch, max_chunks);
#define X(TH, RD, DK, V)                                                                  \
    if (tile_h == TH && rd == RD && dk == DK && vec == V) {                               \
        esi_tile_tab_kernel<TH, RD, DK, V><<<grid, TH * 32, smem, s>>>(tab, group);       \
        return cudaGetLastError();                                                        \
    }
    ESI_TILE_VARIANTS(4)
    ESI_TILE_VARIANTS(8)
    ESI_TILE_VARIANTS(16)
    ESI_TILE_VARIANTS(32)
#undef X
    return cudaErrorInvalidValue;
}

int decay_kind_of(const DecayParams &dp) { return decay_kind(dp); }

cudaError_t launch_tile(const TileArgs &a, int tile_h, bool vec, cudaStream_t s)
{
    const size_t smem = tile_smem_bytes(tile_h, a.batch, a.n_chunks);
    const int rd = a.mp.render_decay ? 1 : 0;
    const int dk = decay_kind(a.dp);
#define X(TH, RD, DK, V)                                                          \
    if (tile_h == TH && rd == RD && dk == DK && vec == V) {                       \
        esi_tile_kernel<TH, RD, DK, V><<<a.n_tiles, TH * 32, smem, s>>>(a);       \
        return cudaGetLastError();                                                \
    }
    ESI_TILE_VARIANTS(4)
    ESI_TILE_VARIANTS(8)
    ESI_TILE_VARIANTS(16)
    ESI_TILE_VARIANTS(32)
#undef X
    return cudaErrorInvalidValue;
}


}  // namespace esi

namespace esi {

__global__ void esi_fill_i64_kernel(long long *dst, long long n, long long value)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = value;
}

cudaError_t launch_fill_i64(long long *dst, long long n, long long value, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const long long blocks = std::min<long long>((n + 255) / 256, 152LL * 8);
    esi_fill_i64_kernel<<<(unsigned)blocks, 256, 0, s>>>(dst, n, value);
    return cudaGetLastError();
}

}  // namespace esi
