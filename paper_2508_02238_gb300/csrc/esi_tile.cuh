// Block-level body of the tile kernel (shared by the single-sensor, batched
// and 32-pixel-row instantiations).
#pragma once

#include "esi_device.cuh"
#include "esi_internal.h"

namespace esi {

constexpr int kStageFrames = 256;   // per-frame constants a tile block keeps in shared memory
#ifndef ESI_GATHER_LANES
#define ESI_GATHER_LANES 4
#endif
constexpr int kGatherLanes = ESI_GATHER_LANES;   // lanes copying one run of a batch

static __host__ __device__ inline int tile_round_up(int v, int m) { return (v + m - 1) / m * m; }

// Shared-memory layout of the tile kernel (dynamic part) for tiles of th
// rows: the gathered batch A, its row-sorted copy B, the run table, and the
// records' offsets within their warp's row runs, whose bytes hold the
// segmented scan's 32 event maps (16 bytes each) per warp while the warps
// walk B (A then receives the next batch).
static __host__ __device__ inline size_t tile_layout(int batch, int n_chunks, int th, size_t *off_b,
                                                     size_t *off_runpre, size_t *off_runoff,
                                                     size_t *off_lpos)
{
    size_t o = (size_t)(batch + 2) * 8;   // batch + the next batch's first record
    *off_b = o;
    o += (size_t)batch * 8;
    *off_runpre = o;
    o += (size_t)tile_round_up(n_chunks + 1, 4) * 4;
    *off_runoff = o;
    o += (size_t)tile_round_up(n_chunks, 4) * 4;
    *off_lpos = o;                   // record: offset inside its warp's row run
    const size_t lbytes = (size_t)tile_round_up(batch, 8) * 2, sbytes = (size_t)th * 32 * 16;
    o += lbytes > sbytes ? lbytes : sbytes;
    return o;
}

// Per-event output: two u32 index arrays beside A and B, after the layout.
static __host__ __device__ inline size_t tile_layout_ev(int batch, int n_chunks, int th, size_t *off_ia,
                                                        size_t *off_ib)
{
    size_t a, b, c, d;
    size_t o = tile_round_up((int)tile_layout(batch, n_chunks, th, &a, &b, &c, &d), 16);
    *off_ia = o;
    o += (size_t)(batch + 2) * 4;
    *off_ib = o;
    o += (size_t)batch * 4;
    return o;
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

// A group of due records with a long same-pixel chain, as a segmented scan.
// Each event is a monotone map of its pixel's state, f(S) = clamp(a S + b,
// lo, hi): Alg. 2 gives (d, d c, S_min, S_max) from S <- clamp((S + c) d),
// Alg. 1 the same without the clamp, Eq. 3 (exp) (d, c) from S <- S d + c.
// Such maps compose into maps of the same form (a >= 0 commutes with the
// clamp): g o f = (a_g a_f, a_g b_f + b_g, clamp(a_g lo_f + b_g, lo_g, hi_g),
// clamp(a_g hi_f + b_g, lo_g, hi_g)), and composition is associative.  The
// group's lanes are permuted so that each pixel's events sit in contiguous
// lanes in arrival order, an inclusive segmented scan composes each lane's
// prefix in log2(chain) shuffle steps, and every lane applies its prefix to
// the state its pixel had when the group started.  The rounding differs from
// the event-by-event loop by a few units in the last place.
// sc: this warp's 32 slots; peers / rank: the lane's same-pixel lanes and
// its place among them; maxr: the longest chain minus one.
template <int DK>
__device__ __forceinline__ float scan_group(float4 *sc, bool valid, unsigned peers, unsigned rank,
                                            float c, float d, float s_mem, unsigned maxr,
                                            const DecayParams &dp, const MapParams &mp)
{
    const int lane = threadIdx.x & 31;
    const bool clamped = mp.s_min > -INFINITY;   // Alg. 2 only
    const bool after = DK == kDecayGeneral && dp.b_mode == kBModeExp;
    // position of each event: its pixel's first position (an exclusive scan
    // of the chain lengths over the pixels' first lanes) plus its rank
    const bool lead = valid && rank == 0u;
    const unsigned len = lead ? (unsigned)__popc(peers) : 0u;
    const unsigned first_pos = warp_inclusive_scan(len) - len;
    const unsigned seg0 = __shfl_sync(kFull, first_pos, valid ? __ffs(peers) - 1 : lane);
    const unsigned starts = __reduce_or_sync(kFull, lead ? (1u << seg0) : 0u);
    const int nv = __popc(__ballot_sync(kFull, valid));
    if (valid) sc[seg0 + rank] = make_float4(d, after ? c : d * c, mp.s_min, mp.s_max);
    __syncwarp();
    float4 q = sc[lane];
    __syncwarp();
    const unsigned le = lane == 31 ? kFull : (2u << lane) - 1u;
    const int seg = lane < nv ? 31 - __clz(starts & le) : lane;   // start of this position's pixel
    for (int o = 1; o <= (int)maxr; o <<= 1) {
        const float pa = __shfl_up_sync(kFull, q.x, o);
        const float pb = __shfl_up_sync(kFull, q.y, o);
        float pl = 0.0f, ph = 0.0f;
        if (clamped) {
            pl = __shfl_up_sync(kFull, q.z, o);
            ph = __shfl_up_sync(kFull, q.w, o);
        }
        if (lane - o >= seg) {
            if (clamped) {
                const float lo = fminf(fmaxf(fmaf(q.x, pl, q.y), q.z), q.w);
                const float hi = fminf(fmaxf(fmaf(q.x, ph, q.y), q.z), q.w);
                q.z = lo;
                q.w = hi;
            }
            q.y = fmaf(q.x, pb, q.y);
            q.x *= pa;
        }
    }
    // back to the lane that holds the event: its prefix applied to the state
    // its pixel had when the group started
    const int src = valid ? (int)(seg0 + rank) : lane;
    const float A = __shfl_sync(kFull, q.x, src);
    const float B = __shfl_sync(kFull, q.y, src);
    float v = fmaf(A, s_mem, B);
    if (clamped) {
        const float lo = __shfl_sync(kFull, q.z, src);
        const float hi = __shfl_sync(kFull, q.w, src);
        v = fminf(fmaxf(v, lo), hi);
    }
    return v;
}

// A row's pixel state in shared memory as one warp walks it: S, F = (float)O
// (for the decay view), O = T - t_base, and a lane mask word per pixel (kept
// zero between groups).
struct RowState {
    float *S;
    float *F;
    long long *O;
    unsigned *P;
};

// Alg. 2 for a group of due records (one per valid lane, time order):
// S += p C; dt = t - T; S *= d(dt); T = t; clamp (Eq. 13).  Alg. 1 and Eq. 3
// run the same loop with infinite clamp bounds, Eq. 3 adding p C after the
// decay.  A record's dt needs only times (the previous record of its pixel in
// the group, or T), so every decay of the group is evaluated at once; only
// S = clamp((S + p C) d) runs in rank order per pixel, S passing from lane to
// lane by shuffle: the same operations in the same order as the sequential
// loop, so the result is bit-identical to it.  A group whose longest
// same-pixel chain has scan_chain records or more is composed by the
// segmented scan instead (scan_group).  Returns S after the lane's event;
// the last record of each pixel writes the pixel's state back.
template <int TWP, int RD, int DK>
__device__ __forceinline__ float apply_group(const RowState &rs, float4 *sc, unsigned long long r,
                                             bool valid, const DecayParams &dp,
                                             const MapParams &mp, int scan_chain)
{
    const int lane = threadIdx.x & 31;
    const int x = (int)((r >> 33) & (unsigned)(TWP - 1));
    const unsigned toff = (unsigned)r;
    // the pixel's state as the group starts (no lane writes it before the
    // write-back below): loaded by every lane while the peers are found
    const float s_mem = rs.S[x];
    const long long o_mem = rs.O[x];
    // lanes holding the same pixel: each sets its bit in the pixel's mask
    // word, reads the word, and clears it for the next group
    if (valid) atomicOr(&rs.P[x], 1u << lane);
    __syncwarp();
    const unsigned peers = valid ? rs.P[x] : 0u;
    __syncwarp();
    if (valid) rs.P[x] = 0u;
    const unsigned below = peers & lanemask_lt();
    const unsigned rank = __popc(below);
    const int prev = below ? 31 - __clz(below) : lane;
    const unsigned t_prev_rec = __shfl_sync(kFull, toff, prev);
    const bool first = valid && rank == 0;
    float s_in = first ? s_mem : 0.0f;
    const long long t_prev = first ? o_mem : (long long)t_prev_rec;
    const float d = valid ? decay_state_k<DK>((long long)toff - t_prev, dp) : 0.0f;
    const float c = ((r >> 32) & 1u) ? mp.C : -mp.C;
    const unsigned maxr = __reduce_max_sync(kFull, valid ? rank : 0u);
    float s_out = 0.0f;
    if ((int)maxr + 1 < scan_chain) {
        for (unsigned k = 0;; ++k) {
            if (valid && rank == k) s_out = event_step<DK>(s_in, c, d, dp, mp);
            if (k == maxr) break;
            const float got = __shfl_sync(kFull, s_out, prev);
            if (valid && rank == k + 1) s_in = got;
        }
    } else {
        s_out = scan_group<DK>(sc, valid, peers, rank, c, d, s_mem, maxr, dp, mp);
    }
    // the last record of each pixel writes its state back
    if (valid && (peers >> lane) == 1u) {
        rs.S[x] = s_out;
        rs.O[x] = (long long)toff;
        if (RD) rs.F[x] = __uint2float_rn(toff);
    }
    __syncwarp();
    return s_out;
}

// Eq. 14 codes of the lane's PPL pixels at a frame (the decay view to the
// frame time when RD): one 32-bit word (PPL = 4), one 16-bit word (PPL = 2)
// when vec, else byte by byte.  fr: the frame at the lane's first pixel.
template <int PPL, int RD, int DK>
__device__ __forceinline__ void emit_codes(const RowState &rs, unsigned char *fr, int nval, float tf_f,
                                           const DecayParams &dp, const MapParams &mp, bool vec)
{
    const int lane = threadIdx.x & 31;
    if constexpr (PPL == 4) {
        const float4 s4 = *reinterpret_cast<const float4 *>(rs.S + 4 * lane);
        float v[4] = {s4.x, s4.y, s4.z, s4.w};
        if (RD) {
            const float4 f4 = *reinterpret_cast<const float4 *>(rs.F + 4 * lane);
            v[0] *= decay_view_k<DK>(tf_f - f4.x, dp);
            v[1] *= decay_view_k<DK>(tf_f - f4.y, dp);
            v[2] *= decay_view_k<DK>(tf_f - f4.z, dp);
            v[3] *= decay_view_k<DK>(tf_f - f4.w, dp);
        }
        unsigned code[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) code[q] = quantize_u8(fmaf(v[q], mp.scale, mp.offs));
        if (vec) {
            if (nval == 4)
                *reinterpret_cast<unsigned *>(fr) =
                    code[0] | (code[1] << 8) | (code[2] << 16) | (code[3] << 24);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (q < nval) fr[q] = (unsigned char)code[q];
        }
    } else if constexpr (PPL == 2) {
        const float2 s2 = *reinterpret_cast<const float2 *>(rs.S + 2 * lane);
        float v0 = s2.x, v1 = s2.y;
        if (RD) {
            const float2 f2 = *reinterpret_cast<const float2 *>(rs.F + 2 * lane);
            v0 *= decay_view_k<DK>(tf_f - f2.x, dp);
            v1 *= decay_view_k<DK>(tf_f - f2.y, dp);
        }
        const unsigned c0 = quantize_u8(fmaf(v0, mp.scale, mp.offs));
        const unsigned c1 = quantize_u8(fmaf(v1, mp.scale, mp.offs));
        if (vec) {
            if (nval == 2) *reinterpret_cast<unsigned short *>(fr) = (unsigned short)(c0 | (c1 << 8));
        } else {
            if (nval > 0) fr[0] = (unsigned char)c0;
            if (nval > 1) fr[1] = (unsigned char)c1;
        }
    } else {
        float v = rs.S[lane];
        if (RD) v *= decay_view_k<DK>(tf_f - rs.F[lane], dp);
        if (nval) fr[0] = (unsigned char)quantize_u8(fmaf(v, mp.scale, mp.offs));
    }
}

// One block per (32 PPL) x TH tile; warp w owns tile row w, lane l owns the
// PPL pixels x = PPL l .. PPL l + PPL - 1 of that row for loads, stores and
// frame codes (PPL = 4: 128-pixel rows; PPL = 2: 64-pixel rows; PPL = 1:
// 32-pixel rows: narrower rows give more independent row walks).
// Events are applied event-parallel: a row's records are in time order, so at
// each frame the due records go 32 at a time, one per lane; lanes holding the
// same pixel (their lane masks gathered in a shared-memory word per pixel)
// apply theirs in arrival order, rank by rank, to the pixel state kept in
// shared memory.  RD: render_decay; DK: decay kind; VEC
// (PPL = 4 or 2): rows start PPL-byte aligned (W % PPL == 0), so a lane's
// pixels move as one float4 / two longlong2 / one 32-bit frame word (PPL = 4)
// or one 16-bit frame word (PPL = 2).  EV: every record's event index is
// carried beside it and S after each event is stored at that index
// (esi_event_states; launched with no frames).  VECRT: the row alignment is
// read from a.W at run time instead of VEC (one instance serves both).
template <int TH, int PPL, int RD, int DK, bool VEC, bool EV = false, bool VECRT = false>
__device__ __forceinline__ void tile_body(const TileArgs &a, int tile)
{
    constexpr int NT = TH * 32;
    constexpr int TWP = 32 * PPL;              // pixels per tile row
    constexpr int XB = (PPL == 4) ? 7 : (PPL == 2) ? 6 : 5;   // bits of x within the row
    static_assert(PPL == 1 || PPL == 2 || PPL == 4, "1, 2 or 4 pixels per lane");
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ unsigned short rcnt[TH][TH];   // [warp][row] counts, then offsets
    constexpr int RB = (TH == 4) ? 2 : (TH == 8) ? 3 : (TH == 16) ? 4 : 5;  // bits of a row index
    __shared__ unsigned rowstart[TH + 1];
    __shared__ unsigned scan_tmp[NT / 32 + 1];
    __shared__ long long s_tnext;
    __shared__ WinInfo swin[kStageFrames];              // this launch's frames, if they fit
    __shared__ __align__(16) float sS[TH][TWP];      // S of the tile's pixels
    __shared__ __align__(16) float sF[TH][TWP];      // (float)(T - t_base)
    __shared__ __align__(16) long long sO[TH][TWP];  // T - t_base
    __shared__ unsigned sPeer[TH][TWP];              // per-pixel lane masks of a group (kept zero)

    const int R = a.batch, n_chunks = a.n_chunks;
    size_t off_b, off_runpre, off_runoff, off_lpos;
    tile_layout(R, n_chunks, TH, &off_b, &off_runpre, &off_runoff, &off_lpos);
    unsigned long long *A = reinterpret_cast<unsigned long long *>(smem);
    unsigned long long *B = reinterpret_cast<unsigned long long *>(smem + off_b);
    unsigned *runpre = reinterpret_cast<unsigned *>(smem + off_runpre);
    unsigned *runoff = reinterpret_cast<unsigned *>(smem + off_runoff);
    unsigned short *lpos = reinterpret_cast<unsigned short *>(smem + off_lpos);
    unsigned *IA = nullptr, *IB = nullptr;
    if constexpr (EV) {
        size_t off_ia, off_ib;
        tile_layout_ev(R, n_chunks, TH, &off_ia, &off_ib);
        IA = reinterpret_cast<unsigned *>(smem + off_ia);
        IB = reinterpret_cast<unsigned *>(smem + off_ib);
    }

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool vec = VECRT ? (a.W % PPL == 0) : VEC;
    const int x0 = (tile % a.tiles_x) * TWP + PPL * lane;
    const int y = (tile / a.tiles_x) * TH + warp;
    const int nval = (y < a.H) ? max(0, min(PPL, a.W - x0)) : 0;
    const long long pix0 = (long long)y * a.W + x0;
    const long long tb = a.t_base;
    const DecayParams dp = a.dp;
    const MapParams mp = a.mp;
    unsigned *rP = sPeer[warp];
    for (int i = lane; i < TWP; i += 32) rP[i] = 0u;
    float *rS = sS[warp];
    float *rF = sF[warp];
    long long *rO = sO[warp];

    // this tile's run in every chunk, in chunk (= arrival) order
    for (int c = tid; c < n_chunks; c += NT) {
        const unsigned h = a.hrow[(size_t)tile * n_chunks + c];
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

    // gather a batch (records b0 .. b0 + nb of this tile, arrival order,
    // plus the next batch's first record) into A with asynchronous copies,
    // so every record of the batch is in flight; the first batch's copies
    // fly while the state loads, each later one while the rows walk the
    // previous batch's sorted copy B
    auto gather = [&](unsigned b0) {
        const int nb = (int)min((unsigned)R, total - min(total, b0));
        const unsigned next = b0 + (unsigned)R >= total ? 0u : 1u;
        if (nb == 0) return;
        const unsigned bend = b0 + (unsigned)nb + next;
        const int cfirst = run_of(runpre, n_chunks, b0);
        const int clast = run_of(runpre, n_chunks, bend - 1u);
        // kGatherLanes lanes per run: a warp instruction copies several
        // runs, each from contiguous addresses
        const int grp = tid / kGatherLanes, sub = tid % kGatherLanes;
        for (int c = cfirst + grp; c <= clast; c += NT / kGatherLanes) {
            const unsigned rs = max(runpre[c], b0), re = min(runpre[c + 1], bend);
            const unsigned long long *src = a.rec + (size_t)c * a.chunk + runoff[c] + (rs - runpre[c]);
            for (unsigned i = sub; i + rs < re; i += kGatherLanes) cp_async8(&A[rs - b0 + i], src + i);
            if constexpr (EV) {
                const unsigned *isrc = a.rec_idx + (size_t)c * a.chunk + runoff[c] + (rs - runpre[c]);
                for (unsigned i = sub; i + rs < re; i += kGatherLanes) cp_async4(&IA[rs - b0 + i], isrc + i);
            }
        }
    };
    gather(0u);

    {
        float s4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        long long o4[4] = {0, 0, 0, 0};
        if (PPL == 4 && vec && nval == 4) {
            const float4 v = *reinterpret_cast<const float4 *>(a.S + pix0);
            const longlong2 t01 = *reinterpret_cast<const longlong2 *>(a.T + pix0);
            const longlong2 t23 = *reinterpret_cast<const longlong2 *>(a.T + pix0 + 2);
            s4[0] = v.x; s4[1] = v.y; s4[2] = v.z; s4[3] = v.w;
            o4[0] = t01.x - tb; o4[1] = t01.y - tb; o4[2] = t23.x - tb; o4[3] = t23.y - tb;
        } else {
#pragma unroll
            for (int q = 0; q < PPL; ++q)
                if (q < nval) {
                    s4[q] = a.S[pix0 + q];
                    o4[q] = a.T[pix0 + q] - tb;
                }
        }
#pragma unroll
        for (int q = 0; q < PPL; ++q) {
            rS[PPL * lane + q] = s4[q];
            rO[PPL * lane + q] = o4[q];
            rF[PPL * lane + q] = RD ? __ll2float_rn(o4[q]) : 0.0f;
        }
    }


    const RowState rs{rS, rF, rO, rP};
    // the segmented scan's 32 slots per warp (the offsets' bytes, free while
    // the warps walk)
    float4 *sScan = reinterpret_cast<float4 *>(smem + off_lpos) + warp * 32;
    auto apply = [&](unsigned long long r, bool valid, unsigned ev_idx) {
        const float s_out = apply_group<TWP, RD, DK>(rs, sScan, r, valid, dp, mp, a.scan_chain);
        if constexpr (EV) {
            if (valid) a.ev_out[ev_idx] = s_out;
        }
    };

    int wi = a.w_begin;
    for (unsigned b0 = 0;; b0 += (unsigned)R) {
        const int nb = (int)min((unsigned)R, total - min(total, b0));
        const bool last = b0 + (unsigned)R >= total;
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
            const int row = valid ? (int)(A[k] >> (33 + XB)) : 0;
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
        // each warp scatters the slice it ranked
        for (int k = s0 + lane; k < s1; k += 32) {
            const unsigned long long r = A[k];
            const int row = (int)(r >> (33 + XB));
            B[rcnt[warp][row] + lpos[k]] = r;
            if constexpr (EV) IB[rcnt[warp][row] + lpos[k]] = IA[k];
        }
        __syncthreads();
        // A (and the offsets) are free: the next batch's copies start now
        if (!last) gather(b0 + (unsigned)R);

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
                apply(r, valid, EV && valid ? IB[k] : 0u);
                const int nv = __popc(vm);
                cur += nv;
                if (nv < 32) break;
            }
            // Eq. 14 codes of the lane's pixels at this frame
            unsigned char *fr =
                (a.frame_outs ? a.frame_outs[wi] : a.frames + (long long)wi * a.P) + pix0;
            emit_codes<PPL, RD, DK>(rs, fr, nval, wv.tf_f, dp, mp, vec);
            ++wi;
        }
        // the rest of this batch's row precedes the next batch's records
        for (; cur < re; cur += 32) {
            const int k = cur + lane;
            const bool valid = k < re;
            apply(valid ? B[k] : 0ull, valid, EV && valid ? IB[k] : 0u);
        }
        if (last) break;
        __syncthreads();  // B, rcnt and the scan slots are rewritten by the next batch
    }

    __syncwarp();
    if (PPL == 4 && vec && nval == 4) {
        const float4 s4 = *reinterpret_cast<const float4 *>(rS + 4 * lane);
        *reinterpret_cast<float4 *>(a.S + pix0) = s4;
        *reinterpret_cast<longlong2 *>(a.T + pix0) =
            make_longlong2(rO[4 * lane] + tb, rO[4 * lane + 1] + tb);
        *reinterpret_cast<longlong2 *>(a.T + pix0 + 2) =
            make_longlong2(rO[4 * lane + 2] + tb, rO[4 * lane + 3] + tb);
    } else {
#pragma unroll
        for (int q = 0; q < PPL; ++q)
            if (q < nval) {
                a.S[pix0 + q] = rS[PPL * lane + q];
                a.T[pix0 + q] = rO[PPL * lane + q] + tb;
            }
    }
}


}  // namespace esi
