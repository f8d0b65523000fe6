// Tile kernel with rows split across warps (128-pixel rows, four pixels per
// lane): the render path's tile kernel.
//
// The batch-walk tile kernel (esi_tile.cuh) binds warp w to tile row w and
// makes every warp wait at each batch's barrier, so a tile lasts as long as
// its busiest row (a hot pixel's row can hold several times the records of
// its neighbours).  Here a block first sorts all of its batches by row into
// a global scratch region (L2-resident), then divides the rows' records into
// pieces of about equal cost, contiguous per warp, splitting a busy row at
// record boundaries.  A piece that is not the first of its row needs the
// state its pixels have at its first record: Alg. 2's event update is a
// monotone clamped-affine map of the state, S -> clamp(a S + b, lo, hi), and
// such maps compose associatively (the clamp of Eq. 13 commutes with a
// non-negative scale), so the pieces before a split are composed into one
// map per pixel while the other warps already walk their own rows; a short
// prefix over each split row's pieces then gives every piece its input
// state, and all pieces replay their records and emit their frames with no
// barrier between warps.  A record's decay d(t - T) needs the time of the
// pixel's previous event: within a piece it is known; for the first event of
// a pixel in a piece it is deferred to the prefix, where T is known.
//
// Rounding: a split row's pieces after the first start from a composed
// state, which differs from the event-by-event result by a few units in the
// last place; rows that are not split give the batch-walk kernel's result
// bit for bit when the segmented scan is off.
#pragma once

#include <cfloat>

#include "esi_tile.cuh"

namespace esi {

constexpr int kSplitMaxBatches = 16;    // batches sorted per round (a round's rows are split together)
constexpr int kSplitMaxPieces = 40;     // pieces of one round (rows + splits)
constexpr int kSplitHalf = 128;         // records per half of a warp's staging ring (at most)
constexpr int kSplitMinPiece = 64;      // no piece shorter than this many records is split off
constexpr float kSplitEmitCost = 8.0f;  // cost of one frame's emission, in records
constexpr float kSplitComposeCost = 1.2f;  // cost of composing a record, in records replayed
constexpr float kSplitRowShare = 1.5f;  // rows above this many warp shares of work are split

// Per split point, the composed map of the piece before it (per pixel) and
// the input state of the piece after it, in the block's batch buffers
// (free once a round is sorted).
struct SplitStore {
    float4 *map;          // (a, b, lo, hi) of the piece's events after each pixel's first
    unsigned *t_first;    // time of each pixel's first event in the piece
    unsigned *t_last;     // time of its last one
    unsigned char *flag;  // bit 0: the pixel has events in the piece; bit 1: first event p > 0
    float *S_in;          // the next piece's input state
    long long *O_in;
};

__host__ __device__ inline int split_store_bytes() { return 128 * (16 + 4 + 4 + 1 + 4 + 8) + 64; }

__device__ __forceinline__ SplitStore split_store(unsigned char *base, int s)
{
    unsigned char *p = base + (size_t)s * split_store_bytes();
    SplitStore st;
    st.map = reinterpret_cast<float4 *>(p);
    st.O_in = reinterpret_cast<long long *>(p + 128 * 16);
    st.S_in = reinterpret_cast<float *>(p + 128 * 24);
    st.t_first = reinterpret_cast<unsigned *>(p + 128 * 28);
    st.t_last = reinterpret_cast<unsigned *>(p + 128 * 32);
    st.flag = p + 128 * 36;
    return st;
}

// (a2, b2, lo2, hi2) o (a1, b1, lo1, hi1): apply the first, then the second.
__device__ __forceinline__ float4 compose_maps(const float4 &g, const float4 &f, bool clamped)
{
    float4 r;
    r.x = g.x * f.x;
    r.y = fmaf(g.x, f.y, g.y);
    if (clamped) {
        r.z = fminf(fmaxf(fmaf(g.x, f.z, g.y), g.z), g.w);
        r.w = fminf(fmaxf(fmaf(g.x, f.w, g.y), g.z), g.w);
    } else {
        r.z = g.z;
        r.w = g.w;
    }
    return r;
}

// The group's prefix maps, lane by lane (the segmented scan of scan_group,
// without applying them): each valid lane gets the composition of its
// pixel's events in the group up to its own.  e: the lane's event map.
__device__ __forceinline__ float4 scan_group_maps(float4 *sc, bool valid, unsigned peers, unsigned rank,
                                                  float4 e, unsigned maxr, bool clamped)
{
    const int lane = threadIdx.x & 31;
    const bool lead = valid && rank == 0u;
    const unsigned len = lead ? (unsigned)__popc(peers) : 0u;
    const unsigned first_pos = warp_inclusive_scan(len) - len;
    const unsigned seg0 = __shfl_sync(kFull, first_pos, valid ? __ffs(peers) - 1 : lane);
    const unsigned starts = __reduce_or_sync(kFull, lead ? (1u << seg0) : 0u);
    const int nv = __popc(__ballot_sync(kFull, valid));
    if (valid) sc[seg0 + rank] = e;
    __syncwarp();
    float4 q = sc[lane];
    __syncwarp();
    const unsigned le = lane == 31 ? kFull : (2u << lane) - 1u;
    const int seg = lane < nv ? 31 - __clz(starts & le) : lane;
    for (int o = 1; o <= (int)maxr; o <<= 1) {
        float4 pq;
        pq.x = __shfl_up_sync(kFull, q.x, o);
        pq.y = __shfl_up_sync(kFull, q.y, o);
        pq.z = clamped ? __shfl_up_sync(kFull, q.z, o) : 0.0f;
        pq.w = clamped ? __shfl_up_sync(kFull, q.w, o) : 0.0f;
        if (lane - o >= seg) q = compose_maps(q, pq, clamped);
    }
    const int src = valid ? (int)(seg0 + rank) : lane;
    float4 r;
    r.x = __shfl_sync(kFull, q.x, src);
    r.y = __shfl_sync(kFull, q.y, src);
    r.z = clamped ? __shfl_sync(kFull, q.z, src) : 0.0f;
    r.w = clamped ? __shfl_sync(kFull, q.w, src) : 0.0f;
    return r;
}

// One group of a piece's records (one per valid lane, time order) composed
// into the piece's per-pixel maps.  The first event of a pixel in the piece
// enters as the identity (its decay waits for the prefix); the others as
// their Alg. 2 / Alg. 1 / Eq. 3 maps.  P: the warp's mask words (kept zero).
template <int DK>
__device__ __forceinline__ void compose_group(const SplitStore &st, unsigned *P, float4 *sc,
                                              unsigned long long r, bool valid,
                                              const DecayParams &dp, const MapParams &mp)
{
    const int lane = threadIdx.x & 31;
    const bool clamped = mp.s_min > -INFINITY;
    const bool after = DK == kDecayGeneral && dp.b_mode == kBModeExp;
    const int x = (int)((r >> 33) & 127u);
    const unsigned toff = (unsigned)r;
    const unsigned char fl = st.flag[x];
    const unsigned last_mem = st.t_last[x];
    if (valid) atomicOr(&P[x], 1u << lane);
    __syncwarp();
    const unsigned peers = valid ? P[x] : 0u;
    __syncwarp();
    if (valid) P[x] = 0u;
    const unsigned below = peers & lanemask_lt();
    const unsigned rank = __popc(below);
    const int prev = below ? 31 - __clz(below) : lane;
    const unsigned t_prev_rec = __shfl_sync(kFull, toff, prev);
    const bool has = (fl & 1u) != 0;
    const bool deferred = valid && rank == 0 && !has;
    const unsigned t_prev = rank == 0 ? last_mem : t_prev_rec;
    const float c = ((r >> 32) & 1u) ? mp.C : -mp.C;
    float4 e = make_float4(1.0f, 0.0f, -FLT_MAX, FLT_MAX);   // identity (finite bounds: 0 * bound stays finite)
    if (valid && !deferred) {
        const float d = decay_state_k<DK>((long long)toff - (long long)t_prev, dp);
        e = make_float4(d, after ? c : d * c, mp.s_min, mp.s_max);
    }
    const unsigned maxr = __reduce_max_sync(kFull, valid ? rank : 0u);
    const float4 q = scan_group_maps(sc, valid, peers, rank, e, maxr, clamped);
    if (deferred) {
        st.t_first[x] = toff;
        st.flag[x] = (unsigned char)(1u | (c > 0.0f ? 2u : 0u));
    }
    if (valid && (peers >> lane) == 1u) {
        const float4 g_old = has ? st.map[x] : make_float4(1.0f, 0.0f, -FLT_MAX, FLT_MAX);
        st.map[x] = compose_maps(q, g_old, clamped);
        st.t_last[x] = toff;
    }
    __syncwarp();
}

// One piece of a row: records [start, end) of the row's records in the
// round.  split_in / split_out: the split store holding its input state /
// receiving its composed maps (-1: none; the first piece of a row reads the
// state from global memory, the last writes it back).  warp_c: the warp that
// composes it (pieces with a split after them); warp_r, phase_r: the warp
// and phase (1 or 3) that replay it.
struct Piece {
    unsigned short row;
    short split_in, split_out;
    signed char warp_c, warp_r, phase_r;
    unsigned start, end;
};

template <int TH, int RD, int DK, bool VEC>
__device__ __forceinline__ void tile_body_split(const TileArgs &a, int tile)
{
    constexpr int PPL = 4;
    constexpr int NT = TH * 32;
    constexpr int NW = TH;
    constexpr int TWP = 128;
    constexpr int XB = 7;
    constexpr int RB = (TH == 4) ? 2 : (TH == 8) ? 3 : 4;
    constexpr int MAXB = kSplitMaxBatches;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ unsigned short rcnt[TH][TH];
    __shared__ unsigned rowstart[TH + 1];
    __shared__ unsigned scan_tmp[NT / 32 + 1];
    __shared__ long long s_tnext;
    __shared__ WinInfo swin[kStageFrames];
    __shared__ __align__(16) float sS[NW][TWP];       // working state of each warp's piece
    __shared__ __align__(16) float sF[NW][TWP];
    __shared__ __align__(16) long long sO[NW][TWP];
    __shared__ unsigned sPeer[NW][TWP];
    __shared__ __align__(16) float4 sScan[NW][32];
    __shared__ unsigned rowoff[TH];                   // records of each row stored so far
    __shared__ unsigned roundoff[TH];                 // ... before this round
    __shared__ Piece pcs[kSplitMaxPieces];
    __shared__ int s_npieces, s_nsplit, s_fend, s_split;
    __shared__ long long s_base;

    const int R = a.batch, n_chunks = a.n_chunks;
    size_t off_b, off_runpre, off_runoff, off_lpos;
    tile_layout(R, n_chunks, TH, &off_b, &off_runpre, &off_runoff, &off_lpos);
    unsigned long long *A = reinterpret_cast<unsigned long long *>(smem);
    unsigned long long *B = reinterpret_cast<unsigned long long *>(smem + off_b);
    unsigned *runpre = reinterpret_cast<unsigned *>(smem + off_runpre);
    unsigned *runoff = reinterpret_cast<unsigned *>(smem + off_runoff);
    unsigned short *lpos = reinterpret_cast<unsigned short *>(smem + off_lpos);
    // after a round is sorted, the batch buffers hold each warp's staging ring
    // (two halves of kSplitHalf records) and the split stores
    unsigned long long *rings = A;
    unsigned half = kSplitHalf;   // a power of two, the rings within the batch buffers
    while (half > 32 && (size_t)NW * 2 * half * 8 > off_runpre) half >>= 1;
    const size_t ring_bytes = (size_t)NW * 2 * half * 8;
    unsigned char *stores = smem + ring_bytes;
    const int max_splits = min(a.max_splits, min(NW - 1, (int)((off_runpre - ring_bytes) /
                                                               (size_t)split_store_bytes())));

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const long long tb = a.t_base;
    const DecayParams dp = a.dp;
    const MapParams mp = a.mp;
    for (int i = lane; i < TWP; i += 32) sPeer[warp][i] = 0u;
    if (tid < TH) rowoff[tid] = 0u;

    for (int c = tid; c < n_chunks; c += NT) {
        const unsigned h = a.hrow[(size_t)tile * n_chunks + c];
        runpre[c] = h & 0xffffu;
        runoff[c] = h >> 16;
    }
    const int nwin = a.w_end - a.w_begin;
    const bool staged = nwin <= kStageFrames;
    if (staged)
        for (int i = tid; i < nwin; i += NT) swin[i] = a.win[a.w_begin + i];
    __syncthreads();
    const unsigned total = block_exclusive_scan<NT>(runpre, n_chunks, scan_tmp);
    if (tid == 0) {
        runpre[n_chunks] = total;
        // the tile's region of the scratch: room for every record in each
        // row's own contiguous part (row r at r * total)
        s_base = 0;
        if (total) {
            const unsigned long long need = (unsigned long long)TH * total;
            const unsigned long long b = atomicAdd(a.srt_top, need);
            if (b + need > a.srt_cap) {
                set_error(a.status, ESI_ERANGE, 3);
                s_base = -1;
            } else {
                s_base = (long long)b;
            }
        }
    }
    __syncthreads();
    if (total == 0 && a.w_end == a.w_begin) return;
    if (s_base < 0) return;
    unsigned long long *srt = a.srt + s_base;

    auto lim_of = [&](int f) -> long long { return staged ? swin[f - a.w_begin].lim : a.win[f].lim; };
    auto tf_of = [&](int f) -> float { return staged ? swin[f - a.w_begin].tf_f : a.win[f].tf_f; };
    // first frame in [lo, hi) with lim >= t
    auto first_frame_at = [&](int lo, int hi, long long t) {
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (lim_of(mid) < t) lo = mid + 1; else hi = mid;
        }
        return lo;
    };

    int f_begin = a.w_begin;
    for (unsigned b0 = 0;;) {
        if (tid < TH) roundoff[tid] = rowoff[tid];
        // ---------------------------------------------------------- sort
        bool last = false;
        for (int nbat = 0; nbat < MAXB && !last; ++nbat, b0 += (unsigned)R) {
            const int nb = (int)min((unsigned)R, total - min(total, b0));
            last = b0 + (unsigned)R >= total;
            const unsigned next = last ? 0u : 1u;
            if (nb > 0) {
                const unsigned bend = b0 + (unsigned)nb + next;
                const int cfirst = run_of(runpre, n_chunks, b0);
                const int clast = run_of(runpre, n_chunks, bend - 1u);
                const int grp = tid / kGatherLanes, sub = tid % kGatherLanes;
                for (int c = cfirst + grp; c <= clast; c += NT / kGatherLanes) {
                    const unsigned rs = max(runpre[c], b0), re = min(runpre[c + 1], bend);
                    const unsigned long long *src =
                        a.rec + (size_t)c * a.chunk + runoff[c] + (rs - runpre[c]);
                    for (unsigned i = sub; i + rs < re; i += kGatherLanes) cp_async8(&A[rs - b0 + i], src + i);
                }
            }
            cp_async_wait_all();
            __syncthreads();
            if (tid == 0) s_tnext = last ? 0x7fffffffffffffffll : (long long)(unsigned)A[nb];
            for (int i = tid; i < TH * TH; i += NT) (&rcnt[0][0])[i] = 0;
            __syncthreads();
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
            for (int k = s0 + lane; k < s1; k += 32) {
                const unsigned long long r = A[k];
                const int row = (int)(r >> (33 + XB));
                B[rcnt[warp][row] + lpos[k]] = r;
            }
            __syncthreads();
            // warp w appends row w's part of the batch to the row's own part
            // of the scratch region (coalesced)
            {
                const unsigned r0 = rowstart[warp], r1 = rowstart[warp + 1];
                unsigned long long *dst = srt + (size_t)warp * total + rowoff[warp];
                for (unsigned k = r0 + lane; k < r1; k += 32) dst[k - r0] = B[k];
                __syncwarp();
                if (lane == 0) rowoff[warp] += r1 - r0;
            }
            __syncthreads();
        }
        const long long tnext = s_tnext;

        // ---------------------------------------------------------- plan
        // frames of this round: those before the next round's first record;
        // a row well above the per-warp share of work is split
        if (warp == 0) {
            const int f_end = tnext == 0x7fffffffffffffffll ? a.w_end : first_frame_at(f_begin, a.w_end, tnext);
            const float nfr = (float)(f_end - f_begin);
            const float c = lane < TH ? (float)(rowoff[lane] - roundoff[lane]) + kSplitEmitCost * nfr : 0.0f;
            float ctot = c, cmax = c;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                ctot += __shfl_xor_sync(kFull, ctot, o);
                cmax = fmaxf(cmax, __shfl_xor_sync(kFull, cmax, o));
            }
            const bool split = max_splits > 0 && cmax > kSplitRowShare * ctot / (float)NW;
            if (!split && lane < TH) {
                // every row whole on its own warp, in phase 1
                Piece pc;
                pc.row = (unsigned short)lane;
                pc.start = 0;
                pc.end = rowoff[lane] - roundoff[lane];
                pc.split_in = pc.split_out = -1;
                pc.warp_c = -1;
                pc.warp_r = (signed char)lane;
                pc.phase_r = 1;
                pcs[lane] = pc;
            }
            if (lane == 0) {
                s_fend = f_end;
                s_npieces = TH;
                s_nsplit = 0;
                s_split = split ? 1 : 0;
            }
        }
        __syncthreads();
        if (s_split && tid == 0) {
            const int f_end = s_fend;
            const float nfr = (float)(f_end - f_begin);
            float ctot = 0.0f;
            for (int r = 0; r < TH; ++r) ctot += (float)(rowoff[r] - roundoff[r]) + kSplitEmitCost * nfr;
            const float Q = ctot / (float)NW;
            // pieces: a row well above the per-warp share is cut into pieces
            // of about one share each
            int np = 0, ns = 0;
            for (int r = 0; r < TH; ++r) {
                const unsigned n = rowoff[r] - roundoff[r];
                const float c = (float)n + kSplitEmitCost * nfr;
                int K = 1;
                if (c > kSplitRowShare * Q && n >= 2u * kSplitMinPiece) {
                    K = (int)ceilf(c / Q);
                    K = min(K, 1 + max_splits - ns);
                    K = min(K, (int)(n / kSplitMinPiece));
                    K = min(K, kSplitMaxPieces - np - (TH - 1 - r));
                    K = max(K, 1);
                }
                for (int k = 0; k < K; ++k) {
                    Piece pc;
                    pc.row = (unsigned short)r;
                    pc.start = (unsigned)((unsigned long long)n * k / K);
                    pc.end = (unsigned)((unsigned long long)n * (k + 1) / K);
                    pc.split_in = (short)(k > 0 ? ns + k - 1 : -1);
                    pc.split_out = (short)(k < K - 1 ? ns + k : -1);
                    pc.warp_c = -1;
                    pc.warp_r = 0;
                    pc.phase_r = 1;
                    pcs[np++] = pc;
                }
                ns += K - 1;
            }
            // schedule: composes (phase 1) and the replays after a split
            // (phase 3) are fixed, the other replays go to whichever phase
            // and warp keeps max(phase 1) + max(phase 3) smallest; largest
            // items first.  A split row's first piece replays in phase 1 (it
            // reads the row's state before the last piece writes it back).
            float L1[NW], L3[NW];
            for (int w = 0; w < NW; ++w) L1[w] = L3[w] = 0.0f;
            auto piece_cost = [&](const Piece &pc) {
                const unsigned n = rowoff[pc.row] - roundoff[pc.row];
                const float len = (float)(pc.end - pc.start);
                return len + kSplitEmitCost * nfr * (n ? len / (float)n : 1.0f);
            };
            // items: 2p = compose of piece p (when a split follows it),
            // 2p + 1 = replay of piece p; sorted by cost, largest first
            short item[kSplitMaxPieces * 2];
            float icost[kSplitMaxPieces * 2];
            int ni = 0;
            for (int p = 0; p < np; ++p) {
                if (pcs[p].split_out >= 0) {
                    item[ni] = (short)(2 * p);
                    icost[ni++] = kSplitComposeCost * (float)(pcs[p].end - pcs[p].start);
                }
                item[ni] = (short)(2 * p + 1);
                icost[ni++] = piece_cost(pcs[p]);
            }
            for (int i = 1; i < ni; ++i) {
                const short it = item[i];
                const float c = icost[i];
                int j = i - 1;
                while (j >= 0 && icost[j] < c) {
                    item[j + 1] = item[j];
                    icost[j + 1] = icost[j];
                    --j;
                }
                item[j + 1] = it;
                icost[j + 1] = c;
            }
            for (int ii = 0; ii < ni; ++ii) {
                const int best = item[ii];
                const float bc = icost[ii];
                Piece &pc = pcs[best >> 1];
                float m1 = 0.0f, m3 = 0.0f;
                for (int w = 0; w < NW; ++w) {
                    m1 = fmaxf(m1, L1[w]);
                    m3 = fmaxf(m3, L3[w]);
                }
                const bool compose_item = !(best & 1);
                const bool in1 = compose_item || pc.split_in < 0;
                const bool in3 = !compose_item && (pc.split_in >= 0 || pc.split_out < 0);
                int bw = 0, bphase = in1 ? 1 : 3;
                float bo = 3.0e38f;
                for (int w = 0; w < NW; ++w) {
                    if (in1) {
                        const float o = fmaxf(m1, L1[w] + bc) + m3;
                        if (o < bo) { bo = o; bw = w; bphase = 1; }
                    }
                    if (in3) {
                        const float o = m1 + fmaxf(m3, L3[w] + bc);
                        if (o < bo) { bo = o; bw = w; bphase = 3; }
                    }
                }
                if (compose_item) {
                    pc.warp_c = (signed char)bw;
                    L1[bw] += bc;
                } else {
                    pc.warp_r = (signed char)bw;
                    pc.phase_r = (signed char)bphase;
                    (bphase == 1 ? L1 : L3)[bw] += bc;
                }
            }
            s_npieces = np;
            s_nsplit = ns;
        }
        __syncthreads();
        const int npieces = s_npieces, nsplit = s_nsplit;
        const int f_end = s_fend;

        // the warp's staging ring: records of the piece's row copied from the
        // scratch region half by half (cp.async), at most two halves in
        // flight; record i sits at slot (i - org) mod 2 kSplitHalf
        unsigned long long *ring = rings + (size_t)warp * 2 * half;
        const unsigned rmask = 2 * half - 1;
        const unsigned long long *rsrc = nullptr;
        unsigned org = 0, rend = 0, issued = 0, ready = 0;
        int pending = 0;
        auto ring_issue = [&]() {
            const unsigned hi = min(rend, issued + half);
            for (unsigned i = issued + lane; i < hi; i += 32) cp_async8(&ring[(i - org) & rmask], rsrc + i);
            cp_async_commit();
            issued = hi;
            ++pending;
        };
        auto ring_open = [&](const unsigned long long *src, unsigned start, unsigned end) {
            rsrc = src;
            org = issued = ready = start;
            rend = end;
            pending = 0;
            if (issued < rend) ring_issue();
            if (issued < rend) ring_issue();
        };
        // records below min(upto, end) readable; refill the half left behind
        auto ring_need = [&](unsigned cur, unsigned upto) {
            upto = min(upto, rend);
            // (the slots of records this far ahead hold records below cur)
            while (issued < upto) ring_issue();
            if (ready < upto) {
                do {
                    if (pending >= 2) cp_async_wait_one(); else cp_async_wait_none();
                    --pending;
                    ready = min(rend, ready + half);
                } while (ready < upto);
                __syncwarp();
            }
            if (issued < rend && issued <= cur + half && pending < 2) ring_issue();
        };
        auto ring_at = [&](unsigned i) -> unsigned long long { return ring[(i - org) & rmask]; };
        auto ring_close = [&]() {
            cp_async_wait_none();
            __syncwarp();
        };

        // replay one piece: its records through Alg. 2, its frames emitted
        auto replay = [&](const Piece &pc) {
            const RowState rs{sS[warp], sF[warp], sO[warp], sPeer[warp]};
            const int r = pc.row;
            const unsigned long long *rrec = srt + (size_t)r * total + roundoff[r];
            const int x0 = tx * TWP + PPL * lane;
            const int y = ty * TH + r;
            const int nval = (y < a.H) ? max(0, min(PPL, a.W - x0)) : 0;
            const long long pix0 = (long long)y * a.W + x0;
            if (pc.split_in < 0) {
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
                    for (int q = 0; q < PPL; ++q)
                        if (q < nval) {
                            s4[q] = a.S[pix0 + q];
                            o4[q] = a.T[pix0 + q] - tb;
                        }
                }
#pragma unroll
                for (int q = 0; q < PPL; ++q) {
                    rs.S[PPL * lane + q] = s4[q];
                    rs.O[PPL * lane + q] = o4[q];
                    rs.F[PPL * lane + q] = RD ? __ll2float_rn(o4[q]) : 0.0f;
                }
            } else {
                const SplitStore st = split_store(stores, pc.split_in);
                for (int i = lane; i < TWP; i += 32) {
                    rs.S[i] = st.S_in[i];
                    rs.O[i] = st.O_in[i];
                    rs.F[i] = RD ? __ll2float_rn(st.O_in[i]) : 0.0f;
                }
            }
            __syncwarp();
            const unsigned end = pc.end;
            // frames: those whose first record not due lies in [start, end)
            // (the last piece also those after all records)
            const bool last_piece = pc.split_out < 0;
            const long long t_lo = pc.start ? (long long)(unsigned)rrec[pc.start - 1] : -1ll;
            const long long t_hi = last_piece ? 0x7fffffffffffffffll : (long long)(unsigned)rrec[end - 1];
            const int fa = pc.start ? first_frame_at(f_begin, f_end, t_lo) : f_begin;
            const int fb = last_piece ? f_end : first_frame_at(fa, f_end, t_hi);
            unsigned cur = pc.start;
            ring_open(rrec, cur, end);
            for (int f = fa; f < fb; ++f) {
                const long long lim = lim_of(f);
                while (cur < end) {
                    ring_need(cur, cur + 32u);
                    const unsigned k = cur + lane;
                    const unsigned long long rv = k < end ? ring_at(k) : 0ull;
                    const bool valid = k < end && (long long)(unsigned)rv <= lim;
                    const unsigned vm = __ballot_sync(kFull, valid);
                    if (vm == 0u) break;
                    apply_group<TWP, RD, DK>(rs, sScan[warp], rv, valid, dp, mp, a.scan_chain);
                    const int nv = __popc(vm);
                    cur += nv;
                    if (nv < 32) break;
                }
                unsigned char *fr = (a.frame_outs ? a.frame_outs[f] : a.frames + (long long)f * a.P) + pix0;
                emit_codes<PPL, RD, DK>(rs, fr, nval, tf_of(f), dp, mp, VEC);
            }
            for (; cur < end; cur += 32) {
                ring_need(cur, cur + 32u);
                const unsigned k = cur + lane;
                apply_group<TWP, RD, DK>(rs, sScan[warp], k < end ? ring_at(k) : 0ull, k < end, dp, mp,
                                         a.scan_chain);
            }
            ring_close();
            if (last_piece) {
                if (VEC && nval == 4) {
                    const float4 s4 = *reinterpret_cast<const float4 *>(rs.S + 4 * lane);
                    *reinterpret_cast<float4 *>(a.S + pix0) = s4;
                    *reinterpret_cast<longlong2 *>(a.T + pix0) =
                        make_longlong2(rs.O[4 * lane] + tb, rs.O[4 * lane + 1] + tb);
                    *reinterpret_cast<longlong2 *>(a.T + pix0 + 2) =
                        make_longlong2(rs.O[4 * lane + 2] + tb, rs.O[4 * lane + 3] + tb);
                } else {
#pragma unroll
                    for (int q = 0; q < PPL; ++q)
                        if (q < nval) {
                            a.S[pix0 + q] = rs.S[PPL * lane + q];
                            a.T[pix0 + q] = rs.O[PPL * lane + q] + tb;
                        }
                }
            }
            __syncwarp();
        };

        // compose one piece's records into its split store
        auto compose = [&](const Piece &pc) {
            const SplitStore st = split_store(stores, pc.split_out);
            for (int i = lane; i < TWP; i += 32) st.flag[i] = 0;
            __syncwarp();
            const unsigned long long *rrec = srt + (size_t)pc.row * total + roundoff[pc.row];
            const unsigned end = pc.end;
            ring_open(rrec, pc.start, end);
            for (unsigned cur = pc.start; cur < end; cur += 32) {
                ring_need(cur, cur + 32u);
                const unsigned k = cur + lane;
                compose_group<DK>(st, sPeer[warp], sScan[warp], k < end ? ring_at(k) : 0ull, k < end, dp, mp);
            }
            ring_close();
        };

        // ---------------------------------------------- phase 1: composes and
        // the replays that need no other piece
        for (int p = 0; p < npieces; ++p)
            if (pcs[p].warp_c == warp) compose(pcs[p]);
        for (int p = 0; p < npieces; ++p)
            if (pcs[p].phase_r == 1 && pcs[p].warp_r == warp) replay(pcs[p]);
        __syncthreads();
        if (nsplit > 0) {
            // ------------------------------------------ phase 2: each split
            // row's pieces in order give the next piece its input state
            for (int i = tid; i < TH * TWP; i += NT) {
                const int r = i / TWP, x = i % TWP;
                int p = 0;
                while (p < npieces && pcs[p].row != r) ++p;
                if (p >= npieces || pcs[p].split_out < 0) continue;   // row not split
                const int px = tx * TWP + x, y = ty * TH + r;
                const bool inside = px < a.W && y < a.H;
                const long long pix = (long long)y * a.W + px;
                float S = inside ? a.S[pix] : 0.0f;
                long long O = inside ? a.T[pix] - tb : 0;
                for (; p < npieces && pcs[p].row == r && pcs[p].split_out >= 0; ++p) {
                    const SplitStore st = split_store(stores, pcs[p].split_out);
                    const unsigned fl = st.flag[x];
                    if (fl & 1u) {
                        const float d1 = decay_state_k<DK>((long long)st.t_first[x] - O, dp);
                        S = event_step<DK>(S, (fl & 2u) ? mp.C : -mp.C, d1, dp, mp);
                        const float4 g = st.map[x];
                        S = fmaf(g.x, S, g.y);
                        if (mp.s_min > -INFINITY) S = fminf(fmaxf(S, g.z), g.w);
                        O = (long long)st.t_last[x];
                    }
                    st.S_in[x] = S;
                    st.O_in[x] = O;
                }
            }
            __syncthreads();
        }
        // ---------------------------------------------- phase 3: the pieces
        // after a split, and the replays moved here to balance the phases
        for (int p = 0; p < npieces; ++p)
            if (pcs[p].phase_r == 3 && pcs[p].warp_r == warp) replay(pcs[p]);
        f_begin = f_end;
        if (last) break;
        __syncthreads();   // the next round reuses the batch buffers
    }
}

}  // namespace esi
