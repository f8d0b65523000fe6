// sm_103a kernels of the ESI hot path.
//
//   esi_bin_kernel   one block per chunk of consecutive events: bulk-copies
//                    the chunk into shared memory (TMA), validates x < W,
//                    y < H, and writes the chunk's events as 8-byte records
//                    stably sorted by pixel tile, plus the chunk's per-tile
//                    (start, count) row.  Events of one tile stay in arrival
//                    (= time) order: ranks come from warp match_any over warp
//                    slices that are themselves in order.
//   esi_tile_kernel  one block per 32 x TH pixel tile, one thread per pixel:
//                    gathers the tile's runs from every chunk in chunk order
//                    (so arrival order is kept), stable-sorts each batch by
//                    row and then by column in shared memory, and lets every
//                    lane walk its own pixel's events through Alg. 2, emitting
//                    the Eq. 14 code of its pixel at every frame time.
//
// Per-pixel independence (each pixel's state depends only on its own
// time-ordered events, Eq. 5 and Alg. 2) is what makes the reorder legal.
#include <algorithm>
#include <cstdint>

#include "esi_device.cuh"
#include "esi_internal.h"

namespace esi {

constexpr int kBinThreads = 256;
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
    return o;
}

size_t bin_smem_bytes(int chunk, int n_tiles)
{
    size_t a, b, c;
    return bin_layout(chunk, n_tiles, &a, &b, &c);
}

__global__ void __launch_bounds__(kBinThreads) esi_bin_kernel(BinArgs a)
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

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long c0 = (long long)blockIdx.x * chunk;
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
    for (int i = tid; i < NW * ntp; i += NT) cnt[i] = 0;
    __syncthreads();
    if (!mbar_wait_bounded(&bar, 0, kWaitLimitNs)) {
        // never read a partial chunk: report, give the copy one more bounded
        // wait so it does not land in reassigned shared memory, and leave
        set_error(a.status, ESI_ETIMEOUT, kWhereBinCopy);
        mbar_wait_bounded(&bar, 0, kWaitLimitNs);
        return;
    }

    const int W = a.W, H = a.H, tiles_x = a.tiles_x, thl = a.th_log2;
    const int th_mask = (1 << thl) - 1;
    const int per = chunk / NW;
    const int s0 = warp * per;
    const int s1 = min(s0 + per, nc);

    // phase 1: per-warp tile counts
    unsigned drop = 0;
    for (int base = s0; base < s1; base += 32) {
        const int k = base + lane;
        int tile = -1;
        if (k < s1) {
            const int4 e = sev[k];
            const int x = e.z & 0xffff, y = (int)((unsigned)e.z >> 16);
            if (x < W && y < H)
                tile = (y >> thl) * tiles_x + (x >> 5);
            else
                ++drop;
        }
        const unsigned m = __match_any_sync(kFull, tile);
        if (tile >= 0 && (m & lanemask_lt()) == 0) cnt[warp * ntp + tile] += (unsigned short)__popc(m);
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
    unsigned *hrow = a.hrow + (size_t)blockIdx.x * n_tiles;
    for (int j = tid; j < n_tiles; j += NT)
        hrow[j] = (tstart[j] << 16) | (tstart[j + 1] - tstart[j]);

    // phase 3: stable scatter into tile order
    for (int base = s0; base < s1; base += 32) {
        const int k = base + lane;
        int tile = -1;
        unsigned long long rec = 0;
        if (k < s1) {
            const int4 e = sev[k];
            const int x = e.z & 0xffff, y = (int)((unsigned)e.z >> 16);
            if (x < W && y < H) {
                tile = (y >> thl) * tiles_x + (x >> 5);
                const long long t = ((long long)(unsigned)e.y << 32) | (unsigned)e.x;
                const unsigned pit = ((unsigned)(y & th_mask) << 5) | (unsigned)(x & 31);
                const bool pos = (signed char)(e.w & 0xff) > 0;
                rec = make_record((unsigned)(t - a.t_base), pit, pos ? 1u : 0u);
            }
        }
        const unsigned m = __match_any_sync(kFull, tile);
        const unsigned rank = __popc(m & lanemask_lt());
        if (tile >= 0) ssort[tstart[tile] + cnt[warp * ntp + tile] + rank] = rec;
        __syncwarp();
        if (tile >= 0 && rank == 0) cnt[warp * ntp + tile] += (unsigned short)__popc(m);
        __syncwarp();
    }
    __syncthreads();

    // phase 4: the chunk's records, tile-sorted, to global memory
    unsigned long long *dst = a.rec + c0;
    for (unsigned i = tid; i < total; i += NT) dst[i] = ssort[i];
    if (tid == 0 && s_drop) atomicAdd(&a.status->dropped, (unsigned long long)s_drop);
}

// Shared-memory layout of the tile kernel (dynamic part).
static __host__ __device__ inline size_t tile_layout(int batch, int n_chunks, size_t *off_b,
                                                     size_t *off_runpre, size_t *off_runoff)
{
    size_t o = (size_t)batch * 8;
    *off_b = o;
    o += (size_t)batch * 8;
    *off_runpre = o;
    o += (size_t)round_up(n_chunks + 1, 4) * 4;
    *off_runoff = o;
    o += (size_t)round_up(n_chunks, 4) * 4;
    return o;
}

size_t tile_smem_bytes(int tile_h, int batch, int n_chunks)
{
    (void)tile_h;
    size_t a, b, c;
    return tile_layout(batch, n_chunks, &a, &b, &c);
}

template <int TH>
__global__ void __launch_bounds__(TH * 32, (TH == 32) ? 1 : 2) esi_tile_kernel(TileArgs a)
{
    constexpr int NT = TH * 32;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ unsigned short rcnt[TH][TH];   // [warp][row]
    __shared__ unsigned short xoff[TH][32];   // [row][x]
    __shared__ unsigned rowstart[TH + 1];
    __shared__ unsigned scan_tmp[NT / 32 + 1];
    __shared__ long long s_tnext;

    const int R = a.batch, n_chunks = a.n_chunks;
    size_t off_b, off_runpre, off_runoff;
    tile_layout(R, n_chunks, &off_b, &off_runpre, &off_runoff);
    unsigned long long *A = reinterpret_cast<unsigned long long *>(smem);
    unsigned long long *B = reinterpret_cast<unsigned long long *>(smem + off_b);
    unsigned *runpre = reinterpret_cast<unsigned *>(smem + off_runpre);
    unsigned *runoff = reinterpret_cast<unsigned *>(smem + off_runoff);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tile = blockIdx.x;
    const int x = (tile % a.tiles_x) * 32 + lane;
    const int y = (tile / a.tiles_x) * TH + warp;
    const bool inb = x < a.W && y < a.H;
    const long long pix = (long long)y * a.W + x;

    float S = 0.0f;
    long long T = 0;
    if (inb) {
        S = a.S[pix];
        T = a.T[pix];
    }

    // this tile's run in every chunk, in chunk (= arrival) order
    for (int c = tid; c < n_chunks; c += NT) {
        const unsigned h = a.hrow[(size_t)c * a.n_tiles + tile];
        runpre[c] = h & 0xffffu;
        runoff[c] = h >> 16;
    }
    __syncthreads();
    const unsigned total = block_exclusive_scan<NT>(runpre, n_chunks, scan_tmp);
    if (tid == 0) runpre[n_chunks] = total;
    __syncthreads();

    const DecayParams dp = a.dp;
    const MapParams mp = a.mp;
    const long long tb = a.t_base;
    int wi = a.w_begin;

    for (unsigned b0 = 0;; b0 += (unsigned)R) {
        const int nb = (int)min((unsigned)R, total - min(total, b0));
        const bool last = b0 + (unsigned)R >= total;

        // gather the batch (records b0 .. b0 + nb of this tile, arrival order)
        for (int i = tid; i < nb; i += NT) {
            const unsigned g = b0 + (unsigned)i;
            int lo = 0, hi = n_chunks;  // largest c with runpre[c] <= g
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (runpre[mid] <= g) lo = mid; else hi = mid;
            }
            A[i] = a.rec[(size_t)lo * a.chunk + runoff[lo] + (g - runpre[lo])];
        }
        if (tid == 0) {
            long long tn = 0x7fffffffffffffffll;
            if (!last) {
                const unsigned g = b0 + (unsigned)R;
                int lo = 0, hi = n_chunks;
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (runpre[mid] <= g) lo = mid; else hi = mid;
                }
                tn = (long long)(unsigned)a.rec[(size_t)lo * a.chunk + runoff[lo] + (g - runpre[lo])];
            }
            s_tnext = tn;
        }
        for (int i = tid; i < TH * TH; i += NT) (&rcnt[0][0])[i] = 0;
        __syncthreads();

        // level 1: stable counting sort of the batch by row (A -> B)
        const int sl = (nb + TH - 1) / TH;
        const int s0 = min(warp * sl, nb), s1 = min(s0 + sl, nb);
        for (int base = s0; base < s1; base += 32) {
            const int k = base + lane;
            const int row = (k < s1) ? (int)(A[k] >> 38) : -1;
            const unsigned m = __match_any_sync(kFull, row);
            if (row >= 0 && (m & lanemask_lt()) == 0) rcnt[warp][row] += (unsigned short)__popc(m);
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
        for (int base = s0; base < s1; base += 32) {
            const int k = base + lane;
            unsigned long long r = 0;
            int row = -1;
            if (k < s1) {
                r = A[k];
                row = (int)(r >> 38);
            }
            const unsigned m = __match_any_sync(kFull, row);
            const unsigned rank = __popc(m & lanemask_lt());
            if (row >= 0) B[rcnt[warp][row] + rank] = r;
            __syncwarp();
            if (row >= 0 && rank == 0) rcnt[warp][row] += (unsigned short)__popc(m);
            __syncwarp();
        }
        __syncthreads();

        // level 2: warp `warp` sorts its row by column (B -> A), stable
        const int rs = (int)rowstart[warp], re = (int)rowstart[warp + 1];
        xoff[warp][lane] = 0;
        __syncwarp();
        for (int base = rs; base < re; base += 32) {
            const int k = base + lane;
            const int xx = (k < re) ? (int)((B[k] >> 33) & 31u) : -1;
            const unsigned m = __match_any_sync(kFull, xx);
            if (xx >= 0 && (m & lanemask_lt()) == 0) xoff[warp][xx] += (unsigned short)__popc(m);
        }
        __syncwarp();
        const unsigned mycnt = xoff[warp][lane];
        const unsigned myoff = (unsigned)rs + warp_inclusive_scan(mycnt) - mycnt;
        __syncwarp();
        xoff[warp][lane] = (unsigned short)myoff;
        __syncwarp();
        for (int base = rs; base < re; base += 32) {
            const int k = base + lane;
            unsigned long long r = 0;
            int xx = -1;
            if (k < re) {
                r = B[k];
                xx = (int)((r >> 33) & 31u);
            }
            const unsigned m = __match_any_sync(kFull, xx);
            const unsigned rank = __popc(m & lanemask_lt());
            if (xx >= 0) A[xoff[warp][xx] + rank] = r;
            __syncwarp();
            if (xx >= 0 && rank == 0) xoff[warp][xx] += (unsigned short)__popc(m);
            __syncwarp();
        }
        __syncwarp();

        // walk: this lane's events of the batch, A[myoff .. myoff + mycnt)
        int cur = (int)myoff;
        const int end = (int)(myoff + mycnt);
        const long long tnext = s_tnext;
        while (wi < a.w_end) {
            const long long tf_abs = a.t_frames[wi];
            const long long tf = tf_abs - tb;
            if (tf >= tnext) break;  // later records of this tile may still be <= tf
            while (cur < end) {
                const unsigned long long r = A[cur];
                const long long t = (long long)(unsigned)r;
                if (t > tf) break;
                esi_apply(S, T, tb + t, (r >> 32) & 1u, dp, mp);
                ++cur;
            }
            if (inb) a.frames[(long long)wi * a.P + pix] = esi_pixel_code(S, T, tf_abs, dp, mp);
            ++wi;
        }
        while (cur < end) {
            const unsigned long long r = A[cur];
            esi_apply(S, T, tb + (long long)(unsigned)r, (r >> 32) & 1u, dp, mp);
            ++cur;
        }
        if (last) break;
        __syncthreads();  // A, B, rcnt are rewritten by the next batch
    }
    if (inb) {
        a.S[pix] = S;
        a.T[pix] = T;
    }
}

cudaError_t set_kernel_attributes()
{
    cudaError_t e;
    const int max_dyn = 200 * 1024;
    e = cudaFuncSetAttribute(esi_bin_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(esi_tile_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(esi_tile_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(esi_tile_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn);
}

cudaError_t launch_bin(const BinArgs &a, int n_chunks, cudaStream_t s)
{
    const size_t smem = bin_smem_bytes(a.chunk, a.n_tiles);
    esi_bin_kernel<<<n_chunks, kBinThreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_tile(const TileArgs &a, int tile_h, cudaStream_t s)
{
    const size_t smem = tile_smem_bytes(tile_h, a.batch, a.n_chunks);
    switch (tile_h) {
    case 8: esi_tile_kernel<8><<<a.n_tiles, 8 * 32, smem, s>>>(a); break;
    case 16: esi_tile_kernel<16><<<a.n_tiles, 16 * 32, smem, s>>>(a); break;
    default: esi_tile_kernel<32><<<a.n_tiles, 32 * 32, smem, s>>>(a); break;
    }
    return cudaGetLastError();
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
