// Device helpers of the ESI kernels: the Alg. 2 update, the Eq. 4 decay, the
// Eq. 14 map, warp/block scans and the bulk-copy (TMA) / mbarrier PTX.
#pragma once

#include <cstdint>

#include "esi_internal.h"

namespace esi {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// ------------------------------------------------------ mbarrier + bulk copy
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// 1-D bulk copy global -> shared through the TMA unit, completing `bytes` of
// transaction count on `bar` (dst, src 16-byte aligned, bytes % 16 == 0),
// with an L2 evict-first hint: for data read exactly once (the events), so
// that it leaves L2 before data a later kernel reads again.
__device__ __forceinline__ void bulk_g2s_stream(void *dst, const void *src, unsigned bytes,
                                                uint64_t *bar)
{
    uint64_t policy;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(policy));
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned phase)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Asynchronous 8-byte global -> shared copy (no register round trip), and
// the wait for all of this thread's outstanding ones.
__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src)
                 : "memory");
}

__device__ __forceinline__ void cp_async4(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// Close the thread's outstanding cp.async copies into one group; wait until
// none of its groups is pending.
__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait_none()
{
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// Wait until at most one of the thread's groups is pending.
__device__ __forceinline__ void cp_async_wait_one()
{
    asm volatile("cp.async.wait_group 1;" ::: "memory");
}

// Wait for phase `phase` of `bar` for at most limit_ns; false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned phase,
                                                  unsigned long long limit_ns)
{
    unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, phase)) {
        if (global_ns() - t0 > limit_ns) return false;
    }
    return true;
}

// Lanes of the warp holding the same key (lanes with valid == false never
// match).  One ballot per key bit: much cheaper here than match.any.
__device__ __forceinline__ unsigned warp_peers(unsigned key, int nbits, bool valid)
{
    unsigned m = __ballot_sync(kFull, valid);
    for (int b = 0; b < nbits; ++b) {
        const bool bit = (key >> b) & 1u;
        const unsigned v = __ballot_sync(kFull, bit);
        m &= bit ? v : ~v;
    }
    return m;
}

template <int NBITS>
__device__ __forceinline__ unsigned warp_peers_n(unsigned key, bool valid)
{
    unsigned m = __ballot_sync(kFull, valid);
#pragma unroll
    for (int b = 0; b < NBITS; ++b) {
        const bool bit = (key >> b) & 1u;
        const unsigned v = __ballot_sync(kFull, bit);
        m &= bit ? v : ~v;
    }
    return m;
}

// ------------------------------------------------------------------- scans
__device__ __forceinline__ unsigned warp_inclusive_scan(unsigned v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned u = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Exclusive scan of one value per thread over the block; returns the prefix
// and writes the total to *total.  tmp holds NT/32 + 1 words.
template <int NT>
__device__ __forceinline__ unsigned block_exclusive_scan1(unsigned v, unsigned *tmp, unsigned *total)
{
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned inc = warp_inclusive_scan(v);
    if (lane == 31) tmp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        unsigned w = (lane < NW) ? tmp[lane] : 0u;
        unsigned wi = warp_inclusive_scan(w);
        if (lane < NW) tmp[lane] = wi - w;
        if (lane == NW - 1) tmp[NW] = wi;
    }
    __syncthreads();
    unsigned r = tmp[warp] + inc - v;
    *total = tmp[NW];
    __syncthreads();
    return r;
}

// In-place exclusive scan of data[0..n) (shared memory); returns the total.
template <int NT>
__device__ __forceinline__ unsigned block_exclusive_scan(unsigned *data, int n, unsigned *tmp)
{
    const int per = (n + NT - 1) / NT;
    const int b0 = min((int)threadIdx.x * per, n), b1 = min(b0 + per, n);
    unsigned s = 0;
    for (int i = b0; i < b1; ++i) s += data[i];
    unsigned total;
    unsigned run = block_exclusive_scan1<NT>(s, tmp, &total);
    for (int i = b0; i < b1; ++i) {
        unsigned d = data[i];
        data[i] = run;
        run += d;
    }
    __syncthreads();
    return total;
}

// ------------------------------------------------------------- the method
// 1 - k dt formed as (1 - k_hi dh) - (error terms) with dt = dh + dl split
// exactly and k_hi dh = p + e exactly (FMA), so that u keeps its relative
// accuracy when it is small (dt near the cutoff).
__device__ __forceinline__ float one_minus_kdt(long long dt, const DecayParams &dp)
{
    if (dt < (1ll << 24)) {
        // dt >= 0 is exact in FP32 here: no 64-bit conversion (slow on this
        // part) and no low part to carry
        const float dh = __int2float_rn((int)dt);
        const float p = dp.k_hi * dh;
        const float e = fmaf(dp.k_hi, dh, -p);
        return fmaxf((1.0f - p) - fmaf(dp.k_lo, dh, e), 0.0f);
    }
    float dh = __ll2float_rn(dt);
    float dl = __ll2float_rn(dt - __float2ll_rn(dh));
    float p = dp.k_hi * dh;
    float e = fmaf(dp.k_hi, dh, -p);
    float u = 1.0f - p;
    float corr = e + fmaf(dp.k_hi, dl, dp.k_lo * dh);
    return fmaxf(u - corr, 0.0f);
}

// exp(-k dt) for Eq. 3 (dt < cutoff, so k dt stays below about 110): with
// dt = dh + dl and k_hi dh = p + e split exactly as above, the small rest
// corr = k dt - p enters as the factor 1 - corr, so d keeps the relative
// accuracy of expf at its FP32 argument.
__device__ __forceinline__ float exp_kdt(long long dt, const DecayParams &dp)
{
    float dh, dl = 0.0f;
    if (dt < (1ll << 24)) {
        dh = __int2float_rn((int)dt);
    } else {
        dh = __ll2float_rn(dt);
        dl = __ll2float_rn(dt - __float2ll_rn(dh));
    }
    const float p = dp.k_hi * dh;
    const float e = fmaf(dp.k_hi, dh, -p);
    const float corr = e + fmaf(dp.k_hi, dl, dp.k_lo * dh);
    return expf(-p) * (1.0f - corr);
}

// Eq. 4 for the state update (accurate powf for non-integer b), or the
// exponential decay of Eq. 3.
__device__ __forceinline__ float decay_state(long long dt, const DecayParams &dp)
{
    if (dt >= dp.cutoff) return 0.0f;
    if (dp.b_mode == 4) return 1.0f;
    if (dp.b_mode == kBModeExp) return exp_kdt(dt, dp);
    float u = one_minus_kdt(dt, dp);
    switch (dp.b_mode) {
    case 1: return u;
    case 2: return u * u;
    case 3: return u * u * u;
    default: return powf(u, dp.b);
    }
}

// Decay kinds the kernels are specialised on.
enum DecayKind { kDecayGeneral = 0, kDecaySquare = 1, kDecayNone = 2 };

// Eq. 4 for the state update, specialised: b = 2 squares, k = 0 gives d = 1.
template <int DK>
__device__ __forceinline__ float decay_state_k(long long dt, const DecayParams &dp)
{
    if (DK == kDecayNone) return 1.0f;
    if (DK == kDecaySquare) {
        if (dt >= dp.cutoff) return 0.0f;
        const float u = one_minus_kdt(dt, dp);
        return u * u;
    }
    return decay_state(dt, dp);
}

// Eq. 4 for the render-time view from an FP32 time difference (exact below
// 2^24 us).  1 - k dt <= 0 gives d = 0; the decision may differ from the FP64
// one only where d is within rounding of 0, and only the 8-bit code uses it.
// Eq. 3's exponential view is exp(-k dt).
template <int DK>
__device__ __forceinline__ float decay_view_k(float dt, const DecayParams &dp)
{
    if (DK == kDecayNone) return 1.0f;
    if (DK == kDecayGeneral && dp.b_mode == kBModeExp) return expf(-dp.k_hi * dt);
    const float u = fmaxf(fmaf(-dp.k_hi, dt, 1.0f), 0.0f);
    if (DK == kDecaySquare) return u * u;
    switch (dp.b_mode) {
    case 1: return u;
    case 3: return u * u * u;
    default: return __powf(u, dp.b);
    }
}

// One event of a pixel (Alg. 2): S <- clamp((S + p C) d) with c = +-C.  The
// general decay kind also runs Eq. 3's order, S d + p C (b_mode kBModeExp);
// Alg. 1 and Eq. 3 come with infinite clamp bounds.
template <int DK>
__device__ __forceinline__ float event_step(float s, float c, float d, const DecayParams &dp,
                                            const MapParams &mp)
{
    float v;
    if (DK == kDecayGeneral) {
        const bool after = dp.b_mode == kBModeExp;
        v = fmaf(s + (after ? 0.0f : c), d, after ? c : 0.0f);
    } else {
        v = (s + c) * d;
    }
    return fminf(fmaxf(v, mp.s_min), mp.s_max);
}

// Round half to even and saturate to [0, 255] in one conversion.
__device__ __forceinline__ unsigned quantize_u8(float x)
{
    unsigned short r;
    asm("cvt.rni.sat.u8.f32 %0, %1;" : "=h"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void set_error(DevStatus *st, int code, int where)
{
    if (atomicCAS(&st->err, 0, code) == 0) st->err_where = where;
}

}  // namespace esi
