// Diagnostics of Sec. III-B (Fig. 4): the noise-accumulation map
// ln(1 + |S|) of a handle's state and per-pixel event counts, from which the
// event-trigger rate map follows (counts over the window).  Both kernels
// stream HBM once: 8 B per pixel for the map, 16 B per event (plus the
// count array) for the counts.
#include <cmath>

#include "esi_api_impl.h"

namespace esi {

namespace {

constexpr int kDiagThreads = 256;

// Blocks for a grid-stride loop over `units` on the handle's device: enough
// to fill every SM several times, no more than the work needs.
int diag_blocks(const esi_handle *h, long long units)
{
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess || sms <= 0)
        sms = 1;
    const long long need = (units + kDiagThreads - 1) / kDiagThreads;
    const long long cap = (long long)sms * 8;
    return (int)(need < 1 ? 1 : need < cap ? need : cap);
}

// N = ln(1 + |S|) per pixel; four pixels per thread through 16-byte loads
// and stores where both arrays allow it.
__global__ void __launch_bounds__(kDiagThreads) esi_noise_map_kernel(const float *__restrict__ S,
                                                                     long long P, float *__restrict__ N,
                                                                     int vec4)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long done = 0;
    if (vec4) {
        const long long P4 = P / 4;
        const float4 *S4 = reinterpret_cast<const float4 *>(S);
        float4 *N4 = reinterpret_cast<float4 *>(N);
        for (long long i = i0; i < P4; i += stride) {
            const float4 s = __ldcs(S4 + i);
            float4 n;
            n.x = log1pf(fabsf(s.x));
            n.y = log1pf(fabsf(s.y));
            n.z = log1pf(fabsf(s.z));
            n.w = log1pf(fabsf(s.w));
            __stcs(N4 + i, n);
        }
        done = P4 * 4;
    }
    for (long long i = done + i0; i < P; i += stride) N[i] = log1pf(fabsf(S[i]));
}

__global__ void __launch_bounds__(kDiagThreads) esi_zero_u32_kernel(unsigned *c, long long n)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) c[i] = 0u;
}

// counts[y W + x] += 1 for every event inside the sensor.  Only the x, y
// word of each 16-byte event is read (the sectors come whole from HBM
// anyway); the adds are fire-and-forget reductions in L2.
__global__ void __launch_bounds__(kDiagThreads) esi_count_kernel(const esi_event *__restrict__ ev,
                                                                 long long n, int W, int H,
                                                                 unsigned *__restrict__ counts)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    const unsigned *words = reinterpret_cast<const unsigned *>(ev);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const unsigned xy = __ldcs(words + 4 * i + 2);
        const int x = (int)(xy & 0xffffu), y = (int)(xy >> 16);
        if (x < W && y < H) atomicAdd(counts + (long long)y * W + x, 1u);
    }
}

}  // namespace

}  // namespace esi

using namespace esi;

extern "C" int esi_noise_map(esi_handle *h, float *out, int out_on_device)
{
    if (!h || !out || (out_on_device != 0 && out_on_device != 1)) return ESI_EINVAL;
    const size_t bytes = (size_t)h->P * sizeof(float);
    float *dst = out;
    if (!out_on_device) {
        int rc = ensure_device(h, &h->diag, &h->diag_cap, bytes);
        if (rc) return rc;
        dst = reinterpret_cast<float *>(h->diag);
    }
    const int vec4 = ((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(h->S)) & 15u) == 0;
    cudaEvent_t ev = nullptr;
    int rc = prof_begin(h, &ev, h->stream);
    if (rc) return rc;
    esi_noise_map_kernel<<<diag_blocks(h, vec4 ? (h->P + 3) / 4 : h->P), kDiagThreads, 0, h->stream>>>(
        h->S, h->P, dst, vec4);
    rc = cuda_fail(h, cudaGetLastError());
    if (!rc) rc = prof_end(h, kKindNoise, ev, h->stream);
    if (rc) return rc;
    if (!out_on_device) {
        rc = cuda_fail(h, cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, h->stream));
        if (rc) return rc;
    }
    return read_status(h);
}

extern "C" int esi_count_events(esi_handle *h, const esi_event *events, size_t n, int events_on_device,
                                uint32_t *counts, int counts_on_device)
{
    if (!h || !counts || (n > 0 && !events)) return ESI_EINVAL;
    if ((events_on_device != 0 && events_on_device != 1) || (counts_on_device != 0 && counts_on_device != 1))
        return ESI_EINVAL;
    if (n > ((size_t)1 << 40)) return ESI_ERANGE;
    // scratch: [counts if on the host][events if on the host], 16-byte aligned
    const size_t cbytes = counts_on_device ? 0 : (((size_t)h->P * 4 + 15) & ~(size_t)15);
    const size_t ebytes = events_on_device ? 0 : n * sizeof(esi_event);
    if (cbytes + ebytes) {
        int rc = ensure_device(h, &h->diag, &h->diag_cap, cbytes + ebytes);
        if (rc) return rc;
    }
    unsigned *dcounts = counts_on_device ? counts : reinterpret_cast<unsigned *>(h->diag);
    const esi_event *dev = events_on_device ? events : reinterpret_cast<const esi_event *>(h->diag + cbytes);
    if (!events_on_device && n > 0) {
        int rc = cuda_fail(h, cudaMemcpyAsync(const_cast<esi_event *>(dev), events, ebytes,
                                              cudaMemcpyHostToDevice, h->stream));
        if (rc) return rc;
    }
    esi_zero_u32_kernel<<<diag_blocks(h, h->P), kDiagThreads, 0, h->stream>>>(dcounts, h->P);
    int rc = cuda_fail(h, cudaGetLastError());
    if (rc) return rc;
    h->launches += 1;
    if (n > 0) {
        cudaEvent_t ev = nullptr;
        rc = prof_begin(h, &ev, h->stream);
        if (rc) return rc;
        esi_count_kernel<<<diag_blocks(h, (long long)n), kDiagThreads, 0, h->stream>>>(dev, (long long)n, h->W,
                                                                                     h->H, dcounts);
        rc = cuda_fail(h, cudaGetLastError());
        if (!rc) rc = prof_end(h, kKindCount, ev, h->stream);
        if (rc) return rc;
    }
    if (!counts_on_device) {
        rc = cuda_fail(h, cudaMemcpyAsync(counts, dcounts, (size_t)h->P * 4, cudaMemcpyDeviceToHost,
                                          h->stream));
        if (rc) return rc;
    }
    return read_status(h);
}
