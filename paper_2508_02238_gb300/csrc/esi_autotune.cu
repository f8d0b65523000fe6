// Launch-shape autotuner (esi_autotune and esi_stream_autotune in esi.h).
//
// Every candidate shape runs the caller's sample through a scratch handle of
// the same sensor and parameters; the render is timed with CUDA events on the
// caller's stream (the first render of a candidate warms it up, the second
// counts).  The fastest shape is cached per (width, height, events-per-frame
// bucket, render mode, decay kind, flags), so that later sensors of the same
// kind reuse it without measuring.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "esi_api_impl.h"

namespace esi {

namespace {

using Key = std::tuple<int, int, int, int, int, int>;
std::mutex g_cache_mu;
std::map<Key, esi_tuning> g_cache;

Key key_of(const AutotuneKey &k)
{
    return Key{k.W, k.H, k.bucket, k.render_decay, k.decay_kind, k.flags};
}

int check_sample(const esi_event *sample, size_t n, const int64_t *t_frames, size_t m)
{
    if (!sample || n == 0 || !t_frames || m == 0) return ESI_EINVAL;
    for (size_t i = 1; i < n; ++i)
        if (sample[i].t_us < sample[i - 1].t_us) return ESI_ETIMEORDER;
    for (size_t w = 1; w < m; ++w)
        if (t_frames[w] < t_frames[w - 1]) return ESI_ETIMEORDER;
    return ESI_OK;
}

}  // namespace

int autotune_bucket(size_t n, size_t m)
{
    return (int)std::lround(std::log2(std::max(1.0, (double)n / (double)m)));
}

int autotune_shapes(const AutotuneKey &key, const esi_params &prm_in, cudaStream_t stream,
                    const esi_event *sample, size_t n, const int64_t *t_frames, size_t m,
                    const std::vector<esi_tuning> &cands, bool force, esi_tuning *best_out)
{
    int rc = check_sample(sample, n, t_frames, m);
    if (rc) return rc;
    if (!force) {
        std::lock_guard<std::mutex> lock(g_cache_mu);
        auto it = g_cache.find(key_of(key));
        if (it != g_cache.end()) {
            *best_out = it->second;
            return ESI_OK;
        }
    }
    // the scratch sensor starts no later than the sample
    esi_params prm = prm_in;
    prm.t_origin_us = std::min<long long>(prm.t_origin_us, std::min<long long>(sample[0].t_us, t_frames[0]));
    esi_handle *sh = nullptr;
    rc = esi_create(key.W, key.H, &prm, stream, &sh);
    if (rc) return rc;
    unsigned char *dframes = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc((void **)&dframes, m * (size_t)sh->P);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        esi_destroy(sh);
        cudaFree(dframes);
        return e == cudaErrorMemoryAllocation ? ESI_ENOMEM : ESI_ECUDA;
    }
    // every render of the scratch handle replays the sample one span later
    const long long span = std::max<long long>(t_frames[m - 1], sample[n - 1].t_us) -
                           std::min<long long>(sample[0].t_us, t_frames[0]) + 1;
    std::vector<esi_event> ev(sample, sample + n);
    std::vector<int64_t> tf(t_frames, t_frames + m);
    long long shift = 0;
    esi_tuning best{};
    float best_ms = 1e30f;
    for (const esi_tuning &cand : cands) {
        if (esi_set_tuning(sh, &cand) != ESI_OK) continue;
        float ms = 0.0f;
        for (int rep = 0; rep < 2 && rc == ESI_OK; ++rep) {
            shift += span;
            for (size_t i = 0; i < n; ++i) ev[i].t_us = sample[i].t_us + shift;
            for (size_t w = 0; w < m; ++w) tf[w] = t_frames[w] + shift;
            rc = esi_push_events(sh, ev.data(), n, 0);
            if (!rc) rc = cuda_fail(sh, cudaEventRecord(e0, sh->stream));
            if (!rc) rc = esi_render_frames(sh, tf.data(), m, dframes, 1);
            if (!rc) rc = cuda_fail(sh, cudaEventRecord(e1, sh->stream));
            if (!rc) rc = cuda_fail(sh, cudaEventSynchronize(e1));
            if (!rc) rc = cuda_fail(sh, cudaEventElapsedTime(&ms, e0, e1));
        }
        if (rc) break;
        if (ms < best_ms) {
            best_ms = ms;
            best = cand;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(dframes);
    esi_destroy(sh);
    if (rc) return rc;
    if (best_ms >= 1e30f) return ESI_ERANGE;
    {
        std::lock_guard<std::mutex> lock(g_cache_mu);
        g_cache[key_of(key)] = best;
    }
    *best_out = best;
    return ESI_OK;
}

}  // namespace esi

using namespace esi;

namespace {

std::vector<esi_tuning> handle_candidates(int flags)
{
    std::vector<esi_tuning> out;
    const int shapes[][2] = {{128, 4}, {128, 8}, {128, 16}, {64, 8}, {64, 16}, {32, 16}, {32, 32}};
    for (auto &sh : shapes) {
        if ((flags & ESI_AUTOTUNE_WIDE_ONLY) && sh[0] != 128) continue;
        for (int chunk : {2048, 4096})
            for (int batch : {2048, 4096})
                for (int mb : {1 << 21, 1 << 22, 1 << 23}) {
                    esi_tuning t{};
                    t.tile_w = sh[0];
                    t.tile_h = sh[1];
                    t.chunk_events = chunk;
                    t.batch_records = batch;
                    t.max_batch_events = mb;
                    out.push_back(t);
                }
    }
    return out;
}

}  // namespace

extern "C" int esi_autotune(esi_handle *h, const esi_event *sample, size_t n,
                            const int64_t *t_frames, size_t m, int flags, esi_tuning *chosen)
{
    if (!h || !chosen) return ESI_EINVAL;
    int rc = check_sample(sample, n, t_frames, m);
    if (rc) return rc;
    const AutotuneKey key{h->W, h->H, autotune_bucket(n, m), h->mp.render_decay,
                          decay_kind_of(h->dp), flags & ESI_AUTOTUNE_WIDE_ONLY};
    esi_tuning best{};
    rc = autotune_shapes(key, h->prm, h->stream, sample, n, t_frames, m, handle_candidates(flags),
                         (flags & ESI_AUTOTUNE_FORCE) != 0, &best);
    if (rc) return rc;
    *chosen = best;
    return esi_set_tuning(h, &best);
}
