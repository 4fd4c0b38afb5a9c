// Host side of the C ABI declared in include/svgf.h: argument validation, workspace layout,
// temporal-state bookkeeping and kernel sequencing.  No device memory is allocated here.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <new>

#include "svgf.h"
#include "svgf_internal.h"

using svgf::Params;

struct svgf_handle {
    svgf_config cfg;
    Params P;
    size_t n_px;
    int n_tiles;
    // workspace
    unsigned char* ws = nullptr;
    size_t ws_bytes = 0;
    // workspace images in the storage precision (float4 or 8-byte records)
    void* hist[2] = {nullptr, nullptr};
    void* mom[2] = {nullptr, nullptr};
    void* cv_a = nullptr;
    void* cv_b = nullptr;
    void* sep = nullptr;
    int* tile_flags = nullptr;
    int* err_word = nullptr;
    // temporal state: slot of the latest frame's history, and whether it holds a history
    int slot = 0;
    int has_history = 0;
    int frame_open = 0;   // a frame's temporal stage ran; its a-trous passes may follow
    unsigned long long launches = 0;
    char last_error[256] = {0};
    // host-buffer staging (svgf_host_submit / svgf_host_wait / svgf_denoise_frame_host): two
    // slots of inputs and outputs for frames t and t + 1 in flight, three G-buffers (frame t's,
    // its predecessor's, and the one being uploaded for t + 1)
    unsigned char* stage = nullptr;
    float* st_noisy[2] = {nullptr, nullptr};
    float2* st_motion[2] = {nullptr, nullptr};
    float* st_rough[2] = {nullptr, nullptr};
    float4* st_out[2] = {nullptr, nullptr};   // rgb_out staging (FP32 in every precision)
    float4* st_gbuf[3] = {nullptr, nullptr, nullptr};
    unsigned long long st_frame = 0;           // frames submitted since binding / reset
    int st_have_prev = 0;
    // copy streams and the events that order uploads, denoise and downloads (created on first use)
    cudaStream_t st_in = nullptr, st_dl = nullptr;
    cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_comp[2] = {nullptr, nullptr},
                ev_out[2] = {nullptr, nullptr};
    // per-kernel event timing
    struct Rec { int kind; cudaEvent_t a, b; };
    static constexpr int kRing = 4096;
    Rec* ring = nullptr;
    int ring_used = 0;
    int prof_on = 0;
    double prof_ms[SVGF_K_COUNT] = {0};
    unsigned long long prof_n[SVGF_K_COUNT] = {0};
    ~svgf_handle() {
        for (int i = 0; i < 2; ++i) {
            if (ev_in[i]) cudaEventDestroy(ev_in[i]);
            if (ev_comp[i]) cudaEventDestroy(ev_comp[i]);
            if (ev_out[i]) cudaEventDestroy(ev_out[i]);
        }
        if (st_in) cudaStreamDestroy(st_in);
        if (st_dl) cudaStreamDestroy(st_dl);
        if (ring) {
            for (int i = 0; i < kRing; ++i) {
                cudaEventDestroy(ring[i].a);
                cudaEventDestroy(ring[i].b);
            }
            delete[] ring;
        }
    }
};

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

svgf_status check_config(const svgf_config* c) {
    if (!c) return SVGF_ERR_INVALID_ARG;
    if (c->width < 1 || c->height < 1 || c->width > 32768 || c->height > 32768)
        return SVGF_ERR_INVALID_ARG;
    if (!(c->alpha > 0.f && c->alpha <= 1.f) || !(c->alpha_moments > 0.f && c->alpha_moments <= 1.f))
        return SVGF_ERR_INVALID_ARG;
    if (!(c->clamp_gamma >= 0.f) || !isfinite(c->clamp_gamma)) return SVGF_ERR_INVALID_ARG;
    if (c->atrous_iters < 0 || c->atrous_iters > 8) return SVGF_ERR_INVALID_ARG;
    if (!(c->sigma_z >= 0.f) || !(c->sigma_n >= 0.f) || !(c->sigma_l >= 0.f)) return SVGF_ERR_INVALID_ARG;
    if (!isfinite(c->sigma_n)) return SVGF_ERR_INVALID_ARG;
    if (c->spatial_mode != SVGF_ATROUS_5X5 && c->spatial_mode != SVGF_SEPARABLE) return SVGF_ERR_INVALID_ARG;
    if (c->inverse_mode != SVGF_INVERSE_EXACT && c->inverse_mode != SVGF_INVERSE_PAPER) return SVGF_ERR_INVALID_ARG;
    if (!(c->luma_k > 0.f) || !isfinite(c->luma_k) || !isfinite(c->inv_weight)) return SVGF_ERR_INVALID_ARG;
    if (c->history_from_pass < -1) return SVGF_ERR_INVALID_ARG;
    if (!(c->depth_rel_tol >= 0.f) || !(c->normal_cos_tol >= -1.f && c->normal_cos_tol <= 1.f))
        return SVGF_ERR_INVALID_ARG;
    if (!(c->disocclusion_weight > 0.f && c->disocclusion_weight <= 1.f)) return SVGF_ERR_INVALID_ARG;
    if (c->max_history < 1 || c->max_history > 65535) return SVGF_ERR_INVALID_ARG;
    if (c->min_temporal_frames < 1 || c->spatial_var_radius < 0 || c->spatial_var_radius > 7)
        return SVGF_ERR_INVALID_ARG;
    if (!(c->eps > 0.f) || !isfinite(c->eps)) return SVGF_ERR_INVALID_ARG;
    if (!(c->roughness_threshold == c->roughness_threshold)) return SVGF_ERR_INVALID_ARG;
    if (c->precision != SVGF_FP32 && c->precision != SVGF_FP16 && c->precision != SVGF_BF16)
        return SVGF_ERR_INVALID_ARG;
    if (c->rectify_mode != SVGF_RECTIFY_CLAMP && c->rectify_mode != SVGF_RECTIFY_CLIP)
        return SVGF_ERR_INVALID_ARG;
    if (c->iter_by_roughness != 0 && c->iter_by_roughness != 1) return SVGF_ERR_INVALID_ARG;
    if (!(c->iter_rough_t0 <= c->iter_rough_t1)) return SVGF_ERR_INVALID_ARG;   // also rejects NaN
    // a budget above atrous_iters means every pass
    if (c->iter_count0 < 0 || c->iter_count0 > 8 || c->iter_count1 < 0 || c->iter_count1 > 8)
        return SVGF_ERR_INVALID_ARG;
    return SVGF_OK;
}

Params make_params(const svgf_config& c) {
    Params P;
    P.W = c.width;
    P.H = c.height;
    P.alpha = c.alpha;
    P.alpha_m = c.alpha_moments;
    P.gamma = c.clamp_gamma;
    P.sigma_z = c.sigma_z;
    P.sigma_n = c.sigma_n;
    P.sigma_l = c.sigma_l;
    P.clamp_enable = c.clamp_enable;
    P.adaptive_start = c.adaptive_start;
    P.rough_thr = c.roughness_threshold;
    P.tonemap = c.tonemap;
    P.luma_k = c.luma_k;
    P.inv_weight = c.inv_weight;
    P.inverse_mode = c.inverse_mode;
    P.depth_rel_tol = c.depth_rel_tol;
    P.normal_tol2 = 2.0f * (1.0f - c.normal_cos_tol);
    P.disocc_w = c.disocclusion_weight;
    P.max_history = (float)c.max_history;
    P.min_temporal = (float)c.min_temporal_frames;
    P.var_radius = c.spatial_var_radius;
    P.eps = c.eps;
    P.rectify_mode = c.rectify_mode;
    P.iter_budget = c.iter_by_roughness;
    P.iter_t0 = c.iter_rough_t0;
    P.iter_t1 = c.iter_rough_t1;
    P.iter_n0 = c.iter_count0;
    P.iter_n1 = c.iter_count1;
    P.iter_all = c.atrous_iters;
    const float cn = -c.sigma_n * 1.4426950408889634f;
    P.tc1 = cn * 0.5f;
    P.tc2 = cn * 0.125f;
    P.tc3 = cn * (1.0f / 24.0f);
    P.tc4 = cn * (1.0f / 64.0f);
    return P;
}

size_t image_bytes(const svgf_handle* h) {
    return align_up(h->n_px * svgf::image_bytes_per_px(h->cfg.precision));
}

// A caller's colour+variance buffer: 16-byte aligned float4 (FP32) or 8-byte aligned records.
bool cv_aligned(const svgf_handle* h, const void* p) {
    return ((uintptr_t)p & (h->cfg.precision == SVGF_FP32 ? 15u : 7u)) == 0;
}

size_t workspace_bytes(const svgf_handle* h) {
    const size_t img = image_bytes(h);
    return 7 * img + align_up((size_t)h->n_tiles * sizeof(int)) + kAlign;
}

svgf_status cuda_fail(svgf_handle* h, cudaError_t e) {
    if (e == cudaSuccess) return SVGF_OK;
    snprintf(h->last_error, sizeof h->last_error, "%s: %s", cudaGetErrorName(e),
             cudaGetErrorString(e));
    return SVGF_ERR_CUDA;
}

// Brackets one launch with the profiling events (when on) and counts it.
struct LaunchScope {
    svgf_handle* h;
    svgf_handle::Rec* r = nullptr;
    cudaStream_t s;
    LaunchScope(svgf_handle* hh, int kind, cudaStream_t ss) : h(hh), s(ss) {
        if (h->prof_on && h->ring_used < svgf_handle::kRing) {
            r = &h->ring[h->ring_used++];
            r->kind = kind;
            cudaEventRecord(r->a, s);
        }
    }
    svgf_status done(cudaError_t e) {
        if (e != cudaSuccess) {
            if (r) --h->ring_used;
            return cuda_fail(h, e);
        }
        if (r) cudaEventRecord(r->b, s);
        ++h->launches;
        return SVGF_OK;
    }
};

// The roughness image is read by the adaptive start (Sec. 3.2) and the pass budget (Sec. 3.5).
bool needs_roughness(const svgf_config& c) { return c.adaptive_start || c.iter_by_roughness; }

bool frame_ok(const svgf_handle* h, const svgf_frame* f) {
    if (!f || !f->noisy_rgb || !f->gbuf_nz || !f->motion) return false;
    if (!aligned16(f->gbuf_nz) || !aligned16(f->prev_gbuf_nz) || ((uintptr_t)f->motion & 7u) ||
        ((uintptr_t)f->noisy_rgb & 3u) || ((uintptr_t)f->roughness & 3u))
        return false;
    if (needs_roughness(h->cfg) && !f->roughness) return false;
    return true;
}

cudaStream_t as_stream(void* s) { return (cudaStream_t)s; }

// Temporal stage into `cv_out`, moments into the new slot; flips the slot.
svgf_status run_temporal(svgf_handle* h, const svgf_frame* f, void* cv_out, cudaStream_t s) {
    const int prev = h->slot, cur = h->slot ^ 1;
    const int hp = h->cfg.history_from_pass;
    const bool hist_from_accum = hp < 0 || hp >= h->cfg.atrous_iters;
    const int have = h->has_history && f->prev_gbuf_nz != nullptr;
    {
        LaunchScope L(h, SVGF_K_TEMPORAL, s);
        svgf_status st = L.done(svgf::launch_temporal(
            h->cfg.precision, h->P, f->noisy_rgb, (const float4*)f->gbuf_nz, (const float4*)f->prev_gbuf_nz,
            (const float2*)f->motion, h->hist[prev], h->mom[prev], have, cv_out, h->mom[cur],
            hist_from_accum ? h->hist[cur] : nullptr, h->tile_flags, s));
        if (st != SVGF_OK) return st;
    }
    {
        LaunchScope L(h, SVGF_K_SPATIAL_VAR, s);
        svgf_status st = L.done(svgf::launch_spatial_variance(
            h->cfg.precision, h->P, (const float4*)f->gbuf_nz, h->mom[cur], h->tile_flags, cv_out, s));
        if (st != SVGF_OK) return st;
    }
    h->slot = cur;
    h->has_history = 1;
    h->frame_open = 1;
    return SVGF_OK;
}

// One a-trous iteration cv_in -> (cv_out | rgb_out with the inverse map fused).
// need (optional): the pass computes only the 32x32 tiles set in it (need_tx tiles a row); for
// the separable mode need_h gives the horizontal pass's tiles.
svgf_status run_atrous(svgf_handle* h, int iter, const svgf_frame* f, const void* cv_in,
                       void* cv_out, float4* rgb_out, cudaStream_t s,
                       const unsigned char* need = nullptr, const unsigned char* need_h = nullptr,
                       int need_tx = 0) {
    const int pr = h->cfg.precision;
    void* hist_out = iter == h->cfg.history_from_pass ? h->hist[h->slot] : nullptr;
    const float* rough = needs_roughness(h->cfg) ? f->roughness : nullptr;
    if (h->cfg.spatial_mode == SVGF_SEPARABLE) {
        {
            LaunchScope L(h, SVGF_K_ATROUS_H, s);
            svgf_status st = L.done(svgf::launch_atrous(pr, h->P, 1, iter, cv_in, (const float4*)f->gbuf_nz,
                                                        rough, h->sep, nullptr, nullptr, s, need_h, need_tx));
            if (st != SVGF_OK) return st;
        }
        LaunchScope L(h, SVGF_K_ATROUS_V, s);
        return L.done(svgf::launch_atrous(pr, h->P, 2, iter, h->sep, (const float4*)f->gbuf_nz, rough,
                                          cv_out, hist_out, rgb_out, s, need, need_tx));
    }
    LaunchScope L(h, SVGF_K_ATROUS_5X5, s);
    return L.done(svgf::launch_atrous(pr, h->P, 0, iter, cv_in, (const float4*)f->gbuf_nz, rough,
                                      cv_out, hist_out, rgb_out, s, need, need_tx));
}

svgf_status run_inverse(svgf_handle* h, const void* cv_in, float4* rgb_out, cudaStream_t s) {
    LaunchScope L(h, SVGF_K_INVERSE, s);
    return L.done(svgf::launch_inverse(h->cfg.precision, h->P, cv_in, rgb_out, s));
}

svgf_status run_frame(svgf_handle* h, const svgf_frame* f, float4* rgb_out, cudaStream_t s) {
    svgf_status st = run_temporal(h, f, h->cv_a, s);
    if (st != SVGF_OK) return st;
    const int n = h->cfg.atrous_iters;
    if (n == 0) return run_inverse(h, h->cv_a, rgb_out, s);
    void* bufs[2] = {h->cv_a, h->cv_b};
    for (int i = 0; i < n; ++i) {
        const bool last = i == n - 1;
        st = run_atrous(h, i, f, bufs[i & 1], last ? nullptr : bufs[(i + 1) & 1],
                        last ? rgb_out : nullptr, s);
        if (st != SVGF_OK) return st;
    }
    return SVGF_OK;
}

size_t staging_bytes(const svgf_handle* h) {
    const size_t n = h->n_px;
    return 2 * (align_up(n * 12) + align_up(n * 8) + align_up(n * 4) + align_up(n * 16)) +
           3 * align_up(n * 16);
}

// Copy streams and ordering events of the host path, created on first use.
cudaError_t host_pipeline(svgf_handle* h) {
    if (h->st_in) return cudaSuccess;
    cudaError_t e = cudaStreamCreateWithFlags(&h->st_in, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->st_dl, cudaStreamNonBlocking);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = cudaEventCreateWithFlags(&h->ev_in[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_comp[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_out[i], cudaEventDisableTiming);
    }
    return e;
}

}  // namespace

extern "C" {

svgf_status svgf_default_config(int width, int height, svgf_config* out) {
    if (!out) return SVGF_ERR_INVALID_ARG;
    svgf_config c;
    memset(&c, 0, sizeof c);
    c.width = width;
    c.height = height;
    c.alpha = 0.2f;
    c.alpha_moments = 0.2f;
    c.clamp_gamma = 1.0f;
    c.atrous_iters = 5;
    c.sigma_z = 1.0f;
    c.sigma_n = 128.0f;
    c.sigma_l = 4.0f;
    c.spatial_mode = SVGF_ATROUS_5X5;
    c.clamp_enable = 1;
    c.adaptive_start = 1;
    c.roughness_threshold = 0.2f;
    c.tonemap = 1;
    c.luma_k = 1.0f;
    c.inv_weight = 1.0f;
    c.inverse_mode = SVGF_INVERSE_EXACT;
    c.history_from_pass = 0;
    c.depth_rel_tol = 0.1f;
    c.normal_cos_tol = 0.9f;
    c.disocclusion_weight = 1e-4f;
    c.max_history = 255;
    c.min_temporal_frames = 4;
    c.spatial_var_radius = 3;
    c.eps = 1e-10f;
    c.precision = SVGF_FP32;
    c.rectify_mode = SVGF_RECTIFY_CLAMP;
    c.iter_by_roughness = 0;
    c.iter_rough_t0 = 0.0f;
    c.iter_rough_t1 = 0.05f;
    c.iter_count0 = 0;
    c.iter_count1 = 1;
    *out = c;
    return (width >= 1 && height >= 1 && width <= 32768 && height <= 32768) ? SVGF_OK
                                                                             : SVGF_ERR_INVALID_ARG;
}

svgf_status svgf_channel_config(int channel, int width, int height, svgf_config* out) {
    if (!out || (channel != SVGF_CHANNEL_INDIRECT_SPECULAR && channel != SVGF_CHANNEL_SHADOW))
        return SVGF_ERR_INVALID_ARG;
    svgf_status st = svgf_default_config(width, height, out);
    if (st != SVGF_OK) return st;
    if (channel == SVGF_CHANNEL_SHADOW) {
        out->tonemap = 0;
        out->roughness_threshold = 6.0f;
    }
    return SVGF_OK;
}

svgf_status svgf_create(const svgf_config* cfg, svgf_handle** out) {
    if (!out) return SVGF_ERR_INVALID_ARG;
    *out = nullptr;
    svgf_status st = check_config(cfg);
    if (st != SVGF_OK) return st;
    svgf_handle* h = new (std::nothrow) svgf_handle;
    if (!h) return SVGF_ERR_INVALID_ARG;
    h->cfg = *cfg;
    h->P = make_params(*cfg);
    h->n_px = (size_t)cfg->width * cfg->height;
    dim3 g = svgf::tile_grid(cfg->width, cfg->height);
    h->n_tiles = (int)(g.x * g.y);
    *out = h;
    return SVGF_OK;
}

svgf_status svgf_destroy(svgf_handle* h) {
    delete h;
    return SVGF_OK;
}

svgf_status svgf_workspace_size(const svgf_handle* h, size_t* bytes) {
    if (!h || !bytes) return SVGF_ERR_INVALID_ARG;
    *bytes = workspace_bytes(h);
    return SVGF_OK;
}

svgf_status svgf_bind_workspace(svgf_handle* h, void* dev, size_t bytes) {
    if (!h || !dev || ((uintptr_t)dev % kAlign) != 0) return SVGF_ERR_INVALID_ARG;
    if (bytes < workspace_bytes(h)) return SVGF_ERR_NO_WORKSPACE;
    unsigned char* p = (unsigned char*)dev;
    const size_t img = image_bytes(h);
    h->ws = p;
    h->ws_bytes = bytes;
    h->hist[0] = p; p += img;
    h->hist[1] = p; p += img;
    h->mom[0] = p; p += img;
    h->mom[1] = p; p += img;
    h->cv_a = p; p += img;
    h->cv_b = p; p += img;
    h->sep = p; p += img;
    h->tile_flags = (int*)p; p += align_up((size_t)h->n_tiles * sizeof(int));
    h->err_word = (int*)p;
    h->slot = 0;
    h->has_history = 0;
    h->frame_open = 0;
    return SVGF_OK;
}

svgf_status svgf_reset_history(svgf_handle* h) {
    if (!h) return SVGF_ERR_INVALID_ARG;
    h->has_history = 0;
    h->frame_open = 0;
    h->st_have_prev = 0;
    return SVGF_OK;
}

svgf_status svgf_reproject_accumulate(svgf_handle* h, const svgf_frame* f, float* cv_out,
                                      void* stream) {
    if (!h) return SVGF_ERR_INVALID_ARG;
    if (!h->ws) return SVGF_ERR_NO_WORKSPACE;
    if (!frame_ok(h, f) || !cv_out || !cv_aligned(h, cv_out)) return SVGF_ERR_INVALID_ARG;
    return run_temporal(h, f, cv_out, as_stream(stream));
}

svgf_status svgf_clamp(svgf_handle* h, const svgf_frame* f, const float* hist_in,
                       float* hist_out, void* stream) {
    if (!h || !f || !f->noisy_rgb || ((uintptr_t)f->noisy_rgb & 3u)) return SVGF_ERR_INVALID_ARG;
    if (!hist_in || !hist_out || !aligned16(hist_in) || !aligned16(hist_out) || hist_in == hist_out)
        return SVGF_ERR_INVALID_ARG;
    LaunchScope L(h, SVGF_K_CLAMP, as_stream(stream));
    return L.done(svgf::launch_clamp(h->P, f->noisy_rgb, (const float4*)hist_in,
                                     (float4*)hist_out, as_stream(stream)));
}

svgf_status svgf_atrous(svgf_handle* h, int iter, const svgf_frame* f, const float* cv_in,
                        float* cv_out, void* stream) {
    if (!h) return SVGF_ERR_INVALID_ARG;
    if (!h->ws) return SVGF_ERR_NO_WORKSPACE;
    if (!frame_ok(h, f) || !cv_in || !cv_out || cv_in == cv_out || !cv_aligned(h, cv_in) ||
        !cv_aligned(h, cv_out))
        return SVGF_ERR_INVALID_ARG;
    if (iter < 0 || iter >= 16) return SVGF_ERR_INVALID_ARG;
    return run_atrous(h, iter, f, cv_in, cv_out, nullptr, as_stream(stream));
}

svgf_status svgf_inverse_tonemap(svgf_handle* h, const float* cv_in, float* rgb_out,
                                 void* stream) {
    if (!h || !cv_in || !rgb_out || !cv_aligned(h, cv_in) || !aligned16(rgb_out))
        return SVGF_ERR_INVALID_ARG;
    if (h->cfg.precision != SVGF_FP32 && (const void*)cv_in == (const void*)rgb_out)
        return SVGF_ERR_INVALID_ARG;
    return run_inverse(h, cv_in, (float4*)rgb_out, as_stream(stream));
}

svgf_status svgf_denoise_frame(svgf_handle* h, const svgf_frame* f, float* rgb_out,
                               void* stream) {
    if (!h) return SVGF_ERR_INVALID_ARG;
    if (!h->ws) return SVGF_ERR_NO_WORKSPACE;
    if (!frame_ok(h, f) || !rgb_out || !aligned16(rgb_out)) return SVGF_ERR_INVALID_ARG;
    return run_frame(h, f, (float4*)rgb_out, as_stream(stream));
}

svgf_status svgf_staging_size(const svgf_handle* h, size_t* bytes) {
    if (!h || !bytes) return SVGF_ERR_INVALID_ARG;
    *bytes = staging_bytes(h);
    return SVGF_OK;
}

svgf_status svgf_bind_staging(svgf_handle* h, void* dev, size_t bytes) {
    if (!h || !dev || ((uintptr_t)dev % kAlign) != 0) return SVGF_ERR_INVALID_ARG;
    if (bytes < staging_bytes(h)) return SVGF_ERR_NO_WORKSPACE;
    const size_t n = h->n_px;
    unsigned char* p = (unsigned char*)dev;
    h->stage = p;
    for (int i = 0; i < 2; ++i) {
        h->st_noisy[i] = (float*)p; p += align_up(n * 12);
        h->st_motion[i] = (float2*)p; p += align_up(n * 8);
        h->st_rough[i] = (float*)p; p += align_up(n * 4);
        h->st_out[i] = (float4*)p; p += align_up(n * 16);
    }
    for (int i = 0; i < 3; ++i) {
        h->st_gbuf[i] = (float4*)p; p += align_up(n * 16);
    }
    h->st_frame = 0;
    h->st_have_prev = 0;
    return SVGF_OK;
}

svgf_status svgf_host_submit(svgf_handle* h, const svgf_frame* hf, float* host_rgb_out,
                             void* stream) {
    if (!h) return SVGF_ERR_INVALID_ARG;
    if (!h->ws || !h->stage) return SVGF_ERR_NO_WORKSPACE;
    if (!hf || !hf->noisy_rgb || !hf->gbuf_nz || !hf->motion || !host_rgb_out)
        return SVGF_ERR_INVALID_ARG;
    if (needs_roughness(h->cfg) && !hf->roughness) return SVGF_ERR_INVALID_ARG;
    cudaError_t e = host_pipeline(h);
    if (e != cudaSuccess) return cuda_fail(h, e);
    cudaStream_t s = as_stream(stream);
    const size_t n = h->n_px;
    const unsigned long long t = h->st_frame;
    const int slot = (int)(t & 1), g = (int)(t % 3), gp = (int)((t + 2) % 3);
    // uploads: this slot's inputs and G-buffer g were last read by frame t - 2's denoise (an
    // event never recorded yet is complete)
    e = cudaStreamWaitEvent(h->st_in, h->ev_comp[slot], 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->st_noisy[slot], hf->noisy_rgb, n * 12, cudaMemcpyHostToDevice, h->st_in);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->st_gbuf[g], hf->gbuf_nz, n * 16, cudaMemcpyHostToDevice, h->st_in);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->st_motion[slot], hf->motion, n * 8, cudaMemcpyHostToDevice, h->st_in);
    if (e == cudaSuccess && hf->roughness)
        e = cudaMemcpyAsync(h->st_rough[slot], hf->roughness, n * 4, cudaMemcpyHostToDevice, h->st_in);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_in[slot], h->st_in);
    // the denoise on the caller's stream, after the uploads and after frame t - 2's download
    // has emptied this slot's output
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ev_in[slot], 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ev_out[slot], 0);
    if (e != cudaSuccess) return cuda_fail(h, e);
    svgf_frame df;
    df.noisy_rgb = h->st_noisy[slot];
    df.gbuf_nz = (const float*)h->st_gbuf[g];
    df.prev_gbuf_nz = h->st_have_prev ? (const float*)h->st_gbuf[gp] : nullptr;
    df.motion = (const float*)h->st_motion[slot];
    df.roughness = hf->roughness ? h->st_rough[slot] : nullptr;
    svgf_status st = run_frame(h, &df, h->st_out[slot], s);
    if (st != SVGF_OK) return st;
    e = cudaEventRecord(h->ev_comp[slot], s);
    // the download on the second copy stream
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->st_dl, h->ev_comp[slot], 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(host_rgb_out, h->st_out[slot], n * 16, cudaMemcpyDeviceToHost, h->st_dl);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_out[slot], h->st_dl);
    if (e != cudaSuccess) return cuda_fail(h, e);
    h->st_frame = t + 1;
    h->st_have_prev = 1;
    return SVGF_OK;
}

svgf_status svgf_host_wait(svgf_handle* h) {
    if (!h) return SVGF_ERR_INVALID_ARG;
    if (!h->st_in) return SVGF_OK;
    cudaError_t e = cudaStreamSynchronize(h->st_dl);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st_in);
    return cuda_fail(h, e);
}

svgf_status svgf_denoise_frame_host(svgf_handle* h, const svgf_frame* hf, float* host_rgb_out,
                                    void* stream) {
    svgf_status st = svgf_host_submit(h, hf, host_rgb_out, stream);
    if (st != SVGF_OK) return st;
    return svgf_host_wait(h);
}

svgf_status svgf_profile_enable(svgf_handle* h, int enable) {
    if (!h) return SVGF_ERR_INVALID_ARG;
    if (enable && !h->ring) {
        h->ring = new (std::nothrow) svgf_handle::Rec[svgf_handle::kRing];
        if (!h->ring) return SVGF_ERR_INVALID_ARG;
        for (int i = 0; i < svgf_handle::kRing; ++i) {
            cudaError_t e = cudaEventCreate(&h->ring[i].a);
            if (e == cudaSuccess) e = cudaEventCreate(&h->ring[i].b);
            if (e != cudaSuccess) {
                for (int j = 0; j < i; ++j) {
                    cudaEventDestroy(h->ring[j].a);
                    cudaEventDestroy(h->ring[j].b);
                }
                delete[] h->ring;
                h->ring = nullptr;
                return cuda_fail(h, e);
            }
        }
    }
    h->prof_on = enable ? 1 : 0;
    return SVGF_OK;
}

svgf_status svgf_profile_read(svgf_handle* h, double* total_ms, unsigned long long* counts,
                              int n_kinds) {
    if (!h || !total_ms || !counts || n_kinds < 1) return SVGF_ERR_INVALID_ARG;
    for (int i = 0; i < h->ring_used; ++i) {
        float ms = 0.f;
        cudaError_t e = cudaEventElapsedTime(&ms, h->ring[i].a, h->ring[i].b);
        if (e != cudaSuccess) return cuda_fail(h, e);
        h->prof_ms[h->ring[i].kind] += ms;
        h->prof_n[h->ring[i].kind] += 1;
    }
    h->ring_used = 0;
    for (int k = 0; k < n_kinds; ++k) {
        total_ms[k] = k < SVGF_K_COUNT ? h->prof_ms[k] : 0.0;
        counts[k] = k < SVGF_K_COUNT ? h->prof_n[k] : 0ull;
    }
    for (int k = 0; k < SVGF_K_COUNT; ++k) {
        h->prof_ms[k] = 0.0;
        h->prof_n[k] = 0;
    }
    return SVGF_OK;
}

svgf_status svgf_history_export(svgf_handle* h, float* hist_rgb, float* moments, void* stream) {
    if (!h) return SVGF_ERR_INVALID_ARG;
    if (!h->ws) return SVGF_ERR_NO_WORKSPACE;
    if (!hist_rgb || !moments || !aligned16(hist_rgb) || !aligned16(moments)) return SVGF_ERR_INVALID_ARG;
    return cuda_fail(h, svgf::launch_state_export(h->cfg.precision, (int)h->n_px, h->hist[h->slot],
                                                  h->mom[h->slot], (float4*)hist_rgb,
                                                  (float4*)moments, as_stream(stream)));
}

svgf_status svgf_history_import(svgf_handle* h, const float* hist_rgb, const float* moments,
                                int has_history, void* stream) {
    if (!h) return SVGF_ERR_INVALID_ARG;
    if (!h->ws) return SVGF_ERR_NO_WORKSPACE;
    if (has_history && (!hist_rgb || !moments || !aligned16(hist_rgb) || !aligned16(moments)))
        return SVGF_ERR_INVALID_ARG;
    if (!has_history) {
        h->has_history = 0;
        return SVGF_OK;
    }
    cudaError_t e = svgf::launch_state_import(h->cfg.precision, (int)h->n_px, (const float4*)hist_rgb,
                                              (const float4*)moments, h->hist[h->slot],
                                              h->mom[h->slot], as_stream(stream));
    if (e != cudaSuccess) return cuda_fail(h, e);
    h->has_history = 1;
    return SVGF_OK;
}

const char* svgf_status_string(svgf_status s) {
    switch (s) {
        case SVGF_OK: return "ok";
        case SVGF_ERR_INVALID_ARG: return "invalid argument";
        case SVGF_ERR_UNSUPPORTED: return "unsupported option";
        case SVGF_ERR_CUDA: return "CUDA error";
        case SVGF_ERR_TIMEOUT: return "device wait timed out";
        case SVGF_ERR_DEVICE_CHECK: return "device-side check failed";
        case SVGF_ERR_NO_WORKSPACE: return "no workspace bound";
    }
    return "unknown status";
}

const char* svgf_last_error(const svgf_handle* h) { return h ? h->last_error : ""; }

unsigned long long svgf_launch_count(const svgf_handle* h) { return h ? h->launches : 0ull; }

}  // extern "C"

// ---- separable iteration without any allocation ---------------------------------------------
// Scratch for the horizontal pass of svgf_atrous_separable_noalloc: a file-scope device array, so
// the call needs no device allocation.  Host code may not use the array's name as an address (on
// the host it names a host-side shadow); the device address is looked up with
// cudaGetSymbolAddress and passed to the kernels.  The lookup is cached per device together with
// the identity of the CUDA context it was made in: a device reset ends that context, and the array
// of the next one may sit elsewhere, so a call in a different context looks the address up again.
static __device__ __align__(256) float4 g_noalloc_scratch[SVGF_NOALLOC_MAX_PIXELS];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
float4* g_noalloc_addr[kMaxDevices] = {nullptr};
unsigned long long g_noalloc_ctx[kMaxDevices] = {0};

// Process-unique identity of the calling thread's current context (cuCtxGetId through the
// runtime's driver entry points, so the library needs no link to the driver library).
cudaError_t current_context_id(unsigned long long* id) {
    using GetCurrent = CUresult (*)(CUcontext*);
    using GetId = CUresult (*)(CUcontext, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    if (!get_current || !get_id) {
        void* a = nullptr;
        void* b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa);
        if (e == cudaSuccess)
            e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb);
        if (e != cudaSuccess) return e;
        if (qa != cudaDriverEntryPointSuccess || qb != cudaDriverEntryPointSuccess || !a || !b)
            return cudaErrorNotSupported;
        get_current = (GetCurrent)a;
        get_id = (GetId)b;
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, id) != CUDA_SUCCESS)
        return cudaErrorDeviceUninitialized;
    return cudaSuccess;
}

// Device address of the scratch array in the current device's current context (looked up on the
// first use in each context).
cudaError_t noalloc_scratch(float4** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    unsigned long long id = 0;
    const bool have_ctx = current_context_id(&id) == cudaSuccess;
    if (!g_noalloc_addr[dev] || !have_ctx || id != g_noalloc_ctx[dev]) {
        // a first use, or another context than the cached address's: look it up (this makes
        // the device's primary context current if no context is)
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        e = current_context_id(&id);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = (float4*)p;
        g_noalloc_ctx[dev] = id;
    }
    *out = g_noalloc_addr[dev];
    return cudaSuccess;
}
}  // namespace

extern "C" svgf_status svgf_atrous_separable_noalloc(svgf_handle* h, int iter,
                                                     const svgf_frame* f, const float* cv_in,
                                                     float* cv_out, void* stream) {
    if (!h) return SVGF_ERR_INVALID_ARG;
    if (h->n_px > (size_t)SVGF_NOALLOC_MAX_PIXELS) {
        snprintf(h->last_error, sizeof h->last_error,
                 "frame of %zu pixels exceeds the no-allocation scratch of %u pixels", h->n_px,
                 (unsigned)SVGF_NOALLOC_MAX_PIXELS);
        return SVGF_ERR_INVALID_ARG;
    }
    if (!frame_ok(h, f) || !cv_in || !cv_out || cv_in == cv_out || !cv_aligned(h, cv_in) ||
        !cv_aligned(h, cv_out))
        return SVGF_ERR_INVALID_ARG;
    if (iter < 0 || iter >= 16) return SVGF_ERR_INVALID_ARG;
    float4* scratch = nullptr;
    cudaError_t e = noalloc_scratch(&scratch);   // float4 slots hold any storage precision's records
    if (e != cudaSuccess) return cuda_fail(h, e);
    cudaStream_t s = as_stream(stream);
    const float* rough = needs_roughness(h->cfg) ? f->roughness : nullptr;
    {
        LaunchScope L(h, SVGF_K_ATROUS_H, s);
        svgf_status st = L.done(svgf::launch_atrous(h->cfg.precision, h->P, 1, iter, cv_in,
                                                    (const float4*)f->gbuf_nz, rough, scratch,
                                                    nullptr, nullptr, s));
        if (st != SVGF_OK) return st;
    }
    LaunchScope L(h, SVGF_K_ATROUS_V, s);
    return L.done(svgf::launch_atrous(h->cfg.precision, h->P, 2, iter, scratch,
                                      (const float4*)f->gbuf_nz, rough, cv_out, nullptr, nullptr, s));
}

// ---- batched streams --------------------------------------------------------------------------

struct svgf_batch {
    svgf_handle** hs = nullptr;
    int n = 0;
    svgf_config cfg;          // the shared configuration (width/height of handle 0)
    int sm_count = 0;
    int atrous_shape = 0;     // tile shape index of the batched a-trous kernel
    int atrous_bps = 0;       // a-trous grid: blocks per SM of the persistent grid, 0 = one per tile
    int stage_bps = 0;        // temporal / spatial-variance grid, same convention
    int use_graph = 0;
    cudaGraphExec_t exec = nullptr;
    char last_error[256] = {0};
    ~svgf_batch() {
        if (exec) cudaGraphExecDestroy(exec);
        delete[] hs;
    }
};

namespace {

// Streams of one batch share what selects the kernels and the launches: the storage precision,
// the spatial mode and the number of passes.  Everything else (tone mapping, thresholds,
// accumulation factors, rectification, ...) is per stream.
bool batch_compatible(const svgf_config& a, const svgf_config& b) {
    return a.precision == b.precision && a.spatial_mode == b.spatial_mode &&
           a.atrous_iters == b.atrous_iters;
}

svgf_status batch_fail(svgf_batch* b, cudaError_t e) {
    if (e == cudaSuccess) return SVGF_OK;
    snprintf(b->last_error, sizeof b->last_error, "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    for (int i = 0; i < b->n; ++i) snprintf(b->hs[i]->last_error, sizeof b->hs[i]->last_error, "%s", b->last_error);
    return SVGF_ERR_CUDA;
}

// Grid of a batched launch: bps blocks per SM walking the tiles with a grid stride, or, for
// bps = 0, one block per tile (the hardware block scheduler then balances uneven tiles).
int grid_for(int total, int sm_count, int bps) {
    if (bps <= 0) return total;
    const long g = (long)sm_count * bps;
    return (int)(total < g ? total : g);
}

// Temporal + spatial-variance stages of one frame for streams [i0, i1); flips their slots.
svgf_status batch_temporal(svgf_batch* b, int i0, int i1, const svgf_frame* frames, cudaStream_t s) {
    svgf::BatchTemporalArgs ta;
    svgf::BatchSpatialArgs sa;
    memset(&ta, 0, sizeof ta);
    memset(&sa, 0, sizeof sa);
    ta.n = sa.n = i1 - i0;
    int total = 0;
    for (int i = i0; i < i1; ++i) {
        svgf_handle* h = b->hs[i];
        const svgf_frame* f = &frames[i];
        const int prev = h->slot, cur = h->slot ^ 1;
        const int hp = h->cfg.history_from_pass;
        const bool hist_from_accum = hp < 0 || hp >= h->cfg.atrous_iters;
        const dim3 g = svgf::tile_grid(h->cfg.width, h->cfg.height);
        svgf::BTemporal& d = ta.s[i - i0];
        d.P = h->P;
        d.noisy = f->noisy_rgb;
        d.gbuf = (const float4*)f->gbuf_nz;
        d.prev_gbuf = (const float4*)f->prev_gbuf_nz;
        d.mv = (const float2*)f->motion;
        d.hist_prev = h->hist[prev];
        d.mom_prev = h->mom[prev];
        d.cv_out = h->cv_a;
        d.mom_out = h->mom[cur];
        d.hist_accum = hist_from_accum ? h->hist[cur] : nullptr;
        d.flags = h->tile_flags;
        d.W = h->cfg.width;
        d.H = h->cfg.height;
        d.tiles_x = (int)g.x;
        d.tile_base = total;
        d.has_history = h->has_history && f->prev_gbuf_nz != nullptr;
        svgf::BSpatial& e = sa.s[i - i0];
        e.P = h->P;
        e.gbuf = d.gbuf;
        e.mom = h->mom[cur];
        e.flags = h->tile_flags;
        e.cv = h->cv_a;
        e.W = d.W;
        e.H = d.H;
        e.tiles_x = d.tiles_x;
        e.tile_base = total;
        total += (int)(g.x * g.y);
    }
    ta.total = sa.total = total;
    svgf_handle* h0 = b->hs[i0];
    ta.uniform = sa.uniform = 1;
    for (int i = i0 + 1; i < i1; ++i) ta.uniform &= svgf::same_params_but_size(b->hs[i]->P, h0->P);
    sa.uniform = ta.uniform;
    ta.P = sa.P = h0->P;
    {
        LaunchScope L(h0, SVGF_K_TEMPORAL, s);
        svgf_status st = L.done(svgf::launch_batch_temporal(b->cfg.precision, ta,
                                                            grid_for(total, b->sm_count, b->stage_bps), s));
        if (st != SVGF_OK) return st;
    }
    {
        LaunchScope L(h0, SVGF_K_SPATIAL_VAR, s);
        svgf_status st = L.done(svgf::launch_batch_spatial(b->cfg.precision, sa,
                                                           grid_for(total, b->sm_count, b->stage_bps), s));
        if (st != SVGF_OK) return st;
    }
    for (int i = i0; i < i1; ++i) {
        svgf_handle* h = b->hs[i];
        h->slot ^= 1;
        h->has_history = 1;
        h->frame_open = 1;
    }
    return SVGF_OK;
}

// One a-trous iteration for streams [i0, i1).  chain = true: the frame's real ping-pong (pass i
// reads cv_a or cv_b by parity, the last pass writes outs[i] through the inverse map); chain =
// false (tuning): every pass reads cv_a and writes cv_b.
svgf_status batch_atrous(svgf_batch* b, int i0, int i1, int iter, const svgf_frame* frames,
                         float* const* outs, bool chain, int shape, int bps, cudaStream_t s) {
    const int n_it = b->cfg.atrous_iters;
    const bool last = chain && iter == n_it - 1;
    const bool sep = b->cfg.spatial_mode == SVGF_SEPARABLE;
    int tx, ty;
    svgf::atrous_shape(shape, &tx, &ty);
    svgf::BatchAtrousArgs a;
    memset(&a, 0, sizeof a);
    a.n = i1 - i0;
    a.iter = iter;
    for (int i = i0; i < i1; ++i) {
        svgf_handle* h = b->hs[i];
        svgf::BAtrous& d = a.s[i - i0];
        d.P = h->P;
        void* in = chain ? ((iter & 1) ? h->cv_b : h->cv_a) : h->cv_a;
        void* out = chain ? ((iter & 1) ? h->cv_a : h->cv_b) : h->cv_b;
        d.cv_in = in;
        d.gbuf = (const float4*)frames[i].gbuf_nz;
        d.rough = needs_roughness(h->cfg) ? frames[i].roughness : nullptr;
        d.cv_out = sep ? h->sep : out;
        d.hist_out = (!sep && iter == h->cfg.history_from_pass) ? h->hist[h->slot] : nullptr;
        d.rgb_out = (!sep && last) ? (float4*)outs[i] : nullptr;
        d.W = h->cfg.width;
        d.H = h->cfg.height;
    }
    a.P = b->hs[i0]->P;
    a.uniform = 1;
    for (int i = i0 + 1; i < i1; ++i) a.uniform &= svgf::same_params_but_size(b->hs[i]->P, a.P);
    // tiles of each stream for the pass's mode: rows spaced as in the per-frame kernel
    auto set_tiles = [&](int mode) {
        const int ys = svgf::atrous_row_spacing(mode, iter), rows = ty * ys;
        int total = 0;
        for (int k = 0; k < a.n; ++k) {
            svgf::BAtrous& d = a.s[k];
            d.tiles_x = (d.W + tx - 1) / tx;
            d.tile_base = total;
            total += d.tiles_x * (((d.H + rows - 1) / rows) * ys);
        }
        a.total = total;
        return grid_for(total, b->sm_count, bps);
    };
    svgf_handle* h0 = b->hs[i0];
    if (!sep) {
        const int grid = set_tiles(0);
        LaunchScope L(h0, SVGF_K_ATROUS_5X5, s);
        return L.done(svgf::launch_batch_atrous(b->cfg.precision, 0, shape, a, grid, s));
    }
    {
        const int grid = set_tiles(1);
        LaunchScope L(h0, SVGF_K_ATROUS_H, s);
        svgf_status st = L.done(svgf::launch_batch_atrous(b->cfg.precision, 1, shape, a, grid, s));
        if (st != SVGF_OK) return st;
    }
    for (int i = i0; i < i1; ++i) {
        svgf_handle* h = b->hs[i];
        svgf::BAtrous& d = a.s[i - i0];
        d.cv_in = h->sep;
        d.cv_out = chain ? ((iter & 1) ? h->cv_a : h->cv_b) : h->cv_b;
        d.hist_out = iter == h->cfg.history_from_pass ? h->hist[h->slot] : nullptr;
        d.rgb_out = last ? (float4*)outs[i] : nullptr;
    }
    const int grid = set_tiles(2);
    LaunchScope L(h0, SVGF_K_ATROUS_V, s);
    return L.done(svgf::launch_batch_atrous(b->cfg.precision, 2, shape, a, grid, s));
}

svgf_status batch_check(svgf_batch* b, const svgf_frame* frames, float* const* outs) {
    if (!b || !frames || !outs) return SVGF_ERR_INVALID_ARG;
    for (int i = 0; i < b->n; ++i) {
        if (!b->hs[i]->ws) return SVGF_ERR_NO_WORKSPACE;
        if (!frame_ok(b->hs[i], &frames[i]) || !outs[i] || !aligned16(outs[i])) return SVGF_ERR_INVALID_ARG;
    }
    return SVGF_OK;
}

svgf_status batch_enqueue(svgf_batch* b, const svgf_frame* frames, float* const* outs, cudaStream_t s) {
    for (int i0 = 0; i0 < b->n; i0 += svgf::kMaxBatch) {
        const int i1 = i0 + svgf::kMaxBatch < b->n ? i0 + svgf::kMaxBatch : b->n;
        svgf_status st = batch_temporal(b, i0, i1, frames, s);
        if (st != SVGF_OK) return st;
        for (int it = 0; it < b->cfg.atrous_iters; ++it) {
            st = batch_atrous(b, i0, i1, it, frames, outs, true, b->atrous_shape, b->atrous_bps, s);
            if (st != SVGF_OK) return st;
        }
    }
    return SVGF_OK;
}

}  // namespace

extern "C" {

svgf_status svgf_batch_create(svgf_handle* const* handles, int n, svgf_batch** out) {
    if (!out) return SVGF_ERR_INVALID_ARG;
    *out = nullptr;
    if (!handles || n < 1 || n > 1024) return SVGF_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
        if (!handles[i]) return SVGF_ERR_INVALID_ARG;
        if (!batch_compatible(handles[i]->cfg, handles[0]->cfg)) return SVGF_ERR_INVALID_ARG;
        for (int j = 0; j < i; ++j)
            if (handles[j] == handles[i]) return SVGF_ERR_INVALID_ARG;
    }
    if (handles[0]->cfg.atrous_iters < 1) return SVGF_ERR_UNSUPPORTED;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return SVGF_ERR_CUDA;
    svgf_batch* b = new (std::nothrow) svgf_batch;
    if (!b) return SVGF_ERR_INVALID_ARG;
    b->hs = new (std::nothrow) svgf_handle*[n];
    if (!b->hs) {
        delete b;
        return SVGF_ERR_INVALID_ARG;
    }
    for (int i = 0; i < n; ++i) b->hs[i] = handles[i];
    b->n = n;
    b->cfg = handles[0]->cfg;
    b->sm_count = sms;
    *out = b;
    return SVGF_OK;
}

svgf_status svgf_batch_destroy(svgf_batch* b) {
    delete b;
    return SVGF_OK;
}

svgf_status svgf_batch_use_graph(svgf_batch* b, int enable) {
    if (!b) return SVGF_ERR_INVALID_ARG;
    b->use_graph = enable ? 1 : 0;
    return SVGF_OK;
}

svgf_status svgf_batch_get_tuning(const svgf_batch* b, int* atrous_shape, int* blocks_per_sm) {
    if (!b || !atrous_shape || !blocks_per_sm) return SVGF_ERR_INVALID_ARG;
    *atrous_shape = b->atrous_shape;
    *blocks_per_sm = b->atrous_bps;
    return SVGF_OK;
}

svgf_status svgf_batch_set_tuning(svgf_batch* b, int atrous_shape, int blocks_per_sm) {
    if (!b || atrous_shape < 0 || atrous_shape >= svgf::kAtrousShapes || blocks_per_sm < 0 ||
        blocks_per_sm > 64)
        return SVGF_ERR_INVALID_ARG;
    b->atrous_shape = atrous_shape;
    b->atrous_bps = blocks_per_sm;
    return SVGF_OK;
}

svgf_status svgf_batch_denoise(svgf_batch* b, const svgf_frame* frames, float* const* outs,
                               void* stream) {
    svgf_status st = batch_check(b, frames, outs);
    if (st != SVGF_OK) return st;
    cudaStream_t s = as_stream(stream);
    if (!b->use_graph) return batch_enqueue(b, frames, outs, s);
    if (s == nullptr || s == cudaStreamLegacy || s == cudaStreamPerThread) return SVGF_ERR_INVALID_ARG;
    // capture this frame's launches, refresh the executable graph with them, launch it
    int saved_prof[1024];
    for (int i = 0; i < b->n; ++i) {
        saved_prof[i] = b->hs[i]->prof_on;
        b->hs[i]->prof_on = 0;   // no event records inside the graph
    }
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return batch_fail(b, e);
    st = batch_enqueue(b, frames, outs, s);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s, &g);
    for (int i = 0; i < b->n; ++i) b->hs[i]->prof_on = saved_prof[i];
    if (st != SVGF_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return batch_fail(b, e);
    if (b->exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(b->exec, g, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
    }
    if (!b->exec) e = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->exec = nullptr;
        return batch_fail(b, e);
    }
    return batch_fail(b, cudaGraphLaunch(b->exec, s));
}

svgf_status svgf_batch_autotune(svgf_batch* b, const svgf_frame* frames, float* const* outs,
                                void* stream, char* report, size_t report_len) {
    svgf_status st = batch_check(b, frames, outs);
    if (st != SVGF_OK) return st;
    cudaStream_t s = as_stream(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return batch_fail(b, ce);
    }
    size_t used = 0;
    if (report && report_len) report[0] = 0;
    float best = 1e30f;
    int best_shape = b->atrous_shape, best_bps = b->atrous_bps;
    for (int i0 = 0; i0 < b->n && st == SVGF_OK; i0 += svgf::kMaxBatch) {
        const int i1 = i0 + svgf::kMaxBatch < b->n ? i0 + svgf::kMaxBatch : b->n;
        st = batch_temporal(b, i0, i1, frames, s);
        if (st != SVGF_OK || i0 > 0) continue;   // candidates are timed on the first chunk
        // the kernel form the batch's launches take (as batch_atrous sets it)
        int uniform = 1;
        for (int i = i0 + 1; i < i1; ++i) uniform &= svgf::same_params_but_size(b->hs[i]->P, b->hs[i0]->P);
        const int form = !uniform ? 2 : svgf::series_only_normal(b->hs[i0]->P.sigma_n) ? 1 : 0;
        for (int shape = 0; shape < svgf::kAtrousShapes && st == SVGF_OK; ++shape) {
            // grids: one block per tile; persistent grids of 1x, 2x, 4x the resident blocks per SM
            const int occ = svgf::batch_atrous_occupancy(b->cfg.precision, b->cfg.spatial_mode == SVGF_SEPARABLE ? 2 : 0,
                                                         shape, form);
            const int kBps[4] = {0, occ > 0 ? occ : 1, 2 * (occ > 0 ? occ : 1), 4 * (occ > 0 ? occ : 1)};
            for (int k = 0; k < 4 && st == SVGF_OK; ++k) {
                // one untimed round, then the timed round: every pass of the frame, cv_a -> cv_b
                float ms = 0.f;
                for (int rep = 0; rep < 2 && st == SVGF_OK; ++rep) {
                    if (rep == 1) cudaEventRecord(e0, s);
                    for (int it = 0; it < b->cfg.atrous_iters && st == SVGF_OK; ++it)
                        st = batch_atrous(b, i0, i1, it, frames, outs, false, shape, kBps[k], s);
                    if (rep == 1) cudaEventRecord(e1, s);
                }
                if (st != SVGF_OK) break;
                ce = cudaEventSynchronize(e1);
                if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
                if (ce != cudaSuccess) {
                    st = batch_fail(b, ce);
                    break;
                }
                int tx, ty;
                svgf::atrous_shape(shape, &tx, &ty);
                if (report && used + 64 < report_len) {
                    if (kBps[k] == 0)
                        used += (size_t)snprintf(report + used, report_len - used,
                                                 "atrous %dx%d, one block per tile: %.4f ms\n", tx, ty, ms);
                    else
                        used += (size_t)snprintf(report + used, report_len - used,
                                                 "atrous %dx%d, %2d blocks/SM: %.4f ms\n", tx, ty, kBps[k], ms);
                }
                if (ms < best) {
                    best = ms;
                    best_shape = shape;
                    best_bps = kBps[k];
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != SVGF_OK) return st;
    b->atrous_shape = best_shape;
    b->atrous_bps = best_bps;
    // the frame's real a-trous chain with the chosen configuration (temporal ran above)
    for (int i0 = 0; i0 < b->n; i0 += svgf::kMaxBatch) {
        const int i1 = i0 + svgf::kMaxBatch < b->n ? i0 + svgf::kMaxBatch : b->n;
        for (int it = 0; it < b->cfg.atrous_iters; ++it) {
            st = batch_atrous(b, i0, i1, it, frames, outs, true, b->atrous_shape, b->atrous_bps, s);
            if (st != SVGF_OK) return st;
        }
    }
    return batch_fail(b, cudaStreamSynchronize(s));
}

}  // extern "C"

// ---- learned part ----------------------------------------------------------------------------

#include "svgf_kpn.h"

struct svgf_kpn {
    float* params = nullptr;
    float* grad = nullptr;
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    int max_px = 0;
    int sm_count = 0;
    long adam_t = 0;
    svgf::kpn::WeightPtrs w;
    // workspace images (max_px pixels each)
    __nv_bfloat16 *x1, *x2, *x3, *dzA, *dzB, *feats;
    float *K, *gK, *loss_sum;   // K, gK: 25 planes [25][pixels]
    float4 *c0, *c1, *c2, *u;
    unsigned char* tile_masks;   // kMaskArrays arrays of mask_stride bytes (one per 32x32 tile)
    size_t mask_stride;
    int* tile_count;
    int* err = nullptr;          // device error word (in the tile-count block of the workspace)
    int err_zeroed = 0;
    char last_error[256] = {0};
};

namespace {

// Tile masks of the fallback: the flagged tiles, then per plain pass (at most 8) the tiles of its
// output and of its horizontal half (separable mode).
constexpr int kMaskArrays = 1 + 2 * 8;

size_t kpn_layout(int max_px, svgf_kpn* k) {
    const size_t n = (size_t)max_px;
    size_t off = 0;
    auto take = [&](size_t bytes) -> size_t {
        const size_t o = off;
        off += align_up(bytes);
        return o;
    };
    const size_t o_fwd0 = take(9 * 32 * 16 * 2), o_fwd1 = take(9 * 32 * 32 * 2),
                 o_fwd2 = take(9 * 32 * 32 * 2), o_fwd3 = take(9 * 32 * 32 * 2);
    const size_t o_dg1 = take(9 * 32 * 32 * 2), o_dg2 = take(9 * 32 * 32 * 2), o_dg3 = take(9 * 32 * 32 * 2);
    const size_t o_b0 = take(128), o_b1 = take(128), o_b2 = take(128), o_b3 = take(128);
    const size_t o_x1 = take(n * 64), o_x2 = take(n * 64), o_x3 = take(n * 64);
    const size_t o_dzA = take(n * 64), o_dzB = take(n * 64), o_feats = take(n * 32);
    const size_t o_K = take(n * 100), o_gK = take(n * 100);
    const size_t o_c0 = take(n * 16), o_c1 = take(n * 16), o_c2 = take(n * 16), o_u = take(n * 16);
    // 32x32 tiles of a frame of n pixels, each side <= 32768: at most n/1024 + 2048 + 1; the
    // fallback's tile masks: the flagged tiles and, per plain pass, the tiles it computes
    const size_t mask_stride = align_up(n / 1024 + 2049);
    const size_t o_loss = take(64), o_count = take(64), o_masks = take(kMaskArrays * mask_stride);
    if (k) {
        unsigned char* b = (unsigned char*)k->x1;   // base passed through x1 by the caller
        k->w.fwd[0] = (__nv_bfloat16*)(b + o_fwd0);
        k->w.fwd[1] = (__nv_bfloat16*)(b + o_fwd1);
        k->w.fwd[2] = (__nv_bfloat16*)(b + o_fwd2);
        k->w.fwd[3] = (__nv_bfloat16*)(b + o_fwd3);
        k->w.dgrad[0] = nullptr;
        k->w.dgrad[1] = (__nv_bfloat16*)(b + o_dg1);
        k->w.dgrad[2] = (__nv_bfloat16*)(b + o_dg2);
        k->w.dgrad[3] = (__nv_bfloat16*)(b + o_dg3);
        k->w.bias[0] = (float*)(b + o_b0);
        k->w.bias[1] = (float*)(b + o_b1);
        k->w.bias[2] = (float*)(b + o_b2);
        k->w.bias[3] = (float*)(b + o_b3);
        k->x1 = (__nv_bfloat16*)(b + o_x1);
        k->x2 = (__nv_bfloat16*)(b + o_x2);
        k->x3 = (__nv_bfloat16*)(b + o_x3);
        k->dzA = (__nv_bfloat16*)(b + o_dzA);
        k->dzB = (__nv_bfloat16*)(b + o_dzB);
        k->feats = (__nv_bfloat16*)(b + o_feats);
        k->K = (float*)(b + o_K);
        k->gK = (float*)(b + o_gK);
        k->c0 = (float4*)(b + o_c0);
        k->c1 = (float4*)(b + o_c1);
        k->c2 = (float4*)(b + o_c2);
        k->u = (float4*)(b + o_u);
        k->loss_sum = (float*)(b + o_loss);
        k->tile_count = (int*)(b + o_count);
        k->err = (int*)(b + o_count) + 4;
        k->tile_masks = b + o_masks;
        k->mask_stride = mask_stride;
    }
    return off;
}

svgf_status kpn_fail(svgf_kpn* k, cudaError_t e) {
    if (e == cudaSuccess) return SVGF_OK;
    snprintf(k->last_error, sizeof k->last_error, "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    return SVGF_ERR_CUDA;
}

bool kpn_batch_ok(const svgf_kpn* k, const void* feats, const float* c0, int B, int H, int W) {
    if (!k || !feats || !c0 || B < 1 || H < 1 || W < 1) return false;
    if ((long)B * H * W > (long)k->max_px) return false;
    return aligned16(feats) && aligned16(c0);
}

// The device error word is zeroed on the stream before the first convolution after creation.
cudaError_t kpn_zero_err(svgf_kpn* k, cudaStream_t s) {
    if (k->err_zeroed) return cudaSuccess;
    const cudaError_t e = cudaMemsetAsync(k->err, 0, sizeof(int), s);
    if (e == cudaSuccess) k->err_zeroed = 1;
    return e;
}

// Forward through the four layers and the two applications (K and c1 kept for backward).
cudaError_t kpn_run_forward(svgf_kpn* k, const __nv_bfloat16* feats, const float4* c0, int B, int H,
                            int W, float4* c2, cudaStream_t s) {
    using namespace svgf::kpn;
    cudaError_t e = kpn_zero_err(k, s);
    if (e == cudaSuccess) e = conv(0, false, feats, k->w, nullptr, k->x1, B, H, W, k->sm_count, s, k->err);
    if (e == cudaSuccess) e = conv(1, false, k->x1, k->w, nullptr, k->x2, B, H, W, k->sm_count, s, k->err);
    if (e == cudaSuccess) e = conv(2, false, k->x2, k->w, nullptr, k->x3, B, H, W, k->sm_count, s, k->err);
    if (e == cudaSuccess) e = conv(3, false, k->x3, k->w, nullptr, k->K, B, H, W, k->sm_count, s, k->err);
    svgf::Params P;
    memset(&P, 0, sizeof P);
    if (e == cudaSuccess) e = apply(k->K, c0, k->c1, B, H, W, 1, P, nullptr, nullptr, s);
    if (e == cudaSuccess) e = apply(k->K, k->c1, c2, B, H, W, 4, P, nullptr, nullptr, s);
    return e;
}

cudaError_t kpn_run_grad(svgf_kpn* k, const __nv_bfloat16* feats, const float4* c0, const float4* T,
                         int B, int H, int W, float* loss_out, cudaStream_t s) {
    using namespace svgf::kpn;
    cudaError_t e = cudaMemsetAsync(k->grad, 0, sizeof(float) * kParamCount, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(k->loss_sum, 0, sizeof(float), s);
    if (e == cudaSuccess) e = kpn_run_forward(k, feats, c0, B, H, W, k->c2, s);
    if (e == cudaSuccess) e = backward_apply(k->K, c0, k->c1, k->c2, T, k->gK, k->u, k->dzA, k->loss_sum, B, H, W, s);
    if (e == cudaSuccess) e = wgrad(3, k->x3, k->dzA, k->grad, B, H, W, k->sm_count, s);
    if (e == cudaSuccess) e = conv(3, true, k->dzA, k->w, k->x3, k->dzB, B, H, W, k->sm_count, s, k->err);
    if (e == cudaSuccess) e = wgrad(2, k->x2, k->dzB, k->grad, B, H, W, k->sm_count, s);
    if (e == cudaSuccess) e = conv(2, true, k->dzB, k->w, k->x2, k->dzA, B, H, W, k->sm_count, s, k->err);
    if (e == cudaSuccess) e = wgrad(1, k->x1, k->dzA, k->grad, B, H, W, k->sm_count, s);
    if (e == cudaSuccess) e = conv(1, true, k->dzA, k->w, k->x1, k->dzB, B, H, W, k->sm_count, s, k->err);
    if (e == cudaSuccess) e = wgrad(0, feats, k->dzB, k->grad, B, H, W, k->sm_count, s);
    if (e == cudaSuccess && loss_out) e = loss_finish(k->loss_sum, loss_out, (long)B * H * W, s);
    return e;
}

}  // namespace

extern "C" {

svgf_status svgf_kpn_workspace_size(int max_pixels, size_t* bytes) {
    if (!bytes || max_pixels < 1) return SVGF_ERR_INVALID_ARG;
    *bytes = kpn_layout(max_pixels, nullptr);
    return SVGF_OK;
}

svgf_status svgf_kpn_create(float* params, float* grad, float* adam_m, float* adam_v,
                            void* workspace, size_t workspace_bytes, int max_pixels,
                            svgf_kpn** out) {
    if (!out) return SVGF_ERR_INVALID_ARG;
    *out = nullptr;
    if (!params || !workspace || max_pixels < 1 || ((uintptr_t)workspace % kAlign) != 0 ||
        ((uintptr_t)params & 3u))
        return SVGF_ERR_INVALID_ARG;
    if ((adam_m || adam_v) && !(adam_m && adam_v && grad)) return SVGF_ERR_INVALID_ARG;
    if (workspace_bytes < kpn_layout(max_pixels, nullptr)) return SVGF_ERR_NO_WORKSPACE;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SVGF_ERR_CUDA;
    svgf_kpn* k = new (std::nothrow) svgf_kpn;
    if (!k) return SVGF_ERR_INVALID_ARG;
    k->params = params;
    k->grad = grad;
    k->adam_m = adam_m;
    k->adam_v = adam_v;
    k->max_px = max_pixels;
    k->sm_count = sms;
    k->x1 = (__nv_bfloat16*)workspace;
    kpn_layout(max_pixels, k);
    *out = k;
    return SVGF_OK;
}

svgf_status svgf_kpn_check_device(svgf_kpn* k, int* word, void* stream) {
    if (!k) return SVGF_ERR_INVALID_ARG;
    int v = 0;
    if (k->err_zeroed) {
        cudaStream_t s = as_stream(stream);
        cudaError_t e = cudaMemcpyAsync(&v, k->err, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess && v != 0) e = cudaMemsetAsync(k->err, 0, sizeof(int), s);
        if (e != cudaSuccess) return kpn_fail(k, e);
    }
    if (word) *word = v;
    if (v == 0) return SVGF_OK;
    return v == svgf::kpn::kErrWaitGaveUp ? SVGF_ERR_TIMEOUT : SVGF_ERR_DEVICE_CHECK;
}

svgf_status svgf_kpn_wait_selftest(svgf_kpn* k, int tries, void* stream) {
    if (!k || tries < 1 || tries > (1 << 20)) return SVGF_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    cudaError_t e = kpn_zero_err(k, s);
    if (e == cudaSuccess) e = svgf::kpn::wait_expiry_probe(tries, k->err, s);
    return e == cudaSuccess ? SVGF_OK : kpn_fail(k, e);
}

svgf_status svgf_kpn_destroy(svgf_kpn* k) {
    delete k;
    return SVGF_OK;
}

svgf_status svgf_kpn_params_changed(svgf_kpn* k, int reset_adam, void* stream) {
    if (!k) return SVGF_ERR_INVALID_ARG;
    if (reset_adam) {
        k->adam_t = 0;
        if (k->adam_m) {
            cudaError_t e = cudaMemsetAsync(k->adam_m, 0, sizeof(float) * svgf::kpn::kParamCount, as_stream(stream));
            if (e == cudaSuccess)
                e = cudaMemsetAsync(k->adam_v, 0, sizeof(float) * svgf::kpn::kParamCount, as_stream(stream));
            if (e != cudaSuccess) return kpn_fail(k, e);
        }
    }
    return kpn_fail(k, svgf::kpn::prep_weights(k->params, k->w, as_stream(stream)));
}

// Checkpoint layout (little-endian): magic, version, parameter count, flags (bit 0: Adam state),
// Adam step count, parameters, then adam_m and adam_v when flagged.
constexpr uint32_t kKpnMagic = 0x504B5653u;   // "SVKP"
constexpr uint32_t kKpnVersion = 1u;
struct KpnCkptHeader {
    uint32_t magic, version, count, flags;
    uint64_t adam_t;
};

svgf_status svgf_kpn_save(svgf_kpn* k, void* host_buf, size_t* bytes, void* stream) {
    if (!k || !bytes) return SVGF_ERR_INVALID_ARG;
    const size_t n = svgf::kpn::kParamCount;
    const bool adam = k->adam_m != nullptr;
    const size_t need = sizeof(KpnCkptHeader) + sizeof(float) * n * (adam ? 3 : 1);
    if (!host_buf) {
        *bytes = need;
        return SVGF_OK;
    }
    if (*bytes < need) {
        *bytes = need;
        return SVGF_ERR_INVALID_ARG;
    }
    KpnCkptHeader hd{kKpnMagic, kKpnVersion, (uint32_t)n, adam ? 1u : 0u, (uint64_t)k->adam_t};
    unsigned char* b = (unsigned char*)host_buf;
    memcpy(b, &hd, sizeof hd);
    float* p = (float*)(b + sizeof hd);
    cudaStream_t s = as_stream(stream);
    cudaError_t e = cudaMemcpyAsync(p, k->params, sizeof(float) * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && adam)
        e = cudaMemcpyAsync(p + n, k->adam_m, sizeof(float) * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && adam)
        e = cudaMemcpyAsync(p + 2 * n, k->adam_v, sizeof(float) * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return kpn_fail(k, e);
    *bytes = need;
    return SVGF_OK;
}

svgf_status svgf_kpn_load(svgf_kpn* k, const void* host_buf, size_t bytes, void* stream) {
    if (!k || !host_buf || bytes < sizeof(KpnCkptHeader)) return SVGF_ERR_INVALID_ARG;
    KpnCkptHeader hd;
    memcpy(&hd, host_buf, sizeof hd);
    const size_t n = svgf::kpn::kParamCount;
    if (hd.magic != kKpnMagic || hd.version != kKpnVersion || hd.count != n || (hd.flags & ~1u))
        return SVGF_ERR_INVALID_ARG;
    const bool adam_in = (hd.flags & 1u) != 0;
    if (bytes < sizeof hd + sizeof(float) * n * (adam_in ? 3 : 1)) return SVGF_ERR_INVALID_ARG;
    const float* p = (const float*)((const unsigned char*)host_buf + sizeof hd);
    cudaStream_t s = as_stream(stream);
    cudaError_t e = cudaMemcpyAsync(k->params, p, sizeof(float) * n, cudaMemcpyHostToDevice, s);
    const bool adam = adam_in && k->adam_m != nullptr;
    if (e == cudaSuccess && adam)
        e = cudaMemcpyAsync(k->adam_m, p + n, sizeof(float) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && adam)
        e = cudaMemcpyAsync(k->adam_v, p + 2 * n, sizeof(float) * n, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return kpn_fail(k, e);
    // without saved moments the optimiser restarts: zeroed moments and step count
    svgf_status st = svgf_kpn_params_changed(k, adam ? 0 : 1, stream);
    if (st != SVGF_OK) return st;
    if (adam) k->adam_t = (long)hd.adam_t;
    return kpn_fail(k, cudaStreamSynchronize(s));
}

svgf_status svgf_kpn_forward(svgf_kpn* k, const void* feats, const float* c0, int B, int H, int W,
                             float* c2_out, void* stream) {
    if (!kpn_batch_ok(k, feats, c0, B, H, W) || !c2_out || !aligned16(c2_out)) return SVGF_ERR_INVALID_ARG;
    return kpn_fail(k, kpn_run_forward(k, (const __nv_bfloat16*)feats, (const float4*)c0, B, H, W,
                                       (float4*)c2_out, as_stream(stream)));
}

svgf_status svgf_kpn_predict(svgf_kpn* k, const void* feats, int B, int H, int W, void* kernels_out,
                             int form, void* stream) {
    if (!k || !feats || !kernels_out || B < 1 || H < 1 || W < 1 || form < 0 || form > 2)
        return SVGF_ERR_INVALID_ARG;
    if ((long)B * H * W > (long)k->max_px || !aligned16(feats) || !aligned16(kernels_out))
        return SVGF_ERR_INVALID_ARG;
    using namespace svgf::kpn;
    cudaStream_t s = as_stream(stream);
    const __nv_bfloat16* x = (const __nv_bfloat16*)feats;
    cudaError_t e = kpn_zero_err(k, s);
    if (form == 0) {
        if (e == cudaSuccess) e = net_forward(x, k->w, kernels_out, B, H, W, k->sm_count, s, k->err);
    } else if (form == 2) {
        if (e == cudaSuccess) e = net_pairs(x, k->w, k->x2, kernels_out, B, H, W, k->sm_count, s, k->err);
    } else {
        if (e == cudaSuccess) e = conv(0, false, x, k->w, nullptr, k->x1, B, H, W, k->sm_count, s, k->err);
        if (e == cudaSuccess) e = conv(1, false, k->x1, k->w, nullptr, k->x2, B, H, W, k->sm_count, s, k->err);
        if (e == cudaSuccess) e = conv(2, false, k->x2, k->w, nullptr, k->x3, B, H, W, k->sm_count, s, k->err);
        if (e == cudaSuccess) e = conv(4, false, k->x3, k->w, nullptr, kernels_out, B, H, W, k->sm_count, s, k->err);
    }
    return kpn_fail(k, e);
}

svgf_status svgf_kpn_grad(svgf_kpn* k, const void* feats, const float* c0, const float* target,
                          int B, int H, int W, float* loss_out, void* stream) {
    if (!kpn_batch_ok(k, feats, c0, B, H, W) || !k->grad || !target || !aligned16(target))
        return SVGF_ERR_INVALID_ARG;
    return kpn_fail(k, kpn_run_grad(k, (const __nv_bfloat16*)feats, (const float4*)c0,
                                    (const float4*)target, B, H, W, loss_out, as_stream(stream)));
}

svgf_status svgf_kpn_train_step(svgf_kpn* k, const void* feats, const float* c0,
                                const float* target, int B, int H, int W, float lr,
                                float* loss_out, void* stream) {
    if (!kpn_batch_ok(k, feats, c0, B, H, W) || !k->grad || !k->adam_m || !target ||
        !aligned16(target) || !(lr > 0.f))
        return SVGF_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    cudaError_t e = kpn_run_grad(k, (const __nv_bfloat16*)feats, (const float4*)c0,
                                 (const float4*)target, B, H, W, loss_out, s);
    if (e != cudaSuccess) return kpn_fail(k, e);
    k->adam_t += 1;
    const double b1 = 0.9, b2 = 0.999;
    const float bc1 = (float)(1.0 - pow(b1, (double)k->adam_t));
    const float bc2 = (float)(1.0 - pow(b2, (double)k->adam_t));
    e = svgf::kpn::adam(k->params, k->grad, k->adam_m, k->adam_v, lr, (float)b1, (float)b2, 1e-8f, bc1, bc2, s);
    if (e == cudaSuccess) e = svgf::kpn::prep_weights(k->params, k->w, s);
    return kpn_fail(k, e);
}

svgf_status svgf_kpn_features(svgf_handle* h, const void* cv, const svgf_frame* f,
                              const float* albedo, void* feats_out, float* c0_out, void* stream) {
    if (!h || !cv || !f || !f->gbuf_nz || !albedo || !feats_out || !cv_aligned(h, cv) ||
        !aligned16(feats_out) || !aligned16(f->gbuf_nz) || (c0_out && !aligned16(c0_out)))
        return SVGF_ERR_INVALID_ARG;
    return cuda_fail(h, svgf::kpn::features(h->cfg.precision, cv, (const float4*)f->gbuf_nz, albedo,
                                            (__nv_bfloat16*)feats_out, (float4*)c0_out, (int)h->n_px,
                                            as_stream(stream)));
}

svgf_status svgf_kpn_apply(svgf_kpn* k, svgf_handle* h, const void* kernels, const float* c0, float* rgb_out,
                           void* stream) {
    if (!k || !h || !kernels || !c0 || !rgb_out) return SVGF_ERR_INVALID_ARG;
    if (!aligned16(kernels) || !aligned16(c0) || !aligned16(rgb_out)) return SVGF_ERR_INVALID_ARG;
    if ((long)h->n_px > (long)k->max_px) return SVGF_ERR_NO_WORKSPACE;
    using namespace svgf::kpn;
    cudaStream_t s = as_stream(stream);
    const int W = h->cfg.width, H = h->cfg.height;
    cudaError_t e = apply_h(kernels, (const float4*)c0, k->c1, 1, H, W, 1, h->P, nullptr, nullptr, s);
    if (e == cudaSuccess) e = apply_h(kernels, k->c1, nullptr, 1, H, W, 4, h->P, (float4*)rgb_out, (const float4*)c0, s);
    return cuda_fail(h, e);
}

svgf_status svgf_kpn_denoise_frame(svgf_kpn* k, svgf_handle* h, const svgf_frame* f,
                                   const float* albedo, float* rgb_out, float detail_threshold,
                                   int* fallback_tiles, void* stream) {
    if (!k || !h) return SVGF_ERR_INVALID_ARG;
    if (!h->ws) return SVGF_ERR_NO_WORKSPACE;
    if (!frame_ok(h, f) || !albedo || !rgb_out || !aligned16(rgb_out)) return SVGF_ERR_INVALID_ARG;
    if ((long)h->n_px > (long)k->max_px) return SVGF_ERR_NO_WORKSPACE;
    if (h->cfg.atrous_iters < 1) return SVGF_ERR_UNSUPPORTED;
    cudaStream_t s = as_stream(stream);
    const int W = h->cfg.width, H = h->cfg.height;
    svgf_status st = run_temporal(h, f, h->cv_a, s);
    if (st != SVGF_OK) return st;
    st = run_atrous(h, 0, f, h->cv_a, h->cv_b, nullptr, s);
    if (st != SVGF_OK) return st;
    using namespace svgf::kpn;
    cudaError_t e = kpn_zero_err(k, s);
    if (e == cudaSuccess)
        e = features(h->cfg.precision, h->cv_b, (const float4*)f->gbuf_nz, albedo, k->feats, k->c0,
                     (int)h->n_px, s);
    // inference: the network layer by layer (faster than the four-layer kernel of
    // svgf_kpn_predict's form 0, whose four-slot accumulator rings tie each layer's issue to its
    // own drain every two rows), the kernels as FP16, pixel-major (64 B per pixel instead of 25
    // FP32 planes)
    if (e == cudaSuccess) e = conv(0, false, k->feats, k->w, nullptr, k->x1, 1, H, W, k->sm_count, s, k->err);
    if (e == cudaSuccess) e = conv(1, false, k->x1, k->w, nullptr, k->x2, 1, H, W, k->sm_count, s, k->err);
    if (e == cudaSuccess) e = conv(2, false, k->x2, k->w, nullptr, k->x3, 1, H, W, k->sm_count, s, k->err);
    if (e == cudaSuccess) e = conv(4, false, k->x3, k->w, nullptr, k->K, 1, H, W, k->sm_count, s, k->err);
    // the two applications (one launch computing both, the dilation-1 result recomputed over
    // the reach of the dilation-4 taps in shared memory, measured slower: 152 against 109 us at
    // 1080p)
    if (e == cudaSuccess) e = apply_h(k->K, k->c0, k->c1, 1, H, W, 1, h->P, nullptr, nullptr, s);
    if (e == cudaSuccess) e = apply_h(k->K, k->c1, nullptr, 1, H, W, 4, h->P, (float4*)rgb_out, k->c0, s);
    if (e != cudaSuccess) return cuda_fail(h, e);
    h->launches += 7;   // features, four convolutions, two applications
    if (fallback_tiles) *fallback_tiles = 0;
    if (!isfinite(detail_threshold)) return SVGF_OK;
    const int ntx = (W + 31) / 32, nty = (H + 31) / 32;
    unsigned char* flags = k->tile_masks;
    e = cudaMemsetAsync(k->tile_count, 0, sizeof(int), s);
    if (e == cudaSuccess) e = tile_flags(k->c0, H, W, detail_threshold, flags, k->tile_count, s);
    if (e == cudaSuccess) ++h->launches;
    int count = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&count, k->tile_count, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(h, e);
    if (fallback_tiles) *fallback_tiles = count;
    if (count == 0) return SVGF_OK;
    // Plain passes 1.. from the pass-0 output (cv_b), the last one into c2 with the inverse map,
    // each on the tiles the flagged tiles depend on: pass i reads its input within 2 step_i
    // pixels (step_i = 2^(i + 1) with the adaptive start), so going back from the flagged tiles
    // each pass's region is the next one's dilated by ceil(2 step_i / 32) tiles (twice in the
    // separable mode: the vertical half reads the horizontal half's output, which reads the
    // input).  A pass that writes the colour history covers the whole frame, and so do the
    // passes before it.
    const int n = h->cfg.atrous_iters;
    const bool sep = h->cfg.spatial_mode == SVGF_SEPARABLE;
    const int hp = h->cfg.history_from_pass;
    const bool regions = hp < 1 || hp >= n;
    auto mask = [&](int j) { return k->tile_masks + (size_t)j * k->mask_stride; };
    const unsigned char* out_m[8] = {nullptr};
    const unsigned char* h_m[8] = {nullptr};
    if (regions) {
        const int lvl = h->cfg.adaptive_start ? 1 : 0;
        out_m[n - 1] = flags;
        for (int i = n - 1; i >= 1 && e == cudaSuccess; --i) {
            const int reach = 2 << (i + lvl);
            const int r = (reach + 31) / 32;
            const unsigned char* src = out_m[i];
            if (sep) {
                e = tile_dilate(src, mask(2 * i - 1), ntx, nty, r, s);
                h_m[i] = mask(2 * i - 1);
                src = h_m[i];
                ++h->launches;
            }
            if (i > 1 && e == cudaSuccess) {
                e = tile_dilate(src, mask(2 * i), ntx, nty, r, s);
                out_m[i - 1] = mask(2 * i);
                ++h->launches;
            }
        }
        if (e != cudaSuccess) return cuda_fail(h, e);
    }
    void* bufs[2] = {h->cv_b, h->cv_a};
    for (int i = 1; i < n; ++i) {
        const bool last = i == n - 1;
        st = run_atrous(h, i, f, bufs[(i - 1) & 1], last ? nullptr : bufs[i & 1],
                        last ? k->c2 : nullptr, s, out_m[i], h_m[i], ntx);
        if (st != SVGF_OK) return st;
    }
    if (n == 1) {
        st = run_inverse(h, h->cv_b, k->c2, s);
        if (st != SVGF_OK) return st;
    }
    ++h->launches;
    return cuda_fail(h, tile_select(k->c2, flags, (float4*)rgb_out, H, W, s));
}

}  // extern "C"
