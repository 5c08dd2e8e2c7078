// extern "C" entry points of gs.h: argument validation, scratch carving,
// and stage launches on the context's stream.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "gs_common.cuh"

namespace gs {

gs_status set_error(gs_context* ctx, gs_status st, const char* fmt, ...) {
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
        va_end(ap);
    }
    return st;
}

gs_status check_launch(gs_context* ctx, const char* what) {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(ctx, GS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return GS_OK;
}

int64_t scan_blocks_for(int64_t n) { return (n + kScanBlock - 1) / kScanBlock; }

namespace {
constexpr int64_t kAlign = 256;
int64_t align_up(int64_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
}  // namespace

ScratchLayout scratch_layout(int64_t ncap, int64_t kcap, int64_t range_warps) {
    ScratchLayout L;
    int64_t off = 0;
    L.status = off;
    off += align_up(kStatusWords * 4);
    L.partials = off;
    off += align_up((scan_blocks_for(ncap) + 1) * 8);
    L.hist = off;
    off += align_up(kSortCtlWords * 4);
    L.lookback = off;
    off += align_up(2 * std::max<int64_t>(sort_partitions_for(kcap), 1) * 256 * 4);
    L.order = off;
    off += align_up((int64_t)kMaxOrderedTiles * 4);
    L.warp_range = off;
    off += align_up(std::max<int64_t>(range_warps ? range_warps : (ncap + kPreThreads - 1) / kPreThreads *
                                                                     (kPreThreads / 32),
                                      1) * 8);
    L.block_range = off;
    off += align_up(std::max<int64_t>(scan_blocks_for(ncap), 1) * 8);
    L.total = off;
    return L;
}

namespace {

bool valid_tile(int t) { return t == 8 || t == 16 || t == 32; }

gs_status check_cam(gs_context* ctx, const gs_camera* cam, const gs_frame* f) {
    if (!cam) return set_error(ctx, GS_ERR_INVALID, "camera is NULL");
    if (cam->width != f->width || cam->height != f->height)
        return set_error(ctx, GS_ERR_INVALID, "camera %dx%d does not match frame %dx%d", cam->width, cam->height,
                         f->width, f->height);
    return GS_OK;
}

gs_status check_scene(gs_context* ctx, const gs_scene* scene, const gs_frame* frame) {
    if (!scene) return set_error(ctx, GS_ERR_INVALID, "scene is NULL");
    if (scene->n < 0 || scene->n > frame->n_capacity)
        return set_error(ctx, GS_ERR_INVALID, "scene n %lld exceeds frame n_capacity %lld", (long long)scene->n,
                         (long long)frame->n_capacity);
    if (scene->sh_degree < 0 || scene->sh_degree > 3)
        return set_error(ctx, GS_ERR_INVALID, "sh_degree %d not in 0..3", scene->sh_degree);
    if (scene->n > 0 && (!scene->means || !scene->scales || !scene->rotations || !scene->opacities || !scene->sh))
        return set_error(ctx, GS_ERR_INVALID, "scene has a NULL array");
    return GS_OK;
}

gs_status check_cfg(gs_context* ctx, const gs_raster_cfg* cfg, const gs_frame* f) {
    if (!cfg) return set_error(ctx, GS_ERR_INVALID, "cfg is NULL");
    if (cfg->tile != f->tile) return set_error(ctx, GS_ERR_INVALID, "cfg tile %d != frame tile %d", cfg->tile, f->tile);
    if (cfg->mode < GS_MODE_3SIGMA || cfg->mode > GS_MODE_PIXEL)
        return set_error(ctx, GS_ERR_INVALID, "mode %d is not a gs_mode", cfg->mode);
    if (cfg->sort_digit_bits != 0 && (cfg->sort_digit_bits < 4 || cfg->sort_digit_bits > 8))
        return set_error(ctx, GS_ERR_INVALID, "sort_digit_bits %d not in {0, 4..8}", cfg->sort_digit_bits);
    return GS_OK;
}

}  // namespace

bool make_view(gs_context* ctx, const gs_frame* f, FrameView* v, unsigned need) {
    if (!f) {
        set_error(ctx, GS_ERR_INVALID, "frame is NULL");
        return false;
    }
    if (!valid_tile(f->tile) || f->width <= 0 || f->height <= 0 || f->n_capacity < 0 || f->key_capacity < 0 ||
        f->key_capacity > GS_MAX_KEYS || f->n_capacity > (int64_t)0xffffffffll) {
        set_error(ctx, GS_ERR_INVALID, "frame sizes invalid (tile %d, %dx%d, n %lld, keys %lld)", f->tile, f->width,
                  f->height, (long long)f->n_capacity, (long long)f->key_capacity);
        return false;
    }
    const bool render_bufs = need == kNeedAll;
    if (!f->proj || !f->counts || !f->keys || !f->vals || !f->scratch ||
        (render_bufs && (!f->ranges || !f->image || !f->final_T || !f->last))) {
        set_error(ctx, GS_ERR_INVALID, "frame has a NULL buffer");
        return false;
    }
    v->ncap = f->n_capacity;
    v->kcap = f->key_capacity;
    v->width = f->width;
    v->height = f->height;
    v->tile = f->tile;
    v->gx = (f->width + f->tile - 1) / f->tile;
    v->gy = (f->height + f->tile - 1) / f->tile;
    float4* proj = reinterpret_cast<float4*>(f->proj);
    v->p0 = proj;
    v->p1 = proj + f->n_capacity;
    v->p2 = proj + 2 * f->n_capacity;
    v->counts = f->counts;
    v->keys0 = f->keys;
    v->vals0 = f->vals;
    v->ranges = reinterpret_cast<uint2*>(f->ranges);
    v->image = f->image;
    v->final_T = f->final_T;
    v->last = f->last;
    const ScratchLayout L = scratch_layout(f->n_capacity, f->key_capacity);
    unsigned char* s = static_cast<unsigned char*>(f->scratch);
    v->status = reinterpret_cast<uint32_t*>(s + L.status);
    v->scan_partials = reinterpret_cast<long long*>(s + L.partials);
    v->sort_hist = reinterpret_cast<uint32_t*>(s + L.hist);
    v->sort_ticket = v->sort_hist + kMaxPasses * 256;
    v->sort_lookback = reinterpret_cast<uint32_t*>(s + L.lookback);
    v->sort_partitions = std::max<int64_t>(sort_partitions_for(f->key_capacity), 1);
    v->tile_order = reinterpret_cast<uint32_t*>(s + L.order);
    v->tile_order_cap = kMaxOrderedTiles;
    v->warp_range = reinterpret_cast<uint2*>(s + L.warp_range);
    v->block_range = reinterpret_cast<uint2*>(s + L.block_range);
    if ((reinterpret_cast<uintptr_t>(f->proj) & 15) || (reinterpret_cast<uintptr_t>(f->keys) & 7) ||
        (reinterpret_cast<uintptr_t>(f->ranges) & 7) || (reinterpret_cast<uintptr_t>(f->scratch) & 15)) {
        set_error(ctx, GS_ERR_INVALID, "frame buffer misaligned (proj/scratch need 16 B, keys/ranges 8 B)");
        return false;
    }
    return true;
}

}  // namespace gs

using namespace gs;

extern "C" {

gs_status gs_create(int device, void* cuda_stream, gs_context** out) {
    if (!out) return GS_ERR_INVALID;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return GS_ERR_CUDA;
    gs_context* ctx = new (std::nothrow) gs_context();
    if (!ctx) return GS_ERR_OOM;
    ctx->device = device;
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    if (cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        delete ctx;
        return GS_ERR_CUDA;
    }
    *out = ctx;
    return GS_OK;
}

void gs_destroy(gs_context* ctx) { delete ctx; }

gs_status gs_set_stream(gs_context* ctx, void* cuda_stream) {
    if (!ctx) return GS_ERR_INVALID;
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    return GS_OK;
}

const char* gs_last_error(const gs_context* ctx) { return ctx ? ctx->err : "context is NULL"; }

int64_t gs_launch_count(const gs_context* ctx) { return ctx ? ctx->launches : 0; }

gs_status gs_frame_sizes(int64_t n_capacity, int32_t width, int32_t height, int32_t tile, int64_t key_capacity,
                         gs_frame_bytes* out) {
    if (!out || !valid_tile(tile) || width <= 0 || height <= 0 || n_capacity < 0 || key_capacity < 0 ||
        key_capacity > GS_MAX_KEYS || n_capacity > (int64_t)0xffffffffll)
        return GS_ERR_INVALID;
    const int64_t gx = (width + tile - 1) / tile, gy = (height + tile - 1) / tile;
    const int64_t hw = (int64_t)width * height;
    out->proj = std::max<int64_t>(3 * n_capacity * 16, 16);
    out->counts = std::max<int64_t>(n_capacity * 4, 4);
    out->keys = std::max<int64_t>(2 * key_capacity * 8, 8);
    out->vals = std::max<int64_t>(2 * key_capacity * 4, 4);
    out->ranges = gx * gy * 8;
    out->image = 3 * hw * 4;
    out->final_T = hw * 4;
    out->last = hw * 4;
    out->scratch = scratch_layout(n_capacity, key_capacity).total;
    return GS_OK;
}

static gs_status enter(gs_context* ctx) {
    if (!ctx) return GS_ERR_INVALID;
    ctx->err[0] = 0;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return set_error(ctx, GS_ERR_CUDA, "cudaSetDevice failed");
    return GS_OK;
}

gs_status gs_preprocess(gs_context* ctx, const gs_scene* scene, const gs_camera* cam, const gs_raster_cfg* cfg,
                        const gs_frame* frame) {
    gs_status st = enter(ctx);
    if (st) return st;
    FrameView v;
    if (!make_view(ctx, frame, &v)) return GS_ERR_INVALID;
    if ((st = check_cam(ctx, cam, frame)) || (st = check_cfg(ctx, cfg, frame))) return st;
    if ((st = check_scene(ctx, scene, frame))) return st;
    return launch_preprocess(ctx, scene, cam, cfg, v);
}

gs_status gs_intersect(gs_context* ctx, const gs_camera* cam, const gs_raster_cfg* cfg, const gs_frame* frame,
                       int64_t* num_keys) {
    gs_status st = enter(ctx);
    if (st) return st;
    FrameView v;
    if (!make_view(ctx, frame, &v)) return GS_ERR_INVALID;
    if ((st = check_cam(ctx, cam, frame)) || (st = check_cfg(ctx, cfg, frame))) return st;
    if ((st = launch_intersect(ctx, cfg, v))) return st;
    if (num_keys) {
        uint32_t flags = 0;
        return gs_read_status(ctx, frame, num_keys, &flags);
    }
    return GS_OK;
}

gs_status gs_sort(gs_context* ctx, const gs_camera* cam, const gs_raster_cfg* cfg, const gs_frame* frame) {
    gs_status st = enter(ctx);
    if (st) return st;
    FrameView v;
    if (!make_view(ctx, frame, &v)) return GS_ERR_INVALID;
    if ((st = check_cam(ctx, cam, frame)) || (st = check_cfg(ctx, cfg, frame))) return st;
    return launch_sort(ctx, v, cfg->sort_digit_bits);
}

gs_status gs_tile_ranges(gs_context* ctx, const gs_camera* cam, const gs_raster_cfg* cfg, const gs_frame* frame) {
    gs_status st = enter(ctx);
    if (st) return st;
    FrameView v;
    if (!make_view(ctx, frame, &v)) return GS_ERR_INVALID;
    if ((st = check_cam(ctx, cam, frame)) || (st = check_cfg(ctx, cfg, frame))) return st;
    return launch_ranges(ctx, v);
}

gs_status gs_render(gs_context* ctx, const gs_camera* cam, const gs_raster_cfg* cfg, const gs_frame* frame) {
    gs_status st = enter(ctx);
    if (st) return st;
    FrameView v;
    if (!make_view(ctx, frame, &v)) return GS_ERR_INVALID;
    if ((st = check_cam(ctx, cam, frame)) || (st = check_cfg(ctx, cfg, frame))) return st;
    return launch_render(ctx, cfg, v);
}

gs_status gs_render_stats(gs_context* ctx, const gs_camera* cam, const gs_raster_cfg* cfg, const gs_frame* frame,
                          uint64_t* evaluated, uint64_t* contributed, uint64_t* executed) {
    gs_status st = enter(ctx);
    if (st) return st;
    FrameView v;
    if (!make_view(ctx, frame, &v)) return GS_ERR_INVALID;
    if ((st = check_cam(ctx, cam, frame)) || (st = check_cfg(ctx, cfg, frame))) return st;
    unsigned long long* counters = reinterpret_cast<unsigned long long*>(v.status + 4);
    if (cudaMemsetAsync(counters, 0, 3 * sizeof(unsigned long long), ctx->stream) != cudaSuccess)
        return set_error(ctx, GS_ERR_CUDA, "render_stats: cudaMemsetAsync failed");
    if ((st = launch_render(ctx, cfg, v, counters))) return st;
    unsigned long long h[3] = {0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(h, counters, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return set_error(ctx, GS_ERR_CUDA, "render_stats: %s", cudaGetErrorString(e));
    if (evaluated) *evaluated = h[0];
    if (contributed) *contributed = h[1];
    if (executed) *executed = h[2];
    return GS_OK;
}

gs_status gs_forward(gs_context* ctx, const gs_scene* scene, const gs_camera* cam, const gs_raster_cfg* cfg,
                     const gs_frame* frame) {
    gs_status st = enter(ctx);
    if (st) return st;
    FrameView v;
    if (!make_view(ctx, frame, &v)) return GS_ERR_INVALID;
    if ((st = check_cam(ctx, cam, frame)) || (st = check_cfg(ctx, cfg, frame))) return st;
    if ((st = check_scene(ctx, scene, frame))) return st;
    if ((st = launch_preprocess(ctx, scene, cam, cfg, v))) return st;
    if ((st = launch_intersect(ctx, cfg, v, true))) return st;
    if ((st = launch_sort(ctx, v, cfg->sort_digit_bits, true))) return st;
    if ((st = launch_ranges(ctx, v))) return st;
    return launch_render(ctx, cfg, v);
}

int64_t gs_backward_work_bytes(int64_t n_capacity) {
    return n_capacity < 0 ? 0 : std::max<int64_t>(backward_work_floats(n_capacity) * 4, 4);
}

gs_status gs_render_backward(gs_context* ctx, const gs_scene* scene, const gs_camera* cam, const gs_raster_cfg* cfg,
                             const gs_frame* frame, const float* dL_dimage, const gs_grads* grads) {
    gs_status st = enter(ctx);
    if (st) return st;
    FrameView v;
    if (!make_view(ctx, frame, &v)) return GS_ERR_INVALID;
    if ((st = check_cam(ctx, cam, frame)) || (st = check_cfg(ctx, cfg, frame))) return st;
    if (!scene || scene->n < 0 || scene->n > frame->n_capacity)
        return set_error(ctx, GS_ERR_INVALID, "scene is NULL or larger than the frame");
    if (!dL_dimage || !grads || !grads->work)
        return set_error(ctx, GS_ERR_INVALID, "dL_dimage, grads or grads->work is NULL");
    if (reinterpret_cast<uintptr_t>(grads->work) & 15)
        return set_error(ctx, GS_ERR_INVALID, "grads->work must be 16-byte aligned");
    if (scene->n > 0 && (!scene->means || !scene->scales || !scene->rotations || !scene->sh || !grads->means ||
                         !grads->scales || !grads->rotations || !grads->opacities || !grads->sh))
        return set_error(ctx, GS_ERR_INVALID, "scene or grads has a NULL array");
    return launch_backward(ctx, scene, cam, cfg, v, dL_dimage, grads);
}

int64_t gs_pup_work_bytes(int64_t n_capacity) { return n_capacity < 0 ? 0 : std::max<int64_t>(n_capacity * 64, 16); }

gs_status gs_pup_accumulate(gs_context* ctx, const gs_scene* scene, const gs_camera* cam, const gs_raster_cfg* cfg,
                            const gs_frame* frame, float* hessian, float* work) {
    gs_status st = enter(ctx);
    if (st) return st;
    FrameView v;
    if (!make_view(ctx, frame, &v)) return GS_ERR_INVALID;
    if ((st = check_cam(ctx, cam, frame)) || (st = check_cfg(ctx, cfg, frame))) return st;
    if ((st = check_scene(ctx, scene, frame))) return st;
    if (!hessian || !work) return set_error(ctx, GS_ERR_INVALID, "pup: hessian and work are required");
    if (reinterpret_cast<uintptr_t>(work) & 15) return set_error(ctx, GS_ERR_INVALID, "pup: work must be 16-byte aligned");
    return launch_pup(ctx, scene, cam, cfg, v, hessian, work);
}

gs_status gs_pup_score(gs_context* ctx, const float* hessian, int64_t n, float* score) {
    gs_status st = enter(ctx);
    if (st) return st;
    if (n < 0 || (n > 0 && (!hessian || !score))) return set_error(ctx, GS_ERR_INVALID, "pup_score: bad arguments");
    return launch_pup_score(ctx, hessian, n, score);
}

gs_status gs_set_sort_wait(gs_context* ctx, uint32_t max_polls, int64_t withhold_partition) {
    if (!ctx) return GS_ERR_INVALID;
    ctx->sort_spin_limit = max_polls ? max_polls : kDefaultSpinLimit;
    ctx->sort_withhold = withhold_partition < 0 ? -1 : withhold_partition;
    return GS_OK;
}

gs_status gs_read_culled(gs_context* ctx, const gs_frame* frame, int64_t* culled) {
    gs_status st = enter(ctx);
    if (st) return st;
    if (!culled) return set_error(ctx, GS_ERR_INVALID, "culled is NULL");
    FrameView v;
    if (!make_view(ctx, frame, &v)) return GS_ERR_INVALID;
    uint32_t w = 0;
    cudaError_t e = cudaMemcpyAsync(&w, v.status + kStatusCulled, sizeof(w), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return set_error(ctx, GS_ERR_CUDA, "read_culled: %s", cudaGetErrorString(e));
    *culled = (int64_t)w;
    return GS_OK;
}

gs_status gs_read_sort_plan(gs_context* ctx, const gs_raster_cfg* cfg, const gs_frame* frame, int32_t* passes,
                            int32_t* digit_bits, int32_t* depth_bits) {
    gs_status st = enter(ctx);
    if (st) return st;
    FrameView v;
    if (!make_view(ctx, frame, &v, kNeedEmit)) return GS_ERR_INVALID;
    if ((st = check_cfg(ctx, cfg, frame))) return st;
    uint32_t w[kStatusWords] = {0};
    cudaError_t e = cudaMemcpyAsync(w, v.status, sizeof(w), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return set_error(ctx, GS_ERR_CUDA, "read_sort_plan: %s", cudaGetErrorString(e));
    const SortPlan P = sort_plan_of(w[kStatusDepthLoN], w[kStatusDepthHi], sort_tile_bits((int64_t)v.gx * v.gy),
                                    sort_digit_max(cfg->sort_digit_bits), true);
    if (passes) *passes = P.passes;
    if (digit_bits) *digit_bits = P.dbits;
    if (depth_bits) *depth_bits = P.w;
    return GS_OK;
}

gs_status gs_sort_plan_for(int64_t tiles, uint32_t least, uint32_t greatest, int32_t sort_digit_bits, int32_t fused,
                           int32_t* passes, int32_t* digit_bits, int32_t* depth_bits, int32_t* start_buffer) {
    if (tiles < 1 || (sort_digit_bits != 0 && (sort_digit_bits < 4 || sort_digit_bits > 8))) return GS_ERR_INVALID;
    // the status-word form: complement of the least bits, greatest bits; both 0 = none recorded
    const uint32_t lo_n = least > greatest ? 0u : ~least;
    const uint32_t hi = least > greatest ? 0u : greatest;
    const SortPlan P = sort_plan_of(lo_n, hi, sort_tile_bits(tiles), sort_digit_max(sort_digit_bits), fused != 0);
    if (passes) *passes = P.passes;
    if (digit_bits) *digit_bits = P.dbits;
    if (depth_bits) *depth_bits = P.w;
    if (start_buffer) *start_buffer = P.start;
    return GS_OK;
}

gs_status gs_read_status(gs_context* ctx, const gs_frame* frame, int64_t* num_keys, uint32_t* flags) {
    gs_status st = enter(ctx);
    if (st) return st;
    FrameView v;
    if (!make_view(ctx, frame, &v)) return GS_ERR_INVALID;
    uint32_t w[3] = {0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(w, v.status, sizeof(w), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return set_error(ctx, GS_ERR_CUDA, "read_status: %s", cudaGetErrorString(e));
    const int64_t K = (int64_t)w[0] | ((int64_t)w[1] << 32);
    if (num_keys) *num_keys = K;
    if (flags) *flags = w[2];
    if (w[2] & GS_FLAG_CAPACITY)
        return set_error(ctx, GS_ERR_CAPACITY, "%lld keys exceed key_capacity %lld", (long long)K,
                         (long long)frame->key_capacity);
    if (w[2] & GS_FLAG_TIMEOUT) return set_error(ctx, GS_ERR_TIMEOUT, "sort look-back wait exceeded its bound");
    if (w[2] & GS_FLAG_KEYRANGE)
        return set_error(ctx, GS_ERR_INVALID, "gs_sort met a key outside the range gs_intersect recorded");
    return GS_OK;
}

}  // extern "C"
