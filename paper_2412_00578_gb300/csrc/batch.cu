// Multi-view batches: entry points gs_batch_sizes, gs_forward_batch,
// gs_batch_status, and the set-up kernel that turns the caller's device array
// of cameras into the per-camera table the stage kernels read.
#include <algorithm>

#include "gs_common.cuh"

namespace gs {
namespace {

constexpr int64_t kAlign = 256;
int64_t align_up(int64_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct BatchLayout {
    ScratchLayout base;
    int64_t table, order, ctl, total;
};

// The batch scratch adds the camera table, a launch order for all of the
// batch's tiles and the counters of the multi-block ordering.
BatchLayout batch_layout(int64_t n_capacity, int64_t max_cams, int64_t kcap, int64_t tile_capacity) {
    BatchLayout L;
    // the multi-view preprocess runs ceil(n / 256) blocks per camera
    L.base = scratch_layout(n_capacity * max_cams, kcap,
                            (n_capacity + kPreThreads - 1) / kPreThreads * (kPreThreads / 32) * max_cams);
    L.table = L.base.total;
    L.order = L.table + align_up(max_cams * (int64_t)sizeof(CamRec));
    L.ctl = L.order + align_up(tile_capacity * 4);
    L.total = L.ctl + align_up(67 * 4);
    return L;
}

// One block.  Thread c < V derives camera c's constants and raster size;
// thread 0 then assigns the tile and pixel offsets in camera order and
// flags a batch that does not fit the frame's capacities.
__global__ void __launch_bounds__(1024) batch_setup_kernel(const gs_camera* __restrict__ cams, int V, int tile,
                                                           long long tile_cap, long long pix_cap,
                                                           CamRec* __restrict__ table, uint32_t* status) {
    __shared__ long long s_tiles[GS_MAX_BATCH_CAMS];
    __shared__ long long s_pix[GS_MAX_BATCH_CAMS];
    const int c = threadIdx.x;
    CamRec R;
    if (c < V) {
        const gs_camera g = cams[c];
        R.k.fx = g.fx;
        R.k.fy = g.fy;
        R.k.cx = g.cx;
        R.k.cy = g.cy;
        R.k.limx = 1.3f * g.tan_fovx;
        R.k.limy = 1.3f * g.tan_fovy;
        R.k.near_z = g.near_z;
        for (int k = 0; k < 12; ++k) R.k.V[k] = g.viewmat[k];
        for (int k = 0; k < 3; ++k) R.k.campos[k] = g.campos[k];
        const bool ok = g.width > 0 && g.height > 0;
        R.width = ok ? g.width : 0;
        R.height = ok ? g.height : 0;
        R.gx = ok ? (g.width + tile - 1) / tile : 0;
        R.gy = ok ? (g.height + tile - 1) / tile : 0;
        s_tiles[c] = (long long)R.gx * R.gy;
        s_pix[c] = (long long)R.width * R.height;
    }
    __syncthreads();
    if (c == 0) {
        long long t = 0, p = 0;
        for (int k = 0; k < V; ++k) {
            const long long a = s_tiles[k], b = s_pix[k];
            s_tiles[k] = t;
            s_pix[k] = p;
            t += a;
            p += b;
        }
        status[3] = (t > tile_cap || p > pix_cap) ? GS_FLAG_BATCH : 0u;
    }
    __syncthreads();
    if (c < V) {
        R.tile_offset = s_tiles[c];
        R.pix_offset = s_pix[c];
        table[c] = R;
    }
}

bool valid_batch(const gs_batch_frame* f) {
    return f && (f->tile == 8 || f->tile == 16 || f->tile == 32) && f->n_capacity >= 0 && f->key_capacity >= 0 &&
           f->key_capacity <= GS_MAX_KEYS && f->max_cams >= 1 && f->max_cams <= GS_MAX_BATCH_CAMS &&
           f->tile_capacity >= 1 && f->tile_capacity <= (int64_t)0x7fffffff && f->pixel_capacity >= 1 &&
           f->n_capacity * f->max_cams <= (int64_t)0xffffffffll;
}

bool make_batch_view(gs_context* ctx, const gs_batch_frame* f, int num_cams, FrameView* v) {
    if (!valid_batch(f)) {
        set_error(ctx, GS_ERR_INVALID, "batch frame sizes invalid");
        return false;
    }
    if (!f->proj || !f->counts || !f->keys || !f->vals || !f->ranges || !f->image || !f->final_T || !f->last ||
        !f->scratch) {
        set_error(ctx, GS_ERR_INVALID, "batch frame has a NULL buffer");
        return false;
    }
    if ((reinterpret_cast<uintptr_t>(f->proj) & 15) || (reinterpret_cast<uintptr_t>(f->keys) & 7) ||
        (reinterpret_cast<uintptr_t>(f->ranges) & 7) || (reinterpret_cast<uintptr_t>(f->scratch) & 15)) {
        set_error(ctx, GS_ERR_INVALID, "batch frame buffer misaligned");
        return false;
    }
    const int64_t stride = f->n_capacity * f->max_cams;  // slots per proj plane
    v->ncap = f->n_capacity * num_cams;                   // slots scanned by this call
    v->kcap = f->key_capacity;
    v->width = 1;
    v->height = 1;
    v->tile = f->tile;
    v->gx = (int)f->tile_capacity;  // global tile index space, one row
    v->gy = 1;
    float4* proj = reinterpret_cast<float4*>(f->proj);
    v->p0 = proj;
    v->p1 = proj + stride;
    v->p2 = proj + 2 * stride;
    v->counts = f->counts;
    v->keys0 = f->keys;
    v->vals0 = f->vals;
    v->ranges = reinterpret_cast<uint2*>(f->ranges);
    v->image = f->image;
    v->final_T = f->final_T;
    v->last = f->last;
    const BatchLayout L = batch_layout(f->n_capacity, f->max_cams, f->key_capacity, f->tile_capacity);
    unsigned char* s = static_cast<unsigned char*>(f->scratch);
    v->status = reinterpret_cast<uint32_t*>(s + L.base.status);
    v->scan_partials = reinterpret_cast<long long*>(s + L.base.partials);
    v->sort_hist = reinterpret_cast<uint32_t*>(s + L.base.hist);
    v->sort_ticket = v->sort_hist + kMaxPasses * 256;
    v->sort_lookback = reinterpret_cast<uint32_t*>(s + L.base.lookback);
    v->sort_partitions = std::max<int64_t>(sort_partitions_for(f->key_capacity), 1);
    v->tile_order = reinterpret_cast<uint32_t*>(s + L.order);
    v->tile_order_cap = f->tile_capacity;
    v->warp_range = reinterpret_cast<uint2*>(s + L.base.warp_range);
    v->block_range = reinterpret_cast<uint2*>(s + L.base.block_range);
    v->order_ctl = reinterpret_cast<uint32_t*>(s + L.ctl);
    v->table = reinterpret_cast<const CamRec*>(s + L.table);
    v->num_cams = num_cams;
    v->cam_stride = f->n_capacity;
    v->pixel_capacity = f->pixel_capacity;
    return true;
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" {

gs_status gs_batch_sizes(int64_t n_capacity, int32_t max_cams, int32_t tile, int64_t tile_capacity,
                         int64_t pixel_capacity, int64_t key_capacity, gs_frame_bytes* out) {
    gs_batch_frame f{};
    f.n_capacity = n_capacity;
    f.key_capacity = key_capacity;
    f.tile_capacity = tile_capacity;
    f.pixel_capacity = pixel_capacity;
    f.max_cams = max_cams;
    f.tile = tile;
    if (!out || !valid_batch(&f)) return GS_ERR_INVALID;
    const int64_t slots = n_capacity * max_cams;
    out->proj = std::max<int64_t>(3 * slots * 16, 16);
    out->counts = std::max<int64_t>(slots * 4, 4);
    out->keys = std::max<int64_t>(2 * key_capacity * 8, 8);
    out->vals = std::max<int64_t>(2 * key_capacity * 4, 4);
    out->ranges = tile_capacity * 8;
    out->image = 3 * pixel_capacity * 4;
    out->final_T = pixel_capacity * 4;
    out->last = pixel_capacity * 4;
    out->scratch = batch_layout(n_capacity, max_cams, key_capacity, tile_capacity).total;
    return GS_OK;
}

gs_status gs_forward_batch(gs_context* ctx, const gs_scene* scene, const gs_camera* cams, int32_t num_cams,
                           const gs_raster_cfg* cfg, const gs_batch_frame* frame) {
    if (!ctx) return GS_ERR_INVALID;
    ctx->err[0] = 0;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return set_error(ctx, GS_ERR_CUDA, "cudaSetDevice failed");
    if (!frame || !cfg || !scene || !cams) return set_error(ctx, GS_ERR_INVALID, "NULL argument");
    if (num_cams < 1 || num_cams > frame->max_cams)
        return set_error(ctx, GS_ERR_INVALID, "num_cams %d not in 1..max_cams (%d)", num_cams, frame->max_cams);
    if (cfg->tile != frame->tile || cfg->mode < GS_MODE_3SIGMA || cfg->mode > GS_MODE_PIXEL ||
        (cfg->sort_digit_bits != 0 && (cfg->sort_digit_bits < 4 || cfg->sort_digit_bits > 8)))
        return set_error(ctx, GS_ERR_INVALID, "bad cfg (tile %d, mode %d, digit bits %d)", cfg->tile, cfg->mode,
                         cfg->sort_digit_bits);
    if (scene->n < 0 || scene->n > frame->n_capacity || scene->sh_degree < 0 || scene->sh_degree > 3)
        return set_error(ctx, GS_ERR_INVALID, "scene n %lld / degree %d do not fit the batch frame",
                         (long long)scene->n, scene->sh_degree);
    if (scene->n > 0 && (!scene->means || !scene->scales || !scene->rotations || !scene->opacities || !scene->sh))
        return set_error(ctx, GS_ERR_INVALID, "scene has a NULL array");
    FrameView v;
    if (!make_batch_view(ctx, frame, num_cams, &v)) return GS_ERR_INVALID;
    batch_setup_kernel<<<1, 1024, 0, ctx->stream>>>(cams, num_cams, frame->tile, frame->tile_capacity,
                                                    frame->pixel_capacity, const_cast<CamRec*>(v.table), v.status);
    ctx->launches += 1;
    gs_status st = check_launch(ctx, "batch_setup");
    if (st) return st;
    if ((st = launch_preprocess(ctx, scene, nullptr, cfg, v))) return st;
    if ((st = launch_intersect(ctx, cfg, v, true))) return st;
    if ((st = launch_sort(ctx, v, cfg->sort_digit_bits, true))) return st;
    if ((st = launch_ranges(ctx, v))) return st;
    return launch_render(ctx, cfg, v);
}

gs_status gs_batch_status(gs_context* ctx, const gs_batch_frame* frame, int64_t* num_keys, uint32_t* flags) {
    if (!ctx) return GS_ERR_INVALID;
    ctx->err[0] = 0;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return set_error(ctx, GS_ERR_CUDA, "cudaSetDevice failed");
    FrameView v;
    if (!make_batch_view(ctx, frame, 1, &v)) return GS_ERR_INVALID;
    uint32_t w[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(w, v.status, sizeof(w), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return set_error(ctx, GS_ERR_CUDA, "batch_status: %s", cudaGetErrorString(e));
    const int64_t K = (int64_t)w[0] | ((int64_t)w[1] << 32);
    if (num_keys) *num_keys = K;
    const uint32_t fl = w[2] | w[3];
    if (flags) *flags = fl;
    if (fl & GS_FLAG_BATCH)
        return set_error(ctx, GS_ERR_INVALID, "batch cameras exceed the frame's tile or pixel capacity");
    if (fl & GS_FLAG_CAPACITY)
        return set_error(ctx, GS_ERR_CAPACITY, "%lld keys exceed key_capacity %lld", (long long)K,
                         (long long)frame->key_capacity);
    if (fl & GS_FLAG_TIMEOUT) return set_error(ctx, GS_ERR_TIMEOUT, "sort look-back wait exceeded its bound");
    if (fl & GS_FLAG_KEYRANGE)
        return set_error(ctx, GS_ERR_INVALID, "gs_sort met a key outside the range gs_intersect recorded");
    return GS_OK;
}

}  // extern "C"
