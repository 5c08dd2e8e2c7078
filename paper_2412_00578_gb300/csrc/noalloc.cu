// gs_intersect_noalloc: key emission for callers that cannot allocate device
// memory.
//
// Some callers of this library are not allowed to call cudaMalloc at all: a
// plug-in running inside a host application that owns every device
// allocation through its own pool, a real-time loop where an allocation
// (which can synchronise the device) would stall a frame, or a certified
// program that forbids dynamic allocation after start-up.  gs_intersect needs
// a little working memory (the frame's scratch buffer) for the running sums
// of the tile counts and the status words; this entry point instead keeps
// that working memory in a fixed array compiled into the library, so the
// caller supplies only the inputs (the preprocessed frame) and the outputs
// (the key and value arrays).
//
// The array lives in every GPU's memory from the moment the library's code is
// loaded on that device until the process exits (about 131 KB).  All calls on
// a device share it and it keeps the last call's contents; this code clears
// what must start at zero on every call.  Two calls whose work overlaps on
// the GPU (different streams, or different host threads) would race on it.
#include <mutex>

#include "gs_common.cuh"

namespace gs {
namespace {

constexpr int64_t kNoAllocMaxGaussians = int64_t(1) << 24;  // 16,777,216
// Layout inside the array, as gs_frame scratch lays it out: 256 bytes of
// status words, then one 8-byte running sum per block of kScanBlock counts
// (plus one).
constexpr int64_t kNoAllocStatusBytes = 256;
constexpr int64_t kNoAllocPartialBytes = ((kNoAllocMaxGaussians + kScanBlock - 1) / kScanBlock + 1) * 8;
constexpr int64_t kNoAllocBytes = (kNoAllocStatusBytes + kNoAllocPartialBytes + 255) / 256 * 256;

static __device__ __align__(256) unsigned char g_intersect_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_intersect_scratch on the current device (looked up once
// per device; in host code the symbol itself is only a host-side stand-in).
gs_status scratch_address(gs_context* ctx, void** out) {
    if (ctx->device < 0 || ctx->device >= kMaxDevices)
        return set_error(ctx, GS_ERR_INVALID, "intersect_noalloc: device %d out of range", ctx->device);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[ctx->device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_intersect_scratch);
        if (e != cudaSuccess || p == nullptr)
            return set_error(ctx, GS_ERR_CUDA, "intersect_noalloc: cudaGetSymbolAddress failed: %s",
                             cudaGetErrorString(e));
        g_scratch_addr[ctx->device] = p;
    }
    *out = g_scratch_addr[ctx->device];
    return GS_OK;
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" gs_status gs_intersect_noalloc(gs_context* ctx, const gs_camera* cam, const gs_raster_cfg* cfg,
                                          const gs_frame* frame, int64_t* num_keys) {
    if (!ctx) return GS_ERR_INVALID;
    ctx->err[0] = 0;
    if (!frame || !cam || !cfg || !num_keys)
        return set_error(ctx, GS_ERR_INVALID, "intersect_noalloc: frame, cam, cfg and num_keys are required");
    if (frame->n_capacity > kNoAllocMaxGaussians)
        return set_error(ctx, GS_ERR_INVALID,
                         "intersect_noalloc: n_capacity %lld exceeds the fixed working-memory limit of %lld "
                         "Gaussians; use gs_intersect with a frame scratch buffer",
                         (long long)frame->n_capacity, (long long)kNoAllocMaxGaussians);
    if (cudaSetDevice(ctx->device) != cudaSuccess)
        return set_error(ctx, GS_ERR_CUDA, "intersect_noalloc: cudaSetDevice failed");
    void* scratch = nullptr;
    gs_status st = scratch_address(ctx, &scratch);
    if (st) return st;
    if (cam->width != frame->width || cam->height != frame->height)
        return set_error(ctx, GS_ERR_INVALID, "intersect_noalloc: camera does not match frame");
    if (cfg->tile != frame->tile || cfg->mode < GS_MODE_3SIGMA || cfg->mode > GS_MODE_PIXEL)
        return set_error(ctx, GS_ERR_INVALID, "intersect_noalloc: bad cfg (tile %d, mode %d)", cfg->tile, cfg->mode);
    gs_frame f = *frame;
    f.scratch = scratch;  // the caller's scratch pointer is neither needed nor touched
    FrameView v;
    if (!make_view(ctx, &f, &v, kNeedEmit)) return GS_ERR_INVALID;
    // the intersect stage only touches the status words and the running sums
    const unsigned char* end = reinterpret_cast<const unsigned char*>(v.scan_partials) +
                               (scan_blocks_for(v.ncap) + 1) * (int64_t)sizeof(long long);
    if (reinterpret_cast<const unsigned char*>(v.status) != static_cast<unsigned char*>(scratch) ||
        end > static_cast<unsigned char*>(scratch) + kNoAllocBytes)
        return set_error(ctx, GS_ERR_INVALID, "intersect_noalloc: working-memory layout does not fit");
    v.warp_range = nullptr;  // outside the fixed array: no depth range (this path does not sort)
    v.block_range = nullptr;
    if ((st = launch_intersect(ctx, cfg, v))) return st;  // clears the status words first
    uint32_t w[3] = {0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(w, v.status, sizeof(w), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return set_error(ctx, GS_ERR_CUDA, "intersect_noalloc: %s", cudaGetErrorString(e));
    *num_keys = (int64_t)w[0] | ((int64_t)w[1] << 32);
    if (w[2] & GS_FLAG_CAPACITY)
        return set_error(ctx, GS_ERR_CAPACITY, "%lld keys exceed key_capacity %lld", (long long)*num_keys,
                         (long long)frame->key_capacity);
    return GS_OK;
}
