// Internal definitions shared by the library's translation units.
//
// Floating-point contract: the library is compiled with -fmad=false, IEEE
// division and square root, and without flush-to-zero, so every float
// operation rounds once unless written as fmaf().  The per-Gaussian values
// that decide tile membership (projected mean, conic, t, depth) and the
// per-pixel blend are evaluated in a fixed operation order, so results are
// reproducible bit for bit by any implementation that follows the same order.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <utility>

#include "gs.h"  // include/ is on the compiler include path

namespace gs {

constexpr int kMaxTile = 32;

// ---------------------------------------------------------------- status words
// scratch layout starts with these words (device):
//   [0] key total K, low 32 bits   [1] K high bits   [2] GS_FLAG_* bits
//   [3] multi-view set-up flags (GS_FLAG_BATCH), written by every batch set-up
//   [4..9] three 64-bit counters of the instrumented blend (gs_render_stats)
//   [10] Gaussians culled by the running preprocess for non-finite
//        parameters or a zero quaternion (accumulated, then moved to [11] and
//        cleared by the scan that follows it)
//   [11] that count for the last preprocessed frame
//   [12] complement of the least and [13] greatest depth bits of the
//        Gaussians the last preprocess gave tiles (written by the scan from
//        the preprocess's per-warp ranges; both 0 when none was recorded);
//        the sort plan follows from them (sort_plan_of)
constexpr int kStatusWords = 16;
constexpr int kStatusCulledAcc = 10;
constexpr int kStatusCulled = 11;
constexpr int kStatusDepthLoN = 12;
constexpr int kStatusDepthHi = 13;
// Bound of one sort look-back wait, in polls (about 32 ns apart).
constexpr uint32_t kDefaultSpinLimit = 1u << 22;

// Camera constants as the kernels use them.
struct CamK {
    float fx, fy, cx, cy, limx, limy, near_z;
    float V[12];
    float campos[3];
};

// One camera of a multi-view batch (device table built by the batch set-up
// kernel): constants, raster size, and where its tiles and pixels start in
// the batch's global tile index space and packed image buffers.
struct CamRec {
    CamK k;
    int width, height, gx, gy;
    long long tile_offset;
    long long pix_offset;
};

struct FrameView {
    int64_t ncap, kcap;
    int width, height, tile, gx, gy;
    float4* p0;  // u, v, opacity, depth
    float4* p1;  // a, b, c, t
    float4* p2;  // r, g, b, radius bits
    int32_t* counts;
    uint64_t* keys0;  // buffer 0; the sort's buffer 1 follows at keys0 + kcap
    uint32_t* vals0;  // alike
    uint2* ranges;
    float* image;
    float* final_T;
    uint32_t* last;
    uint32_t* status;
    long long* scan_partials;  // one per scan block + 1
    // depth-bit ranges (complement of the least, greatest) of the Gaussians
    // given tiles: one per preprocess warp, then one per scan block; both
    // nullptr where the frame has no scratch (the range is then not recorded)
    uint2* warp_range = nullptr;
    uint2* block_range = nullptr;
    uint32_t* sort_hist;       // [kMaxPasses][256]
    uint32_t* sort_ticket;     // [kMaxPasses]
    uint32_t* sort_lookback;   // [2][sort_partitions][256] look-back words, see sort.cu
    int64_t sort_partitions;   // partitions the look-back table holds
    uint32_t* tile_order;      // [tile_order_cap] the blend's tile launch order
    int64_t tile_order_cap = 0;
    uint32_t* order_ctl = nullptr;  // [67] class counts, class bases, done counter (multi-block ordering)
    // multi-view batches only (table == nullptr for a single camera)
    const CamRec* table = nullptr;
    int num_cams = 1;
    int64_t cam_stride = 0;    // Gaussian slots per camera in proj/counts
    int64_t pixel_capacity = 0;
};

// ---------------------------------------------------------------- scan / sort geometry
constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;  // counts per thread (rounds per emit block)
constexpr int kScanBlock = kScanThreads * kScanItems;

constexpr int kSortThreads = 512;
constexpr int kSortItems = 8;
constexpr int kSortPartition = kSortThreads * kSortItems;  // keys per onesweep partition
constexpr int kMaxPasses = 12;
// Sort control words at the start of the sort's scratch: [kMaxPasses][256]
// digit totals, a partition ticket per pass, a ranking-method word per pass,
// and the histogram kernel's block-completion counter.
constexpr int kSortCtlWords = kMaxPasses * 256 + 2 * kMaxPasses + 1;

// ---------------------------------------------------------------- elementary functions
// Natural logarithm: frexp range reduction to m in [sqrt(1/2), sqrt(2)),
// log x = e ln2 + 2 atanh(s), s = (m-1)/(m+1), atanh series through s^11/11;
// ln2 split into a 15-bit head (exact products with the exponent) and a tail.
__device__ __forceinline__ float gs_logf(float x) {
    if (isnan(x)) return x;
    if (!(x > 0.0f)) return -INFINITY;
    if (isinf(x)) return x;
    int e;
    float m = frexpf(x, &e);
    if (m < 0.70710677f) {
        m = m * 2.0f;
        e = e - 1;
    }
    const float s = (m - 1.0f) / (m + 1.0f);
    const float s2 = s * s;
    float p = 1.0f / 11.0f;
    p = fmaf(p, s2, 1.0f / 9.0f);
    p = fmaf(p, s2, 1.0f / 7.0f);
    p = fmaf(p, s2, 1.0f / 5.0f);
    p = fmaf(p, s2, 1.0f / 3.0f);
    p = fmaf(p, s2, 1.0f);
    const float lm = (2.0f * s) * p;
    const float fe = (float)e;
    return fmaf(fe, 0.693145751953125f, fmaf(fe, 1.42860682030941723e-06f, lm));
}

// Exponential: x = k ln2 + r (Cody-Waite, same ln2 split), e^r by its Taylor
// polynomial to degree 7 (Horner), scaled by 2^k.
__device__ __forceinline__ float gs_expf(float x) {
    if (isnan(x)) return x;
    if (x < -104.0f) return 0.0f;
    if (x > 89.0f) return INFINITY;
    const float k = rintf(x * 1.44269502f);
    float r = fmaf(-k, 0.693145751953125f, x);
    r = fmaf(-k, 1.42860682030941723e-06f, r);
    float p = 1.0f / 5040.0f;
    p = fmaf(p, r, 1.0f / 720.0f);
    p = fmaf(p, r, 1.0f / 120.0f);
    p = fmaf(p, r, 1.0f / 24.0f);
    p = fmaf(p, r, 1.0f / 6.0f);
    p = fmaf(p, r, 0.5f);
    p = fmaf(p, r, 1.0f);
    p = fmaf(p, r, 1.0f);
    return ldexpf(p, (int)k);
}

// gs_expf for the blend, where x = -q/2 with 0 <= q <= t <= 2 ln 255: the same
// reduction and polynomial, with the final scaling by 2^k done as an add to
// the exponent field, which is exactly ldexpf whenever the result is a normal
// number (x >= -80 here).  Any other x takes gs_expf itself, so the value is
// gs_expf(x) bit for bit for every input.
__device__ __forceinline__ float gs_expf_blend(float x) {
    if (!(x >= -80.0f && x <= 88.0f)) return gs_expf(x);
    const float k = rintf(x * 1.44269502f);
    float r = fmaf(-k, 0.693145751953125f, x);
    r = fmaf(-k, 1.42860682030941723e-06f, r);
    float p = 1.0f / 5040.0f;
    p = fmaf(p, r, 1.0f / 720.0f);
    p = fmaf(p, r, 1.0f / 120.0f);
    p = fmaf(p, r, 1.0f / 24.0f);
    p = fmaf(p, r, 1.0f / 6.0f);
    p = fmaf(p, r, 0.5f);
    p = fmaf(p, r, 1.0f);
    p = fmaf(p, r, 1.0f);
    return __int_as_float(__float_as_int(p) + ((int)k << 23));
}

// floor(x) as an int clamped to [lo, hi], safe for any finite or infinite x.
__device__ __forceinline__ int floor_clamp(float x, int lo, int hi) {
    const float f = floorf(x);
    if (!(f >= (float)lo)) return lo;
    if (f > (float)hi) return hi;
    return (int)f;
}

// ---------------------------------------------------------------- ptx helpers
__device__ __forceinline__ uint32_t ld_relaxed_gpu(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_gpu(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}


// ---------------------------------------------------------------- warp scan
__device__ __forceinline__ long long warp_incl_scan(long long v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// ---------------------------------------------------------------- programmatic dependent launch
// A frame's kernels are launched so that each can be scheduled while its
// predecessor in the stream finishes (launch_pdl).  Every such kernel first
// lets its own successor be scheduled, then waits until its predecessor has
// completed and that grid's writes are visible, before it touches memory.
// The successor is scheduled only once every block of this grid has started,
// so waiting blocks never hold back blocks of the grid they wait for.  For a
// kernel launched without the attribute both instructions do nothing.
__device__ __forceinline__ void pdl_begin() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(cudaStream_t stream, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

namespace {
// n zero words (a kernel rather than a memset, so the launch chain stays
// programmatic).
__global__ void __launch_bounds__(256) zero_words_kernel(uint32_t* __restrict__ p, int64_t n) {
    pdl_begin();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = 0u;
}
}  // namespace

inline unsigned zero_blocks(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 1024)); }

}  // namespace gs

// ---------------------------------------------------------------- context
struct gs_context {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    int64_t launches = 0;
    uint32_t sort_spin_limit = gs::kDefaultSpinLimit;  // gs_set_sort_wait
    int64_t sort_withhold = -1;                        // gs_set_sort_wait: partition that does not publish
    char err[512] = {0};
};

namespace gs {
// host helpers (api.cu)
gs_status set_error(gs_context* ctx, gs_status st, const char* fmt, ...);
gs_status check_launch(gs_context* ctx, const char* what);
// Buffers a stage needs (make_view rejects a NULL one among them).
constexpr unsigned kNeedAll = 0xffu;
constexpr unsigned kNeedEmit = 1u;  // proj, counts, keys, vals only
bool make_view(gs_context* ctx, const gs_frame* f, FrameView* v, unsigned need = kNeedAll);
int sort_tile_bits(int64_t tiles);

// A frame's sort plan (see sort.cu): pass count, bits per digit, depth bits
// kept and the least depth bits, from status words [14] and [15].  At most
// dmax bits per digit, at least two passes and at most kMaxPasses, an even
// count unless `fused` (a chain that also runs the emit may start the passes
// from either buffer); without a recorded range (both words zero) the whole
// depth word is kept.
struct SortPlan {
    int passes, dbits, w;
    uint32_t dmin;
    int start;  // buffer the emit writes and the first pass reads
};
__host__ __device__ inline SortPlan sort_plan_of(uint32_t lo_n, uint32_t hi, int tile_bits, int dmax, bool fused) {
    SortPlan P;
    if ((lo_n | hi) == 0u) {
        P.dmin = 0u;
        P.w = 32;
    } else {
        P.dmin = ~lo_n;
        uint32_t span = hi - P.dmin;
        P.w = 0;
        while (span) {
            ++P.w;
            span >>= 1;
        }
    }
    const int total = tile_bits + P.w;
    int p = (total + dmax - 1) / dmax;
    p = p < 2 ? 2 : (p > kMaxPasses ? kMaxPasses : p);
    if (!fused) p += p & 1;
    P.passes = p;
    P.dbits = (total + P.passes - 1) / P.passes;
    P.start = P.passes & 1;  // so that the last pass writes buffer 0
    return P;
}
// The most passes any plan of a frame with these tiles can need.
inline int sort_max_passes(int tile_bits, int dmax, bool fused) {
    int p = (32 + tile_bits + dmax - 1) / dmax;
    p = p < 2 ? 2 : (p > kMaxPasses ? kMaxPasses : p);
    if (!fused) p += p & 1;
    return p;
}
// Bits per digit at most: the override when it is 4..8, else 8.
inline int sort_digit_max(int digit_override) {
    return (digit_override >= 4 && digit_override <= 8) ? digit_override : 8;
}

struct ScratchLayout {
    int64_t status, partials, hist, lookback, order, warp_range, block_range, total;
};
// Frames with more tiles than this blend them in index order.
constexpr unsigned kMaxOrderedTiles = 1u << 15;
// range_warps: preprocess warps of the largest launch (0: one per 32 slots)
ScratchLayout scratch_layout(int64_t ncap, int64_t kcap, int64_t range_warps = 0);
constexpr int kPreThreads = 256;  // preprocess block size
int64_t sort_partitions_for(int64_t kcap);
int64_t scan_blocks_for(int64_t n);

// launchers (one per translation unit); all enqueue on ctx->stream
gs_status launch_preprocess(gs_context* ctx, const gs_scene* s, const gs_camera* cam, const gs_raster_cfg* cfg,
                            const FrameView& v);
// fused: the call runs intersect and sort back to back (gs_forward,
// gs_forward_batch), so the emit may write the buffer the sort plan starts
// from; otherwise the emitted pairs are in buffer 0 and the plan is even.
gs_status launch_intersect(gs_context* ctx, const gs_raster_cfg* cfg, const FrameView& v, bool fused = false);
gs_status launch_sort(gs_context* ctx, const FrameView& v, int digit_override = 0, bool fused = false);
// identifyTileRanges, then the blend's heaviest-first tile launch order
// (for frames of at most kMaxOrderedTiles tiles).
gs_status launch_ranges(gs_context* ctx, const FrameView& v);
gs_status launch_render(gs_context* ctx, const gs_raster_cfg* cfg, const FrameView& v,
                        unsigned long long* stats = nullptr);
gs_status launch_backward(gs_context* ctx, const gs_scene* s, const gs_camera* cam, const gs_raster_cfg* cfg,
                          const FrameView& v, const float* dL_dimg, const gs_grads* g);
int64_t backward_work_floats(int64_t ncap);
gs_status launch_pup(gs_context* ctx, const gs_scene* s, const gs_camera* cam, const gs_raster_cfg* cfg,
                     const FrameView& v, float* hessian, float* work);
gs_status launch_pup_score(gs_context* ctx, const float* hessian, int64_t n, float* score);
}  // namespace gs
