// identifyTileRanges and render (Sec. 3.2.2, Sec. 3.2.3).
//
// ranges: one thread per sorted key; a thread whose tile differs from its
// predecessor's closes the previous range and opens its own.
//
// blend: one CTA per tile, one thread per pixel.  The tile's Gaussians are
// brought into shared memory in batches of one per thread (a gather of the
// 48-byte 2D state by sorted index), then every pixel walks the batch in
// depth order.  Per pixel (Eqs. render_alpha, 2d_gaussian_scalar,
// contribution): dx = px - u, dy = py - v, e = (2b) dy, f = (c dy) dy,
// q = fma(dx, fma(a, dx, e), f); a Gaussian counts iff q <= t (alpha >= 1/255);
// alpha = min(0.99, sigma exp(-q/2)); T' = T (1 - alpha); if T' < 1e-4 the
// pixel stops before adding it; else C = fma(c, alpha T, C), T = T'.
// The CTA leaves the loop as soon as every pixel has stopped
// (__syncthreads_count vote before each batch).
#include "gs_common.cuh"

namespace gs {
namespace {

__device__ __forceinline__ uint32_t frame_keys_r(const uint32_t* status) {
    return (status[2] & GS_FLAG_CAPACITY) ? 0u : status[0];
}

__global__ void __launch_bounds__(256) ranges_kernel(const uint64_t* __restrict__ keys,
                                                     const uint32_t* __restrict__ status, uint2* __restrict__ ranges) {
    const uint32_t K = frame_keys_r(status);
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= K) return;
    const uint32_t tile = (uint32_t)(keys[i] >> 32);
    if (i == 0) {
        ranges[tile].x = 0;
    } else {
        const uint32_t prev = (uint32_t)(keys[i - 1] >> 32);
        if (prev != tile) {
            ranges[prev].y = i;
            ranges[tile].x = i;
        }
    }
    if (i == K - 1) ranges[tile].y = K;
}

struct BlendArgs {
    const uint2* ranges;
    const uint32_t* vals;
    const float4* p0;
    const float4* p1;
    const float4* p2;
    float* image;
    float* final_T;
    uint32_t* last;
    int width, height, gx;
    float bg0, bg1, bg2;
};

template <int T>
__global__ void __launch_bounds__(T* T) blend_kernel(const BlendArgs A) {
    constexpr int NT = T * T;
    __shared__ float4 s_g0[NT];  // u, v, a, 2b
    __shared__ float4 s_g1[NT];  // c, t, opacity, -
    __shared__ float4 s_g2[NT];  // r, g, b, -
    const int tile = blockIdx.x;
    const int tx = tile % A.gx, ty = tile / A.gx;
    const int px = tx * T + (int)(threadIdx.x % T);
    const int py = ty * T + (int)(threadIdx.x / T);
    const bool inside = px < A.width && py < A.height;
    const float pxf = (float)px, pyf = (float)py;
    const uint2 rg = A.ranges[tile];
    const int n = (int)(rg.y - rg.x);
    float Tr = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
    uint32_t last = 0;
    bool done = !inside;
    for (int b0 = 0; b0 < n; b0 += NT) {
        if (__syncthreads_count(done) == NT) break;
        const int j = b0 + (int)threadIdx.x;
        if (j < n) {
            const uint32_t id = A.vals[rg.x + j];
            const float4 q0 = A.p0[id];
            const float4 q1 = A.p1[id];
            const float4 q2 = A.p2[id];
            s_g0[threadIdx.x] = make_float4(q0.x, q0.y, q1.x, q1.y + q1.y);
            s_g1[threadIdx.x] = make_float4(q1.z, q1.w, q0.z, 0.0f);
            s_g2[threadIdx.x] = q2;
        }
        __syncthreads();
        if (!done) {
            const int cnt = min(NT, n - b0);
            for (int k = 0; k < cnt; ++k) {
                const float4 g0 = s_g0[k];
                const float4 g1 = s_g1[k];
                const float dx = pxf - g0.x;
                const float dy = pyf - g0.y;
                const float e = g0.w * dy;
                const float f = (g1.x * dy) * dy;
                const float q = fmaf(dx, fmaf(g0.z, dx, e), f);
                if (!(q <= g1.y)) continue;
                const float g = gs_expf(-0.5f * q);
                const float alpha = fminf(0.99f, g1.z * g);
                const float Tn = Tr * (1.0f - alpha);
                if (Tn < 1e-4f) {
                    done = true;
                    break;
                }
                const float w = alpha * Tr;
                const float4 c = s_g2[k];
                C0 = fmaf(c.x, w, C0);
                C1 = fmaf(c.y, w, C1);
                C2 = fmaf(c.z, w, C2);
                Tr = Tn;
                last = (uint32_t)(b0 + k + 1);
            }
        }
    }
    if (inside) {
        const size_t HW = (size_t)A.width * A.height;
        const size_t o = (size_t)py * A.width + px;
        A.image[o] = fmaf(Tr, A.bg0, C0);
        A.image[HW + o] = fmaf(Tr, A.bg1, C1);
        A.image[2 * HW + o] = fmaf(Tr, A.bg2, C2);
        A.final_T[o] = Tr;
        A.last[o] = last;
    }
}

}  // namespace

gs_status launch_ranges(gs_context* ctx, const FrameView& v) {
    const size_t tiles = (size_t)v.gx * v.gy;
    if (cudaMemsetAsync(v.ranges, 0, tiles * sizeof(uint2), ctx->stream) != cudaSuccess)
        return set_error(ctx, GS_ERR_CUDA, "tile_ranges: cudaMemsetAsync failed");
    if (v.kcap == 0) return GS_OK;
    const int64_t blocks = (v.kcap + 255) / 256;
    ranges_kernel<<<(unsigned)blocks, 256, 0, ctx->stream>>>(v.keys0, v.status, v.ranges);
    ctx->launches += 1;
    return check_launch(ctx, "tile_ranges");
}

gs_status launch_render(gs_context* ctx, const gs_raster_cfg* cfg, const FrameView& v) {
    BlendArgs A;
    A.ranges = v.ranges;
    A.vals = v.vals0;
    A.p0 = v.p0;
    A.p1 = v.p1;
    A.p2 = v.p2;
    A.image = v.image;
    A.final_T = v.final_T;
    A.last = v.last;
    A.width = v.width;
    A.height = v.height;
    A.gx = v.gx;
    A.bg0 = cfg->bg[0];
    A.bg1 = cfg->bg[1];
    A.bg2 = cfg->bg[2];
    const unsigned tiles = (unsigned)(v.gx * v.gy);
    if (tiles == 0) return GS_OK;
    switch (v.tile) {
        case 8: blend_kernel<8><<<tiles, 64, 0, ctx->stream>>>(A); break;
        case 16: blend_kernel<16><<<tiles, 256, 0, ctx->stream>>>(A); break;
        case 32: blend_kernel<32><<<tiles, 1024, 0, ctx->stream>>>(A); break;
        default: return set_error(ctx, GS_ERR_INVALID, "render: tile %d not supported", v.tile);
    }
    ctx->launches += 1;
    return check_launch(ctx, "render");
}

}  // namespace gs
