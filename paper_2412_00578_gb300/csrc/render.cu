// identifyTileRanges and render (Sec. 3.2.2, Sec. 3.2.3).
//
// ranges: four sorted keys per thread; a key whose tile differs from its
// predecessor's closes the previous range and opens its own.
//
// blend: one CTA per tile, one thread per pixel, each warp owning an 8 x 4
// pixel sub-tile.  The tile's Gaussians are brought into shared memory in
// batches of one per thread (a gather of the 48-byte 2D state by sorted
// index); the loading thread also computes which sub-tiles the Gaussian's
// ellipse can reach.  Each warp then takes a batch in two phases: it walks,
// in depth order, only the Gaussians whose mask has its bit (ballot +
// find-first-set) and records per pixel which of them pass the in-ellipse
// test; then every lane blends its own passing Gaussians in order, the lanes
// of the warp working on different Gaussians at once.  Every pixel still
// takes every Gaussian that reaches it in the same order with the same
// arithmetic.  Per pixel (Eqs. render_alpha, 2d_gaussian_scalar,
// contribution): dx = px - u, dy = py - v, e = (2b) dy, f = (c dy) dy,
// q = fma(dx, fma(a, dx, e), f); a Gaussian counts iff q <= t (alpha >= 1/255);
// alpha = min(0.99, sigma exp(-q/2)); T' = T (1 - alpha); if T' < 1e-4 the
// pixel stops before adding it; else C = fma(c, alpha T, C), T = T'.
// The CTA leaves the loop as soon as every pixel has stopped
// (__syncthreads_count vote before each batch).
#include <algorithm>

#include "blend_common.cuh"

namespace gs {
namespace {

// Keys present in the buffer (see sort.cu): none when the emit was skipped,
// a sort wait gave up or the sort met a key outside the recorded range.
__device__ __forceinline__ uint32_t frame_keys_r(const uint32_t* status) {
    return ((status[2] & (GS_FLAG_CAPACITY | GS_FLAG_TIMEOUT | GS_FLAG_KEYRANGE)) || status[3]) ? 0u : status[0];
}

// Four consecutive keys per thread (two 16-byte loads when the buffer is
// 16-byte aligned) plus the key before them: a key whose tile differs from its
// predecessor's closes the previous range and opens its own, and writes
// [0, 0) for the empty tiles between the two.  The whole grid writes [0, 0)
// for the tiles before the first key's and after the last key's (all tiles
// when there are no keys).  Every word of the ranges is written exactly
// once, so no zero-fill precedes the kernel.
__global__ void __launch_bounds__(256) ranges_kernel(const uint64_t* __restrict__ keys,
                                                     const uint32_t* __restrict__ status, uint2* __restrict__ ranges,
                                                     uint32_t tiles) {
    pdl_begin();
    const uint32_t K = frame_keys_r(status);
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    const uint32_t i0 = g * 4u;
    const uint32_t t_first = K ? (uint32_t)(keys[0] >> 32) : tiles;
    const uint32_t t_last = K ? (uint32_t)(keys[K - 1] >> 32) : tiles;
    for (uint32_t t = g; t < t_first; t += stride) ranges[t] = make_uint2(0u, 0u);
    for (uint32_t t = t_last + 1u + g; t < tiles; t += stride) ranges[t] = make_uint2(0u, 0u);
    if (i0 >= K) return;
    uint32_t t[4];
    // the frame only guarantees 8-byte alignment of keys: vector loads only
    // from a 16-byte aligned buffer
    if (i0 + 4u <= K && (reinterpret_cast<uintptr_t>(keys) & 15u) == 0u) {
        const ulonglong2 a = *reinterpret_cast<const ulonglong2*>(keys + i0);
        const ulonglong2 b = *reinterpret_cast<const ulonglong2*>(keys + i0 + 2);
        t[0] = (uint32_t)(a.x >> 32);
        t[1] = (uint32_t)(a.y >> 32);
        t[2] = (uint32_t)(b.x >> 32);
        t[3] = (uint32_t)(b.y >> 32);
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) t[j] = i0 + j < K ? (uint32_t)(keys[i0 + j] >> 32) : 0u;
    }
    uint32_t prev = i0 > 0 ? (uint32_t)(keys[i0 - 1] >> 32) : 0xffffffffu;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t i = i0 + j;
        if (i >= K) break;
        if (i == 0) {
            ranges[t[j]].x = 0;
        } else if (prev != t[j]) {
            ranges[prev].y = i;
            ranges[t[j]].x = i;
            for (uint32_t e = prev + 1; e < t[j]; ++e) ranges[e] = make_uint2(0u, 0u);
        }
        if (i == K - 1) ranges[t[j]].y = K;
        prev = t[j];
    }
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
    unsigned long long* stats;  // [3]: defined, contributing, executed pair counts (stats variant)
    const CamRec* table;        // multi-view (else nullptr)
    int num_cams;
    int64_t cam_stride;
    int64_t pixel_capacity;
    const uint32_t* order;      // tile of each CTA (heaviest first), or nullptr for tile = CTA
    unsigned tiles;             // CTAs launched (tiles of the frame, or the batch's tile capacity)
};

// Camera owning global tile g of a multi-view batch: the last camera whose
// first tile is <= g (tile offsets ascend with the camera index).
__device__ __forceinline__ int camera_of_tile(const CamRec* table, int num_cams, long long g) {
    int lo = 0, hi = num_cams - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (table[mid].tile_offset <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Launch order of the blend's tiles, heaviest first: a counting sort of the
// tiles by floor(log2(entries)), descending (one block, one shared-memory
// atomic per warp and class).  Tiles are
// independent, so the order changes only when each tile's CTA starts; it keeps
// the few tiles with thousands of entries from starting last and leaving the
// rest of the GPU idle while they finish.
__global__ void __launch_bounds__(1024) tile_order_kernel(const uint2* __restrict__ ranges, uint32_t tiles,
                                                         uint32_t* __restrict__ order) {
    pdl_begin();
    __shared__ uint32_t cnt[33];
    __shared__ uint32_t base[33];
    __shared__ uint8_t s_cls[kMaxOrderedTiles];  // class of each tile, read once from ranges
    const uint32_t lane = threadIdx.x & 31u;
    if (threadIdx.x < 33) cnt[threadIdx.x] = 0;
    // Class 0 = heaviest (clz of the entry count), 32 = empty.
    for (uint32_t t0 = 0; t0 < tiles; t0 += 4u * blockDim.x) {
        uint2 r[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t t = t0 + (uint32_t)u * blockDim.x + threadIdx.x;
            r[u] = t < tiles ? ranges[t] : make_uint2(0u, 0u);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t t = t0 + (uint32_t)u * blockDim.x + threadIdx.x;
            const uint32_t n = r[u].y - r[u].x;
            if (t < tiles) s_cls[t] = (uint8_t)(n ? __clz(n) : 32);
        }
    }
    __syncthreads();
    // lanes of a warp with the same class add to its counter once
    for (uint32_t t0 = 0; t0 < tiles; t0 += blockDim.x) {
        const uint32_t t = t0 + threadIdx.x;
        const uint32_t cls = t < tiles ? s_cls[t] : 64u;
        const uint32_t peers = __match_any_sync(0xffffffffu, cls);
        if (t < tiles && lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&cnt[cls], (uint32_t)__popc(peers));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int k = 0; k < 33; ++k) {
            base[k] = run;
            run += cnt[k];
        }
    }
    __syncthreads();
    for (uint32_t t0 = 0; t0 < tiles; t0 += blockDim.x) {
        const uint32_t t = t0 + threadIdx.x;
        const uint32_t cls = t < tiles ? s_cls[t] : 64u;
        const uint32_t peers = __match_any_sync(0xffffffffu, cls);
        const uint32_t leader = (uint32_t)(__ffs(peers) - 1);
        uint32_t b = 0;
        if (t < tiles && lane == leader) b = atomicAdd(&base[cls], (uint32_t)__popc(peers));
        b = __shfl_sync(0xffffffffu, b, leader);
        if (t < tiles) order[b + (uint32_t)__popc(peers & ((1u << lane) - 1u))] = t;
    }
}

// The same heaviest-first order for more tiles than one block holds (a
// multi-view batch): many blocks count the tiles per class (shared-memory
// counters, one global atomic per class and block); the last block to finish
// turns the counts into class bases; a second launch places every tile in
// its class's segment (warp-aggregated atomics, so the order within a class
// is arbitrary: tiles are independent and the order changes no output).
// ctl: [0, 33) class counts, [33, 66) class bases, [66] blocks done; zero at launch.
__global__ void __launch_bounds__(256) order_count_kernel(const uint2* __restrict__ ranges, uint32_t tiles,
                                                          uint32_t* __restrict__ ctl) {
    pdl_begin();
    __shared__ uint32_t cnt[33];
    __shared__ bool s_last;
    if (threadIdx.x < 33) cnt[threadIdx.x] = 0;
    __syncthreads();
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < tiles; t += gridDim.x * blockDim.x) {
        const uint2 r = ranges[t];
        const uint32_t n = r.y - r.x;
        atomicAdd(&cnt[n ? __clz(n) : 32], 1u);
    }
    __syncthreads();
    if (threadIdx.x < 33 && cnt[threadIdx.x]) atomicAdd(&ctl[threadIdx.x], cnt[threadIdx.x]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&ctl[66], 1u) == gridDim.x - 1;
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        uint32_t run = 0;
        for (int k = 0; k < 33; ++k) {
            ctl[33 + k] = run;
            run += __ldcg(&ctl[k]);
        }
    }
}

__global__ void __launch_bounds__(256) order_place_kernel(const uint2* __restrict__ ranges, uint32_t tiles,
                                                          uint32_t* __restrict__ ctl, uint32_t* __restrict__ order) {
    pdl_begin();
    const uint32_t lane = threadIdx.x & 31u;
    for (uint32_t t0 = blockIdx.x * blockDim.x; t0 < tiles; t0 += gridDim.x * blockDim.x) {
        const uint32_t t = t0 + threadIdx.x;
        uint32_t cls = 64u;
        if (t < tiles) {
            const uint2 r = ranges[t];
            const uint32_t n = r.y - r.x;
            cls = n ? __clz(n) : 32u;
        }
        const uint32_t peers = __match_any_sync(0xffffffffu, cls);
        const uint32_t leader = (uint32_t)(__ffs(peers) - 1);
        uint32_t b = 0;
        if (t < tiles && lane == leader) b = atomicAdd(&ctl[33 + cls], (uint32_t)__popc(peers));
        b = __shfl_sync(0xffffffffu, b, leader);
        if (t < tiles) order[b + (uint32_t)__popc(peers & ((1u << lane) - 1u))] = t;
    }
}

template <int T, bool kStats, bool kMulti>
__global__ void __launch_bounds__(T* T, T == 32 ? 1 : (T == 16 ? 4 : 16)) blend_kernel(const BlendArgs A) {
    pdl_begin();
    constexpr int NT = T * T;
    constexpr int NB = NT < 256 ? NT : 256;  // Gaussians per shared-memory batch
    constexpr int NSX = T / kSubW;
    __shared__ float4 s_g0[NB];  // u, v, a, 2b
    __shared__ float4 s_g1[NB];  // c, t, opacity, -
    __shared__ float4 s_g2[NB];  // r, g, b, -
    __shared__ uint32_t s_mask[NB];
    __shared__ uint32_t s_pass[NT / 32][NB / 32][32];  // per warp, chunk, lane: passing entries
    const int tile = A.order ? (int)A.order[blockIdx.x] : (int)blockIdx.x;  // global tile index
    if ((unsigned)tile >= A.tiles) return;  // an order never written by gs_tile_ranges
    int gx = A.gx, width = A.width, height = A.height, local = tile;
    float* image = A.image;
    float* final_T = A.final_T;
    uint32_t* last_out = A.last;
    const float4* p0 = A.p0;
    const float4* p1 = A.p1;
    const float4* p2 = A.p2;
    if (kMulti) {
        const int cam = camera_of_tile(A.table, A.num_cams, tile);
        const CamRec& R = A.table[cam];
        if ((long long)tile >= R.tile_offset + (long long)R.gx * R.gy) return;  // beyond the last camera
        if (R.pix_offset + (long long)R.width * R.height > A.pixel_capacity) return;
        gx = R.gx;
        width = R.width;
        height = R.height;
        local = (int)(tile - R.tile_offset);
        image += 3 * R.pix_offset;
        final_T += R.pix_offset;
        last_out += R.pix_offset;
        p0 += (int64_t)cam * A.cam_stride;
        p1 += (int64_t)cam * A.cam_stride;
        p2 += (int64_t)cam * A.cam_stride;
    }
    const int tx = local % gx, ty = local / gx;
    const int warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
    const uint32_t my_bit = 1u << warp;
    const int px = tx * T + (warp % NSX) * kSubW + (lane & (kSubW - 1));
    const int py = ty * T + (warp / NSX) * kSubH + (lane >> 3);
    const bool inside = px < width && py < height;
    const float pxf = (float)px, pyf = (float)py;
    const float ox = (float)(tx * T), oy = (float)(ty * T);
    const uint2 rg = A.ranges[tile];
    const int n = (int)(rg.y - rg.x);
    float Tr = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
    uint32_t last = 0;
    bool done = !inside;
    uint32_t stop_pos = 0, n_exec = 0, n_contrib = 0;
    // Software pipeline over the batches: while the warps work on batch i,
    // each loading thread already has batch i+1's 2D state in flight and
    // batch i+2's index requested.
    const bool loader = (int)threadIdx.x < NB;
    uint32_t id_next = 0, id_next2 = 0;
    float4 q0 = make_float4(0.f, 0.f, 0.f, 0.f), q1 = q0, q2 = q0;
    if (loader) {
        if ((int)threadIdx.x < n) {
            const uint32_t id = A.vals[rg.x + threadIdx.x];
            q0 = p0[id];
            q1 = p1[id];
            q2 = p2[id];
        }
        if (NB + (int)threadIdx.x < n) id_next = A.vals[rg.x + NB + threadIdx.x];
    }
    for (int b0 = 0; b0 < n; b0 += NB) {
        if (__syncthreads_count(done) == NT) break;
        if (loader && b0 + (int)threadIdx.x < n) {
            s_g0[threadIdx.x] = make_float4(q0.x, q0.y, q1.x, q1.y + q1.y);
            s_g1[threadIdx.x] = make_float4(q1.z, q1.w, q0.z, 0.0f);
            s_g2[threadIdx.x] = q2;
            s_mask[threadIdx.x] = subtile_mask<T>(q0.x, q0.y, q1.x, q1.y, q1.z, q1.w, ox, oy);
        }
        __syncthreads();
        if (loader) {
            if (b0 + NB + (int)threadIdx.x < n) {
                q0 = p0[id_next];
                q1 = p1[id_next];
                q2 = p2[id_next];
            }
            if (b0 + 2 * NB + (int)threadIdx.x < n) id_next2 = A.vals[rg.x + b0 + 2 * NB + threadIdx.x];
            id_next = id_next2;
        }
        if (__all_sync(0xffffffffu, done)) continue;
        const int cnt = min(NB, n - b0);
        const int nch = (cnt + 31) >> 5;
        // Phase 1: the in-ellipse test of every entry whose mask reaches this
        // warp's sub-tile, for every pixel still running; bit j of chunk c
        // records that entry 32 c + j passes for this lane's pixel.
        for (int c = 0; c < nch; ++c) {
            const int c0 = c * 32;
            uint32_t bits = __ballot_sync(0xffffffffu, c0 + lane < cnt && (s_mask[c0 + lane] & my_bit));
            uint32_t pass = 0;
            // two entries per step (the second repeats the first when only
            // one is left): half the loop overhead, two independent chains
            while (bits) {
                const int j = __ffs(bits) - 1;
                bits &= bits - 1u;
                const int j2 = bits ? __ffs(bits) - 1 : j;
                bits &= bits - 1u;
                if (done) continue;
                const float4 g0 = s_g0[c0 + j];
                const float4 g1 = s_g1[c0 + j];
                const float4 h0 = s_g0[c0 + j2];
                const float4 h1 = s_g1[c0 + j2];
                const float dx = pxf - g0.x, dy = pyf - g0.y;
                const float ex = pxf - h0.x, ey = pyf - h0.y;
                const float q = fmaf(dx, fmaf(g0.z, dx, g0.w * dy), (g1.x * dy) * dy);
                const float q2 = fmaf(ex, fmaf(h0.z, ex, h0.w * ey), (h1.x * ey) * ey);
                if (kStats) n_exec += (j2 != j) ? 2u : 1u;
                if (q <= g1.y) pass |= 1u << j;
                if (q2 <= h1.y) pass |= 1u << j2;
            }
            s_pass[warp][c][lane] = pass;
        }
        __syncwarp();
        // Phase 2: each lane blends its own passing entries in list order (q
        // recomputed with the same operations) until its pixel stops, so the
        // warp's iterations follow its busiest pixel, not the union of all.
        int c = 0;
        uint32_t cur = s_pass[warp][0][lane];
        for (;;) {
            while (cur == 0u && c + 1 < nch) cur = s_pass[warp][++c][lane];
            const bool have = cur != 0u && !done;
            if (!__any_sync(0xffffffffu, have)) break;
            if (!have) continue;
            const int k = c * 32 + __ffs(cur) - 1;
            cur &= cur - 1u;
            const float4 g0 = s_g0[k];
            const float4 g1 = s_g1[k];
            const float dx = pxf - g0.x;
            const float dy = pyf - g0.y;
            const float e = g0.w * dy;
            const float f = (g1.x * dy) * dy;
            const float q = fmaf(dx, fmaf(g0.z, dx, e), f);
            const float g = gs_expf_blend(-0.5f * q);
            const float alpha = fminf(0.99f, g1.z * g);
            const float Tn = Tr * (1.0f - alpha);
            if (Tn < 1e-4f) {
                done = true;
                stop_pos = (uint32_t)(b0 + k + 1);
                continue;
            }
            const float w = alpha * Tr;
            const float4 col = s_g2[k];
            C0 = fmaf(col.x, w, C0);
            C1 = fmaf(col.y, w, C1);
            C2 = fmaf(col.z, w, C2);
            Tr = Tn;
            last = (uint32_t)(b0 + k + 1);
            if (kStats) ++n_contrib;
        }
        __syncwarp();
    }
    if (inside) {
        const size_t HW = (size_t)width * height;
        const size_t o = (size_t)py * width + px;
        image[o] = fmaf(Tr, A.bg0, C0);
        image[HW + o] = fmaf(Tr, A.bg1, C1);
        image[2 * HW + o] = fmaf(Tr, A.bg2, C2);
        final_T[o] = Tr;
        last_out[o] = last;
    }
    if (kStats) {
        // pairs the tile-list definition evaluates: every entry up to the stop
        const uint32_t n_def = !inside ? 0u : (stop_pos ? stop_pos : (uint32_t)n);
        const uint32_t e = __reduce_add_sync(0xffffffffu, n_def);
        const uint32_t c = __reduce_add_sync(0xffffffffu, n_contrib);
        const uint32_t x = __reduce_add_sync(0xffffffffu, n_exec);
        if (lane == 0) {
            atomicAdd(A.stats, (unsigned long long)e);
            atomicAdd(A.stats + 1, (unsigned long long)c);
            atomicAdd(A.stats + 2, (unsigned long long)x);
        }
    }
}

}  // namespace

gs_status launch_ranges(gs_context* ctx, const FrameView& v) {
    const size_t tiles = (size_t)v.gx * v.gy;
    if (tiles > 0) {
        // 4 keys per thread; at least enough threads to clear the tiles in a few strides
        const int64_t blocks =
            std::max<int64_t>((v.kcap + 1023) / 1024, std::min<int64_t>(((int64_t)tiles + 255) / 256, 1024));
        (void)launch_pdl(ctx->stream, ranges_kernel, dim3((unsigned)blocks), dim3(256), 0, v.keys0, v.status,
                         v.ranges, (uint32_t)tiles);
        ctx->launches += 1;
    }
    // the blend's launch order, from the ranges just found
    if (tiles > 0 && tiles <= kMaxOrderedTiles) {
        (void)launch_pdl(ctx->stream, tile_order_kernel, dim3(1), dim3(1024), 0, v.ranges, (uint32_t)tiles,
                         v.tile_order);
        ctx->launches += 1;
    } else if (tiles > 0 && v.order_ctl && (int64_t)tiles <= v.tile_order_cap) {
        (void)launch_pdl(ctx->stream, zero_words_kernel, dim3(1), dim3(256), 0, v.order_ctl, (int64_t)67);
        const unsigned blocks = (unsigned)std::min<size_t>((tiles + 255) / 256, (size_t)ctx->num_sms * 4);
        (void)launch_pdl(ctx->stream, order_count_kernel, dim3(blocks), dim3(256), 0, v.ranges, (uint32_t)tiles,
                         v.order_ctl);
        (void)launch_pdl(ctx->stream, order_place_kernel, dim3(blocks), dim3(256), 0, v.ranges, (uint32_t)tiles,
                         v.order_ctl, v.tile_order);
        ctx->launches += 3;
    }
    return check_launch(ctx, "tile_ranges");
}

gs_status launch_render(gs_context* ctx, const gs_raster_cfg* cfg, const FrameView& v, unsigned long long* stats) {
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
    A.stats = stats;
    A.table = v.table;
    A.num_cams = v.num_cams;
    A.cam_stride = v.cam_stride;
    A.pixel_capacity = v.pixel_capacity;
    const unsigned tiles = (unsigned)(v.gx * v.gy);
    if (tiles == 0) return GS_OK;
    // written by launch_ranges
    A.order = (tiles <= kMaxOrderedTiles || (v.order_ctl && (int64_t)tiles <= v.tile_order_cap)) ? v.tile_order
                                                                                                   : nullptr;
    A.tiles = tiles;
#define GS_BLEND_LAUNCH(T_, S_, M_) \
    (void)launch_pdl(ctx->stream, blend_kernel<T_, S_, M_>, dim3(tiles), dim3(T_ * T_), 0, A)
#define GS_BLEND_TILES(S_, M_)                                                             \
    switch (v.tile) {                                                                      \
        case 8: GS_BLEND_LAUNCH(8, S_, M_); break;                                         \
        case 16: GS_BLEND_LAUNCH(16, S_, M_); break;                                       \
        case 32: GS_BLEND_LAUNCH(32, S_, M_); break;                                       \
        default: return set_error(ctx, GS_ERR_INVALID, "render: tile %d not supported", v.tile); \
    }
    if (v.table) {
        if (stats) { GS_BLEND_TILES(true, true) } else { GS_BLEND_TILES(false, true) }
    } else {
        if (stats) { GS_BLEND_TILES(true, false) } else { GS_BLEND_TILES(false, false) }
    }
#undef GS_BLEND_TILES
#undef GS_BLEND_LAUNCH
    ctx->launches += 1;
    return check_launch(ctx, "render");
}

}  // namespace gs
