// InclusiveSum + duplicateWithKeys (Sec. 3.2.2).
//
// Three launches:
//   scan_reduce  each block sums 1024 tile counts (int64 partial per block);
//   scan_top     one block turns the partials into exclusive block offsets,
//                stores the key total K in the frame status and flags a
//                capacity overflow;
//   emit         each block re-reads its 1024 counts, scans them in shared
//                memory round by round (so per-Gaussian offsets are never
//                stored in HBM), and every Gaussian with tiles writes its
//                (tile << 32 | depth bits, index) pairs at its offset: a
//                whole rectangle known in advance directly, any other tile
//                set recomputed with the localization function the count
//                used (those are queued per warp and searched after the
//                rounds); in buffer 0, or (for a fused forward call) in the
//                buffer the sort plan starts from (scan_top's offsets say
//                which).
#include "tiles.cuh"

namespace gs {
namespace {

// Each block sums its kScanBlock counts and reduces its share of the
// preprocess's per-warp depth ranges (an even split of the n_warps slots
// over the blocks, independent of which Gaussians a warp held); one barrier
// serves both reductions.
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const int32_t* __restrict__ counts, int64_t n,
                                                                   long long* __restrict__ partials,
                                                                   const uint2* __restrict__ warp_range,
                                                                   int64_t n_warps, uint2* __restrict__ block_range) {
    pdl_begin();
    constexpr int kWarps = kScanThreads / 32;
    __shared__ long long s_sum[kWarps];
    __shared__ uint2 s_range[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint2 r = make_uint2(0u, 0u);
    if (warp_range) {
        const int64_t w0 = n_warps * blockIdx.x / gridDim.x, w1 = n_warps * (blockIdx.x + 1) / gridDim.x;
        for (int64_t w = w0 + threadIdx.x; w < w1; w += kScanThreads) {
            const uint2 x = warp_range[w];
            r.x = max(r.x, x.x);
            r.y = max(r.y, x.y);
        }
    }
    const int64_t base = (int64_t)blockIdx.x * kScanBlock;
    long long sum = 0;
#pragma unroll 4
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        if (i < n) sum += counts[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    r.x = __reduce_max_sync(0xffffffffu, r.x);
    r.y = __reduce_max_sync(0xffffffffu, r.y);
    if (lane == 0) {
        s_sum[warp] = sum;
        s_range[warp] = r;
    }
    __syncthreads();
    if (warp == 0) {
        long long t = lane < kWarps ? s_sum[lane] : 0;
        uint2 m = lane < kWarps ? s_range[lane] : make_uint2(0u, 0u);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        m.x = __reduce_max_sync(0xffffffffu, m.x);
        m.y = __reduce_max_sync(0xffffffffu, m.y);
        if (lane == 0) {
            partials[blockIdx.x] = t;
            if (warp_range) block_range[blockIdx.x] = m;
        }
    }
}

__global__ void __launch_bounds__(1024) scan_top_kernel(long long* __restrict__ partials, int64_t nblocks,
                                                        int64_t kcap, uint32_t* __restrict__ status, bool clear3,
                                                        const uint2* __restrict__ block_range, bool fused,
                                                        int tile_bits, int dmax, uint32_t* __restrict__ sort_ctl) {
    pdl_begin();
    // a fused chain's sort control words (histograms, tickets) start at zero
    if (sort_ctl)
        for (int i = threadIdx.x; i < kSortCtlWords; i += blockDim.x) sort_ctl[i] = 0u;
    // Thread t takes a contiguous run of the partials: one pass sums its run
    // and reduces the matching depth ranges, one block scan of the sums and
    // one reduction of the ranges (sharing two barriers) give every run its
    // offset, and a second pass writes the offsets.
    __shared__ long long s_sum[32];
    __shared__ uint2 s_range[32];
    __shared__ long long s_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t per = (nblocks + blockDim.x - 1) / blockDim.x;
    const int64_t b_lo = min((int64_t)threadIdx.x * per, nblocks), b_hi = min(b_lo + per, nblocks);
    long long sum = 0;
    uint2 r = make_uint2(0u, 0u);
    for (int64_t b = b_lo; b < b_hi; ++b) {
        sum += partials[b];
        if (block_range) {
            const uint2 x = block_range[b];
            r.x = max(r.x, x.x);
            r.y = max(r.y, x.y);
        }
    }
    const long long inc = warp_incl_scan(sum, lane);
    r.x = __reduce_max_sync(0xffffffffu, r.x);
    r.y = __reduce_max_sync(0xffffffffu, r.y);
    if (lane == 31) s_sum[warp] = inc;
    if (lane == 0) s_range[warp] = r;
    __syncthreads();
    if (warp == 0) {
        const bool w = lane < (int)(blockDim.x >> 5);
        const long long ws = warp_incl_scan(w ? s_sum[lane] : 0ll, lane);
        uint2 m = w ? s_range[lane] : make_uint2(0u, 0u);
        m.x = __reduce_max_sync(0xffffffffu, m.x);
        m.y = __reduce_max_sync(0xffffffffu, m.y);
        if (w) s_sum[lane] = ws;
        if (lane == 0) {
            status[kStatusDepthLoN] = m.x;
            status[kStatusDepthHi] = m.y;
            // A fused call whose sort plan starts from buffer 1 has the emit
            // write there: buffer 1 is buffer 0 displaced by the key capacity
            // (keys and values alike), so every block offset starts at kcap.
            const SortPlan P = sort_plan_of(m.x, m.y, tile_bits, dmax, true);
            s_base = (fused && P.start) ? (long long)kcap : 0ll;
        }
    }
    __syncthreads();
    long long run = s_base + (warp > 0 ? s_sum[warp - 1] : 0ll) + (inc - sum);
    for (int64_t b = b_lo; b < b_hi; ++b) {
        const long long v = partials[b];
        partials[b] = run;
        run += v;
    }
    const long long s_carry = s_sum[(blockDim.x >> 5) - 1];  // the key total K
    if (threadIdx.x == 0) {
        const long long K = s_carry;
        // words 0..2 (and 3 for a single camera; a batch's set-up kernel has
        // just written its word 3) start this frame's status afresh
        status[0] = (uint32_t)(K & 0xffffffffll);
        status[1] = (uint32_t)(K >> 32);
        status[2] = K > kcap ? GS_FLAG_CAPACITY : 0u;
        if (clear3) {
            status[3] = 0u;
            // the preprocess that produced these counts has completed: keep
            // its culled count and start the next frame's at zero
            status[kStatusCulled] = status[kStatusCulledAcc];
            status[kStatusCulledAcc] = 0u;
        }
    }
}

struct EmitArgs {
    const int32_t* counts;
    const long long* partials;  // exclusive offset of each scan block
    const float4* p0;
    const float4* p1;
    const float4* p2;
    const uint32_t* status;
    uint64_t* keys;  // buffer 0; buffer 1 follows at keys + kcap (vals alike)
    uint32_t* vals;
    int64_t n;
    int mode;
    Grid grid;
    const CamRec* table;  // multi-view (else nullptr)
    int64_t cam_stride;   // Gaussian slots per camera
};

struct KeyWriter {
    uint64_t* keys;
    uint32_t* vals;
    long long pos;
    long long end;  // one past this Gaussian's last slot (offset + counted tiles)
    uint32_t depth_bits;
    uint32_t id;
    int gx;
    uint32_t tile0;  // first global tile of this camera (multi-view), else 0
    __device__ __forceinline__ void put(uint32_t tile) {
        if (pos < end) {  // the recount always equals the count; never write past it regardless
            keys[pos] = ((uint64_t)(tile0 + tile) << 32) | depth_bits;
            vals[pos] = id;
        }
        ++pos;
    }
    // AccuTile line callback: rows -> line k is tile row ty = k, span over tx;
    // columns -> line k is tile column tx = k, span over ty.
    __device__ __forceinline__ void operator()(int k, int jmin, int jmax, bool rows) {
        if (rows) {
            for (int j = jmin; j <= jmax; ++j) put((uint32_t)(k * gx + j));
        } else {
            for (int j = jmin; j <= jmax; ++j) put((uint32_t)(j * gx + k));
        }
    }
};

// One instantiation per tile mode, so each mode's kernel holds only its own
// tile-set code (and its registers are allocated for that code alone).
template <bool kMulti, int kMode>
__global__ void __launch_bounds__(kScanThreads, 4) emit_kernel(const EmitArgs A) {
    pdl_begin();
    constexpr bool kDefer = kMode == GS_MODE_ACCUTILE || kMode == GS_MODE_TBC || kMode == GS_MODE_PIXEL;
    constexpr int kWarps = kScanThreads / 32;
    __shared__ int s_tot[kScanItems][kWarps];
    // Gaussians whose tiles are not a whole rectangle known in advance
    // (AccuTile: all but whole single lines; tile-based culling and
    // pixel-exact tiles: those that keep fewer tiles than their candidate
    // rectangle holds), queued per warp as (slot in block, key offset in
    // block) and handled together after the rounds
    __shared__ int2 s_q[kDefer ? kWarps : 1][kDefer ? kScanBlock / kWarps : 1];
    if (A.status[2] & GS_FLAG_CAPACITY) return;  // keys do not fit: emit nothing
    if (kMulti && A.status[3]) return;           // cameras do not fit the batch frame
    // The block's 1024 slots are taken in 4 rounds of 256 consecutive ones
    // (one per thread), so the 2D-state loads of a round are coalesced and
    // neighbouring threads write neighbouring key ranges.  A slot is a
    // Gaussian (single view) or a (camera, Gaussian) pair, camera-major.
    // Software pipeline: the four rounds' counts are loaded up front, and
    // while a round is processed the next round's 2D state is already in
    // flight, so the rounds do not wait on memory one after another.  The
    // slots' offsets come from one scan of all four rounds before the first
    // (lane prefixes by warp shuffles, warp totals exchanged once), so the
    // rounds themselves need no barrier.  Offsets within the block fit 32
    // bits: the emit runs only when K <= key_capacity < 2^30.
    const long long carry = A.partials[blockIdx.x];
    const int64_t block0 = (int64_t)blockIdx.x * kScanBlock;
    int cnt[kScanItems];
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) {
        const int64_t i = block0 + (int64_t)r * kScanThreads + threadIdx.x;
        cnt[r] = i < A.n ? A.counts[i] : 0;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int excl[kScanItems];  // slot offset within the block
    {
#pragma unroll
        for (int r = 0; r < kScanItems; ++r) {
            int inc = cnt[r];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            excl[r] = inc - cnt[r];
            if (lane == 31) s_tot[r][warp] = inc;
        }
        __syncthreads();
        int before = 0;  // the block's earlier rounds
#pragma unroll
        for (int r = 0; r < kScanItems; ++r) {
            int wpre = 0, rtot = 0;
#pragma unroll
            for (int w = 0; w < kScanThreads / 32; ++w) {
                const int t = s_tot[r][w];
                rtot += t;
                if (w < warp) wpre += t;
            }
            excl[r] += before + wpre;
            before += rtot;
        }
    }
    // grid, first global tile and Gaussian id of slot i (its camera's, in a
    // multi-view batch)
    auto slot_frame = [&](int64_t i, Grid& grid, uint32_t& tile0, uint32_t& id) {
        grid = A.grid;
        tile0 = 0;
        id = (uint32_t)i;
        if (kMulti) {
            const int64_t cam = i / A.cam_stride;
            const CamRec& R = A.table[cam];
            grid.gx = R.gx;
            grid.gy = R.gy;
            grid.W = R.width;
            grid.H = R.height;
            tile0 = (uint32_t)R.tile_offset;
            id = (uint32_t)(i - cam * A.cam_stride);
        }
    };
    int qn = 0;  // queued slots of this warp
    constexpr bool three = kMode == GS_MODE_3SIGMA;
    float4 q0 = make_float4(0.f, 0.f, 0.f, 0.f), q1 = q0;
    int rad = 0;
    if (cnt[0] > 0) {
        const int64_t i = block0 + threadIdx.x;
        q0 = A.p0[i];
        if (three) rad = __float_as_int(A.p2[i].w);
        else q1 = A.p1[i];
    }
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) {
        const int64_t i = block0 + (int64_t)r * kScanThreads + threadIdx.x;
        const int c = cnt[r];
        float4 n0 = make_float4(0.f, 0.f, 0.f, 0.f), n1 = n0;
        int nrad = 0;
        if (r + 1 < kScanItems && cnt[r + 1] > 0) {
            const int64_t in = i + kScanThreads;
            n0 = A.p0[in];
            if (three) nrad = __float_as_int(A.p2[in].w);
            else n1 = A.p1[in];
        }
        const long long off = carry + excl[r];
        bool defer = false;
        if (c > 0) {
            Grid grid;
            uint32_t tile0, id;
            slot_frame(i, grid, tile0, id);
            KeyWriter W{A.keys, A.vals, off, off + c, __float_as_uint(q0.w), id, grid.gx, tile0};
            if (three) {
                Rect R;
                if (sigma3_rect(q0.x, q0.y, rad, grid, R))
                    for (int ty = R.y0; ty <= R.y1; ++ty)
                        for (int tx = R.x0; tx <= R.x1; ++tx) W.put((uint32_t)(ty * grid.gx + tx));
            } else {
                const Ellipse E{q0.x, q0.y, q1.x, q1.y, q1.z, q1.w};
                Snug S;
                if (snugbox(E, grid, S)) {
                    // tiles x0..x1 of rows y0..y1, row-major: the order in
                    // which every mode's tile function puts a whole rectangle
                    auto rect = [&](int x0, int x1, int y0, int y1) {
                        for (int ty = y0; ty <= y1; ++ty)
                            for (int tx = x0; tx <= x1; ++tx) W.put((uint32_t)(ty * grid.gx + tx));
                    };
                    if (kMode == GS_MODE_SNUGBOX) {
                        rect(S.R.x0, S.R.x1, S.R.y0, S.R.y1);
                    } else if (kMode == GS_MODE_TBC) {
                        // the count is the kept tiles of the SnugBox rectangle
                        if (c == (S.R.x1 - S.R.x0 + 1) * (S.R.y1 - S.R.y0 + 1)) rect(S.R.x0, S.R.x1, S.R.y0, S.R.y1);
                        else defer = true;
                    } else if (kMode == GS_MODE_PIXEL) {
                        // the count is the kept tiles of the pixel box's tile range
                        PixBox P;
                        if (pixel_box(S, grid, P) && c == (P.tx1 - P.tx0 + 1) * (P.ty1 - P.ty0 + 1))
                            rect(P.tx0, P.tx1, P.ty0, P.ty1);
                        else
                            defer = true;
                    } else {
                        int k, j0, j1;
                        bool rows;
                        if (accutile_whole_line(S, grid, k, j0, j1, rows)) W(k, j0, j1, rows);
                        else defer = true;
                    }
                }
            }
        }
        if (kDefer) {
            const unsigned m = __ballot_sync(0xffffffffu, defer);
            if (defer) s_q[warp][qn + __popc(m & ((1u << lane) - 1u))] = make_int2(r * kScanThreads + threadIdx.x, excl[r]);
            qn += __popc(m);
        }
        q0 = n0;
        q1 = n1;
        rad = nrad;
    }
    if (kDefer && qn > 0) {
        // one lane per queued Gaussian: the warp runs the tile searches of all
        // four rounds side by side instead of once per round
        __syncwarp();
        for (int b = 0; b < qn; b += 32) {
            if (b + lane < qn) {
                const int2 it = s_q[warp][b + lane];
                const int64_t i = block0 + it.x;
                const float4 a0 = A.p0[i], a1 = A.p1[i];
                const long long off = carry + it.y;
                Grid grid;
                uint32_t tile0, id;
                slot_frame(i, grid, tile0, id);
                KeyWriter W{A.keys, A.vals, off, off + A.counts[i], __float_as_uint(a0.w), id, grid.gx, tile0};
                const Ellipse E{a0.x, a0.y, a1.x, a1.y, a1.z, a1.w};
                Snug S;
                if (snugbox(E, grid, S)) {
                    auto put = [&](int tx, int ty) { W.put((uint32_t)(ty * grid.gx + tx)); };
                    if (kMode == GS_MODE_TBC) tbc_tiles(E, S, grid, put);
                    else if (kMode == GS_MODE_PIXEL) pixel_tiles(E, S, grid, put);
                    else accutile_sweep(E, S, grid, W);
                }
            }
        }
    }
}

}  // namespace

gs_status launch_intersect(gs_context* ctx, const gs_raster_cfg* cfg, const FrameView& v, bool fused) {
    const int64_t nb = scan_blocks_for(v.ncap);
    // preprocess warps that stored a depth range: ceil(n / 256) blocks (per camera)
    const int64_t per_cam = v.table ? v.cam_stride : v.ncap;
    const int64_t n_warps = (per_cam + kPreThreads - 1) / kPreThreads * (kPreThreads / 32) * (v.table ? v.num_cams : 1);
    if (nb > 0) {
        (void)launch_pdl(ctx->stream, scan_reduce_kernel, dim3((unsigned)nb), dim3(kScanThreads), 0, v.counts, v.ncap,
                         v.scan_partials, (const uint2*)v.warp_range, n_warps, v.block_range);
        ctx->launches += 1;
    }
    (void)launch_pdl(ctx->stream, scan_top_kernel, dim3(1), dim3(1024), 0, v.scan_partials, nb, v.kcap, v.status,
                     v.table == nullptr, (const uint2*)(v.warp_range ? v.block_range : nullptr), fused,
                     sort_tile_bits((int64_t)v.gx * v.gy), sort_digit_max(cfg->sort_digit_bits),
                     fused ? v.sort_hist : nullptr);
    ctx->launches += 1;
    if (nb > 0) {
        EmitArgs A;
        A.counts = v.counts;
        A.partials = v.scan_partials;
        A.p0 = v.p0;
        A.p1 = v.p1;
        A.p2 = v.p2;
        A.status = v.status;
        A.keys = v.keys0;
        A.vals = v.vals0;
        A.n = v.ncap;
        A.mode = cfg->mode;
        A.grid = Grid{(float)v.tile, v.gx, v.gy, v.width, v.height};
        A.table = v.table;
        A.cam_stride = v.cam_stride;
#define GS_EMIT(M_)                                                                                          \
    (v.table ? launch_pdl(ctx->stream, emit_kernel<true, M_>, dim3((unsigned)nb), dim3(kScanThreads), 0, A)     \
             : launch_pdl(ctx->stream, emit_kernel<false, M_>, dim3((unsigned)nb), dim3(kScanThreads), 0, A))
        switch (cfg->mode) {
            case GS_MODE_3SIGMA: (void)GS_EMIT(GS_MODE_3SIGMA); break;
            case GS_MODE_SNUGBOX: (void)GS_EMIT(GS_MODE_SNUGBOX); break;
            case GS_MODE_TBC: (void)GS_EMIT(GS_MODE_TBC); break;
            case GS_MODE_PIXEL: (void)GS_EMIT(GS_MODE_PIXEL); break;
            default: (void)GS_EMIT(GS_MODE_ACCUTILE); break;
        }
#undef GS_EMIT
        ctx->launches += 1;
    }
    return check_launch(ctx, "intersect");
}

}  // namespace gs
