// RadixSort (Sec. 3.2.2): stable least-significant-digit radix sort of the
// (key, value) pairs, onesweep style.
//
//   sort_hist   one read of the keys builds the digit histograms of every
//               pass at once (shared-memory counters, one global atomic per
//               bin per block) and clears the first look-back table; the
//               last block to finish picks each pass's ranking method from
//               the finished histogram (below).
//   sort_pass   one launch per digit, at most two CTAs per SM that stay
//               resident: each takes 4096-key partitions by atomic ticket
//               until none is left (so partitions are processed in ticket
//               order and every predecessor is held by a running or finished
//               CTA), ranks a partition's keys by digit stably (the lanes of
//               a warp holding equal digits find each other, then per-warp
//               counters), publishes its per-digit counts, and resolves its
//               global offsets by decoupled look-back over its predecessors'
//               published counts.  Keys are staged in shared memory in digit
//               order so each digit's run is written to HBM contiguously.
//               Every wait on a predecessor is bounded; when the bound is
//               reached the block records GS_FLAG_TIMEOUT and proceeds, so
//               no kernel can hang.
//
// Bits sorted: ceil(log2(tiles)) tile bits plus the w depth bits that the
// frame's depths span.  The preprocess records the least (dmin) and greatest
// depth bits of the Gaussians it gave tiles; every key is ordered by its
// image (tile << w) | (depth bits - dmin), which is strictly increasing in
// the key over the frame's keys, so sorting the images sorts the keys.  The
// first pass turns each key it reads into its image, the passes in between
// move images, and the last pass writes each key back in full.  The plan
// (pass count P, digit width) is a function of the status words, evaluated
// alike by every block of every sort kernel (sort_plan_of); the host launches
// the most passes any plan of the frame can need and the launches past P
// return at once.  The passes alternate between buffers 0 and 1 and the last
// one writes buffer 0: a
// stand-alone gs_sort (whose keys gs_intersect left in buffer 0) rounds P up
// to even, while gs_forward's chain lets the emit write buffer 1 when P is
// odd (the scan's offsets say where).
//
// Finding the lanes with equal digits: warp match costs more the more
// distinct digits a warp holds; a shared-memory atomicOr of each lane's bit
// into its digit's word costs more the more lanes share a digit.  Both give
// the same peer masks, so the ranks (and the sort) do not depend on the
// choice.  A pass whose digits are spread out (collision probability
// sum_d (n_d / K)^2 at most 1/8) ranks by atomicOr, a concentrated one (a
// depth byte of a frame at nearly one depth, the top tile bits of a tile-heavy
// digit) by match.
#include <algorithm>

#include "gs_common.cuh"

namespace gs {
namespace {

constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagPrefix = 2u << 30;
constexpr uint32_t kCountMask = (1u << 30) - 1;
constexpr uint32_t kNoDigit = 0xffffffffu;
constexpr int kLookWindow = 16;  // predecessors inspected per look-back step

// Keys present in the buffer: none when the emit was skipped (keys over
// capacity, or batch cameras over the frame's tile/pixel capacity), none
// once a look-back wait has given up (the pass that gave up may have placed
// keys wrongly, so no later pass, range or blend reads them), and none when
// a key lies outside the recorded range.
__device__ __forceinline__ uint32_t frame_keys(const uint32_t* status) {
    return ((status[2] & (GS_FLAG_CAPACITY | GS_FLAG_TIMEOUT | GS_FLAG_KEYRANGE)) || status[3]) ? 0u : status[0];
}

using DevPlan = SortPlan;

__device__ __forceinline__ DevPlan device_plan(const uint32_t* status, int tile_bits, int dmax, bool fused) {
    return sort_plan_of(status[kStatusDepthLoN], status[kStatusDepthHi], tile_bits, dmax, fused);
}

// The key's image (tile << w) | (depth bits - dmin), whose digits the passes sort.
__device__ __forceinline__ uint64_t plan_image(uint64_t k, const DevPlan& P) {
    return ((k >> 32) << P.w) | (uint64_t)((uint32_t)k - P.dmin);
}
// The key of an image.
__device__ __forceinline__ uint64_t plan_key(uint64_t im, const DevPlan& P) {
    const uint32_t rel = P.w < 32 ? (uint32_t)im & ((1u << P.w) - 1u) : (uint32_t)im;
    return ((im >> P.w) << 32) | (uint64_t)(rel + P.dmin);
}

struct HistArgs {
    const uint64_t* keys;  // buffer 0; buffer 1 follows at keys + kcap
    int64_t kcap;
    bool fused;
    uint32_t* status;
    uint32_t* hist;        // [passes][256]
    uint32_t* lookback0;   // first pass's table, cleared here
    uint32_t* method;      // [passes]: 1 = rank by warp match, 0 = by atomicOr
    uint32_t* done;        // blocks finished (zero at launch)
    int tile_bits, dmax;
};

constexpr uint32_t kRankMatch = 1u;

__global__ void __launch_bounds__(256) sort_hist_kernel(const HistArgs A) {
    pdl_begin();
    __shared__ uint32_t sh[kMaxPasses * 256];
    const DevPlan P = device_plan(A.status, A.tile_bits, A.dmax, A.fused);
    const uint64_t* keys = A.keys + (P.start ? A.kcap : 0);
    for (int i = threadIdx.x; i < P.passes * 256; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const uint32_t K = frame_keys(A.status);
    const uint32_t mask = (1u << P.dbits) - 1u;
    const uint32_t stride = gridDim.x * blockDim.x;
    // a key outside the recorded range (or past the tile bits) has no image
    const uint32_t wmask = P.w < 32 ? ~((1u << P.w) - 1u) : 0u;
    bool bad = false;
    auto count = [&](uint64_t key) {
        bad |= ((((uint32_t)key - P.dmin) & wmask) != 0u) || ((key >> 32) >> A.tile_bits) != 0ull;
        const uint64_t im = plan_image(key, P);
        for (int p = 0; p < P.passes; ++p) atomicAdd(&sh[p * 256 + (uint32_t)((im >> (p * P.dbits)) & mask)], 1u);
    };
    // four keys per thread and step, all loaded before any is counted
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3u * stride < K; i += 4u * stride) {
        uint64_t key[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) key[u] = keys[i + (uint32_t)u * stride];
#pragma unroll
        for (int u = 0; u < 4; ++u) count(key[u]);
    }
    for (; i < K; i += stride) count(keys[i]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(A.status + 2, GS_FLAG_KEYRANGE);
    // clear the look-back words of the partitions the first pass will use
    const uint32_t words = ((K + kSortPartition - 1) / kSortPartition) * 256u;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < words; i += stride) A.lookback0[i] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < P.passes * 256; i += blockDim.x)
        if (sh[i]) atomicAdd(&A.hist[i], sh[i]);
    // The last block to finish sees every block's counts and sets the
    // passes' ranking methods (warp w handles passes w, w + 8, ...).
    __shared__ bool s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(A.done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int lane = threadIdx.x & 31;
    const double kk = (double)K * (double)K;
    for (int p = threadIdx.x >> 5; p < P.passes; p += blockDim.x >> 5) {
        double sq = 0.0;
        for (int d = lane; d < 256; d += 32) {
            const double c = (double)__ldcg(A.hist + p * 256 + d);
            sq += c * c;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
        if (lane == 0) A.method[p] = (sq * 8.0 > kk) ? kRankMatch : 0u;
    }
}

struct PassArgs {
    uint64_t* keys;  // buffer 0 (the result); buffer 1 follows at keys + kcap
    uint32_t* vals;  // alike
    int64_t kcap;
    bool fused;
    uint32_t* status;
    const uint32_t* hist;   // this pass's 256 digit totals
    uint32_t* lookback;     // this pass's table [partitions][256]
    uint32_t* lookback_next;// next pass's table: this block clears its own row
    uint32_t* ticket;
    const uint32_t* method; // this pass's ranking method (set by sort_hist)
    int pass, tile_bits, dmax;
    uint32_t spin_limit;    // polls per look-back wait before it gives up
    int64_t withhold;       // partition that never publishes (wait-expiry test), else -1
};

struct PassSmem {
    union {
        // keys and values in digit order, staged for the write-out
        struct {
            uint64_t keys[kSortPartition];
            uint32_t vals[kSortPartition];
        } st;
        // ranking by atomicOr (before staging): per warp, three rotating
        // arrays of 256 peer words, so one __syncwarp per round suffices
        uint32_t peer[kSortThreads / 32][3][256];
    };
    // per (warp, digit): while ranking, the warp's keys with that digit so
    // far; after the digit scan, the staging slot of the warp's first key
    // with that digit (the digit's block offset plus the earlier warps' keys)
    uint32_t wbase[kSortThreads / 32][256];
    uint32_t gbase[256];
    unsigned long long warp_tmp[32];
    uint32_t part;
};

// Exclusive scan of one 64-bit value per thread over the block.
__device__ __forceinline__ unsigned long long block_excl_scan_u64(unsigned long long v, unsigned long long* s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (int)(blockDim.x >> 5);
    unsigned long long inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = lane < nwarps ? s_warp[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nwarps) s_warp[lane] = w;
    }
    __syncthreads();
    const unsigned long long r = (warp > 0 ? s_warp[warp - 1] : 0ull) + inc - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kSortThreads, 2) sort_pass_kernel(const PassArgs A) {
    pdl_begin();
    const DevPlan P = device_plan(A.status, A.tile_bits, A.dmax, A.fused);
    if (A.pass >= P.passes) return;  // the plan needs fewer passes
    // pass p reads buffer (start + p) mod 2 and writes the other one
    const int64_t src = ((P.start + A.pass) & 1) ? A.kcap : 0;
    const int64_t dst = A.kcap - src;
    const uint64_t* kin = A.keys + src;
    const uint32_t* vin = A.vals + src;
    uint64_t* kout = A.keys + dst;
    uint32_t* vout = A.vals + dst;
    const int shift = A.pass * P.dbits;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PassSmem& S = *reinterpret_cast<PassSmem*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool by_match = __ldg(A.method) == kRankMatch;  // uniform over the launch
    const uint32_t t = tid;
    const bool digit_thread = t < 256;
    const uint32_t hist_t = digit_thread ? __ldg(A.hist + t) : 0u;  // loaded early, used after ranking
    const uint32_t K = frame_keys(A.status);
    const uint32_t nparts = (K + kSortPartition - 1) / kSortPartition;
    // Persistent: at most two CTAs per SM, each taking partitions by ticket
    // until none is left.  A ticket's predecessors are held by CTAs that are
    // running or done, so every look-back wait ends.
    for (;;) {
        if (tid == 0) S.part = atomicAdd(A.ticket, 1u);
        {
            uint4* c4 = reinterpret_cast<uint4*>(&S.wbase[0][0]);
            constexpr int n4 = (int)(sizeof(S.wbase) / sizeof(uint4));
#pragma unroll
            for (int i = tid; i < n4; i += kSortThreads) c4[i] = make_uint4(0u, 0u, 0u, 0u);
            if (!by_match) {
                uint4* p4 = reinterpret_cast<uint4*>(&S.peer[0][0][0]);
                constexpr int np4 = (int)(sizeof(S.peer) / sizeof(uint4));
#pragma unroll
                for (int i = tid; i < np4; i += kSortThreads) p4[i] = make_uint4(0u, 0u, 0u, 0u);
            }
        }
        __syncthreads();
        const uint32_t part = S.part;
        if (part >= nparts) break;
        const uint32_t base = part * kSortPartition;
        const uint32_t mask = (1u << P.dbits) - 1u;
        const bool first = A.pass == 0, last = A.pass == P.passes - 1;
        auto digit = [&](uint64_t im) { return (uint32_t)((im >> shift) & mask); };

        // Load: warp w owns keys [base + 32 I w, base + 32 I (w+1)) (I items per
        // thread); round r reads 32 consecutive keys, so (warp, round, lane) order
        // is input order.
        uint64_t key[kSortItems];
        uint32_t val[kSortItems];
#pragma unroll
        for (int r = 0; r < kSortItems; ++r) {
            const uint32_t idx = base + warp * (kSortItems * 32) + r * 32 + lane;
            const bool ok = idx < K;
            key[r] = ok ? kin[idx] : 0ull;
            val[r] = ok ? vin[idx] : 0u;
        }
        if (first) {
#pragma unroll
            for (int r = 0; r < kSortItems; ++r) key[r] = plan_image(key[r], P);
        }
        // Rank within the warp, round by round: lanes with equal digits in a round
        // find each other (warp match, or each lane ORs its bit into its digit's
        // word and reads the word back); the lowest of them adds the group's size
        // to the warp's counter for that digit, and the counter's old value plus
        // the number of lower lanes in the group is each key's rank among the
        // warp's keys with that digit.  A __syncwarp separates one round's
        // counter updates from the next round's.  With atomicOr, round r uses
        // array r mod 3 and clears its words of round r-1 after the round's
        // __syncwarp (every lane has read them before it), so an array is clean
        // again, behind another __syncwarp, when round r+2 uses it.
        const uint32_t lt_mask = (1u << lane) - 1u;
        uint32_t rank[kSortItems];  // kNoDigit past the last key
        uint32_t dprev = kNoDigit;
#pragma unroll
        for (int r = 0; r < kSortItems; ++r) {
            const uint32_t idx = base + warp * (kSortItems * 32) + r * 32 + lane;
            const uint32_t d = idx < K ? digit(key[r]) : kNoDigit;
            uint32_t peers;
            if (by_match) {
                __syncwarp();
                peers = __match_any_sync(0xffffffffu, d);
            } else {
                if (d != kNoDigit) atomicOr(&S.peer[warp][r % 3][d], 1u << lane);
                __syncwarp();
                peers = d != kNoDigit ? S.peer[warp][r % 3][d] : 0u;
                if (dprev != kNoDigit) S.peer[warp][(r + 2) % 3][dprev] = 0u;
                dprev = d;
            }
            const uint32_t lt = __popc(peers & lt_mask);
            uint32_t before = 0u;
            if (d != kNoDigit && lt == 0) before = atomicAdd(&S.wbase[warp][d], (uint32_t)__popc(peers));
            const int leader = peers ? __ffs(peers) - 1 : lane;
            before = __shfl_sync(0xffffffffu, before, leader);
            rank[r] = d != kNoDigit ? before + lt : kNoDigit;
        }
        __syncthreads();
        // Per digit (threads 0..255, thread t <-> digit t): block total and
        // published aggregate.  The other threads feed zeros to the block scan.
        uint32_t tot = 0;
        if (digit_thread) {
#pragma unroll
            for (int w = 0; w < kSortThreads / 32; ++w) tot += S.wbase[w][t];
            if ((int64_t)part != A.withhold)
                st_relaxed_gpu(A.lookback + (size_t)part * 256 + t, (part == 0 ? kFlagPrefix : kFlagAgg) | tot);
            // clear this partition's row of the next pass's table (that table's last
            // user was the previous pass, which has completed)
            if (A.lookback_next) A.lookback_next[(size_t)part * 256 + t] = 0;
        }
        // one scan for both the block's digit offsets (low 16 bits, at most 4096)
        // and the digits' global starts (high bits)
        const unsigned long long packed =
            ((unsigned long long)hist_t << 16) | (unsigned long long)tot;
        const unsigned long long sc = block_excl_scan_u64(packed, S.warp_tmp);
        const uint32_t boff = (uint32_t)(sc & 0xffffull);
        const uint32_t dstart = (uint32_t)(sc >> 16);
        // Per digit: the staging slot of each warp's first key with the digit.
        // The counters are read in batches of 8 warps ahead of the stores: the
        // compiler cannot tell that the stores miss the words still to be read,
        // so a read after a store would wait for it.
        if (digit_thread) {
            constexpr int kBatch = 8;
            static_assert((kSortThreads / 32) % kBatch == 0, "warps come in batches of 8");
            uint32_t run = boff;
#pragma unroll
            for (int w0 = 0; w0 < kSortThreads / 32; w0 += kBatch) {
                uint32_t c[kBatch];
#pragma unroll
                for (int w = 0; w < kBatch; ++w) c[w] = S.wbase[w0 + w][t];
#pragma unroll
                for (int w = 0; w < kBatch; ++w) {
                    S.wbase[w0 + w][t] = run;
                    run += c[w];
                }
            }
        }
        __syncthreads();
        // Stage in digit order (positions are block-local, so this does not wait
        // for the look-back, and it frees the key registers before it).  All
        // positions are computed before the first store, so the reads overlap.
        uint32_t pos[kSortItems];
#pragma unroll
        for (int r = 0; r < kSortItems; ++r)
            pos[r] = rank[r] != kNoDigit ? S.wbase[warp][digit(key[r])] + rank[r] : kNoDigit;
#pragma unroll
        for (int r = 0; r < kSortItems; ++r) {
            if (pos[r] != kNoDigit) {
                S.st.keys[pos[r]] = key[r];
                S.st.vals[pos[r]] = val[r];
            }
        }
        if (digit_thread) {
            uint32_t prefix = 0;
            if (part > 0) {
                // Look back over the predecessors' published words, kLookWindow at
                // a time (all loads in flight together): add aggregates until an
                // inclusive prefix is found; on a word not yet published, poll it
                // again (bounded).
                int64_t j = (int64_t)part - 1;
                uint32_t spins = 0;
                bool found = false;
                while (!found && j >= 0) {
                    uint32_t w[kLookWindow];
#pragma unroll
                    for (int m = 0; m < kLookWindow; ++m)
                        w[m] = (j - m >= 0) ? ld_relaxed_gpu(A.lookback + (size_t)(j - m) * 256 + t) : kFlagPrefix;
                    int m = 0;  // words consumed from this window
#pragma unroll
                    for (int mm = 0; mm < kLookWindow; ++mm) {
                        const uint32_t flag = w[mm] & ~kCountMask;
                        if (flag == 0) break;  // not yet published: poll again from here
                        prefix += w[mm] & kCountMask;
                        ++m;
                        if (flag == kFlagPrefix) {
                            found = true;
                            break;
                        }
                    }
                    j -= m;
                    if (!found && m < kLookWindow && j >= 0) {
                        if (++spins > A.spin_limit) {
                            atomicOr(A.status + 2, GS_FLAG_TIMEOUT);
                            break;
                        }
                        __nanosleep(32);
                    }
                }
                if ((int64_t)part != A.withhold)
                    st_relaxed_gpu(A.lookback + (size_t)part * 256 + t, kFlagPrefix | (prefix + tot));
            }
            S.gbase[t] = dstart + prefix - boff;  // modular: gbase + staging index = output index
        }
        __syncthreads();
        const uint32_t nvalid = min((uint32_t)kSortPartition, K - base);
        auto put = [&](uint32_t i) {
            const uint64_t im = S.st.keys[i];
            const uint32_t o = S.gbase[digit(im)] + i;
            if (o < K) {  // always true unless a look-back wait timed out (flagged above)
                kout[o] = last ? plan_key(im, P) : im;
                vout[o] = S.st.vals[i];
            }
        };
        if (nvalid == (uint32_t)kSortPartition) {
#pragma unroll
            for (int u = 0; u < kSortItems; ++u) put(tid + (uint32_t)u * kSortThreads);
        } else {
            for (uint32_t i = tid; i < nvalid; i += kSortThreads) put(i);
        }
        __syncthreads();  // the next partition reuses the staging memory
    }
}

}  // namespace

int sort_tile_bits(int64_t tiles) {
    int b = 0;
    while ((int64_t(1) << b) < tiles) ++b;
    return b;
}


int64_t sort_partitions_for(int64_t kcap) { return (kcap + kSortPartition - 1) / kSortPartition; }

gs_status launch_sort(gs_context* ctx, const FrameView& v, int digit_override, bool fused) {
    // at most 8 bits per digit, or at most digit_override when it is 4..8;
    // launches for the longest plan (all 32 depth bits kept)
    const int tile_bits = sort_tile_bits((int64_t)v.gx * v.gy);
    const int dmax = sort_digit_max(digit_override);
    const int passes = sort_max_passes(tile_bits, dmax, fused);
    static bool attr_done[64] = {false};
    if (!attr_done[ctx->device & 63]) {
        if (cudaFuncSetAttribute(sort_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(PassSmem)) != cudaSuccess)
            return set_error(ctx, GS_ERR_CUDA, "sort: cannot raise dynamic shared memory to %d bytes",
                             (int)sizeof(PassSmem));
        attr_done[ctx->device & 63] = true;
    }
    // histograms and tickets start at zero (a fused chain's scan has cleared them)
    if (!fused) {
        (void)launch_pdl(ctx->stream, zero_words_kernel, dim3(zero_blocks(kSortCtlWords)), dim3(256), 0, v.sort_hist,
                         (int64_t)kSortCtlWords);
        ctx->launches += 1;
    }
    if (v.kcap == 0) return GS_OK;
    // persistent pass grid: two CTAs per SM at most, never more than the partitions
    const int64_t parts = std::min<int64_t>(sort_partitions_for(v.kcap), (int64_t)ctx->num_sms * 2);
    const size_t table = (size_t)v.sort_partitions * 256;
    uint32_t* method = v.sort_hist + kMaxPasses * 256 + kMaxPasses;
    HistArgs H{v.keys0, v.kcap, fused, v.status, v.sort_hist, v.sort_lookback, method, method + kMaxPasses,
               tile_bits, dmax};
    int hblocks = (int)std::min<int64_t>((v.kcap + 2047) / 2048, (int64_t)ctx->num_sms * 8);
    if (hblocks < 1) hblocks = 1;
    (void)launch_pdl(ctx->stream, sort_hist_kernel, dim3(hblocks), dim3(256), 0, H);
    ctx->launches += 1;
    for (int p = 0; p < passes; ++p) {
        PassArgs A;
        const bool even = (p % 2) == 0;
        A.keys = v.keys0;
        A.vals = v.vals0;
        A.kcap = v.kcap;
        A.fused = fused;
        A.status = v.status;
        A.hist = v.sort_hist + p * 256;
        A.lookback = v.sort_lookback + (even ? 0 : table);
        A.lookback_next = (p + 1 < passes) ? v.sort_lookback + (even ? table : 0) : nullptr;
        A.ticket = v.sort_hist + kMaxPasses * 256 + p;
        A.method = method + p;
        A.pass = p;
        A.tile_bits = tile_bits;
        A.dmax = dmax;
        A.spin_limit = ctx->sort_spin_limit;
        A.withhold = ctx->sort_withhold;
        (void)launch_pdl(ctx->stream, sort_pass_kernel, dim3((unsigned)parts), dim3(kSortThreads), sizeof(PassSmem), A);
        ctx->launches += 1;
    }
    return check_launch(ctx, "sort");
}

}  // namespace gs
