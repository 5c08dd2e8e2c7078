/*
 * gs.h — C ABI of the GB300 (sm_103a) 3D Gaussian Splatting tile rasterizer
 * with Speedy-Splat Gaussian-to-tile localization.
 *
 * The pipeline follows the six functions of the 3D-GS forward renderer
 * (Sec. 3.2 and Table 1 of Speedy-Splat, arXiv 2412.00578):
 *   gs_preprocess   per-Gaussian projection, colour and tile count  (Sec. 3.2.1)
 *   gs_intersect    InclusiveSum + duplicateWithKeys                 (Sec. 3.2.2)
 *   gs_sort         RadixSort of the (tile | depth) keys             (Sec. 3.2.2)
 *   gs_tile_ranges  identifyTileRanges                               (Sec. 3.2.2)
 *   gs_render       front-to-back alpha blending per pixel           (Sec. 3.2.3)
 * with the tile-localization mode chosen per call: the 3D-GS 3-sigma square
 * (Eq. radius), SnugBox (Sec. 4.1.1) or AccuTile (Sec. 4.1.2, Algorithm 1).
 *
 * Conventions for every entry point:
 *   - All array arguments are DEVICE pointers owned by the caller, except
 *     where a comment says "host".  The library never allocates device memory;
 *     gs_frame_sizes() tells the caller what to allocate.
 *   - Every call is asynchronous on the context's CUDA stream, except the ones
 *     documented as synchronising (gs_intersect with a non-NULL num_keys,
 *     gs_read_status).
 *   - Errors are returned as gs_status; gs_last_error() gives a message.  No
 *     call aborts, throws or traps.  Errors detected on the device (key
 *     capacity exceeded, a bounded wait that ran out) are recorded in the
 *     frame's status words and reported by gs_read_status().
 *   - One context per host thread.
 */
#ifndef GS_H_
#define GS_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gs_status {
    GS_OK = 0,
    GS_ERR_INVALID = 1,   /* bad argument (null pointer, size, mode, tile)        */
    GS_ERR_OOM = 2,       /* reserved: the library does not allocate device memory */
    GS_ERR_CAPACITY = 3,  /* more keys than gs_frame.key_capacity                 */
    GS_ERR_CUDA = 4,      /* a CUDA runtime call failed                            */
    GS_ERR_TIMEOUT = 5    /* a bounded device-side wait gave up                    */
} gs_status;

typedef enum gs_mode {
    GS_MODE_3SIGMA = 0,   /* 3D-GS square of radius ceil(3 sqrt(lambda_max)), Eq. radius */
    GS_MODE_SNUGBOX = 1,  /* tight box of the opacity-aware ellipse, Sec. 4.1.1       */
    GS_MODE_ACCUTILE = 2, /* exact tiles of that ellipse, Sec. 4.1.2, Algorithm 1     */
    GS_MODE_TBC = 3,      /* tile-based culling, the StopThePop ablation of App. A.4:
                             SnugBox tiles kept iff min of q over the tile <= t      */
    GS_MODE_PIXEL = 4     /* pixel-exact: tiles holding an image pixel with q <= t
                             (the blend's own test), so tile set = pixel set        */
} gs_mode;

/* Device status word flags (gs_read_status). */
#define GS_FLAG_CAPACITY 1u   /* keys did not fit: nothing was emitted            */
#define GS_FLAG_TIMEOUT  2u   /* a sort look-back wait exceeded its bound         */
#define GS_FLAG_BATCH    4u   /* batch cameras exceed the frame's tile or pixel capacity */
#define GS_FLAG_KEYRANGE 8u   /* gs_sort met a key outside the range gs_intersect recorded */

/* Gaussian parameter set G_i = {mu, s, r, h, sigma} (Sec. 3.1), planar
 * structure of arrays, float32, device memory, read only.
 *   means     [3][n]       x plane, y plane, z plane
 *   scales    [3][n]       activated (exp applied)
 *   rotations [4][n]       quaternion w, x, y, z (normalised by the kernel)
 *   opacities [n]          activated (sigmoid applied)
 *   sh        [16][3][n]   coefficient k, channel c at sh[(k*3 + c)*n + i];
 *                          only the first (sh_degree+1)^2 coefficients are read */
typedef struct gs_scene {
    int64_t n;
    int32_t sh_degree;  /* 0..3 */
    const float* means;
    const float* scales;
    const float* rotations;
    const float* opacities;
    const float* sh;
} gs_scene;

/* Pinhole camera (host struct, passed by pointer, copied by value).  OpenCV
 * axes: x right, y down, z forward.  Pixel (i, j) sits at the point (i, j).
 * viewmat is the row-major 3x4 world-to-camera transform [R | t]; campos
 * the camera centre in world coordinates (for the SH view direction).
 * Gaussians with view depth <= near_z are culled. */
typedef struct gs_camera {
    int32_t width, height;
    float fx, fy, cx, cy;
    float tan_fovx, tan_fovy;
    float near_z;
    float viewmat[12];
    float campos[3];
} gs_camera;

/* Raster configuration: tile edge (8, 16 or 32 pixels), gs_mode, background,
 * and the radix sort's digit width (0 = automatic: at most 8 bits per pass;
 * 4..8 = at most that many bits per pass; the pass count then follows on the
 * device from the frame's depth range, see gs_sort).  The digit width changes
 * speed only, never the sorted result. */
typedef struct gs_raster_cfg {
    int32_t tile;
    int32_t mode;
    float bg[3];
    int32_t sort_digit_bits;
} gs_raster_cfg;

/* Per-frame buffers, all device memory owned by the caller, sized by
 * gs_frame_sizes() for (n_capacity, width, height, tile, key_capacity);
 * zero-fill scratch once after allocating it (see gs_read_culled).
 * Layouts:
 *   proj     [3][n_capacity][4] float: plane 0 = (u, v, opacity, depth),
 *            plane 1 = conic (a, b, c) and t = 2 log(255 sigma),
 *            plane 2 = (r, g, b, radius as int32 bits).  Written only for
 *            Gaussians with a non-zero tile count.
 *   counts   [n_capacity] int32: tiles touched in the preprocessed mode.
 *   keys     [2][key_capacity] uint64: (tile id << 32) | float bits of depth.
 *   vals     [2][key_capacity] uint32: Gaussian index.
 *            After gs_sort the sorted pairs are in keys[0..K), vals[0..K).
 *   ranges   [tiles][2] uint32: [start, end) of each tile in the sorted list.
 *   image    [3][height][width] float, final_T [height][width] float,
 *   last     [height][width] uint32: 1-based position, in its tile's list, of
 *            the last Gaussian that contributed to the pixel (0: none).
 *   scratch  library working memory (status words, scan partials, sort
 *            histograms and look-back tables, the render's tile launch
 *            order); contents are private. */
typedef struct gs_frame {
    int64_t n_capacity;
    int64_t key_capacity;   /* <= GS_MAX_KEYS */
    int32_t width, height, tile;
    float* proj;
    int32_t* counts;
    uint64_t* keys;
    uint32_t* vals;
    uint32_t* ranges;
    float* image;
    float* final_T;
    uint32_t* last;
    void* scratch;
} gs_frame;

#define GS_MAX_KEYS ((int64_t)((1u << 30) - 1))

/* Byte sizes of the gs_frame buffers (host output). */
typedef struct gs_frame_bytes {
    int64_t proj, counts, keys, vals, ranges, image, final_T, last, scratch;
} gs_frame_bytes;

typedef struct gs_context gs_context;

/* Create a context bound to CUDA device `device` and stream `cuda_stream`
 * (a cudaStream_t; NULL = legacy default stream).  *out receives the
 * context; free it with gs_destroy.  Allocates host memory only. */
gs_status gs_create(int device, void* cuda_stream, gs_context** out);
void gs_destroy(gs_context* ctx);
gs_status gs_set_stream(gs_context* ctx, void* cuda_stream);
/* Message of the last error on this context (never NULL). */
const char* gs_last_error(const gs_context* ctx);
/* Number of kernels this context has launched so far. */
int64_t gs_launch_count(const gs_context* ctx);

/* Sizes of the per-frame buffers.  Returns GS_ERR_INVALID for tile not in
 * {8,16,32}, non-positive sizes, or key_capacity > GS_MAX_KEYS. */
gs_status gs_frame_sizes(int64_t n_capacity, int32_t width, int32_t height, int32_t tile, int64_t key_capacity,
                         gs_frame_bytes* out);

/* Preprocess (Sec. 3.2.1): for each Gaussian, view transform and near cull,
 * projected mean and depth, Sigma3D = R S S^T R^T, Sigma2D = J W Sigma3D W^T J^T
 * (+0.3 I), its inverse (the conic), t = 2 log(255 sigma) (Sec. 4.1), the 3D-GS
 * radius, the SH colour, and the number of tiles touched in cfg->mode.
 * Writes frame->proj (for counted Gaussians) and frame->counts[0..n), and in
 * frame->scratch the depth-bit range of the Gaussians given tiles, which
 * gs_intersect records for the sort (see gs_sort). */
gs_status gs_preprocess(gs_context* ctx, const gs_scene* scene, const gs_camera* cam, const gs_raster_cfg* cfg,
                        const gs_frame* frame);

/* InclusiveSum of the counts and duplicateWithKeys (Sec. 3.2.2): recomputes
 * each Gaussian's tiles in cfg->mode (which must be the mode the counts were
 * made with) and writes one (key, value) pair per (Gaussian, tile) into
 * keys[0]/vals[0], Gaussians in index order.  The key total K is kept on the
 * device.  If K > key_capacity nothing is emitted and GS_FLAG_CAPACITY is set.
 * num_keys: NULL for a fully asynchronous call; otherwise the call
 * synchronises the stream, stores K (host) and returns GS_ERR_CAPACITY if
 * K exceeds the capacity. */
gs_status gs_intersect(gs_context* ctx, const gs_camera* cam, const gs_raster_cfg* cfg, const gs_frame* frame,
                       int64_t* num_keys);

/* RadixSort (Sec. 3.2.2): stable LSD radix sort of the K pairs by key, in
 * onesweep passes, result in keys[0]/vals[0].  Uses frame->scratch and
 * keys[1]/vals[1].  The passes cover ceil(log2(tiles)) tile bits plus only
 * as many depth bits as the frame's depths span: gs_preprocess records the
 * least and greatest depth bits of the Gaussians it gave tiles, and the sort
 * orders each key by (tile, depth bits - least), an order-preserving map of
 * the K keys, so the result is the sort by the full key.  The pass count is
 * therefore chosen on the device (the launches beyond it return at once);
 * here it is even, so that passes alternating between the two buffers end in
 * keys[0] (gs_forward, which also runs the emit, allows an odd count by
 * having the emit write keys[1]).  The keys sorted must be the ones
 * gs_intersect emitted after the frame's gs_preprocess: a key outside the
 * recorded range sets GS_FLAG_KEYRANGE, the later stages see no keys, and
 * gs_read_status returns GS_ERR_INVALID. */
gs_status gs_sort(gs_context* ctx, const gs_camera* cam, const gs_raster_cfg* cfg, const gs_frame* frame);

/* identifyTileRanges (Sec. 3.2.2): ranges[tile] = [start, end) of the tile's
 * entries in the sorted keys; [0, 0) for empty tiles.  Also records, in
 * frame->scratch, the order in which gs_render launches the tiles (heaviest
 * first; frames of up to 32768 tiles). */
gs_status gs_tile_ranges(gs_context* ctx, const gs_camera* cam, const gs_raster_cfg* cfg, const gs_frame* frame);

/* render (Sec. 3.2.3, Eqs. render_alpha, 2d_gaussian_scalar, contribution):
 * for each pixel, walk its tile's Gaussians front to back; a Gaussian counts
 * where q <= t (alpha >= 1/255), alpha = min(0.99, sigma exp(-q/2)); stop
 * before a Gaussian that would bring the transmittance below 1e-4; finally
 * add T * bg.  Writes image, final_T and last.  Tiles are processed in the
 * order the frame's last gs_tile_ranges recorded (heaviest first); the order
 * does not change any output.  Requires gs_tile_ranges on the sorted keys. */
gs_status gs_render(gs_context* ctx, const gs_camera* cam, const gs_raster_cfg* cfg, const gs_frame* frame);

/* Instrumented render: the same blend as gs_render (same outputs), which
 * also counts, over all pixels: *evaluated = the (pixel, Gaussian) pairs the
 * tile-list definition evaluates (each entry of the pixel's tile list up to
 * and including the one that stops the pixel), *contributed = the pairs that
 * add to the colour, *executed = the pairs whose in-ellipse test the kernel
 * actually evaluated after its in-tile culling (a pixel that stops part-way
 * through a 256-entry batch has the rest of that batch tested too).
 * Synchronises the stream; host outputs, nullable.  States the blend's
 * algorithmic work; not for timing. */
gs_status gs_render_stats(gs_context* ctx, const gs_camera* cam, const gs_raster_cfg* cfg, const gs_frame* frame,
                          uint64_t* evaluated, uint64_t* contributed, uint64_t* executed);

/* The five stages above in one call, with no host synchronisation.  The
 * results equal the stage-by-stage calls'; the one difference is where the
 * emitted pairs wait for the sort: when the sort plan has an odd number of
 * passes the emit writes keys[1]/vals[1], so the sort needs no extra pass
 * to end in keys[0]/vals[0]. */
gs_status gs_forward(gs_context* ctx, const gs_scene* scene, const gs_camera* cam, const gs_raster_cfg* cfg,
                     const gs_frame* frame);

/* Gradients of the render (device, caller-owned), planar like gs_scene:
 *   means [3][n], scales [3][n], rotations [4][n], opacities [n], sh [16][3][n]
 *   (overwritten), means2d [2][n] (nullable, overwritten): dL/d(u, v), the
 *   view-space gradient used by densification heuristics,
 *   score [n] (nullable): the efficient pruning score of Sec. 4.2.1,
 *   sum over pixels and channels of (dC/dg_i)^2, is ADDED to it so views can
 *   be accumulated,
 *   work: library scratch of gs_backward_work_bytes(n_capacity) bytes,
 *   16-byte aligned (GS_ERR_INVALID otherwise). */
typedef struct gs_grads {
    float* means;
    float* scales;
    float* rotations;
    float* opacities;
    float* sh;
    float* means2d;
    float* score;
    float* work;
} gs_grads;

/* Bytes of gs_grads.work for a frame of n_capacity Gaussians. */
int64_t gs_backward_work_bytes(int64_t n_capacity);

/* Render backward (Sec. 4.2, 4.2.1): given dL/dimage ([3][height][width],
 * device) for the image the frame holds (a completed gs_forward of this
 * scene, camera and cfg), write dL/d(means, scales, rotations, opacities,
 * sh), optionally dL/d(u, v), and add the pruning score.  Per pixel, the
 * tile list is walked back to front from its last contributor; threshold,
 * 0.99 clamp and stop decisions are those of the forward.  Accumulation uses
 * atomics, so results are reproducible to rounding, not bit for bit. */
gs_status gs_render_backward(gs_context* ctx, const gs_scene* scene, const gs_camera* cam, const gs_raster_cfg* cfg,
                             const gs_frame* frame, const float* dL_dimage, const gs_grads* grads);

/* PUP sensitivity (the pruning score the paper builds on, Sec. 4.2, Eq.
 * pup_score): U_i = log det H_i with
 *   H_i = sum over views, pixels p and channels of
 *         grad_{mu_i, s_i} C(p) grad_{mu_i, s_i} C(p)^T,
 * the 6 x 6 block of the Gauss-Newton Hessian of the image with respect to
 * the mean and the (activated) scale of Gaussian i, taken through its 2D
 * value g_i(p) (the colour's view dependence is held fixed).  Memory: 21
 * floats per Gaussian for H (the symmetric 6 x 6), against one for the
 * efficient score of gs_render_backward.
 * gs_pup_accumulate adds one view's terms to hessian ([21][n] device floats,
 * row-major upper triangle in the order mu_x mu_y mu_z s_0 s_1 s_2) for the
 * frame's completed forward render of this scene, camera and cfg; work is
 * gs_pup_work_bytes(n_capacity) bytes of device scratch, 16-byte aligned.
 * gs_pup_score writes U_i to score[n] (-inf where H_i is not positive
 * definite, e.g. a Gaussian seen from a single view: rank <= 5). */
int64_t gs_pup_work_bytes(int64_t n_capacity);
gs_status gs_pup_accumulate(gs_context* ctx, const gs_scene* scene, const gs_camera* cam, const gs_raster_cfg* cfg,
                            const gs_frame* frame, float* hessian, float* work);
gs_status gs_pup_score(gs_context* ctx, const float* hessian, int64_t n, float* score);

/* gs_intersect for callers that cannot allocate device memory (a plug-in
 * whose host application owns all GPU allocations, a real-time loop that must
 * not stall on an allocation, a program that forbids allocation after
 * start-up).  The paper has no counterpart: this is a deployment variant of
 * gs_intersect.  It does the same work and writes the same keys[0]/vals[0],
 * but keeps its working memory (running sums of the counts and status words)
 * in a fixed array built into the library instead of frame->scratch, which
 * may be NULL and is never touched.  Of the frame's buffers only proj,
 * counts, keys and vals are used and must be non-NULL; ranges, image,
 * final_T and last may be NULL.
 *   - Limit: frame->n_capacity <= 16,777,216 (GS_ERR_INVALID beyond, with a
 *     message); the array takes about 131 KB on every device that loads the
 *     library, until the process exits.
 *   - num_keys (host) is required: the call synchronises the stream and
 *     returns K there (GS_ERR_CAPACITY if K > key_capacity, nothing emitted).
 *     The frame's own status words are not written, so the later stages
 *     (gs_sort ...) need gs_intersect.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress).
 *   - Allocates nothing; all calls on a device share the array and it keeps
 *     the last call's contents (the call clears what must start at zero), so
 *     calls whose GPU work overlaps (other streams or host threads) race. */
gs_status gs_intersect_noalloc(gs_context* ctx, const gs_camera* cam, const gs_raster_cfg* cfg, const gs_frame* frame,
                               int64_t* num_keys);

/* ---------------------------------------------------------------- multi-view
 * Many cameras of one scene in one batch: each stage is one launch over all
 * cameras.  Tiles of all cameras share one global index space (camera c's
 * tiles start at the sum of the earlier cameras' tile counts), so the keys of
 * every camera go through one sort, one range pass and one blend launch.
 * Grid sizes come from the frame's capacities and the per-camera layout is
 * built on the device from a device array of cameras, so a captured CUDA
 * graph of gs_forward_batch replays for new camera poses (same or smaller
 * total tiles and pixels) after the caller rewrites that array.
 * Buffers (device, caller-owned), for capacities n_capacity (Gaussian slots
 * per camera), max_cams, tile_capacity (>= total tiles of one call),
 * pixel_capacity (>= total pixels of one call), key_capacity:
 *   proj [3][max_cams * n_capacity][4], counts [max_cams * n_capacity],
 *   keys [2][key_capacity], vals [2][key_capacity] (value = index in the scene),
 *   ranges [tile_capacity][2],
 *   image [3 * pixel_capacity]: camera c's [3][H_c][W_c] image starts at
 *   3 * P_c where P_c = sum of W*H over cameras before c; final_T and last
 *   [pixel_capacity]: camera c's [H_c][W_c] plane starts at P_c. */
#define GS_MAX_BATCH_CAMS 1024

typedef struct gs_batch_frame {
    int64_t n_capacity;
    int64_t key_capacity;
    int64_t tile_capacity;
    int64_t pixel_capacity;
    int32_t max_cams;
    int32_t tile;
    float* proj;
    int32_t* counts;
    uint64_t* keys;
    uint32_t* vals;
    uint32_t* ranges;
    float* image;
    float* final_T;
    uint32_t* last;
    void* scratch;
} gs_batch_frame;

/* Byte sizes of the gs_batch_frame buffers (fields as in gs_frame_bytes). */
gs_status gs_batch_sizes(int64_t n_capacity, int32_t max_cams, int32_t tile, int64_t tile_capacity,
                         int64_t pixel_capacity, int64_t key_capacity, gs_frame_bytes* out);

/* The forward of Sec. 3.2 for num_cams cameras of one scene (cams: DEVICE
 * array of num_cams gs_camera structs, read when the work runs).  Same
 * per-camera results as gs_forward on each camera (same keys in the camera's
 * tiles, same images, bit for bit).  No host synchronisation.  If the cameras
 * exceed tile_capacity or pixel_capacity nothing is rendered and
 * GS_FLAG_BATCH is set; if the keys exceed key_capacity, GS_FLAG_CAPACITY. */
gs_status gs_forward_batch(gs_context* ctx, const gs_scene* scene, const gs_camera* cams, int32_t num_cams,
                           const gs_raster_cfg* cfg, const gs_batch_frame* frame);

/* Synchronise and read a batch frame's key total and GS_FLAG_* bits
 * (host outputs, nullable); returns GS_ERR_CAPACITY / GS_ERR_TIMEOUT /
 * GS_ERR_INVALID (for GS_FLAG_BATCH) when a flag is set. */
gs_status gs_batch_status(gs_context* ctx, const gs_batch_frame* frame, int64_t* num_keys, uint32_t* flags);

/* Synchronise the stream and read the frame's device status: the key total
 * K and the GS_FLAG_* bits (both host outputs, nullable).  Returns
 * GS_ERR_CAPACITY or GS_ERR_TIMEOUT if the corresponding flag is set.
 * After GS_FLAG_TIMEOUT the frame holds no keys for the later sort passes,
 * gs_tile_ranges and gs_render (the image is the background); the context
 * stays usable and the next frame starts afresh. */
gs_status gs_read_status(gs_context* ctx, const gs_frame* frame, int64_t* num_keys, uint32_t* flags);

/* Synchronise and read how many Gaussians the frame's last gs_preprocess
 * culled because a parameter was NaN or infinite or the quaternion was zero
 * (*culled, host).  The count is taken over by gs_intersect, so read it after
 * that call.  Its first value after the scratch buffer was allocated is
 * valid only if the buffer was zero-filled once (the library keeps the word
 * consistent afterwards). */
gs_status gs_read_culled(gs_context* ctx, const gs_frame* frame, int64_t* culled);

/* The sort plan for the keys gs_intersect last emitted into the frame, with
 * cfg's sort_digit_bits: the number of onesweep passes gs_forward runs (a
 * stand-alone gs_sort runs the next even number), the bits per digit at that
 * count, and how many depth bits the keys keep (their depths' span; 32 when
 * nothing was recorded).  All three outputs are host pointers and nullable.
 * Synchronises the stream. */
gs_status gs_read_sort_plan(gs_context* ctx, const gs_raster_cfg* cfg, const gs_frame* frame, int32_t* passes,
                            int32_t* digit_bits, int32_t* depth_bits);

/* The same plan as a pure host function of its inputs (no context, no
 * device): a frame of `tiles` tiles whose keys' depth bits lie in
 * [least, greatest] (least > greatest: no range recorded, all 32 depth bits
 * kept), at most `sort_digit_bits` bits per digit (0 = 8), for gs_forward
 * (fused != 0) or a stand-alone gs_sort (even pass count).  Outputs (host,
 * nullable): the pass count, bits per digit, depth bits kept, and the buffer
 * (0 or 1) the emit writes and the first pass reads.  GS_ERR_INVALID for
 * tiles < 1 or a digit width outside {0, 4..8}. */
gs_status gs_sort_plan_for(int64_t tiles, uint32_t least, uint32_t greatest, int32_t sort_digit_bits, int32_t fused,
                           int32_t* passes, int32_t* digit_bits, int32_t* depth_bits, int32_t* start_buffer);

/* Failure detection of the sort's bounded waits.  Each decoupled look-back
 * wait of gs_sort gives up after max_polls polls (0 = the default, 4,194,304,
 * far beyond any wait of a correct run) and then sets GS_FLAG_TIMEOUT.  If
 * withhold_partition >= 0, that key partition (4096 keys) of every sort pass
 * never publishes its digit counts, so the wait of the partition after it
 * must run out: a test uses this, with a small max_polls, to exercise the
 * timeout path without any fault.  -1 restores normal publishing.  Applies
 * to later gs_sort / gs_forward / gs_forward_batch calls on this context. */
gs_status gs_set_sort_wait(gs_context* ctx, uint32_t max_polls, int64_t withhold_partition);

#ifdef __cplusplus
}
#endif

#endif /* GS_H_ */
