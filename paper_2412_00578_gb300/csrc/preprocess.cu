// preprocess (Sec. 3.2.1): one thread per Gaussian.
//
// Reads the planar parameter arrays with coalesced 4-byte loads (a warp reads
// 128 contiguous bytes of each plane), computes the 2D state and the tile
// count of the requested mode, and only for Gaussians that touch at least one
// tile reads the SH coefficients (192 of the 236 bytes of a Gaussian; they are
// prefetched into L2 early, one prefetch per line and warp, so the late loads
// do not wait on HBM) and writes the 48-byte 2D state.  Gaussians that are culled or off-screen cost
// their 44 bytes of geometry and opacity plus a 4-byte count.
#include "tiles.cuh"

namespace gs {
namespace {

struct PreArgs {
    const float* means;
    const float* scales;
    const float* rots;
    const float* opac;
    const float* sh;
    int64_t n;      // Gaussians in the scene
    int64_t ncap;   // counts written for [0, ncap)
    int sh_coeffs;  // (degree + 1)^2
    int mode;
    Grid grid;
    CamK cam;
    float4* p0;
    float4* p1;
    float4* p2;
    int32_t* counts;
    const CamRec* table;  // multi-view: per-camera constants (else nullptr)
    int num_cams;
    uint32_t* culled;     // count of non-finite / zero-quaternion Gaussians (nullable)
    uint2* warp_range;    // per warp: complement of the least, greatest depth bits
};

// Real SH normalisation constants, from their closed forms:
// 1/(2 sqrt(pi)), sqrt(3/(4pi)), sqrt(15/(4pi)), sqrt(5/(16pi)), sqrt(15/(16pi)),
// sqrt(35/(32pi)), sqrt(105/(4pi)), sqrt(21/(32pi)), sqrt(7/(16pi)), sqrt(105/(16pi)).
constexpr float kC0 = 0.28209479177387814f;
constexpr float kC1 = 0.4886025119029199f;
constexpr float kC2a = 1.0925484305920792f;
constexpr float kC2c = 0.31539156525252005f;
constexpr float kC2e = 0.5462742152960396f;
constexpr float kC3a = 0.5900435899266435f;
constexpr float kC3b = 2.890611442640554f;
constexpr float kC3c = 0.4570457994644658f;
constexpr float kC3d = 0.3731763325901154f;
constexpr float kC3f = 1.445305721320277f;

__device__ __forceinline__ void sh_basis16(float x, float y, float z, float Y[16]) {
    Y[0] = kC0;
    Y[1] = (-kC1) * y;
    Y[2] = kC1 * z;
    Y[3] = (-kC1) * x;
    const float xx = x * x, yy = y * y, zz = z * z;
    const float xy = x * y, yz = y * z, xz = x * z;
    Y[4] = kC2a * xy;
    Y[5] = (-kC2a) * yz;
    Y[6] = kC2c * ((2.0f * zz - xx) - yy);
    Y[7] = (-kC2a) * xz;
    Y[8] = kC2e * (xx - yy);
    Y[9] = ((-kC3a) * y) * (3.0f * xx - yy);
    Y[10] = (kC3b * xy) * z;
    Y[11] = ((-kC3c) * y) * ((4.0f * zz - xx) - yy);
    Y[12] = (kC3d * z) * ((2.0f * zz - 3.0f * xx) - 3.0f * yy);
    Y[13] = ((-kC3c) * x) * ((4.0f * zz - xx) - yy);
    Y[14] = (kC3f * z) * (xx - yy);
    Y[15] = ((-kC3a) * x) * (xx - 3.0f * yy);
}

// Gaussian i seen by camera C (grid g); writes slot o of the outputs.
// Returns the depth bits of a Gaussian given tiles, else 0 (a counted
// depth is above the near plane, so its bits are never 0).
template <int kMode>
__device__ __forceinline__ uint32_t preprocess_one(const PreArgs& A, const CamK& C, const Grid& grid, int64_t i,
                                                   int64_t o) {
    int count = 0;
    uint32_t depth_bits = 0u;
    if (i < A.n) {
        const int64_t n = A.n;
        const float mx = __ldg(A.means + i), my = __ldg(A.means + n + i), mz = __ldg(A.means + 2 * n + i);
        const float s0 = __ldg(A.scales + i), s1 = __ldg(A.scales + n + i), s2 = __ldg(A.scales + 2 * n + i);
        const float qw = __ldg(A.rots + i), qx = __ldg(A.rots + n + i), qy = __ldg(A.rots + 2 * n + i),
                    qz = __ldg(A.rots + 3 * n + i);
        const float sigma = __ldg(A.opac + i);
        bool ok = isfinite(mx) && isfinite(my) && isfinite(mz) && isfinite(s0) && isfinite(s1) && isfinite(s2) &&
                  isfinite(qw) && isfinite(qx) && isfinite(qy) && isfinite(qz) && isfinite(sigma);
        // view transform
        const float px = ((C.V[0] * mx + C.V[1] * my) + C.V[2] * mz) + C.V[3];
        const float py = ((C.V[4] * mx + C.V[5] * my) + C.V[6] * mz) + C.V[7];
        const float pz = ((C.V[8] * mx + C.V[9] * my) + C.V[10] * mz) + C.V[11];
        // Start moving the SH coefficients of Gaussians that may be seen into
        // L2 now: their loads come after the long geometry computation and
        // then hit L2.  A warp's 32 Gaussians share each coefficient plane's
        // 128-byte line(s), so its lanes split the prefetches of the first and
        // last Gaussian's address in every plane; a warp whose Gaussians all
        // lie behind the camera or far outside the view prefetches nothing.
        // (Performance only: every colour is still read from memory.)
        {
            const bool maybe = pz > C.near_z && fabsf(px) < (3.0f * C.limx) * pz && fabsf(py) < (3.0f * C.limy) * pz;
            const unsigned act = __activemask();
            const unsigned want = __ballot_sync(act, maybe);
            const int planes = 3 * A.sh_coeffs;
            if (act == 0xffffffffu) {
                if (want) {
                    const int lane = (int)(threadIdx.x & 31);
                    const int64_t first = i - lane;
                    const int64_t last = min(first + 31, n - 1);
                    for (int m = lane; m < 2 * planes; m += 32) {
                        const float* a = A.sh + (int64_t)(m >> 1) * n + ((m & 1) ? last : first);
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
                    }
                }
            } else if (maybe) {
                for (int k = 0; k < planes; ++k)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(A.sh + (int64_t)k * n + i));
            }
        }
        const float n2 = ((qw * qw + qx * qx) + qy * qy) + qz * qz;
        if (A.culled && !(ok && n2 > 0.0f)) atomicAdd(A.culled, 1u);  // rare: no aggregation
        ok = ok && (pz > C.near_z);
        ok = ok && (n2 > 0.0f);
        if (ok) {
            // quotients by one denominator are products with its reciprocal
            // (1/z, 1/|q|, 1/det, 1/|mu - campos|), as the oracle computes them
            const float iz = 1.0f / pz;
            const float xz = px * iz;
            const float yz = py * iz;
            const float u = C.fx * xz + C.cx;
            const float v = C.fy * yz + C.cy;
            // rotation from the normalised quaternion
            const float nq = sqrtf(n2);
            const float inq = 1.0f / nq;
            const float w = qw * inq, x = qx * inq, y = qy * inq, z = qz * inq;
            float R[9];
            R[0] = 1.0f - 2.0f * (y * y + z * z);
            R[1] = 2.0f * (x * y - w * z);
            R[2] = 2.0f * (x * z + w * y);
            R[3] = 2.0f * (x * y + w * z);
            R[4] = 1.0f - 2.0f * (x * x + z * z);
            R[5] = 2.0f * (y * z - w * x);
            R[6] = 2.0f * (x * z - w * y);
            R[7] = 2.0f * (y * z + w * x);
            R[8] = 1.0f - 2.0f * (x * x + y * y);
            // Sigma3D = (R S)(R S)^T
            float M[9];
            const float sc[3] = {s0, s1, s2};
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int k = 0; k < 3; ++k) M[3 * r + k] = R[3 * r + k] * sc[k];
            float S3[9];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    S3[3 * r + c] = (M[3 * r] * M[3 * c] + M[3 * r + 1] * M[3 * c + 1]) + M[3 * r + 2] * M[3 * c + 2];
            // Jacobian at the clamped mean
            const float tx = fminf(C.limx, fmaxf(-C.limx, xz)) * pz;
            const float ty = fminf(C.limy, fmaxf(-C.limy, yz)) * pz;
            const float iz2 = iz * iz;
            const float j00 = C.fx * iz;
            const float j02 = -((C.fx * tx) * iz2);
            const float j11 = C.fy * iz;
            const float j12 = -((C.fy * ty) * iz2);
            float T0[3], T1[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                T0[k] = j00 * C.V[k] + j02 * C.V[8 + k];
                T1[k] = j11 * C.V[4 + k] + j12 * C.V[8 + k];
            }
            float U0[3], U1[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                U0[c] = (T0[0] * S3[c] + T0[1] * S3[3 + c]) + T0[2] * S3[6 + c];
                U1[c] = (T1[0] * S3[c] + T1[1] * S3[3 + c]) + T1[2] * S3[6 + c];
            }
            const float c00 = (U0[0] * T0[0] + U0[1] * T0[1]) + U0[2] * T0[2];
            const float c01 = (U0[0] * T1[0] + U0[1] * T1[1]) + U0[2] * T1[2];
            const float c11 = (U1[0] * T1[0] + U1[1] * T1[1]) + U1[2] * T1[2];
            const float sxx = c00 + 0.3f;
            const float syy = c11 + 0.3f;
            const float sxy = c01;
            const float det = sxx * syy - sxy * sxy;
            if (det > 0.0f) {
                const float idet = 1.0f / det;
                const float a = syy * idet;
                const float b = (-sxy) * idet;
                const float c = sxx * idet;
                if (isfinite(u) && isfinite(v) && isfinite(a) && isfinite(b) && isfinite(c)) {
                    const float t = 2.0f * gs_logf(255.0f * sigma);
                    const float mid = 0.5f * (sxx + syy);
                    const float disc = fmaxf(0.1f, mid * mid - det);
                    const float l1 = mid + sqrtf(disc);
                    const float rad = ceilf(3.0f * sqrtf(l1));
                    const int radius = (rad >= 0.0f && rad < 1073741824.0f) ? (int)rad : (1 << 30);
                    const Ellipse E{u, v, a, b, c, t};
                    count = tile_count(kMode, E, radius, grid);  // kMode is a constant: one mode's code
                    if (count > 0) {
                        // SH colour, read only for Gaussians that touch a tile
                        const float d0 = mx - C.campos[0], d1 = my - C.campos[1], d2 = mz - C.campos[2];
                        const float len = sqrtf((d0 * d0 + d1 * d1) + d2 * d2);
                        const float ilen = 1.0f / len;
                        float Y[16];
                        sh_basis16(d0 * ilen, d1 * ilen, d2 * ilen, Y);
                        float rgb[3];
#pragma unroll
                        for (int ch = 0; ch < 3; ++ch) {
                            // issue all of the channel's coefficient loads before
                            // accumulating (same summation order as a plain loop)
                            float h[16];
#pragma unroll
                            for (int k = 0; k < 16; ++k)
                                h[k] = k < A.sh_coeffs ? __ldg(A.sh + (int64_t)(k * 3 + ch) * n + i) : 0.0f;
                            float acc = Y[0] * h[0];
#pragma unroll
                            for (int k = 1; k < 16; ++k)
                                if (k < A.sh_coeffs) acc = acc + Y[k] * h[k];
                            acc = acc + 0.5f;
                            rgb[ch] = acc < 0.0f ? 0.0f : acc;
                        }
                        A.p0[o] = make_float4(u, v, sigma, pz);
                        depth_bits = __float_as_uint(pz);
                        A.p1[o] = make_float4(a, b, c, t);
                        A.p2[o] = make_float4(rgb[0], rgb[1], rgb[2], __int_as_float(radius));
                    }
                }
            }
        }
    }
    A.counts[o] = count;
    return depth_bits;
}

// Least and greatest depth bits of the warp's Gaussians with tiles, stored
// (as the complement of the least, and the greatest) in the warp's slot; the
// scan reduces the slots and the sort keeps only the bits they span.
__device__ __forceinline__ void record_depth_range(uint2* out, uint32_t db) {
    const uint32_t lo_n = __reduce_max_sync(0xffffffffu, db ? ~db : 0u);
    const uint32_t hi = __reduce_max_sync(0xffffffffu, db);
    if ((threadIdx.x & 31) == 0 && out)
        out[(int64_t)blockIdx.x * (kPreThreads / 32) + (threadIdx.x >> 5)] = make_uint2(lo_n, hi);
}

// One instantiation per tile mode, so each kernel holds only its mode's tile count.
template <int kMode>
__global__ void __launch_bounds__(kPreThreads, 4) preprocess_kernel(const PreArgs A) {
    pdl_begin();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t db = i < A.ncap ? preprocess_one<kMode>(A, A.cam, A.grid, i, i) : 0u;
    record_depth_range(A.warp_range, db);
}

// Multi-view: block b handles Gaussian chunk b / V for camera b % V, so the
// cameras of one chunk run back to back and re-read its parameters from L2.
template <int kMode>
__global__ void __launch_bounds__(kPreThreads, 4) preprocess_multiview_kernel(const PreArgs A) {
    const int cam = (int)(blockIdx.x % (unsigned)A.num_cams);
    const int64_t i = (int64_t)(blockIdx.x / (unsigned)A.num_cams) * blockDim.x + threadIdx.x;
    uint32_t db = 0u;
    if (i < A.ncap) {
        const CamRec& R = A.table[cam];
        const Grid g{A.grid.T, R.gx, R.gy, R.width, R.height};
        db = preprocess_one<kMode>(A, R.k, g, i, (int64_t)cam * A.ncap + i);
    }
    record_depth_range(A.warp_range, db);
}

}  // namespace

gs_status launch_preprocess(gs_context* ctx, const gs_scene* s, const gs_camera* cam, const gs_raster_cfg* cfg,
                            const FrameView& v) {
    PreArgs A;
    A.means = s->means;
    A.scales = s->scales;
    A.rots = s->rotations;
    A.opac = s->opacities;
    A.sh = s->sh;
    A.n = s->n;
    A.ncap = v.ncap;
    A.sh_coeffs = (s->sh_degree + 1) * (s->sh_degree + 1);
    A.mode = cfg->mode;
    A.grid = Grid{(float)v.tile, v.gx, v.gy, v.width, v.height};
    if (cam) {  // single camera: constants travel as kernel parameters
        A.cam.fx = cam->fx;
        A.cam.fy = cam->fy;
        A.cam.cx = cam->cx;
        A.cam.cy = cam->cy;
        A.cam.limx = 1.3f * cam->tan_fovx;
        A.cam.limy = 1.3f * cam->tan_fovy;
        A.cam.near_z = cam->near_z;
        for (int k = 0; k < 12; ++k) A.cam.V[k] = cam->viewmat[k];
        for (int k = 0; k < 3; ++k) A.cam.campos[k] = cam->campos[k];
    }
    A.p0 = v.p0;
    A.p1 = v.p1;
    A.p2 = v.p2;
    A.counts = v.counts;
    A.table = v.table;
    A.num_cams = v.num_cams;
    A.culled = v.table ? nullptr : v.status + kStatusCulledAcc;
    A.warp_range = v.warp_range;
    const int threads = kPreThreads;
    if (v.table) {
        A.ncap = v.cam_stride;
        if (A.ncap == 0 || v.num_cams == 0) return GS_OK;
        const int64_t blocks = (A.ncap + threads - 1) / threads * v.num_cams;
        switch (cfg->mode) {
            case GS_MODE_3SIGMA: preprocess_multiview_kernel<GS_MODE_3SIGMA><<<(unsigned)blocks, threads, 0, ctx->stream>>>(A); break;
            case GS_MODE_SNUGBOX: preprocess_multiview_kernel<GS_MODE_SNUGBOX><<<(unsigned)blocks, threads, 0, ctx->stream>>>(A); break;
            case GS_MODE_TBC: preprocess_multiview_kernel<GS_MODE_TBC><<<(unsigned)blocks, threads, 0, ctx->stream>>>(A); break;
            case GS_MODE_PIXEL: preprocess_multiview_kernel<GS_MODE_PIXEL><<<(unsigned)blocks, threads, 0, ctx->stream>>>(A); break;
            default: preprocess_multiview_kernel<GS_MODE_ACCUTILE><<<(unsigned)blocks, threads, 0, ctx->stream>>>(A); break;
        }
        ctx->launches += 1;
        return check_launch(ctx, "preprocess_multiview");
    }
    if (v.ncap == 0) return GS_OK;
    const int64_t blocks = (v.ncap + threads - 1) / threads;
#define GS_PRE(M_) (void)launch_pdl(ctx->stream, preprocess_kernel<M_>, dim3((unsigned)blocks), dim3(threads), 0, A)
    switch (cfg->mode) {
        case GS_MODE_3SIGMA: GS_PRE(GS_MODE_3SIGMA); break;
        case GS_MODE_SNUGBOX: GS_PRE(GS_MODE_SNUGBOX); break;
        case GS_MODE_TBC: GS_PRE(GS_MODE_TBC); break;
        case GS_MODE_PIXEL: GS_PRE(GS_MODE_PIXEL); break;
        default: GS_PRE(GS_MODE_ACCUTILE); break;
    }
#undef GS_PRE
    ctx->launches += 1;
    return check_launch(ctx, "preprocess");
}

}  // namespace gs
