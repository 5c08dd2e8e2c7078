// Render backward (Sec. 4.2) and the efficient pruning score (Sec. 4.2.1).
//
// blend_backward: one CTA per tile, one thread per pixel (warp = 8 x 4
// sub-tile, as in the forward).  Each pixel walks its tile list backwards
// from its last contributor, recomputing q and alpha with the forward's
// exact float operations (so every inclusion decision is the forward's), and
// recovering the transmittance in front of each contributor as
// T_i = T_{i+1} / (1 - alpha_i), starting from the stored final T.  With B
// the colour behind the current Gaussian seen through it (B = bg after the
// last contributor, B <- alpha c + (1 - alpha) B moving forward):
//   dL/dc = G alpha T,  dL/dalpha = sum_ch G_ch T (c_ch - B_ch),
//   unclamped alpha = sigma g: dL/dsigma = dL/dalpha g,
//   dL/dq = -dL/dalpha sigma g / 2, q = a dx^2 + 2 b dx dy + c dy^2,
//   score += sum_ch (sigma T (c_ch - B_ch))^2   (dC/dg squared).
// The warp sums its lanes' ten values per Gaussian (halving shuffle
// exchanges) and adds them with three vector atomics into the Gaussian's
// 12-float row of the work array.
//
// preprocess_backward: one thread per Gaussian, carries the 2D sums to
// mu, s, q, h, sigma through the conic inverse, Sigma2D = J W Sigma3D W^T J^T
// (with the x/z, y/z clamp), Sigma3D = R S S^T R^T, the quaternion
// normalisation and the SH colour (including the view-direction term).
#include "blend_common.cuh"

namespace gs {
namespace {

constexpr int kWork = 10;     // du dv da db dc dsigma dr dg db score
constexpr int kWorkRow = 12;  // floats per Gaussian row of the work array (three 16-byte groups)

struct BwdArgs {
    const uint2* ranges;
    const uint32_t* vals;
    const float4* p0;
    const float4* p1;
    const float4* p2;
    const float* final_T;
    const uint32_t* last;
    const float* dL_dimg;  // [3][H][W]
    float* work;           // [ncap][kWorkRow], row = the kWork values and 2 pad
    int64_t ncap;
    int width, height, gx;
    float bg0, bg1, bg2;
};

// kPup: instead of the gradients, accumulate the PUP sensitivity terms of
// Sec. 4.2 (Eq. pup_score): per Gaussian, the 15 entries of the symmetric
// 5x5 matrix sum_p w_p G5 G5^T, where G5 = dg/d(u, v, a, b, c) at the pixel
// and w_p = sum_ch (dC_ch/dg)^2 (zero where alpha is clamped), into a
// 16-float row.
template <int T, bool kPup>
__global__ void __launch_bounds__(T* T, T == 32 ? 1 : (T == 16 ? 4 : 12)) blend_backward_kernel(const BwdArgs A) {
    constexpr int kNV = kPup ? 15 : kWork;       // values per (pixel, Gaussian) pair
    constexpr int kRow = kPup ? 16 : kWorkRow;   // floats per Gaussian row
    constexpr int NT = T * T;
    constexpr int NB = NT < 256 ? NT : 256;
    constexpr int NSX = T / kSubW;
    __shared__ float4 s_g0[NB];  // u, v, a, 2b
    __shared__ float4 s_g1[NB];  // c, t, opacity, b
    __shared__ float4 s_g2[NB];  // r, g, b, -
    __shared__ uint32_t s_mask[NB];
    __shared__ uint32_t s_id[NB];
    __shared__ int s_maxlast;
    const int tile = blockIdx.x;
    const int tx = tile % A.gx, ty = tile / A.gx;
    const int warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
    const uint32_t my_bit = 1u << warp;
    const int px = tx * T + (warp % NSX) * kSubW + (lane & (kSubW - 1));
    const int py = ty * T + (warp / NSX) * kSubH + (lane >> 3);
    const bool inside = px < A.width && py < A.height;
    const float pxf = (float)px, pyf = (float)py;
    const float ox = (float)(tx * T), oy = (float)(ty * T);
    const uint2 rg = A.ranges[tile];
    const size_t HW = (size_t)A.width * A.height;
    const size_t o = (size_t)py * A.width + px;
    int my_last = 0;
    float Tr = 1.0f, G0 = 0.0f, G1 = 0.0f, G2 = 0.0f;
    if (inside) {
        my_last = (int)A.last[o];
        Tr = A.final_T[o];
        if (!kPup) {
            G0 = A.dL_dimg[o];
            G1 = A.dL_dimg[HW + o];
            G2 = A.dL_dimg[2 * HW + o];
        }
    }
    float B0 = A.bg0, B1 = A.bg1, B2 = A.bg2;
    if (threadIdx.x == 0) s_maxlast = 0;
    __syncthreads();
    atomicMax(&s_maxlast, my_last);
    __syncthreads();
    const int top = s_maxlast;  // positions [0, top) matter to some pixel
    for (int b1 = top; b1 > 0; b1 -= NB) {
        const int b0 = max(0, b1 - NB);
        const int cnt = b1 - b0;
        __syncthreads();
        if ((int)threadIdx.x < cnt) {
            const int j = b0 + (int)threadIdx.x;
            const uint32_t id = A.vals[rg.x + j];
            const float4 q0 = A.p0[id];
            const float4 q1 = A.p1[id];
            s_g0[threadIdx.x] = make_float4(q0.x, q0.y, q1.x, q1.y + q1.y);
            s_g1[threadIdx.x] = make_float4(q1.z, q1.w, q0.z, q1.y);
            s_g2[threadIdx.x] = A.p2[id];
            s_id[threadIdx.x] = id;
            s_mask[threadIdx.x] = subtile_mask<T>(q0.x, q0.y, q1.x, q1.y, q1.z, q1.w, ox, oy);
        }
        __syncthreads();
        // walk this batch backwards, 32 entries per ballot
        for (int c1 = cnt; c1 > 0; c1 -= 32) {
            const int c0 = max(0, c1 - 32);
            const int k_l = c0 + lane;
            uint32_t bits = __ballot_sync(0xffffffffu, k_l < c1 && (s_mask[k_l] & my_bit));
            while (bits) {
                const int hb = 31 - __clz(bits);
                bits &= ~(1u << hb);
                const int k = c0 + hb;
                const int pos = b0 + k;  // 0-based position in the tile list
                float v[16];
                bool has = false;
                if (pos < my_last) {
                    const float4 g0 = s_g0[k];
                    const float4 g1 = s_g1[k];
                    const float dx = pxf - g0.x;
                    const float dy = pyf - g0.y;
                    const float e = g0.w * dy;
                    const float f = (g1.x * dy) * dy;
                    const float q = fmaf(dx, fmaf(g0.z, dx, e), f);
                    if (q <= g1.y) {
                        has = true;
                        const float g = gs_expf_blend(-0.5f * q);
                        const float raw = g1.z * g;
                        const float alpha = fminf(0.99f, raw);
                        const float Tb = __fdividef(Tr, 1.0f - alpha);
                        const float4 col = s_g2[k];
                        const float w = alpha * Tb;
                        const float d0 = Tb * (col.x - B0), d1 = Tb * (col.y - B1), d2 = Tb * (col.z - B2);
                        if (kPup) {
#pragma unroll
                            for (int m = 0; m < 16; ++m) v[m] = 0.0f;
                            if (raw <= 0.99f) {
                                const float s0 = g1.z * d0, s1 = g1.z * d1, s2 = g1.z * d2;
                                const float wp = s0 * s0 + s1 * s1 + s2 * s2;
                                const float hg = -0.5f * g;
                                const float a = g0.z, b = g1.w, c = g1.x;
                                const float G5[5] = {hg * (-2.0f * (a * dx + b * dy)), hg * (-2.0f * (b * dx + c * dy)),
                                                     hg * (dx * dx), hg * (2.0f * dx * dy), hg * (dy * dy)};
                                int m = 0;
#pragma unroll
                                for (int r = 0; r < 5; ++r)
#pragma unroll
                                    for (int q2 = r; q2 < 5; ++q2) v[m++] = wp * G5[r] * G5[q2];
                            }
                        } else {
                        v[6] = G0 * w;
                        v[7] = G1 * w;
                        v[8] = G2 * w;
                        const float dL_dalpha = G0 * d0 + G1 * d1 + G2 * d2;
                        if (raw <= 0.99f) {
                            v[5] = dL_dalpha * g;
                            const float dL_dq = dL_dalpha * g1.z * (-0.5f * g);
                            const float a = g0.z, b = g1.w, c = g1.x;
                            v[2] = dL_dq * dx * dx;
                            v[3] = dL_dq * 2.0f * dx * dy;
                            v[4] = dL_dq * dy * dy;
                            v[0] = dL_dq * (-2.0f * a * dx - 2.0f * b * dy);
                            v[1] = dL_dq * (-2.0f * b * dx - 2.0f * c * dy);
                            const float s0 = g1.z * d0, s1 = g1.z * d1, s2 = g1.z * d2;
                            v[9] = s0 * s0 + s1 * s1 + s2 * s2;
                        } else {
                            v[0] = v[1] = v[2] = v[3] = v[4] = v[5] = v[9] = 0.0f;
                        }
                        }
                        B0 = alpha * col.x + (1.0f - alpha) * B0;
                        B1 = alpha * col.y + (1.0f - alpha) * B1;
                        B2 = alpha * col.z + (1.0f - alpha) * B2;
                        Tr = Tb;
                    }
                }
                const uint32_t hm = __ballot_sync(0xffffffffu, has);
                if (hm != 0u && __popc(hm) <= 16) {
                    // up to sixteen pixels took this Gaussian: each adds its own values (cheaper
                    // than the warp reduction below at these counts)
                    if (has) {
                        float* row = A.work + (size_t)s_id[k] * kRow;
                        atomicAdd(reinterpret_cast<float4*>(row), make_float4(v[0], v[1], v[2], v[3]));
                        atomicAdd(reinterpret_cast<float4*>(row + 4), make_float4(v[4], v[5], v[6], v[7]));
                        if (kPup) {
                            atomicAdd(reinterpret_cast<float4*>(row + 8), make_float4(v[8], v[9], v[10], v[11]));
                            atomicAdd(reinterpret_cast<float4*>(row + 12), make_float4(v[12], v[13], v[14], 0.0f));
                        } else {
                            atomicAdd(reinterpret_cast<float2*>(row + 8), make_float2(v[8], v[9]));
                        }
                    }
                } else if (hm != 0u) {
                    // Warp sum of the 10 values by halving exchanges: after
                    // the steps over lane bits 4 and 3 each lane keeps 4 of 16
                    // (zero-padded) values, group lane >> 3; three more steps
                    // complete the sums.  Lanes 0, 8 and 16 then add groups
                    // 0..3, 4..7 and 8..9 to the Gaussian's row with one vector
                    // atomic each.
                    float w[16];
#pragma unroll
                    for (int m = 0; m < 16; ++m) w[m] = (m < kNV && has) ? v[m] : 0.0f;
                    const bool up16 = (lane & 16) != 0;
#pragma unroll
                    for (int m = 0; m < 8; ++m) {
                        const float send = up16 ? w[m] : w[m + 8];
                        const float keep = up16 ? w[m + 8] : w[m];
                        w[m] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
                    }
                    const bool up8 = (lane & 8) != 0;
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const float send = up8 ? w[m] : w[m + 4];
                        const float keep = up8 ? w[m + 4] : w[m];
                        w[m] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
                    }
#pragma unroll
                    for (int off = 4; off > 0; off >>= 1)
#pragma unroll
                        for (int m = 0; m < 4; ++m) w[m] += __shfl_xor_sync(0xffffffffu, w[m], off);
                    float* row = A.work + (size_t)s_id[k] * kRow;
                    if (lane == 0) atomicAdd(reinterpret_cast<float4*>(row), make_float4(w[0], w[1], w[2], w[3]));
                    else if (lane == 8) atomicAdd(reinterpret_cast<float4*>(row + 4), make_float4(w[0], w[1], w[2], w[3]));
                    else if (kPup && lane == 16) atomicAdd(reinterpret_cast<float4*>(row + 8), make_float4(w[0], w[1], w[2], w[3]));
                    else if (kPup && lane == 24) atomicAdd(reinterpret_cast<float4*>(row + 12), make_float4(w[0], w[1], w[2], w[3]));
                    else if (!kPup && lane == 16) atomicAdd(reinterpret_cast<float2*>(row + 8), make_float2(w[0], w[1]));
                }
            }
        }
    }
}

struct PreBwdArgs {
    const float* means;
    const float* scales;
    const float* rots;
    const float* sh;
    const int32_t* counts;
    const float* work;
    int64_t n, ncap;
    int sh_coeffs;
    float fx, fy, limx, limy;
    float V[12];
    float campos[3];
    float* g_means;
    float* g_scales;
    float* g_rots;
    float* g_opac;
    float* g_sh;
    float* g_means2d;  // nullable
    float* score;      // nullable (+=)
};

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

__device__ void sh_eval(float x, float y, float z, float Y[16], float dY[16][3]) {
    const float xx = x * x, yy = y * y, zz = z * z, xy = x * y, yz = y * z, xz = x * z;
    Y[0] = kC0;
    Y[1] = -kC1 * y;
    Y[2] = kC1 * z;
    Y[3] = -kC1 * x;
    Y[4] = kC2a * xy;
    Y[5] = -kC2a * yz;
    Y[6] = kC2c * (2.0f * zz - xx - yy);
    Y[7] = -kC2a * xz;
    Y[8] = kC2e * (xx - yy);
    Y[9] = -kC3a * y * (3.0f * xx - yy);
    Y[10] = kC3b * xy * z;
    Y[11] = -kC3c * y * (4.0f * zz - xx - yy);
    Y[12] = kC3d * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
    Y[13] = -kC3c * x * (4.0f * zz - xx - yy);
    Y[14] = kC3f * z * (xx - yy);
    Y[15] = -kC3a * x * (xx - 3.0f * yy);
    const float g[16][3] = {{0, 0, 0},
                            {0, -kC1, 0},
                            {0, 0, kC1},
                            {-kC1, 0, 0},
                            {kC2a * y, kC2a * x, 0},
                            {0, -kC2a * z, -kC2a * y},
                            {-2 * kC2c * x, -2 * kC2c * y, 4 * kC2c * z},
                            {-kC2a * z, 0, -kC2a * x},
                            {2 * kC2e * x, -2 * kC2e * y, 0},
                            {-6 * kC3a * xy, -kC3a * (3 * xx - 3 * yy), 0},
                            {kC3b * yz, kC3b * xz, kC3b * xy},
                            {2 * kC3c * xy, -kC3c * (4 * zz - xx - 3 * yy), -8 * kC3c * yz},
                            {-6 * kC3d * xz, -6 * kC3d * yz, kC3d * (6 * zz - 3 * xx - 3 * yy)},
                            {-kC3c * (4 * zz - 3 * xx - yy), 2 * kC3c * xy, -8 * kC3c * xz},
                            {2 * kC3f * xz, -2 * kC3f * yz, kC3f * (xx - yy)},
                            {-kC3a * (3 * xx - 3 * yy), 6 * kC3a * xy, 0}};
#pragma unroll
    for (int k = 0; k < 16; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) dY[k][j] = g[k][j];
}

// Projection of one Gaussian as the backward chain needs it (Sec. 3.2.1):
// view-space mean, normalised quaternion and rotation, M = R S, Sigma3D,
// T = J W and the 2D covariance, with the x/z, y/z clamp state.
struct ProjChain {
    float x, y, z, tx, ty, nq;
    bool clx, cly;
    float qn[4];
    float Rm[3][3], M[3][3], S3[3][3], T[2][3], TS[2][3];
    float sxx, sxy, syy;
};

__device__ __forceinline__ void chain_setup(ProjChain& P, const float* V, float fx, float fy, float limx, float limy,
                                            const float mu[3], const float sc[3], const float q[4]) {
    float p[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) p[r] = V[4 * r] * mu[0] + V[4 * r + 1] * mu[1] + V[4 * r + 2] * mu[2] + V[4 * r + 3];
    P.x = p[0], P.y = p[1], P.z = p[2];
    P.nq = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const float qw = q[0] / P.nq, qx = q[1] / P.nq, qy = q[2] / P.nq, qz = q[3] / P.nq;
    P.qn[0] = qw, P.qn[1] = qx, P.qn[2] = qy, P.qn[3] = qz;
    const float R[3][3] = {{1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy)},
                           {2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx)},
                           {2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)}};
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            P.Rm[r][k] = R[r][k];
            P.M[r][k] = R[r][k] * sc[k];
        }
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            P.S3[r][c] = P.M[r][0] * P.M[c][0] + P.M[r][1] * P.M[c][1] + P.M[r][2] * P.M[c][2];
    const float z = P.z;
    const float xz = P.x / z, yz = P.y / z;
    P.clx = xz < -limx || xz > limx;
    P.cly = yz < -limy || yz > limy;
    P.tx = fminf(limx, fmaxf(-limx, xz)) * z;
    P.ty = fminf(limy, fmaxf(-limy, yz)) * z;
    const float z2 = z * z;
    const float J[2][3] = {{fx / z, 0.0f, -fx * P.tx / z2}, {0.0f, fy / z, -fy * P.ty / z2}};
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) P.T[r][k] = J[r][0] * V[k] + J[r][1] * V[4 + k] + J[r][2] * V[8 + k];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            P.TS[r][c] = P.T[r][0] * P.S3[0][c] + P.T[r][1] * P.S3[1][c] + P.T[r][2] * P.S3[2][c];
    P.sxx = P.TS[0][0] * P.T[0][0] + P.TS[0][1] * P.T[0][1] + P.TS[0][2] * P.T[0][2] + 0.3f;
    P.sxy = P.TS[0][0] * P.T[1][0] + P.TS[0][1] * P.T[1][1] + P.TS[0][2] * P.T[1][2];
    P.syy = P.TS[1][0] * P.T[1][0] + P.TS[1][1] * P.T[1][1] + P.TS[1][2] * P.T[1][2] + 0.3f;
}

// Chain from gradients with respect to (u, v) and the conic (a, b, c) to
// the mean (dmu, through the projection and the Jacobian J) and to M = R S
// (dM, from which the scale and rotation gradients follow).
__device__ __forceinline__ void chain_apply(const ProjChain& P, const float* V, float fx, float fy, float gu, float gv,
                                            float ga, float gb, float gc, float dmu[3], float dM[3][3]) {
    const float x = P.x, y = P.y, z = P.z, tx = P.tx, ty = P.ty;
    const float z2 = z * z, z3 = z2 * z;
    const float sxx = P.sxx, sxy = P.sxy, syy = P.syy;
    const float det = sxx * syy - sxy * sxy;
    const float id = 1.0f / det, id2 = id * id;
    const float g_sxx = ga * (-syy * syy * id2) + gb * (sxy * syy * id2) + gc * (id - sxx * syy * id2);
    const float g_syy = ga * (id - sxx * syy * id2) + gb * (sxy * sxx * id2) + gc * (-sxx * sxx * id2);
    const float g_sxy = ga * (2.0f * sxy * syy * id2) + gb * (-id - 2.0f * sxy * sxy * id2) + gc * (2.0f * sxy * sxx * id2);
    const float G2[2][2] = {{g_sxx, 0.5f * g_sxy}, {0.5f * g_sxy, g_syy}};
    float G3[3][3], dT[2][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            G3[r][c] = P.T[0][r] * (G2[0][0] * P.T[0][c] + G2[0][1] * P.T[1][c]) +
                       P.T[1][r] * (G2[1][0] * P.T[0][c] + G2[1][1] * P.T[1][c]);
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) dT[r][c] = 2.0f * (G2[r][0] * P.TS[0][c] + G2[r][1] * P.TS[1][c]);
    float dJ[2][3];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) dJ[r][k] = dT[r][0] * V[4 * k] + dT[r][1] * V[4 * k + 1] + dT[r][2] * V[4 * k + 2];
    float dp[3] = {0.0f, 0.0f, 0.0f};
    dp[2] += dJ[0][0] * (-fx / z2) + dJ[1][1] * (-fy / z2);
    if (!P.clx) {
        dp[0] += dJ[0][2] * (-fx / z2);
        dp[2] += dJ[0][2] * (2.0f * fx * x / z3);
    } else {
        dp[2] += dJ[0][2] * (fx * (tx / z) / z2);
    }
    if (!P.cly) {
        dp[1] += dJ[1][2] * (-fy / z2);
        dp[2] += dJ[1][2] * (2.0f * fy * y / z3);
    } else {
        dp[2] += dJ[1][2] * (fy * (ty / z) / z2);
    }
    dp[0] += gu * fx / z;
    dp[1] += gv * fy / z;
    dp[2] += gu * (-fx * x / z2) + gv * (-fy * y / z2);
#pragma unroll
    for (int k = 0; k < 3; ++k) dmu[k] = V[k] * dp[0] + V[4 + k] * dp[1] + V[8 + k] * dp[2];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            dM[r][k] = 2.0f * (G3[r][0] * P.M[0][k] + G3[r][1] * P.M[1][k] + G3[r][2] * P.M[2][k]);
}

__global__ void __launch_bounds__(256, 4) preprocess_backward_kernel(const PreBwdArgs A) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    const int64_t n = A.n;
    float gr[kWork];
    {
        const float* row = A.work + (size_t)i * kWorkRow;
        const float4 a = *reinterpret_cast<const float4*>(row);
        const float4 b = *reinterpret_cast<const float4*>(row + 4);
        const float2 c = *reinterpret_cast<const float2*>(row + 8);
        gr[0] = a.x, gr[1] = a.y, gr[2] = a.z, gr[3] = a.w;
        gr[4] = b.x, gr[5] = b.y, gr[6] = b.z, gr[7] = b.w;
        gr[8] = c.x, gr[9] = c.y;
    }
    if (A.score) A.score[i] += gr[9];
    if (A.g_means2d) {
        A.g_means2d[i] = gr[0];
        A.g_means2d[n + i] = gr[1];
    }
    A.g_opac[i] = gr[5];
    bool any = A.counts[i] > 0;
    if (!any) {
        for (int k = 0; k < 3; ++k) A.g_means[k * n + i] = 0.0f, A.g_scales[k * n + i] = 0.0f;
        for (int k = 0; k < 4; ++k) A.g_rots[k * n + i] = 0.0f;
        for (int k = 0; k < 48; ++k) A.g_sh[(int64_t)k * n + i] = 0.0f;
        return;
    }
    const float mu[3] = {A.means[i], A.means[n + i], A.means[2 * n + i]};
    const float sc[3] = {A.scales[i], A.scales[n + i], A.scales[2 * n + i]};
    const float q[4] = {A.rots[i], A.rots[n + i], A.rots[2 * n + i], A.rots[3 * n + i]};
    ProjChain P;
    chain_setup(P, A.V, A.fx, A.fy, A.limx, A.limy, mu, sc, q);
    const float nq = P.nq, qw = P.qn[0], qx = P.qn[1], qy = P.qn[2], qz = P.qn[3];
    float dmu[3], dM[3][3];
    chain_apply(P, A.V, A.fx, A.fy, gr[0], gr[1], gr[2], gr[3], gr[4], dmu, dM);
    const auto& Rm = P.Rm;
    float dR[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        A.g_scales[k * n + i] = dM[0][k] * Rm[0][k] + dM[1][k] * Rm[1][k] + dM[2][k] * Rm[2][k];
#pragma unroll
        for (int r = 0; r < 3; ++r) dR[r][k] = dM[r][k] * sc[k];
    }
    float dqn[4];
    dqn[0] = 2 * (-qz * dR[0][1] + qy * dR[0][2] + qz * dR[1][0] - qx * dR[1][2] - qy * dR[2][0] + qx * dR[2][1]);
    dqn[1] = 2 * (qy * dR[0][1] + qz * dR[0][2] + qy * dR[1][0] - 2 * qx * dR[1][1] - qw * dR[1][2] + qz * dR[2][0] +
                  qw * dR[2][1] - 2 * qx * dR[2][2]);
    dqn[2] = 2 * (-2 * qy * dR[0][0] + qx * dR[0][1] + qw * dR[0][2] + qx * dR[1][0] + qz * dR[1][2] - qw * dR[2][0] +
                  qz * dR[2][1] - 2 * qy * dR[2][2]);
    dqn[3] = 2 * (-2 * qz * dR[0][0] - qw * dR[0][1] + qx * dR[0][2] + qw * dR[1][0] - 2 * qz * dR[1][1] +
                  qy * dR[1][2] + qx * dR[2][0] + qy * dR[2][1]);
    const float qn[4] = {qw, qx, qy, qz};
    const float dot = qn[0] * dqn[0] + qn[1] * dqn[1] + qn[2] * dqn[2] + qn[3] * dqn[3];
#pragma unroll
    for (int k = 0; k < 4; ++k) A.g_rots[k * n + i] = (dqn[k] - qn[k] * dot) / nq;
    // SH colour and its view-direction term
    const float d0 = mu[0] - A.campos[0], d1 = mu[1] - A.campos[1], d2 = mu[2] - A.campos[2];
    const float len = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
    const float dir[3] = {d0 / len, d1 / len, d2 / len};
    float Y[16], dY[16][3];
    sh_eval(dir[0], dir[1], dir[2], Y, dY);
    float ddir[3] = {0.0f, 0.0f, 0.0f};
    for (int ch = 0; ch < 3; ++ch) {
        float h[16];
        float raw = 0.5f;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            h[k] = k < A.sh_coeffs ? A.sh[(int64_t)(k * 3 + ch) * n + i] : 0.0f;
            raw += Y[k] * h[k];
        }
        const float graw = raw >= 0.0f ? gr[6 + ch] : 0.0f;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            A.g_sh[(int64_t)(k * 3 + ch) * n + i] = k < A.sh_coeffs ? Y[k] * graw : 0.0f;
#pragma unroll
            for (int j = 0; j < 3; ++j) ddir[j] += graw * dY[k][j] * h[k];
        }
    }
    const float dd = dir[0] * ddir[0] + dir[1] * ddir[1] + dir[2] * ddir[2];
#pragma unroll
    for (int k = 0; k < 3; ++k) A.g_means[k * n + i] = dmu[k] + (ddir[k] - dir[k] * dd) / len;
}


// ---------------------------------------------------------------- PUP sensitivity (Sec. 4.2, Eq. pup_score)
// H_i = sum over views, pixels and channels of grad_{mu,s} C grad_{mu,s} C^T,
// through the 2D Gaussian value g_i(p): grad_{mu,s} C_ch(p) =
// dC_ch/dg * J_i^T G5(p), with G5 = dg/d(u, v, a, b, c) and J_i the 5 x 6
// Jacobian of (u, v, a, b, c) with respect to (mu, s).  So
// H_i += J_i^T (sum_p w_p G5 G5^T) J_i per view; the blend pass above sums the
// 5 x 5 matrix, this pass applies J_i (its five rows are the projection chain
// applied to unit gradients) and adds the 21 entries of the symmetric 6 x 6
// matrix to hessian[21][n] (row-major upper triangle, order mu_x mu_y mu_z
// s_0 s_1 s_2).
struct PupArgs {
    const float* means;
    const float* scales;
    const float* rots;
    const int32_t* counts;
    const float* work;  // [ncap][16]
    int64_t n;
    float fx, fy, limx, limy;
    float V[12];
    float* hessian;     // [21][n], +=
};

__global__ void __launch_bounds__(256, 3) pup_jacobian_kernel(const PupArgs A) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n || A.counts[i] <= 0) return;
    const int64_t n = A.n;
    float M5[5][5];
    {
        const float* row = A.work + (size_t)i * 16;
        int m = 0;
#pragma unroll
        for (int r = 0; r < 5; ++r)
#pragma unroll
            for (int c = r; c < 5; ++c) {
                M5[r][c] = row[m];
                M5[c][r] = row[m];
                ++m;
            }
    }
    const float mu[3] = {A.means[i], A.means[n + i], A.means[2 * n + i]};
    const float sc[3] = {A.scales[i], A.scales[n + i], A.scales[2 * n + i]};
    const float q[4] = {A.rots[i], A.rots[n + i], A.rots[2 * n + i], A.rots[3 * n + i]};
    ProjChain P;
    chain_setup(P, A.V, A.fx, A.fy, A.limx, A.limy, mu, sc, q);
    float Jt[5][6];  // row k: d(2D parameter k)/d(mu, s)
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        float dmu[3], dM[3][3];
        chain_apply(P, A.V, A.fx, A.fy, k == 0 ? 1.0f : 0.0f, k == 1 ? 1.0f : 0.0f, k == 2 ? 1.0f : 0.0f,
                    k == 3 ? 1.0f : 0.0f, k == 4 ? 1.0f : 0.0f, dmu, dM);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Jt[k][a] = dmu[a];
            Jt[k][3 + a] = dM[0][a] * P.Rm[0][a] + dM[1][a] * P.Rm[1][a] + dM[2][a] * P.Rm[2][a];
        }
    }
    float MJ[5][6];  // M5 Jt
#pragma unroll
    for (int k = 0; k < 5; ++k)
#pragma unroll
        for (int b = 0; b < 6; ++b) {
            float acc = 0.0f;
#pragma unroll
            for (int l = 0; l < 5; ++l) acc += M5[k][l] * Jt[l][b];
            MJ[k][b] = acc;
        }
    int e = 0;
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
        for (int b = a; b < 6; ++b) {
            float acc = 0.0f;
#pragma unroll
            for (int k = 0; k < 5; ++k) acc += Jt[k][a] * MJ[k][b];
            A.hessian[(int64_t)e * n + i] += acc;
            ++e;
        }
}

// U_i = log det H_i in double precision, by an LDL^T factorisation (no
// square roots): the pivots d_j are positive exactly when H_i is positive
// definite, and log det H_i = sum_j log d_j, taken as one logarithm of the
// pivots' mantissa product (each in [1/2, 1), so no underflow) plus their
// summed binary exponents times ln 2.  One reciprocal per pivot replaces the
// divisions.  -inf where H_i is not positive definite (e.g. a Gaussian seen
// from one view only: its 6 x 6 block has rank 5 at most).
__global__ void __launch_bounds__(256) pup_logdet_kernel(const float* __restrict__ hessian, int64_t n,
                                                        float* __restrict__ score) {
    // A positive definite matrix has a positive diagonal: checked from the
    // six diagonal entries alone (entry (a, a) is row a's first of the packed
    // upper triangle), which settles every Gaussian no view reached (H = 0).
    // The rest of the block's Gaussians are factorised by its lowest threads,
    // so the FP64 work runs in full warps.
    __shared__ uint32_t s_idx[256];
    __shared__ int s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * blockDim.x;
    {
        const int64_t j = base + threadIdx.x;
        if (j < n) {
            bool diag = true;
            constexpr int kDiag[6] = {0, 6, 11, 15, 18, 20};
#pragma unroll
            for (int a = 0; a < 6; ++a) diag = diag && (hessian[(int64_t)kDiag[a] * n + j] > 0.0f);
            if (diag) s_idx[atomicAdd(&s_cnt, 1)] = threadIdx.x;
            else score[j] = -INFINITY;
        }
    }
    __syncthreads();
    if ((int)threadIdx.x >= s_cnt) return;
    const int64_t i = base + s_idx[threadIdx.x];
    double A[6][6];
    {
        int e = 0;
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
            for (int b = a; b < 6; ++b) {
                A[b][a] = (double)hessian[(int64_t)e * n + i];  // lower triangle
                ++e;
            }
    }
    double L[6][6];  // unit lower triangular factor (below the diagonal)
    double d[6];
    bool pd = true;
    double mant = 1.0;
    int expo = 0;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        double v[6];  // v_k = L[j][k] d_k
#pragma unroll
        for (int k = 0; k < j; ++k) v[k] = L[j][k] * d[k];
        double dj = A[j][j];
#pragma unroll
        for (int k = 0; k < j; ++k) dj = fma(-L[j][k], v[k], dj);
        pd = pd && (dj > 0.0);
        d[j] = dj;
        int ej;
        const double mj = frexp(dj, &ej);
        mant *= mj;
        expo += ej;
        const double inv = __drcp_rn(dj);
#pragma unroll
        for (int r = j + 1; r < 6; ++r) {
            double x = A[r][j];
#pragma unroll
            for (int k = 0; k < j; ++k) x = fma(-L[r][k], v[k], x);
            L[r][j] = x * inv;
        }
    }
    const double logdet = log(mant) + (double)expo * 0.69314718055994530942;
    score[i] = pd ? (float)logdet : -INFINITY;
}

}  // namespace

int64_t backward_work_floats(int64_t ncap) { return (int64_t)kWorkRow * ncap; }

gs_status launch_pup(gs_context* ctx, const gs_scene* s, const gs_camera* cam, const gs_raster_cfg* cfg,
                     const FrameView& v, float* hessian, float* work) {
    if (cudaMemsetAsync(work, 0, (size_t)v.ncap * 16 * sizeof(float), ctx->stream) != cudaSuccess)
        return set_error(ctx, GS_ERR_CUDA, "pup: cudaMemsetAsync(work) failed");
    BwdArgs B{};
    B.ranges = v.ranges;
    B.vals = v.vals0;
    B.p0 = v.p0;
    B.p1 = v.p1;
    B.p2 = v.p2;
    B.final_T = v.final_T;
    B.last = v.last;
    B.dL_dimg = nullptr;
    B.work = work;
    B.ncap = v.ncap;
    B.width = v.width;
    B.height = v.height;
    B.gx = v.gx;
    B.bg0 = cfg->bg[0];
    B.bg1 = cfg->bg[1];
    B.bg2 = cfg->bg[2];
    const unsigned tiles = (unsigned)(v.gx * v.gy);
    switch (v.tile) {
        case 8: blend_backward_kernel<8, true><<<tiles, 64, 0, ctx->stream>>>(B); break;
        case 16: blend_backward_kernel<16, true><<<tiles, 256, 0, ctx->stream>>>(B); break;
        case 32: blend_backward_kernel<32, true><<<tiles, 1024, 0, ctx->stream>>>(B); break;
        default: return set_error(ctx, GS_ERR_INVALID, "pup: tile %d not supported", v.tile);
    }
    ctx->launches += 1;
    gs_status st = check_launch(ctx, "pup blend");
    if (st || s->n == 0) return st;
    PupArgs P;
    P.means = s->means;
    P.scales = s->scales;
    P.rots = s->rotations;
    P.counts = v.counts;
    P.work = work;
    P.n = s->n;
    P.fx = cam->fx;
    P.fy = cam->fy;
    P.limx = 1.3f * cam->tan_fovx;
    P.limy = 1.3f * cam->tan_fovy;
    for (int k = 0; k < 12; ++k) P.V[k] = cam->viewmat[k];
    P.hessian = hessian;
    pup_jacobian_kernel<<<(unsigned)((s->n + 255) / 256), 256, 0, ctx->stream>>>(P);
    ctx->launches += 1;
    return check_launch(ctx, "pup jacobian");
}

gs_status launch_pup_score(gs_context* ctx, const float* hessian, int64_t n, float* score) {
    if (n == 0) return GS_OK;
    pup_logdet_kernel<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(hessian, n, score);  // 256: s_idx
    ctx->launches += 1;
    return check_launch(ctx, "pup logdet");
}

gs_status launch_backward(gs_context* ctx, const gs_scene* s, const gs_camera* cam, const gs_raster_cfg* cfg,
                          const FrameView& v, const float* dL_dimg, const gs_grads* g) {
    const int64_t work_bytes = backward_work_floats(v.ncap) * (int64_t)sizeof(float);
    if (cudaMemsetAsync(g->work, 0, (size_t)work_bytes, ctx->stream) != cudaSuccess)
        return set_error(ctx, GS_ERR_CUDA, "render_backward: cudaMemsetAsync(work) failed");
    BwdArgs B;
    B.ranges = v.ranges;
    B.vals = v.vals0;
    B.p0 = v.p0;
    B.p1 = v.p1;
    B.p2 = v.p2;
    B.final_T = v.final_T;
    B.last = v.last;
    B.dL_dimg = dL_dimg;
    B.work = g->work;
    B.ncap = v.ncap;
    B.width = v.width;
    B.height = v.height;
    B.gx = v.gx;
    B.bg0 = cfg->bg[0];
    B.bg1 = cfg->bg[1];
    B.bg2 = cfg->bg[2];
    const unsigned tiles = (unsigned)(v.gx * v.gy);
    switch (v.tile) {
        case 8: blend_backward_kernel<8, false><<<tiles, 64, 0, ctx->stream>>>(B); break;
        case 16: blend_backward_kernel<16, false><<<tiles, 256, 0, ctx->stream>>>(B); break;
        case 32: blend_backward_kernel<32, false><<<tiles, 1024, 0, ctx->stream>>>(B); break;
        default: return set_error(ctx, GS_ERR_INVALID, "render_backward: tile %d not supported", v.tile);
    }
    ctx->launches += 1;
    gs_status st = check_launch(ctx, "blend_backward");
    if (st) return st;
    if (s->n == 0) return GS_OK;
    PreBwdArgs P;
    P.means = s->means;
    P.scales = s->scales;
    P.rots = s->rotations;
    P.sh = s->sh;
    P.counts = v.counts;
    P.work = g->work;
    P.n = s->n;
    P.ncap = v.ncap;
    P.sh_coeffs = (s->sh_degree + 1) * (s->sh_degree + 1);
    P.fx = cam->fx;
    P.fy = cam->fy;
    P.limx = 1.3f * cam->tan_fovx;
    P.limy = 1.3f * cam->tan_fovy;
    for (int k = 0; k < 12; ++k) P.V[k] = cam->viewmat[k];
    for (int k = 0; k < 3; ++k) P.campos[k] = cam->campos[k];
    P.g_means = g->means;
    P.g_scales = g->scales;
    P.g_rots = g->rotations;
    P.g_opac = g->opacities;
    P.g_sh = g->sh;
    P.g_means2d = g->means2d;
    P.score = g->score;
    const int64_t blocks = (s->n + 255) / 256;
    preprocess_backward_kernel<<<(unsigned)blocks, 256, 0, ctx->stream>>>(P);
    ctx->launches += 1;
    return check_launch(ctx, "preprocess_backward");
}

}  // namespace gs
