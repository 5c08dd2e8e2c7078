// Per-warp culling inside a tile, shared by the forward and backward blend.
#pragma once

#include "gs_common.cuh"

namespace gs {

// Sub-tile of one warp: 8 columns x 4 rows of pixels.
constexpr int kSubW = 8;
constexpr int kSubH = 4;

// Conservative mask of the warp sub-tiles of a T x T tile (origin ox, oy) that
// the ellipse q <= t can reach, in two steps.
//
// Box: extents hx = sqrt(t c / D), hy = sqrt(t a / D), widened by
// 1 px + 0.1 % so that rounding in D, in the extents and in the per-pixel q can
// never drop a pixel whose q <= t, select the sub-tiles the ellipse's bounding
// box meets.  Conics too close to singular (b^2 >= 0.999 a c) or non-finite
// extents get every sub-tile; a Gaussian with t < 0 reaches no pixel
// (q >= 0 > t).
//
// Rectangle minimum: each box sub-tile is then kept only if the minimum of
// q(dx, dy) = a dx^2 + 2 b dx dy + c dy^2 over the rectangle spanned by its
// pixel offsets [lx, hx] x [ly, hy] is at most 1.01 t.  The offsets are
// computed exactly as the blend computes a pixel's dx and dy (pixel coordinate
// minus centre, one FP32 subtraction), and rounding is monotone, so every
// pixel's (dx, dy) lies in that rectangle.  If the centre is inside, the
// minimum is 0.  Otherwise the minimum of this convex form lies on a face of
// the rectangle whose outer side holds the centre (at a constrained minimiser
// the gradient points into the rectangle, and convexity then puts the centre
// beyond the face); there are at most two such faces, and along a face
// dx = X the minimum is at dy = clamp(-b X / c, ly, hy) (symmetrically for a
// face dy = Y).  With b^2 < 0.999 a c the relative rounding error of both the
// blend's q and this minimum is below 2e-3, so the 1 % margin keeps every
// sub-tile with a pixel whose q <= t; the reciprocals are approximate because
// an error in the clamped point changes q only to second order.
template <int T>
__device__ __forceinline__ uint32_t subtile_mask(float u, float v, float a, float b, float c, float t, float ox,
                                                 float oy) {
    constexpr int NSX = T / kSubW, NSY = T / kSubH;
    constexpr uint32_t kAll = (NSX * NSY == 32) ? 0xffffffffu : ((1u << (NSX * NSY)) - 1u);
    constexpr int kExactMax = 12;  // larger boxes keep the box mask
    if (t < 0.0f) return 0u;
    const float ac = a * c;
    const float bb = b * b;
    const float D = ac - bb;
    if (!(bb < 0.999f * ac) || !(D > 0.0f)) return kAll;
    const float hx = sqrtf((t * c) / D);
    const float hy = sqrtf((t * a) / D);
    if (!isfinite(hx) || !isfinite(hy)) return kAll;
    const float mx = hx + (1.0f + 1e-3f * hx);
    const float my = hy + (1.0f + 1e-3f * hy);
    const float x0 = (u - ox) - mx, x1 = (u - ox) + mx;
    const float y0 = (v - oy) - my, y1 = (v - oy) + my;
    if (x1 < 0.0f || y1 < 0.0f || x0 >= (float)T || y0 >= (float)T) return 0u;
    const int sx0 = x0 <= 0.0f ? 0 : (int)(x0 * (1.0f / kSubW));
    const int sx1 = x1 >= (float)(T - 1) ? NSX - 1 : (int)(x1 * (1.0f / kSubW));
    const int sy0 = y0 <= 0.0f ? 0 : (int)(y0 * (1.0f / kSubH));
    const int sy1 = y1 >= (float)(T - 1) ? NSY - 1 : (int)(y1 * (1.0f / kSubH));
    const uint32_t row = ((2u << sx1) - 1u) & ~((1u << sx0) - 1u);
    uint32_t m = 0;
    if ((sx1 - sx0 + 1) * (sy1 - sy0 + 1) > kExactMax || !(a > 1e-20f && a < 1e20f && c > 1e-20f && c < 1e20f)) {
        for (int sy = sy0; sy <= sy1; ++sy) m |= row << (sy * NSX);
        return m;
    }
    const float ia = __fdividef(1.0f, a), ic = __fdividef(1.0f, c);
    const float b2 = b + b;
    const float tt = 1.01f * t;
    for (int sy = sy0; sy <= sy1; ++sy) {
        const float ly = (oy + (float)(sy * kSubH)) - v;
        const float hy_ = (oy + (float)(sy * kSubH + kSubH - 1)) - v;
        const bool outy = ly > 0.0f || hy_ < 0.0f;
        const float Y = ly > 0.0f ? ly : hy_;
        const float nbY = -b * Y;
        const float cYY = (c * Y) * Y;
        for (int sx = sx0; sx <= sx1; ++sx) {
            const float lx = (ox + (float)(sx * kSubW)) - u;
            const float hx_ = (ox + (float)(sx * kSubW + kSubW - 1)) - u;
            const bool outx = lx > 0.0f || hx_ < 0.0f;
            float qmin = 0.0f;
            if (outx || outy) {
                qmin = INFINITY;
                if (outx) {  // face dx = X, minimise over dy
                    const float X = lx > 0.0f ? lx : hx_;
                    const float d = fminf(fmaxf((-b * X) * ic, ly), hy_);
                    qmin = fmaf(X, fmaf(a, X, b2 * d), (c * d) * d);
                }
                if (outy) {  // face dy = Y, minimise over dx
                    const float d = fminf(fmaxf(nbY * ia, lx), hx_);
                    qmin = fminf(qmin, fmaf(d, fmaf(a, d, b2 * Y), cYY));
                }
            }
            if (qmin <= tt) m |= 1u << (sy * NSX + sx);
        }
    }
    return m;
}

}  // namespace gs
