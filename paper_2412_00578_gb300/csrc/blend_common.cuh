// Per-warp culling inside a tile, shared by the forward and backward blend.
#pragma once

#include "gs_common.cuh"

namespace gs {

// Sub-tile of one warp: 8 columns x 4 rows of pixels.
constexpr int kSubW = 8;
constexpr int kSubH = 4;

// Conservative mask of the warp sub-tiles of a T x T tile (origin ox, oy) that
// the ellipse q <= t can reach.  Extents hx = sqrt(t c / D), hy = sqrt(t a / D)
// are widened by 1 px + 0.1 % so that rounding in D, in the extents and in the
// per-pixel q can never drop a pixel whose q <= t; conics too close to
// singular (b^2 >= 0.999 a c) or non-finite extents get every sub-tile.  A
// Gaussian with t < 0 reaches no pixel (q >= 0 > t).
template <int T>
__device__ __forceinline__ uint32_t subtile_mask(float u, float v, float a, float b, float c, float t, float ox,
                                                 float oy) {
    constexpr int NSX = T / kSubW, NSY = T / kSubH;
    constexpr uint32_t kAll = (NSX * NSY == 32) ? 0xffffffffu : ((1u << (NSX * NSY)) - 1u);
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
    for (int sy = sy0; sy <= sy1; ++sy) m |= row << (sy * NSX);
    return m;
}

}  // namespace gs
