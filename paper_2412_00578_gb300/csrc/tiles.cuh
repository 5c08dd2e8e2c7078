// Gaussian-to-tile localization: the 3D-GS 3-sigma square (Eq. radius),
// SnugBox (Sec. 4.1.1) and AccuTile (Sec. 4.1.2, Algorithm 1), as device
// functions shared by the counting pass (preprocess) and the emitting pass
// (duplicateWithKeys), plus tile-based culling (App. A.4) and pixel-exact
// tiles.  Both passes call the same functions, so the count always equals the
// number of keys emitted; where the emit writes a whole rectangle without
// them, the count or a shared predicate (accutile_whole_line) has already
// shown that the function's result is that rectangle.
#pragma once

#include "gs_common.cuh"

namespace gs {

// 2D Gaussian in the form the localization needs: centre (u, v), conic
// [[a b][b c]] and threshold t = 2 log(255 sigma) so that alpha >= 1/255
// <=> q = a xd^2 + 2 b xd yd + c yd^2 <= t (Eq. simplified_ellipse).
struct Ellipse {
    float u, v, a, b, c, t;
};

struct Grid {
    float T;      // tile edge, pixels (8, 16 or 32)
    int gx, gy;   // tiles per row, per column
    int W = 0, H = 0;  // image size in pixels (the pixel-exact mode keeps pixels inside it)
    // 1/T.  T is a power of two, so x * invT is the exactly scaled x / T,
    // bit for bit the IEEE quotient, at the cost of one multiply.
    __host__ __device__ float invT() const { return T == 8.0f ? 0.125f : (T == 16.0f ? 0.0625f : 0.03125f); }
};

// 3D-GS rectangle: min = trunc((mu - r)/T), max (exclusive) =
// trunc((mu + r + T - 1)/T), both clamped to [0, G].
__device__ __forceinline__ int trunc_clamp(float x, int G) {
    if (!(x > 0.0f)) return 0;
    if (x >= (float)G) return G;
    return (int)x;
}

struct Rect {
    int x0, x1, y0, y1;  // inclusive bounds
};

__device__ __forceinline__ bool sigma3_rect(float u, float v, int radius, const Grid& g, Rect& R) {
    const float r = (float)radius;
    R.x0 = trunc_clamp((u - r) * g.invT(), g.gx);
    R.x1 = trunc_clamp(((u + r) + (g.T - 1.0f)) * g.invT(), g.gx) - 1;
    R.y0 = trunc_clamp((v - r) * g.invT(), g.gy);
    R.y1 = trunc_clamp(((v + r) + (g.T - 1.0f)) * g.invT(), g.gy) - 1;
    return R.x1 >= R.x0 && R.y1 >= R.y0;
}

// SnugBox: half-extents hx = sqrt(t c / D), hy = sqrt(t a / D), D = a c - b^2
// (Eqs. ellipse_intersect + bbox_args), tile rectangle floor(edge / T)
// clamped to the grid, empty if the box misses the grid.
struct Snug {
    float D, hx, hy, x0, x1, y0, y1;
    Rect R;
};

__device__ __forceinline__ bool snugbox(const Ellipse& E, const Grid& g, Snug& S) {
    if (!(E.t > 0.0f)) return false;
    const float D = E.a * E.c - E.b * E.b;
    if (!(D > 0.0f)) return false;
    S.D = D;
    S.hx = sqrtf((E.t * E.c) / D);
    S.hy = sqrtf((E.t * E.a) / D);
    S.x0 = E.u - S.hx;
    S.x1 = E.u + S.hx;
    S.y0 = E.v - S.hy;
    S.y1 = E.v + S.hy;
    if (!(S.x1 >= 0.0f) || !(S.y1 >= 0.0f) || !(S.x0 < (float)g.gx * g.T) || !(S.y0 < (float)g.gy * g.T))
        return false;
    S.R.x0 = floor_clamp(S.x0 * g.invT(), 0, g.gx - 1);
    S.R.x1 = floor_clamp(S.x1 * g.invT(), 0, g.gx - 1);
    S.R.y0 = floor_clamp(S.y0 * g.invT(), 0, g.gy - 1);
    S.R.y1 = floor_clamp(S.y1 * g.invT(), 0, g.gy - 1);
    return true;
}

// AccuTile sweep over the shorter side of the SnugBox tile rectangle.
// For each swept line k (a tile row, or a tile column), the ellipse's
// extent inside the line comes from the SnugBox extreme point when that
// point lies inside it, otherwise from the ellipse's intersections with the
// line's two boundaries; each boundary is intersected once and reused by the
// next line.  emit(k, jmin, jmax, rows) is called once per non-empty line
// with the inclusive span of tiles; returns the tile count.
// Edge rules: a boundary is intersected only if it lies inside the SnugBox
// span; the discriminant is clamped at 0; a line with neither an extreme
// point nor an intersection falls back to the SnugBox edges; a line whose
// extent lies entirely outside the rectangle's tile span contributes nothing.
template <class Emit>
__device__ __forceinline__ int accutile_sweep(const Ellipse& E, const Snug& S, const Grid& g, Emit&& emit) {
    const bool rows = (S.R.y1 - S.R.y0) <= (S.R.x1 - S.R.x0);
    const float ms = rows ? E.v : E.u;
    const float me = rows ? E.u : E.v;
    const float as = rows ? E.a : E.c;
    const float cs = rows ? E.c : E.a;
    const float s_lo = rows ? S.y0 : S.x0;
    const float s_hi = rows ? S.y1 : S.x1;
    const float e_lo = rows ? S.x0 : S.y0;
    const float e_hi = rows ? S.x1 : S.y1;
    const float h_e = rows ? S.hx : S.hy;
    const int k0 = rows ? S.R.y0 : S.R.x0;
    const int k1 = rows ? S.R.y1 : S.R.x1;
    const int j0 = rows ? S.R.x0 : S.R.y0;
    const int j1 = rows ? S.R.x1 : S.R.y1;
    const float bc = E.b / cs;
    const float pmin_s = ms + bc * h_e;
    const float pmax_s = ms - bc * h_e;
    const float at = as * E.t;
    const float nb0 = -E.b;
    auto isect = [&](float L, float& lo, float& hi) {
        const float d = L - ms;
        float disc = at - (S.D * d) * d;
        if (disc < 0.0f) disc = 0.0f;
        const float sq = sqrtf(disc);
        const float nb = nb0 * d;
        lo = me + (nb - sq) / as;
        hi = me + (nb + sq) / as;
    };
    int cnt = 0;
    float lo_l = 0.0f, lo_r = 0.0f;
    bool have_lo = false;
    const float Llo = (float)k0 * g.T;
    if (Llo >= s_lo) {
        isect(Llo, lo_l, lo_r);
        have_lo = true;
    }
    for (int k = k0; k <= k1; ++k) {
        const float rlo = (float)k * g.T;
        const float rhi = (float)(k + 1) * g.T;
        float hi_l = 0.0f, hi_r = 0.0f;
        const bool have_hi = rhi <= s_hi;
        if (have_hi) isect(rhi, hi_l, hi_r);
        float emin, emax;
        if (pmin_s >= rlo && pmin_s < rhi) emin = e_lo;
        else if (have_lo && have_hi) emin = fminf(lo_l, hi_l);
        else if (have_lo) emin = lo_l;
        else if (have_hi) emin = hi_l;
        else emin = e_lo;
        if (pmax_s >= rlo && pmax_s < rhi) emax = e_hi;
        else if (have_lo && have_hi) emax = fmaxf(lo_r, hi_r);
        else if (have_lo) emax = lo_r;
        else if (have_hi) emax = hi_r;
        else emax = e_hi;
        const float qmin = emin * g.invT();
        const float qmax = emax * g.invT();
        const float fmn = floorf(qmin);
        const float fmx = floorf(qmax);
        const int jmin = floor_clamp(qmin, j0, j1);
        const int jmax = floor_clamp(qmax, j0, j1);
        if (fmn <= (float)j1 && fmx >= (float)j0 && jmax >= jmin) {
            cnt += jmax - jmin + 1;
            emit(k, jmin, jmax, rows);
        }
        lo_l = hi_l;
        lo_r = hi_r;
        have_lo = have_hi;
    }
    return cnt;
}

// The cases where accutile_sweep's result is its single line, whole: a
// rectangle one tile line thick on its shorter side whose two boundaries both
// lie outside the SnugBox span.  Neither boundary is then intersected, so the
// line's extent is the SnugBox edges, which floor to exactly the rectangle's
// span (the same products and clamps as in snugbox).  On true, (k, j0, j1,
// rows) is the sweep's one emit call.
__device__ __forceinline__ bool accutile_whole_line(const Snug& S, const Grid& g, int& k, int& j0, int& j1,
                                                    bool& rows) {
    rows = (S.R.y1 - S.R.y0) <= (S.R.x1 - S.R.x0);
    k = rows ? S.R.y0 : S.R.x0;
    if (k != (rows ? S.R.y1 : S.R.x1)) return false;
    const float s_lo = rows ? S.y0 : S.x0;
    const float s_hi = rows ? S.y1 : S.x1;
    if ((float)k * g.T >= s_lo || (float)(k + 1) * g.T <= s_hi) return false;
    j0 = rows ? S.R.x0 : S.R.y0;
    j1 = rows ? S.R.x1 : S.R.y1;
    return true;
}

struct NoEmit {
    __device__ __forceinline__ void operator()(int, int, int, bool) const {}
};

// q at offset (dx, dy) from the centre, in the blend's operation order.
__device__ __forceinline__ float qpix(const Ellipse& E, float dx, float dy) {
    return fmaf(dx, fmaf(E.a, dx, (E.b + E.b) * dy), (E.c * dy) * dy);
}

// Tile-based culling (StopThePop, App. A.4): does q reach t on the closed
// square [X0, X1] x [Y0, Y1]?  0 if the centre is inside; otherwise the
// minimum lies on a face facing the centre, along face dx = X at
// dy = clamp(-b X / c), along face dy = Y at dx = clamp(-b Y / a).
__device__ __forceinline__ bool tile_reaches(const Ellipse& E, float X0, float X1, float Y0, float Y1) {
    const float dx0 = X0 - E.u, dx1 = X1 - E.u;
    const float dy0 = Y0 - E.v, dy1 = Y1 - E.v;
    const bool outx = dx0 > 0.0f || dx1 < 0.0f;
    const bool outy = dy0 > 0.0f || dy1 < 0.0f;
    if (!outx && !outy) return true;
    float qmin = INFINITY;
    if (outx) {
        const float X = dx0 > 0.0f ? dx0 : dx1;
        const float d = fminf(fmaxf(((-E.b) * X) / E.c, dy0), dy1);
        qmin = fminf(qmin, qpix(E, X, d));
    }
    if (outy) {
        const float Y = dy0 > 0.0f ? dy0 : dy1;
        const float d = fminf(fmaxf(((-E.b) * Y) / E.a, dx0), dx1);
        qmin = fminf(qmin, qpix(E, d, Y));
    }
    return qmin <= E.t;
}

// Candidate tiles of the SnugBox rectangle kept by tile_reaches, row-major;
// put(tx, ty) per kept tile; returns the count.
template <class Put>
__device__ __forceinline__ int tbc_tiles(const Ellipse& E, const Snug& S, const Grid& g, Put&& put) {
    int cnt = 0;
    for (int ty = S.R.y0; ty <= S.R.y1; ++ty)
        for (int tx = S.R.x0; tx <= S.R.x1; ++tx)
            if (tile_reaches(E, (float)tx * g.T, (float)(tx + 1) * g.T, (float)ty * g.T, (float)(ty + 1) * g.T)) {
                put(tx, ty);
                ++cnt;
            }
    return cnt;
}

// Pixel-exact tiles: tiles holding an image pixel with q <= t (the blend's
// test).  The pixels considered are those of the SnugBox widened by one pixel
// on each side, clipped to the image.  Per pixel row the passing pixels form
// one run around the row's chord centre xc = u - b dy / a (q restricted to a
// row is a parabola with its minimum there): the run is seeded at the pixel
// nearest xc (or its neighbour), and each end is found by testing pixels
// from the chord's root estimate outwards or inwards, so every decision is
// the blend's own q <= t.  A tile row whose pixel rows give tile spans that
// do not overlap or touch (possible only for needles thinner than a pixel)
// is settled by testing its tiles' pixels one by one.  Row-major;
// put(tx, ty) per kept tile.
struct PixBox {
    int x0, x1, y0, y1;      // pixels considered (inclusive)
    int tx0, tx1, ty0, ty1;  // tiles holding them (inclusive)
};

// The pixels pixel_tiles considers (the SnugBox widened by one pixel on each
// side, clipped to the image) and their tile range; false when no pixel is
// left.  Every tile pixel_tiles keeps lies in that range.
__device__ __forceinline__ bool pixel_box(const Snug& S, const Grid& g, PixBox& P) {
    auto lo_px = [](float e, int n) {
        const float f = floorf(e) - 1.0f;
        return f < 0.0f ? 0 : (f > (float)n ? n : (int)f);
    };
    auto hi_px = [](float e, int n) {
        const float f = floorf(e) + 1.0f;
        return f < 0.0f ? -1 : (f > (float)(n - 1) ? n - 1 : (int)f);
    };
    P.x0 = lo_px(S.x0, g.W);
    P.x1 = hi_px(S.x1, g.W);
    P.y0 = lo_px(S.y0, g.H);
    P.y1 = hi_px(S.y1, g.H);
    if (P.x0 > P.x1 || P.y0 > P.y1) return false;
    const int T = (int)g.T;
    P.tx0 = P.x0 / T;
    P.tx1 = P.x1 / T;
    P.ty0 = P.y0 / T;
    P.ty1 = P.y1 / T;
    return true;
}

template <class Put>
__device__ __forceinline__ int pixel_tiles(const Ellipse& E, const Snug& S, const Grid& g, Put&& put) {
    PixBox P;
    if (!pixel_box(S, g, P)) return 0;
    const int x0 = P.x0, x1 = P.x1, y0 = P.y0, y1 = P.y1;
    const int T = (int)g.T;
    const int tx0 = P.tx0, tx1 = P.tx1, ty0 = P.ty0, ty1 = P.ty1;
    auto clampi = [](float f, int lo, int hi) { return !(f >= (float)lo) ? lo : (f > (float)hi ? hi : (int)f); };
    int cnt = 0;
    for (int ty = ty0; ty <= ty1; ++ty) {
        const int py0 = max(y0, ty * T), py1 = min(y1, ty * T + T - 1);
        int hl = 1 << 30, hh = -1;
        bool gap = false;
        for (int py = py0; py <= py1 && !gap; ++py) {
            const float dy = (float)py - E.v;
            auto pass = [&](int px) { return qpix(E, (float)px - E.u, dy) <= E.t; };
            const float xc = E.u + ((-E.b) * dy) / E.a;
            int s = clampi(floorf(xc + 0.5f), x0, x1);
            if (!pass(s)) {
                s = clampi((float)s + ((float)s <= xc ? 1.0f : -1.0f), x0, x1);
                if (!pass(s)) continue;  // no pixel of this row reaches the ellipse
            }
            const float disc = (E.b * dy) * (E.b * dy) - E.a * ((E.c * dy) * dy - E.t);
            const float half = disc > 0.0f ? sqrtf(disc) / E.a : 0.0f;
            int L = clampi(ceilf(xc - half), x0, s);
            if (pass(L)) {
                while (L > x0 && pass(L - 1)) --L;
            } else {
                while (!pass(L)) ++L;  // ends at s at the latest
            }
            int R = clampi(floorf(xc + half), s, x1);
            if (pass(R)) {
                while (R < x1 && pass(R + 1)) ++R;
            } else {
                while (!pass(R)) --R;
            }
            const int a = L / T, b = R / T;
            if (hh < 0) {
                hl = a;
                hh = b;
            } else if (a > hh + 1 || b < hl - 1) {
                gap = true;
            } else {
                hl = min(hl, a);
                hh = max(hh, b);
            }
        }
        if (!gap) {
            for (int tx = hl; tx <= hh; ++tx) put(tx, ty);
            cnt += hh >= 0 ? hh - hl + 1 : 0;
            continue;
        }
        for (int tx = tx0; tx <= tx1; ++tx) {
            const int px0 = max(x0, tx * T), px1 = min(x1, tx * T + T - 1);
            bool hit = false;
            for (int py = py0; py <= py1 && !hit; ++py) {
                const float dy = (float)py - E.v;
                for (int px = px0; px <= px1; ++px)
                    if (qpix(E, (float)px - E.u, dy) <= E.t) {
                        hit = true;
                        break;
                    }
            }
            if (hit) {
                put(tx, ty);
                ++cnt;
            }
        }
    }
    return cnt;
}

struct NoPut {
    __device__ __forceinline__ void operator()(int, int) const {}
};

// Tile count of one Gaussian in `mode` (0 when culled).
__device__ __forceinline__ int tile_count(int mode, const Ellipse& E, int radius, const Grid& g) {
    if (mode == GS_MODE_3SIGMA) {
        Rect R;
        if (!sigma3_rect(E.u, E.v, radius, g, R)) return 0;
        return (R.x1 - R.x0 + 1) * (R.y1 - R.y0 + 1);
    }
    Snug S;
    if (!snugbox(E, g, S)) return 0;
    if (mode == GS_MODE_SNUGBOX) return (S.R.x1 - S.R.x0 + 1) * (S.R.y1 - S.R.y0 + 1);
    if (mode == GS_MODE_TBC) return tbc_tiles(E, S, g, NoPut{});
    if (mode == GS_MODE_PIXEL) return pixel_tiles(E, S, g, NoPut{});
    int k, j0, j1;
    bool rows;
    if (accutile_whole_line(S, g, k, j0, j1, rows)) return j1 - j0 + 1;
    return accutile_sweep(E, S, g, NoEmit{});
}

}  // namespace gs
