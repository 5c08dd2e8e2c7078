// CPU oracle for the Speedy-Splat tile rasterizer.
//
// TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, sequential CPU
// implementation of what the rasterizer computes, written from the paper's
// definitions.  Only the test suite, the package's smoke check and the
// benchmark's CPU-baseline leg may load it; the product path never does.  It
// shares no code, header or constant table with the CUDA library.
//
// Precision: every routine is a template over R = float or double.
//   * R = double is the reference of record: libm log/exp, the formulas of
//     Sec. 3.2 and Sec. 4.1 evaluated in FP64.
//   * R = float follows the documented single-precision operation order
//     (left-to-right sums, one rounding per operation, fused multiply-add
//     only where written as fma(), IEEE division and square root, no
//     flush-to-zero).  Built with -ffp-contract=off so the compiler adds no
//     contractions.  In this precision log and exp are the project's own
//     routines (below), so results do not depend on the C library.
//
// Parity status of each function is stated in its comment ("pinned by ...").
// Readings of points where the paper is silent are marked "Reading:".

#include <algorithm>
#include <array>
#include <cmath>
#include <limits>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <vector>

namespace {

// ---------------------------------------------------------------- elementary
// Natural logarithm in single precision by frexp range reduction and the
// atanh series: x = m 2^e with m in [sqrt(1/2), sqrt(2)),
// log x = e ln2 + 2 atanh(s), s = (m - 1)/(m + 1), |s| <= 0.1716, and
// atanh(s)/s = sum_k s^(2k)/(2k+1), truncated after s^10/11 (remainder below
// 1e-10 relative).  ln2 is split Cody-Waite style into hi (15 significant
// bits, so e*hi is exact) + lo.  Pinned by tests against FP64 log (<= 2 ulp).
const float kLn2Hi = 0.693145751953125f;        // round(ln2 * 2^15) / 2^15
const float kLn2Lo = 1.42860682030941723e-06f;  // ln2 - kLn2Hi
const float kSqrtHalf = 0.70710677f;

float log_f32(float x) {
    if (std::isnan(x)) return x;
    if (!(x > 0.0f)) return -INFINITY;
    if (std::isinf(x)) return x;
    int e = 0;
    float m = std::frexp(x, &e);  // x = m * 2^e, m in [0.5, 1)
    if (m < kSqrtHalf) {
        m = m * 2.0f;
        e = e - 1;
    }
    float s = (m - 1.0f) / (m + 1.0f);
    float s2 = s * s;
    float p = 1.0f / 11.0f;
    p = std::fma(p, s2, 1.0f / 9.0f);
    p = std::fma(p, s2, 1.0f / 7.0f);
    p = std::fma(p, s2, 1.0f / 5.0f);
    p = std::fma(p, s2, 1.0f / 3.0f);
    p = std::fma(p, s2, 1.0f);
    float lm = (2.0f * s) * p;
    float fe = static_cast<float>(e);
    return std::fma(fe, kLn2Hi, std::fma(fe, kLn2Lo, lm));
}

// Exponential in single precision: Cody-Waite argument reduction
// x = k ln2 + r, |r| <= ln2/2, then the Taylor polynomial of e^r to degree 7
// in Horner form (truncation error r^8/8! < 6e-9 relative), scaled by 2^k.
// Pinned by tests against FP64 exp (<= 2 ulp).
const float kLog2e = 1.44269502f;

float exp_f32(float x) {
    if (std::isnan(x)) return x;
    if (x < -104.0f) return 0.0f;
    if (x > 89.0f) return INFINITY;
    float k = std::rint(x * kLog2e);
    float r = std::fma(-k, kLn2Hi, x);
    r = std::fma(-k, kLn2Lo, r);
    float p = 1.0f / 5040.0f;
    p = std::fma(p, r, 1.0f / 720.0f);
    p = std::fma(p, r, 1.0f / 120.0f);
    p = std::fma(p, r, 1.0f / 24.0f);
    p = std::fma(p, r, 1.0f / 6.0f);
    p = std::fma(p, r, 0.5f);
    p = std::fma(p, r, 1.0f);
    p = std::fma(p, r, 1.0f);
    return std::ldexp(p, static_cast<int>(k));
}

template <typename R> struct Elem;
template <> struct Elem<double> {
    static double log(double x) { return std::log(x); }
    static double exp(double x) { return std::exp(x); }
};
template <> struct Elem<float> {
    static float log(float x) { return log_f32(x); }
    static float exp(float x) { return exp_f32(x); }
};

template <typename R> R K(double v) { return static_cast<R>(v); }

// ---------------------------------------------------------------- SH basis
// Real spherical harmonics up to degree 3 in the 3D-GS index order
// (l = 0..3, m = -l..l), Condon-Shortley phase kept.  Normalisation constants
// are computed from their closed forms sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) and
// the usual associated-Legendre factors.  Pinned by tests against scipy's
// complex spherical harmonics.
struct ShConst {
    double c0, c1, c2[5], c3[7];
    ShConst() {
        const double pi = 3.14159265358979323846;
        c0 = 0.5 * std::sqrt(1.0 / pi);
        c1 = std::sqrt(3.0 / (4.0 * pi));
        const double a = std::sqrt(15.0 / (4.0 * pi));
        c2[0] = a;
        c2[1] = -a;
        c2[2] = std::sqrt(5.0 / (16.0 * pi));
        c2[3] = -a;
        c2[4] = std::sqrt(15.0 / (16.0 * pi));
        const double b = std::sqrt(35.0 / (32.0 * pi));
        const double c = std::sqrt(21.0 / (32.0 * pi));
        c3[0] = -b;
        c3[1] = std::sqrt(105.0 / (4.0 * pi));
        c3[2] = -c;
        c3[3] = std::sqrt(7.0 / (16.0 * pi));
        c3[4] = -c;
        c3[5] = std::sqrt(105.0 / (16.0 * pi));
        c3[6] = -b;
    }
};
const ShConst kSh;

// Basis values Y[0..15] at the unit direction (x, y, z).
template <typename R> void sh_basis(R x, R y, R z, R Y[16]) {
    Y[0] = K<R>(kSh.c0);
    Y[1] = K<R>(-kSh.c1) * y;
    Y[2] = K<R>(kSh.c1) * z;
    Y[3] = K<R>(-kSh.c1) * x;
    R xx = x * x, yy = y * y, zz = z * z;
    R xy = x * y, yz = y * z, xz = x * z;
    Y[4] = K<R>(kSh.c2[0]) * xy;
    Y[5] = K<R>(kSh.c2[1]) * yz;
    Y[6] = K<R>(kSh.c2[2]) * ((R(2) * zz - xx) - yy);
    Y[7] = K<R>(kSh.c2[3]) * xz;
    Y[8] = K<R>(kSh.c2[4]) * (xx - yy);
    Y[9] = (K<R>(kSh.c3[0]) * y) * (R(3) * xx - yy);
    Y[10] = (K<R>(kSh.c3[1]) * xy) * z;
    Y[11] = (K<R>(kSh.c3[2]) * y) * ((R(4) * zz - xx) - yy);
    Y[12] = (K<R>(kSh.c3[3]) * z) * ((R(2) * zz - R(3) * xx) - R(3) * yy);
    Y[13] = (K<R>(kSh.c3[4]) * x) * ((R(4) * zz - xx) - yy);
    Y[14] = (K<R>(kSh.c3[5]) * z) * (xx - yy);
    Y[15] = (K<R>(kSh.c3[6]) * x) * (xx - R(3) * yy);
}

// ---------------------------------------------------------------- inputs
struct SceneIn {
    int64_t n;
    int sh_degree;
    const float *means, *scales, *rots, *opac, *sh;  // planar SoA
};

template <typename R> struct Cam {
    int width, height;
    R fx, fy, cx, cy, tan_fovx, tan_fovy, near_z;
    R V[3][4];
    R campos[3];
};

template <typename R> Cam<R> make_cam(int width, int height, const float* cf) {
    Cam<R> c;
    c.width = width;
    c.height = height;
    c.fx = cf[0]; c.fy = cf[1]; c.cx = cf[2]; c.cy = cf[3];
    c.tan_fovx = cf[4]; c.tan_fovy = cf[5]; c.near_z = cf[6];
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 4; ++k) c.V[r][k] = cf[7 + 4 * r + k];
    for (int k = 0; k < 3; ++k) c.campos[k] = cf[19 + k];
    return c;
}

// ---------------------------------------------------------------- preprocess
// Per-Gaussian 2D state (Sec. 3.2.1).
template <typename R> struct Proj {
    bool valid = false;
    R u = 0, v = 0, depth = 0, opacity = 0;
    R a = 0, b = 0, c = 0, t = 0;  // conic = Sigma2D^-1 = [[a b][b c]], t = 2 log(255 sigma)
    R rgb[3] = {0, 0, 0};
    R cov[3] = {0, 0, 0};          // dilated Sigma2D: xx, xy, yy
    int32_t radius = 0;            // 3-sigma radius, Eq. (radius)
};

template <typename R> Proj<R> preprocess_one(const SceneIn& s, int64_t i, const Cam<R>& cam) {
    Proj<R> P;
    const int64_t n = s.n;
    R mu[3] = {R(s.means[i]), R(s.means[n + i]), R(s.means[2 * n + i])};
    R sc[3] = {R(s.scales[i]), R(s.scales[n + i]), R(s.scales[2 * n + i])};
    R q[4] = {R(s.rots[i]), R(s.rots[n + i]), R(s.rots[2 * n + i]), R(s.rots[3 * n + i])};
    R sigma = R(s.opac[i]);
    // Reading: non-finite parameters are culled.
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(mu[k]) || !std::isfinite(sc[k])) return P;
    for (int k = 0; k < 4; ++k)
        if (!std::isfinite(q[k])) return P;
    if (!std::isfinite(sigma)) return P;

    // Viewing transform W: p = V[:, :3] mu + V[:, 3].
    R p[3];
    for (int r = 0; r < 3; ++r)
        p[r] = ((cam.V[r][0] * mu[0] + cam.V[r][1] * mu[1]) + cam.V[r][2] * mu[2]) + cam.V[r][3];
    // Reading: near-plane cull at view depth near_z (0.2); no other frustum test.
    if (!(p[2] > cam.near_z)) return P;

    // Perspective projection of the mean (pixel (i, j) at point (i, j)).
    // Reading: quotients by one denominator are products with its reciprocal
    // (1/z here; 1/|q|, 1/det and 1/|mu - campos| below).
    R iz = R(1) / p[2];
    R xz = p[0] * iz;
    R yz = p[1] * iz;
    R u = cam.fx * xz + cam.cx;
    R v = cam.fy * yz + cam.cy;

    // Rotation matrix R_i from the normalised quaternion (w, x, y, z).
    R n2 = ((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]) + q[3] * q[3];
    if (!(n2 > R(0))) return P;
    R nq = std::sqrt(n2);
    R inq = R(1) / nq;
    R w = q[0] * inq, x = q[1] * inq, y = q[2] * inq, z = q[3] * inq;
    R Rm[3][3];
    Rm[0][0] = R(1) - R(2) * (y * y + z * z);
    Rm[0][1] = R(2) * (x * y - w * z);
    Rm[0][2] = R(2) * (x * z + w * y);
    Rm[1][0] = R(2) * (x * y + w * z);
    Rm[1][1] = R(1) - R(2) * (x * x + z * z);
    Rm[1][2] = R(2) * (y * z - w * x);
    Rm[2][0] = R(2) * (x * z - w * y);
    Rm[2][1] = R(2) * (y * z + w * x);
    Rm[2][2] = R(1) - R(2) * (x * x + y * y);

    // Sigma3D = R S S^T R^T = M M^T with M = R S (Sec. 3.2.1).
    R M[3][3];
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) M[r][k] = Rm[r][k] * sc[k];
    R S3[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            S3[r][c] = (M[r][0] * M[c][0] + M[r][1] * M[c][1]) + M[r][2] * M[c][2];

    // Jacobian of the perspective map at the (clamped) mean.
    // Reading: x/z and y/z are clamped to +-1.3 tan(fov) before use (3D-GS).
    R limx = R(1.3) * cam.tan_fovx;
    R limy = R(1.3) * cam.tan_fovy;
    R tx = std::min(limx, std::max(-limx, xz)) * p[2];
    R ty = std::min(limy, std::max(-limy, yz)) * p[2];
    R iz2 = iz * iz;
    R j00 = cam.fx * iz;
    R j02 = -((cam.fx * tx) * iz2);
    R j11 = cam.fy * iz;
    R j12 = -((cam.fy * ty) * iz2);

    // T = J W (2x3); the zero entries of J contribute nothing.
    R T[2][3];
    for (int k = 0; k < 3; ++k) {
        T[0][k] = j00 * cam.V[0][k] + j02 * cam.V[2][k];
        T[1][k] = j11 * cam.V[1][k] + j12 * cam.V[2][k];
    }
    // Sigma2D = T Sigma3D T^T (the 2x2 block of J W Sigma3D W^T J^T).
    R U[2][3];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c)
            U[r][c] = (T[r][0] * S3[0][c] + T[r][1] * S3[1][c]) + T[r][2] * S3[2][c];
    R s00 = (U[0][0] * T[0][0] + U[0][1] * T[0][1]) + U[0][2] * T[0][2];
    R s01 = (U[0][0] * T[1][0] + U[0][1] * T[1][1]) + U[0][2] * T[1][2];
    R s11 = (U[1][0] * T[1][0] + U[1][1] * T[1][1]) + U[1][2] * T[1][2];

    // Reading: low-pass dilation Sigma2D + 0.3 I, no opacity compensation.
    R sxx = s00 + R(0.3);
    R syy = s11 + R(0.3);
    R sxy = s01;
    R det = sxx * syy - sxy * sxy;
    if (!(det > R(0))) return P;
    R idet = R(1) / det;
    R a = syy * idet;
    R b = (-sxy) * idet;
    R c = sxx * idet;
    if (!std::isfinite(u) || !std::isfinite(v) || !std::isfinite(a) || !std::isfinite(b) || !std::isfinite(c))
        return P;

    // Opacity threshold: alpha >= 1/255  <=>  q <= t, t = 2 log(255 sigma) (Sec. 4.1).
    R t = R(2) * Elem<R>::log(R(255) * sigma);

    // 3D-GS radius r = ceil(3 sqrt(lambda_max)) of the dilated Sigma2D (Eq. radius).
    R mid = R(0.5) * (sxx + syy);
    R disc = std::max(R(0.1), mid * mid - det);
    R l1 = mid + std::sqrt(disc);
    R rad = std::ceil(R(3) * std::sqrt(l1));

    // View-dependent colour from W and h (degree <= 3), clamped at 0 after +0.5.
    R d0 = mu[0] - cam.campos[0], d1 = mu[1] - cam.campos[1], d2 = mu[2] - cam.campos[2];
    R len = std::sqrt((d0 * d0 + d1 * d1) + d2 * d2);
    R ilen = R(1) / len;
    R Y[16];
    sh_basis<R>(d0 * ilen, d1 * ilen, d2 * ilen, Y);
    int nc = (s.sh_degree + 1) * (s.sh_degree + 1);
    for (int ch = 0; ch < 3; ++ch) {
        R acc = Y[0] * R(s.sh[(0 * 3 + ch) * n + i]);
        for (int k = 1; k < nc; ++k) acc = acc + Y[k] * R(s.sh[(k * 3 + ch) * n + i]);
        acc = acc + R(0.5);
        P.rgb[ch] = std::max(acc, R(0));
    }

    P.valid = true;
    P.u = u; P.v = v; P.depth = p[2]; P.opacity = sigma;
    P.a = a; P.b = b; P.c = c; P.t = t;
    P.cov[0] = sxx; P.cov[1] = sxy; P.cov[2] = syy;
    P.radius = (rad >= R(0) && rad < R(1 << 30)) ? static_cast<int32_t>(rad) : (1 << 30);
    return P;
}

// ---------------------------------------------------------------- tile sets
struct Grid {
    int T;       // tile edge in pixels
    int gx, gy;  // tiles per row / column
    int W = 0, H = 0;  // image size in pixels (0: gx T by gy T)
    int width() const { return W > 0 ? W : gx * T; }
    int height() const { return H > 0 ? H : gy * T; }
};


inline int clamp_floor(double v, int lo, int hi) {
    // floor(v) clamped to [lo, hi], evaluated without overflowing int.
    double f = std::floor(v);
    if (!(f >= lo)) return lo;  // also maps NaN to lo
    if (f > hi) return hi;
    return static_cast<int>(f);
}

// 3D-GS rectangle (Fig. 2a): min = trunc((mu - r)/T), max_excl = trunc((mu + r + T - 1)/T),
// both clamped to [0, G].  Reading: kept verbatim as the paper's baseline.
template <typename R, typename Emit> int64_t sigma3_tiles(const Proj<R>& P, const Grid& g, Emit&& emit) {
    if (!P.valid) return 0;
    const R T = R(g.T);
    const R r = R(P.radius);
    auto tr = [](R x, int G) {
        if (!(x > R(0))) return 0;
        if (x >= R(G)) return G;
        return static_cast<int>(x);  // truncation toward zero
    };
    int x0 = tr((P.u - r) / T, g.gx);
    int x1 = tr((P.u + r + (T - R(1))) / T, g.gx);
    int y0 = tr((P.v - r) / T, g.gy);
    int y1 = tr((P.v + r + (T - R(1))) / T, g.gy);
    int64_t cnt = int64_t(x1 - x0) * int64_t(y1 - y0);
    if (cnt <= 0) return 0;
    for (int ty = y0; ty < y1; ++ty)
        for (int tx = x0; tx < x1; ++tx) emit(tx, ty);
    return cnt;
}

// SnugBox (Sec. 4.1.1): axis-aligned bounding box of the ellipse
// a xd^2 + 2 b xd yd + c yd^2 = t.  Substituting x_args (Eq. bbox_args) into
// Eq. ellipse_intersect gives the half-extents hy = sqrt(t a / D),
// hx = sqrt(t c / D), D = a c - b^2.
template <typename R> struct Snug {
    bool ok = false;
    R D, hx, hy, x0, x1, y0, y1;
    int tx0, tx1, ty0, ty1;  // inclusive tile rectangle (Reading: floor, clamp, empty if outside)
};

template <typename R> Snug<R> snugbox(const Proj<R>& P, const Grid& g) {
    Snug<R> S;
    if (!P.valid || !(P.t > R(0))) return S;
    R D = P.a * P.c - P.b * P.b;
    if (!(D > R(0))) return S;
    S.D = D;
    S.hx = std::sqrt((P.t * P.c) / D);
    S.hy = std::sqrt((P.t * P.a) / D);
    S.x0 = P.u - S.hx;
    S.x1 = P.u + S.hx;
    S.y0 = P.v - S.hy;
    S.y1 = P.v + S.hy;
    const R T = R(g.T);
    if (!(S.x1 >= R(0)) || !(S.y1 >= R(0)) || !(S.x0 < R(g.gx) * T) || !(S.y0 < R(g.gy) * T)) return S;
    S.tx0 = clamp_floor(double(S.x0 / T), 0, g.gx - 1);
    S.tx1 = clamp_floor(double(S.x1 / T), 0, g.gx - 1);
    S.ty0 = clamp_floor(double(S.y0 / T), 0, g.gy - 1);
    S.ty1 = clamp_floor(double(S.y1 / T), 0, g.gy - 1);
    S.ok = true;
    return S;
}

template <typename R, typename Emit> int64_t snugbox_tiles(const Proj<R>& P, const Grid& g, Emit&& emit) {
    Snug<R> S = snugbox(P, g);
    if (!S.ok) return 0;
    for (int ty = S.ty0; ty <= S.ty1; ++ty)
        for (int tx = S.tx0; tx <= S.tx1; ++tx) emit(tx, ty);
    return int64_t(S.tx1 - S.tx0 + 1) * int64_t(S.ty1 - S.ty0 + 1);
}

// AccuTile (Sec. 4.1.2, Algorithm 1): sweep the shorter side of the SnugBox
// tile rectangle.  Written for rows; columns are the mirror image (x <-> y,
// a <-> c), as App. A.1 states.  For each row the ellipse's extent is taken
// from the SnugBox extreme point if it lies inside the row, otherwise from
// the intersections of the ellipse with the row's two boundary lines
// (Eq. ellipse_intersect), each boundary line intersected once and reused by
// the next row.
//
// Readings: a boundary line is intersected only if it lies within the
// SnugBox span (Algorithm 1's "line >= B_b" / "line <= B_t" tests); the
// discriminant is clamped at 0 near tangency; "point in row r" means its
// coordinate lies in [rT, (r+1)T); a row left with neither an extreme point
// nor a boundary intersection (possible only through rounding) falls back
// to the SnugBox edge; tile indices are floor(x/T) clamped to the SnugBox
// rectangle, and a row whose extent lies entirely beyond that rectangle's
// tile span (only possible when the rectangle was clipped at the image edge)
// contributes no tiles.
//
// dir: 0 = shorter side, 1 = rows, 2 = columns.
template <typename R, typename Emit>
int64_t accutile_tiles(const Proj<R>& P, const Grid& g, int dir, Emit&& emit) {
    Snug<R> S = snugbox(P, g);
    if (!S.ok) return 0;
    const R T = R(g.T);
    bool rows = (dir == 1) || (dir == 0 && (S.ty1 - S.ty0) <= (S.tx1 - S.tx0));
    // Swept axis s, extent axis e.  For rows: s = y, e = x.
    const R ms = rows ? P.v : P.u;       // centre on the swept axis
    const R me = rows ? P.u : P.v;       // centre on the extent axis
    const R as = rows ? P.a : P.c;       // coefficient of the extent-axis square
    const R cs = rows ? P.c : P.a;       // coefficient of the swept-axis square
    const R s_lo = rows ? S.y0 : S.x0;   // SnugBox span on the swept axis
    const R s_hi = rows ? S.y1 : S.x1;
    const R e_lo = rows ? S.x0 : S.y0;   // SnugBox span on the extent axis
    const R e_hi = rows ? S.x1 : S.y1;
    const R h_e = rows ? S.hx : S.hy;
    const int k0 = rows ? S.ty0 : S.tx0, k1 = rows ? S.ty1 : S.tx1;  // swept tile range
    const int j0 = rows ? S.tx0 : S.ty0, j1 = rows ? S.tx1 : S.ty1;  // extent tile range
    // Extreme points along the extent axis (SnugBox min/max points):
    // at e = me -+ h_e the swept coordinate is ms +- (b / cs) h_e.
    const R bc = P.b / cs;
    const R pmin_s = ms + bc * h_e;  // swept coordinate of the minimum-extent point
    const R pmax_s = ms - bc * h_e;  // swept coordinate of the maximum-extent point
    // Intersections of the line (swept coordinate = L) with the ellipse.
    auto isect = [&](R L, R& lo, R& hi) {
        R d = L - ms;
        R disc = as * P.t - (S.D * d) * d;
        if (disc < R(0)) disc = R(0);
        R sq = std::sqrt(disc);
        R nb = (-P.b) * d;
        lo = me + (nb - sq) / as;
        hi = me + (nb + sq) / as;
    };
    int64_t cnt = 0;
    R lo_l = 0, lo_r = 0;
    bool have_lo = false;
    R Llo = R(k0) * T;
    if (Llo >= s_lo) {
        isect(Llo, lo_l, lo_r);
        have_lo = true;
    }
    for (int k = k0; k <= k1; ++k) {
        R rlo = R(k) * T;
        R rhi = R(k + 1) * T;
        R hi_l = 0, hi_r = 0;
        bool have_hi = false;
        if (rhi <= s_hi) {
            isect(rhi, hi_l, hi_r);
            have_hi = true;
        }
        R emin, emax;
        if (pmin_s >= rlo && pmin_s < rhi) emin = e_lo;
        else if (have_lo && have_hi) emin = std::min(lo_l, hi_l);
        else if (have_lo) emin = lo_l;
        else if (have_hi) emin = hi_l;
        else emin = e_lo;
        if (pmax_s >= rlo && pmax_s < rhi) emax = e_hi;
        else if (have_lo && have_hi) emax = std::max(lo_r, hi_r);
        else if (have_lo) emax = lo_r;
        else if (have_hi) emax = hi_r;
        else emax = e_hi;
        // Convert: tile index floor(e/T).  A row whose extent lies wholly
        // outside the rectangle's tile span contributes nothing (clamping it
        // would add a tile the ellipse does not touch); otherwise clamp.
        double fmin = std::floor(double(emin / T));
        double fmax = std::floor(double(emax / T));
        int jmin = clamp_floor(double(emin / T), j0, j1);
        int jmax = clamp_floor(double(emax / T), j0, j1);
        if (fmin <= double(j1) && fmax >= double(j0) && jmax >= jmin) {
            cnt += jmax - jmin + 1;
            for (int j = jmin; j <= jmax; ++j) {
                if (rows) emit(j, k);
                else emit(k, j);
            }
        }
        lo_l = hi_l;
        lo_r = hi_r;
        have_lo = have_hi;
    }
    return cnt;
}

// q at offset (dx, dy) from the centre, in the blend's operation order
// (render, Sec. 3.2.3): fma(dx, fma(a, dx, (2b) dy), (c dy) dy).
template <typename R> R qpix(const Proj<R>& P, R dx, R dy) {
    return std::fma(dx, std::fma(P.a, dx, (P.b + P.b) * dy), (P.c * dy) * dy);
}

// StopThePop tile-based culling (the paper's App. A.4 ablation; described
// there, not printed).  Candidate tiles are those of an opacity-aware box
// (Reading: the SnugBox rectangle); each candidate is kept iff the
// Gaussian's alpha reaches 1/255 somewhere on the tile's closed square, i.e.
// the minimum of q over [kx T, (kx+1) T] x [ky T, (ky+1) T] is <= t.  Reading
// of the minimum: 0 if the centre lies in the square; otherwise the minimum
// of this convex form lies on a face of the square facing the centre, and
// along a face dx = X it is at dy = clamp(-b X / c) (symmetrically for a face
// dy = Y); at most two faces face the centre.
template <typename R> bool tile_reaches(const Proj<R>& P, R X0, R X1, R Y0, R Y1) {
    const R dx0 = X0 - P.u, dx1 = X1 - P.u;
    const R dy0 = Y0 - P.v, dy1 = Y1 - P.v;
    const bool outx = dx0 > R(0) || dx1 < R(0);
    const bool outy = dy0 > R(0) || dy1 < R(0);
    if (!outx && !outy) return true;  // q = 0 <= t
    R qmin = std::numeric_limits<R>::infinity();
    if (outx) {
        const R X = dx0 > R(0) ? dx0 : dx1;
        const R d = std::min(std::max(((-P.b) * X) / P.c, dy0), dy1);
        qmin = std::min(qmin, qpix(P, X, d));
    }
    if (outy) {
        const R Y = dy0 > R(0) ? dy0 : dy1;
        const R d = std::min(std::max(((-P.b) * Y) / P.a, dx0), dx1);
        qmin = std::min(qmin, qpix(P, d, Y));
    }
    return qmin <= P.t;
}

template <typename R, typename Emit> int64_t tbc_tiles(const Proj<R>& P, const Grid& g, Emit&& emit) {
    Snug<R> S = snugbox(P, g);
    if (!S.ok) return 0;
    const R T = R(g.T);
    int64_t cnt = 0;
    for (int ty = S.ty0; ty <= S.ty1; ++ty)
        for (int tx = S.tx0; tx <= S.tx1; ++tx)
            if (tile_reaches(P, R(tx) * T, R(tx + 1) * T, R(ty) * T, R(ty + 1) * T)) {
                emit(tx, ty);
                ++cnt;
            }
    return cnt;
}

// Pixel-exact tiles (the tile-set contract "tiles holding a pixel with
// alpha >= 1/255" made literal): tile (tx, ty) is kept iff one of its pixels
// inside the image has q <= t, with q evaluated exactly as the blend
// evaluates it.  Written as its definition: every pixel of the SnugBox,
// widened by one pixel on each side (so that rounding in the box can never
// hide a pixel the blend would take), is tested.
template <typename R, typename Emit> int64_t pixel_tiles(const Proj<R>& P, const Grid& g, Emit&& emit) {
    Snug<R> S = snugbox(P, g);
    if (!S.ok) return 0;
    const int W = g.width(), H = g.height();
    // floor(edge) -+ 1, clamped to the image (in double, so any float fits)
    auto lo_px = [](double e, int n) { const double f = std::floor(e) - 1.0; return f < 0.0 ? 0 : (f > n ? n : int(f)); };
    auto hi_px = [](double e, int n) { const double f = std::floor(e) + 1.0; return f < 0.0 ? -1 : (f > n - 1 ? n - 1 : int(f)); };
    const int x0 = lo_px(double(S.x0), W), x1 = hi_px(double(S.x1), W);
    const int y0 = lo_px(double(S.y0), H), y1 = hi_px(double(S.y1), H);
    if (x0 > x1 || y0 > y1) return 0;
    const int tx0 = x0 / g.T, tx1 = x1 / g.T, ty0 = y0 / g.T, ty1 = y1 / g.T;
    std::vector<uint8_t> hit(size_t(tx1 - tx0 + 1) * size_t(ty1 - ty0 + 1), 0);
    for (int py = y0; py <= y1; ++py)
        for (int px = x0; px <= x1; ++px)
            if (qpix(P, R(px) - P.u, R(py) - P.v) <= P.t)
                hit[size_t(py / g.T - ty0) * size_t(tx1 - tx0 + 1) + size_t(px / g.T - tx0)] = 1;
    int64_t cnt = 0;
    for (int ty = ty0; ty <= ty1; ++ty)
        for (int tx = tx0; tx <= tx1; ++tx)
            if (hit[size_t(ty - ty0) * size_t(tx1 - tx0 + 1) + size_t(tx - tx0)]) {
                emit(tx, ty);
                ++cnt;
            }
    return cnt;
}

template <typename R, typename Emit>
int64_t mode_tiles(int mode, const Proj<R>& P, const Grid& g, Emit&& emit) {
    if (mode == 0) return sigma3_tiles(P, g, emit);
    if (mode == 1) return snugbox_tiles(P, g, emit);
    if (mode == 3) return tbc_tiles(P, g, emit);
    if (mode == 4) return pixel_tiles(P, g, emit);
    return accutile_tiles(P, g, 0, emit);
}

// Brute-force continuous-exact tile set (FP64 only): tile (kx, ky) belongs
// to the Gaussian iff the minimum of q over the closed square
// [kx T, (kx+1) T] x [ky T, (ky+1) T] is <= t.  The minimum of a positive
// definite quadratic over a box is 0 if the centre is inside, otherwise it
// lies on an edge, where q restricted to the edge is a parabola minimised by
// clamping its vertex into the edge.
double qform(double a, double b, double c, double xd, double yd) {
    return a * xd * xd + 2.0 * b * xd * yd + c * yd * yd;
}
double min_q_on_box(double u, double v, double a, double b, double c, double X0, double X1, double Y0, double Y1) {
    if (u >= X0 && u <= X1 && v >= Y0 && v <= Y1) return 0.0;
    double best = INFINITY;
    for (double X : {X0, X1}) {  // vertical edges: minimise over y
        double xd = X - u;
        double yd = -(b / c) * xd;
        double y = std::min(Y1, std::max(Y0, v + yd));
        best = std::min(best, qform(a, b, c, xd, y - v));
    }
    for (double Y : {Y0, Y1}) {  // horizontal edges: minimise over x
        double yd = Y - v;
        double xd = -(b / a) * yd;
        double x = std::min(X1, std::max(X0, u + xd));
        best = std::min(best, qform(a, b, c, x - u, yd));
    }
    return best;
}

// ---------------------------------------------------------------- blend
// Front-to-back compositing of one pixel over an ordered list (Eqs.
// render_alpha, 2d_gaussian_scalar, contribution).
// Readings: the inclusion test alpha >= 1/255 is evaluated as q <= t (the
// same numbers that drive SnugBox/AccuTile); alpha = min(0.99, sigma g);
// stop before adding a Gaussian that would drive T below 1e-4; background
// added as T * bg.
//   dx = px - u, dy = py - v, e = (2b) dy, f = (c dy) dy,
//   q = fma(dx, fma(a, dx, e), f)
template <typename R> struct Pixel {
    R C[3] = {0, 0, 0};
    R T = R(1);
    uint32_t last = 0;
    uint32_t contributed = 0;  // Gaussians that added to C
};

template <typename R>
bool blend_step(Pixel<R>& px, const Proj<R>& P, R pxf, R pyf, uint32_t pos) {
    // returns false when the pixel is finished (stop rule hit)
    R dx = pxf - P.u;
    R dy = pyf - P.v;
    R e = (P.b + P.b) * dy;
    R f = (P.c * dy) * dy;
    R q = std::fma(dx, std::fma(P.a, dx, e), f);
    if (!(q <= P.t)) return true;
    R g = Elem<R>::exp(R(-0.5) * q);
    R alpha = std::min(R(0.99), P.opacity * g);
    R Tn = px.T * (R(1) - alpha);
    if (Tn < R(1e-4)) return false;
    R w = alpha * px.T;
    for (int ch = 0; ch < 3; ++ch) px.C[ch] = std::fma(P.rgb[ch], w, px.C[ch]);
    px.T = Tn;
    px.last = pos;
    px.contributed += 1;
    return true;
}

// ---------------------------------------------------------------- pipelines
// (With -fopenmp the independent per-Gaussian and per-pixel-row loops below
// run on all host cores; the arithmetic and every result are the same.)
template <typename R> std::vector<Proj<R>> preprocess_all(const SceneIn& s, const Cam<R>& cam) {
    std::vector<Proj<R>> out(static_cast<size_t>(s.n));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < s.n; ++i) out[i] = preprocess_one<R>(s, i, cam);
    return out;
}

Grid make_grid(int width, int height, int T) {
    Grid g;
    g.T = T;
    g.gx = (width + T - 1) / T;
    g.gy = (height + T - 1) / T;
    g.W = width;
    g.H = height;
    return g;
}

template <typename R>
int render_impl(const SceneIn& s, int width, int height, const float* camf, int tile, int mode, const float* bg,
                int64_t key_cap, uint64_t* keys_unsorted, uint32_t* vals_unsorted, uint64_t* keys_sorted,
                uint32_t* vals_sorted, int64_t* num_keys, uint32_t* ranges, double* image, double* final_T,
                uint32_t* last, int64_t* pair_counts) {
    Cam<R> cam = make_cam<R>(width, height, camf);
    Grid g = make_grid(width, height, tile);
    std::vector<Proj<R>> P = preprocess_all<R>(s, cam);
    // Count (preprocess) and emit (duplicateWithKeys), Sec. 3.2.2: keys in
    // Gaussian-id order; key = tile index in the high 32 bits, depth bits low.
    std::vector<uint64_t> keys;
    std::vector<uint32_t> vals;
    for (int64_t i = 0; i < s.n; ++i) {
        float depth_f = static_cast<float>(P[i].depth);
        uint32_t dbits;
        std::memcpy(&dbits, &depth_f, 4);
        mode_tiles<R>(mode, P[i], g, [&](int tx, int ty) {
            uint64_t tid = uint64_t(ty) * uint64_t(g.gx) + uint64_t(tx);
            keys.push_back((tid << 32) | uint64_t(dbits));
            vals.push_back(static_cast<uint32_t>(i));
        });
    }
    int64_t K = static_cast<int64_t>(keys.size());
    *num_keys = K;
    if (K > key_cap) return 3;
    for (int64_t k = 0; k < K; ++k) {
        keys_unsorted[k] = keys[k];
        vals_unsorted[k] = vals[k];
    }
    // RadixSort equivalent: stable sort by key, ties keep emission order.
    std::vector<int64_t> order(static_cast<size_t>(K));
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) { return keys[x] < keys[y]; });
    for (int64_t k = 0; k < K; ++k) {
        keys_sorted[k] = keys[order[k]];
        vals_sorted[k] = vals[order[k]];
    }
    // identifyTileRanges: [start, end) per tile, empty tiles [0, 0).
    const int64_t G = int64_t(g.gx) * g.gy;
    for (int64_t t = 0; t < 2 * G; ++t) ranges[t] = 0;
    for (int64_t k = 0; k < K; ++k) {
        uint32_t tid = static_cast<uint32_t>(keys_sorted[k] >> 32);
        if (k == 0 || static_cast<uint32_t>(keys_sorted[k - 1] >> 32) != tid) ranges[2 * tid] = uint32_t(k);
        if (k == K - 1 || static_cast<uint32_t>(keys_sorted[k + 1] >> 32) != tid) ranges[2 * tid + 1] = uint32_t(k + 1);
    }
    // render: each pixel walks its tile's list front to back.  pair_counts
    // (nullable) receives the pairs the walk evaluates (every entry up to and
    // including the one that stops the pixel) and the pairs that add colour.
    const int64_t HW = int64_t(width) * height;
    int64_t evaluated = 0, contributed = 0;
#pragma omp parallel for schedule(dynamic, 2) reduction(+ : evaluated, contributed)
    for (int py = 0; py < height; ++py) {
        for (int px = 0; px < width; ++px) {
            int64_t tid = int64_t(py / tile) * g.gx + (px / tile);
            uint32_t start = ranges[2 * tid], end = ranges[2 * tid + 1];
            Pixel<R> pix;
            uint32_t k = start;
            for (; k < end; ++k) {
                if (!blend_step<R>(pix, P[vals_sorted[k]], R(px), R(py), k - start + 1)) {
                    ++k;  // the stopping entry was evaluated too
                    break;
                }
            }
            evaluated += k - start;
            contributed += pix.contributed;
            int64_t o = int64_t(py) * width + px;
            for (int ch = 0; ch < 3; ++ch) image[ch * HW + o] = double(std::fma(pix.T, R(bg[ch]), pix.C[ch]));
            final_T[o] = double(pix.T);
            last[o] = pix.last;
        }
    }
    if (pair_counts) {
        pair_counts[0] = evaluated;
        pair_counts[1] = contributed;
    }
    return 0;
}

// Tile-free image: every pixel scans all Gaussians in (depth, id) order.
// This is the plain definition of Eq. contribution and does not depend on any
// tile mode; used to check that a mode's tile lists lose nothing.
template <typename R>
void render_notile_impl(const SceneIn& s, int width, int height, const float* camf, const float* bg, double* image,
                        double* final_T, int literal_exp, int64_t* decisions_differ) {
    Cam<R> cam = make_cam<R>(width, height, camf);
    std::vector<Proj<R>> P = preprocess_all<R>(s, cam);
    std::vector<int64_t> order;
    for (int64_t i = 0; i < s.n; ++i)
        if (P[i].valid) order.push_back(i);
    std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) {
        float dx = float(P[x].depth), dy = float(P[y].depth);
        return dx < dy;
    });
    const int64_t HW = int64_t(width) * height;
    int64_t differ = 0;
    for (int py = 0; py < height; ++py) {
        for (int px = 0; px < width; ++px) {
            Pixel<R> pix;
            R pxf = R(px), pyf = R(py);
            uint32_t pos = 0;
            for (int64_t idx : order) {
                const Proj<R>& G = P[idx];
                ++pos;
                if (literal_exp) {
                    // Literal test of Eq. render_alpha: sigma exp(-q/2) >= 1/255.
                    R dx = pxf - G.u, dy = pyf - G.v;
                    R q = G.a * dx * dx + R(2) * G.b * dx * dy + G.c * dy * dy;
                    bool lit = G.opacity * Elem<R>::exp(R(-0.5) * q) >= R(1) / R(255);
                    bool thr = q <= G.t;
                    if (lit != thr) ++differ;
                }
                if (!blend_step<R>(pix, G, pxf, pyf, pos)) break;
            }
            int64_t o = int64_t(py) * width + px;
            for (int ch = 0; ch < 3; ++ch) image[ch * HW + o] = double(std::fma(pix.T, R(bg[ch]), pix.C[ch]));
            final_T[o] = double(pix.T);
        }
    }
    if (decisions_differ) *decisions_differ = differ;
}

// ---------------------------------------------------------------- backward
// Gradients of L = sum_p sum_ch dL/dC_ch(p) C_ch(p) with respect to every
// Gaussian parameter (Sec. 4.2: the render backward aggregates per-pixel
// gradients into the 2D parameters, then a per-Gaussian pass carries them to
// mu, s, r, h, sigma).  Also the efficient pruning score (Sec. 4.2.1):
// score_i = sum_p sum_ch (dC_ch(p) / dg_i(p))^2, with dC/dg = sigma dC/dalpha
// where alpha = sigma g is not clamped at 0.99, else 0.  Threshold, stop and
// clamp decisions are held fixed (they are piecewise constant).
//
// Blend part, per pixel: with contributors i in front-to-back order,
// transmittance T_i before i and T_f after the last,
//   dC/dc_i = alpha_i T_i,
//   dC/dalpha_i = T_i (c_i - B_i),  B_last = bg,  B_{i-1} = alpha_i c_i + (1 - alpha_i) B_i,
// (B_i is the colour behind i seen through i's hole), then
//   dalpha/dsigma = g, dalpha/dg = sigma, dg/dq = -g/2,
//   q = a dx^2 + 2 b dx dy + c dy^2, dx = px - u, dy = py - v.
struct Grad2D {
    double u = 0, v = 0, a = 0, b = 0, c = 0, sigma = 0, rgb[3] = {0, 0, 0}, score = 0;
};

template <typename R> struct Contrib {
    uint32_t idx;
    R alpha, g, T, q, dx, dy;
    bool clamped;
};

void blend_backward_pixel(const std::vector<Proj<double>>& P, const uint32_t* list, uint32_t len, double pxf,
                          double pyf, const double* G, const float* bg, std::vector<Grad2D>& acc) {
    // forward replay (records each contributor's alpha and T)
    std::vector<Contrib<double>> cs;
    double T = 1.0;
    for (uint32_t k = 0; k < len; ++k) {
        const Proj<double>& g = P[list[k]];
        double dx = pxf - g.u, dy = pyf - g.v;
        double q = std::fma(dx, std::fma(g.a, dx, (g.b + g.b) * dy), (g.c * dy) * dy);
        if (!(q <= g.t)) continue;
        double gg = std::exp(-0.5 * q);
        double raw = g.opacity * gg;
        double alpha = std::min(0.99, raw);
        double Tn = T * (1.0 - alpha);
        if (Tn < 1e-4) break;
        cs.push_back({list[k], alpha, gg, T, q, dx, dy, raw > 0.99});
        T = Tn;
    }
    double B[3] = {bg[0], bg[1], bg[2]};
    for (size_t m = cs.size(); m-- > 0;) {
        const Contrib<double>& e = cs[m];
        const Proj<double>& g = P[e.idx];
        Grad2D& A = acc[e.idx];
        double dC_dalpha[3], dL_dalpha = 0.0;
        for (int ch = 0; ch < 3; ++ch) {
            dC_dalpha[ch] = e.T * (g.rgb[ch] - B[ch]);
            dL_dalpha += G[ch] * dC_dalpha[ch];
            A.rgb[ch] += G[ch] * e.alpha * e.T;
        }
        if (!e.clamped) {
            A.sigma += dL_dalpha * e.g;
            double dL_dq = dL_dalpha * g.opacity * (-0.5 * e.g);
            A.a += dL_dq * e.dx * e.dx;
            A.b += dL_dq * 2.0 * e.dx * e.dy;
            A.c += dL_dq * e.dy * e.dy;
            A.u += dL_dq * (-2.0 * g.a * e.dx - 2.0 * g.b * e.dy);
            A.v += dL_dq * (-2.0 * g.b * e.dx - 2.0 * g.c * e.dy);
            for (int ch = 0; ch < 3; ++ch) {
                double dCdg = g.opacity * dC_dalpha[ch];
                A.score += dCdg * dCdg;
            }
        }
        for (int ch = 0; ch < 3; ++ch) B[ch] = e.alpha * g.rgb[ch] + (1.0 - e.alpha) * B[ch];
    }
}

// PUP sensitivity (Sec. 4.2, Eq. pup_score), FP64, one view added to
// hess[21][n] (row-major upper triangle of the symmetric 6 x 6 block over
// mu_x mu_y mu_z s_0 s_1 s_2).  Reading: the image's gradient with respect
// to (mu_i, s_i) is taken through the 2D Gaussian value g_i(p), with the
// colour's view dependence held fixed:
//   grad C_ch(p) = dC_ch/dg_i * grad_{mu,s} g_i(p),
// dC_ch/dg_i = sigma_i T_i (c_i,ch - B_ch) from the back-to-front walk of the
// backward (zero where alpha is clamped at 0.99), and grad_{mu,s} g_i(p) =
// J_i^T dg/d(u, v, a, b, c), where J_i, the Jacobian of (u, v, a, b, c) with
// respect to (mu, s), is taken by central differences of this file's own
// forward projection (steps h and h/2 on the float parameter, Richardson
// extrapolated), not by the analytic chain.
void pup_jacobian_fd(const SceneIn& s, int64_t i, const Cam<double>& cam, double J[5][6]) {
    float mu[3] = {s.means[i], s.means[s.n + i], s.means[2 * s.n + i]};
    float sc[3] = {s.scales[i], s.scales[s.n + i], s.scales[2 * s.n + i]};
    float q[4] = {s.rots[i], s.rots[s.n + i], s.rots[2 * s.n + i], s.rots[3 * s.n + i]};
    float op = s.opac[i];
    float sh[48];
    for (int k = 0; k < 48; ++k) sh[k] = 0.0f;
    auto state = [&](double out[5]) {
        float m3[3] = {mu[0], mu[1], mu[2]};
        SceneIn one{1, 0, m3, sc, q, &op, sh};
        Proj<double> P = preprocess_one<double>(one, 0, cam);
        out[0] = P.u; out[1] = P.v; out[2] = P.a; out[3] = P.b; out[4] = P.c;
    };
    for (int j = 0; j < 6; ++j) {
        float* x = j < 3 ? &mu[j] : &sc[j - 3];
        const float x0 = *x;
        const double h = std::max(std::fabs(double(x0)) * 1e-3, 1e-5);
        double d[2][5];
        for (int r = 0; r < 2; ++r) {
            const double step = r == 0 ? h : h / 2;
            double fp[5], fm[5];
            *x = float(double(x0) + step);
            const double xp = *x;
            state(fp);
            *x = float(double(x0) - step);
            const double xm = *x;
            state(fm);
            *x = x0;
            for (int k = 0; k < 5; ++k) d[r][k] = (fp[k] - fm[k]) / (xp - xm);
        }
        for (int k = 0; k < 5; ++k) J[k][j] = (4.0 * d[1][k] - d[0][k]) / 3.0;
    }
}

void pup_view(const SceneIn& s, int width, int height, const float* camf, int tile, int mode, const float* bg,
              double* hess) {
    const int64_t n = s.n;
    Cam<double> cam = make_cam<double>(width, height, camf);
    Grid g = make_grid(width, height, tile);
    std::vector<Proj<double>> P = preprocess_all<double>(s, cam);
    std::vector<uint64_t> keys;
    std::vector<uint32_t> vals;
    for (int64_t i = 0; i < n; ++i) {
        float depth_f = static_cast<float>(P[i].depth);
        uint32_t dbits;
        std::memcpy(&dbits, &depth_f, 4);
        mode_tiles<double>(mode, P[i], g, [&](int tx, int ty) {
            keys.push_back(((uint64_t(ty) * uint64_t(g.gx) + uint64_t(tx)) << 32) | uint64_t(dbits));
            vals.push_back(static_cast<uint32_t>(i));
        });
    }
    std::vector<int64_t> order(keys.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return keys[a] < keys[b]; });
    std::vector<std::vector<uint32_t>> lists(size_t(g.gx) * size_t(g.gy));
    for (int64_t k : order) lists[keys[k] >> 32].push_back(vals[k]);
    std::vector<std::array<double, 30>> J(static_cast<size_t>(n));
    std::vector<char> haveJ(size_t(n), 0);
    for (int py = 0; py < height; ++py)
        for (int px = 0; px < width; ++px) {
            const auto& L = lists[size_t(py / tile) * size_t(g.gx) + size_t(px / tile)];
            std::vector<Contrib<double>> cs;
            double T = 1.0;
            for (uint32_t id : L) {
                const Proj<double>& G = P[id];
                double dx = px - G.u, dy = py - G.v;
                double q = std::fma(dx, std::fma(G.a, dx, (G.b + G.b) * dy), (G.c * dy) * dy);
                if (!(q <= G.t)) continue;
                double gg = std::exp(-0.5 * q);
                double raw = G.opacity * gg;
                double alpha = std::min(0.99, raw);
                double Tn = T * (1.0 - alpha);
                if (Tn < 1e-4) break;
                cs.push_back({id, alpha, gg, T, q, dx, dy, raw > 0.99});
                T = Tn;
            }
            double B[3] = {bg[0], bg[1], bg[2]};
            for (size_t m = cs.size(); m-- > 0;) {
                const Contrib<double>& e = cs[m];
                const Proj<double>& G = P[e.idx];
                if (!e.clamped) {
                    double w = 0.0;
                    for (int ch = 0; ch < 3; ++ch) {
                        const double dCdg = G.opacity * e.T * (G.rgb[ch] - B[ch]);
                        w += dCdg * dCdg;
                    }
                    if (!haveJ[e.idx]) {
                        double Jm[5][6];
                        pup_jacobian_fd(s, e.idx, cam, Jm);
                        for (int k = 0; k < 30; ++k) J[e.idx][k] = Jm[k / 6][k % 6];
                        haveJ[e.idx] = 1;
                    }
                    // dg/d(u, v, a, b, c) at this pixel
                    const double hg = -0.5 * e.g;
                    const double g5[5] = {hg * (-2.0 * (G.a * e.dx + G.b * e.dy)), hg * (-2.0 * (G.b * e.dx + G.c * e.dy)),
                                          hg * e.dx * e.dx, hg * 2.0 * e.dx * e.dy, hg * e.dy * e.dy};
                    double g6[6];
                    for (int j = 0; j < 6; ++j) {
                        g6[j] = 0.0;
                        for (int k = 0; k < 5; ++k) g6[j] += J[e.idx][k * 6 + j] * g5[k];
                    }
                    int el = 0;
                    for (int a = 0; a < 6; ++a)
                        for (int b = a; b < 6; ++b) hess[int64_t(el++) * n + e.idx] += w * g6[a] * g6[b];
                }
                for (int ch = 0; ch < 3; ++ch) B[ch] = e.alpha * G.rgb[ch] + (1.0 - e.alpha) * B[ch];
            }
        }
}

// Derivatives of the SH basis (in the order of sh_basis) with respect to
// the unit direction (x, y, z): dY[k][0..2].
void sh_basis_grad(double x, double y, double z, double dY[16][3]) {
    const double C1 = kSh.c1, A2 = kSh.c2[0], C2 = kSh.c2[2], E2 = kSh.c2[4];
    const double A3 = -kSh.c3[0], B3 = kSh.c3[1], C3 = -kSh.c3[2], D3 = kSh.c3[3], F3 = kSh.c3[5];
    const double xx = x * x, yy = y * y, zz = z * z;
    double g[16][3] = {
        {0, 0, 0},
        {0, -C1, 0},
        {0, 0, C1},
        {-C1, 0, 0},
        {A2 * y, A2 * x, 0},
        {0, -A2 * z, -A2 * y},
        {-2 * C2 * x, -2 * C2 * y, 4 * C2 * z},
        {-A2 * z, 0, -A2 * x},
        {2 * E2 * x, -2 * E2 * y, 0},
        {-6 * A3 * x * y, -A3 * (3 * xx - 3 * yy), 0},
        {B3 * y * z, B3 * x * z, B3 * x * y},
        {2 * C3 * x * y, -C3 * (4 * zz - xx - 3 * yy), -8 * C3 * y * z},
        {-6 * D3 * x * z, -6 * D3 * y * z, D3 * (6 * zz - 3 * xx - 3 * yy)},
        {-C3 * (4 * zz - 3 * xx - yy), 2 * C3 * x * y, -8 * C3 * x * z},
        {2 * F3 * x * z, -2 * F3 * y * z, F3 * (xx - yy)},
        {-A3 * (3 * xx - 3 * yy), 6 * A3 * x * y, 0},
    };
    for (int k = 0; k < 16; ++k)
        for (int j = 0; j < 3; ++j) dY[k][j] = g[k][j];
}

// Per-Gaussian chain from the 2D gradients to mu, s, q, h, sigma (FP64).
// out: [59] = dmu[3] ds[3] dq[4] dsigma dh[16][3] (h as sh[k][ch]).
void preprocess_backward_one(const SceneIn& s, int64_t i, const Cam<double>& cam, const Grad2D& gr, double* out) {
    for (int k = 0; k < 59; ++k) out[k] = 0.0;
    const int64_t n = s.n;
    double mu[3] = {s.means[i], s.means[n + i], s.means[2 * n + i]};
    double sc[3] = {s.scales[i], s.scales[n + i], s.scales[2 * n + i]};
    double q[4] = {s.rots[i], s.rots[n + i], s.rots[2 * n + i], s.rots[3 * n + i]};
    double p[3];
    for (int r = 0; r < 3; ++r)
        p[r] = cam.V[r][0] * mu[0] + cam.V[r][1] * mu[1] + cam.V[r][2] * mu[2] + cam.V[r][3];
    const double x = p[0], y = p[1], z = p[2];
    double nq = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double qw = q[0] / nq, qx = q[1] / nq, qy = q[2] / nq, qz = q[3] / nq;
    double Rm[3][3] = {{1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy)},
                       {2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx)},
                       {2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)}};
    double M[3][3], S3[3][3];
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) M[r][k] = Rm[r][k] * sc[k];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) S3[r][c] = M[r][0] * M[c][0] + M[r][1] * M[c][1] + M[r][2] * M[c][2];
    const double limx = 1.3 * cam.tan_fovx, limy = 1.3 * cam.tan_fovy;
    const double xz = x / z, yz = y / z;
    const bool clx = xz < -limx || xz > limx, cly = yz < -limy || yz > limy;
    const double tx = std::min(limx, std::max(-limx, xz)) * z, ty = std::min(limy, std::max(-limy, yz)) * z;
    const double fx = cam.fx, fy = cam.fy;
    double J[2][3] = {{fx / z, 0, -fx * tx / (z * z)}, {0, fy / z, -fy * ty / (z * z)}};
    double T[2][3];
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 3; ++k) T[r][k] = J[r][0] * cam.V[0][k] + J[r][1] * cam.V[1][k] + J[r][2] * cam.V[2][k];
    double TS[2][3];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c) TS[r][c] = T[r][0] * S3[0][c] + T[r][1] * S3[1][c] + T[r][2] * S3[2][c];
    const double sxx = TS[0][0] * T[0][0] + TS[0][1] * T[0][1] + TS[0][2] * T[0][2] + 0.3;
    const double sxy = TS[0][0] * T[1][0] + TS[0][1] * T[1][1] + TS[0][2] * T[1][2];
    const double syy = TS[1][0] * T[1][0] + TS[1][1] * T[1][1] + TS[1][2] * T[1][2] + 0.3;
    const double det = sxx * syy - sxy * sxy, d2 = det * det;
    // conic (a, b, c) -> Sigma2D (sxx, sxy, syy); sxy is one variable
    const double g_sxx = gr.a * (-syy * syy / d2) + gr.b * (sxy * syy / d2) + gr.c * (1.0 / det - sxx * syy / d2);
    const double g_syy = gr.a * (1.0 / det - sxx * syy / d2) + gr.b * (sxy * sxx / d2) + gr.c * (-sxx * sxx / d2);
    const double g_sxy = gr.a * (2.0 * sxy * syy / d2) + gr.b * (-1.0 / det - 2.0 * sxy * sxy / d2) +
                         gr.c * (2.0 * sxy * sxx / d2);
    // Sigma2D = T Sigma3D T^T: with G2 = [[g_sxx, g_sxy/2], [g_sxy/2, g_syy]],
    // dL/dSigma3D = T^T G2 T, dL/dT = 2 G2 T Sigma3D
    const double G2[2][2] = {{g_sxx, 0.5 * g_sxy}, {0.5 * g_sxy, g_syy}};
    double G3[3][3], dT[2][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0;
            for (int m = 0; m < 2; ++m)
                for (int k = 0; k < 2; ++k) acc += T[m][r] * G2[m][k] * T[k][c];
            G3[r][c] = acc;
        }
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c) dT[r][c] = 2.0 * (G2[r][0] * TS[0][c] + G2[r][1] * TS[1][c]);
    // T = J W -> dL/dJ = dL/dT W^T
    double dJ[2][3];
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 3; ++k) dJ[r][k] = dT[r][0] * cam.V[k][0] + dT[r][1] * cam.V[k][1] + dT[r][2] * cam.V[k][2];
    // J entries as functions of the camera-space mean (with the clamp)
    double dp[3] = {0, 0, 0};
    dp[2] += dJ[0][0] * (-fx / (z * z)) + dJ[1][1] * (-fy / (z * z));
    if (!clx) {
        dp[0] += dJ[0][2] * (-fx / (z * z));
        dp[2] += dJ[0][2] * (2.0 * fx * x / (z * z * z));
    } else {
        dp[2] += dJ[0][2] * (fx * (tx / z) / (z * z));
    }
    if (!cly) {
        dp[1] += dJ[1][2] * (-fy / (z * z));
        dp[2] += dJ[1][2] * (2.0 * fy * y / (z * z * z));
    } else {
        dp[2] += dJ[1][2] * (fy * (ty / z) / (z * z));
    }
    // projected mean
    dp[0] += gr.u * fx / z;
    dp[1] += gr.v * fy / z;
    dp[2] += gr.u * (-fx * x / (z * z)) + gr.v * (-fy * y / (z * z));
    double dmu[3];
    for (int k = 0; k < 3; ++k) dmu[k] = cam.V[0][k] * dp[0] + cam.V[1][k] * dp[1] + cam.V[2][k] * dp[2];
    // Sigma3D = M M^T -> dL/dM = 2 G3 M; M = R S
    double dM[3][3];
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) dM[r][k] = 2.0 * (G3[r][0] * M[0][k] + G3[r][1] * M[1][k] + G3[r][2] * M[2][k]);
    double ds[3], dR[3][3];
    for (int k = 0; k < 3; ++k) {
        ds[k] = dM[0][k] * Rm[0][k] + dM[1][k] * Rm[1][k] + dM[2][k] * Rm[2][k];
        for (int r = 0; r < 3; ++r) dR[r][k] = dM[r][k] * sc[k];
    }
    // R(q) for the unit quaternion (w, x, y, z)
    double dqn[4];
    dqn[0] = 2 * (-qz * dR[0][1] + qy * dR[0][2] + qz * dR[1][0] - qx * dR[1][2] - qy * dR[2][0] + qx * dR[2][1]);
    dqn[1] = 2 * (qy * dR[0][1] + qz * dR[0][2] + qy * dR[1][0] - 2 * qx * dR[1][1] - qw * dR[1][2] + qz * dR[2][0] +
                  qw * dR[2][1] - 2 * qx * dR[2][2]);
    dqn[2] = 2 * (-2 * qy * dR[0][0] + qx * dR[0][1] + qw * dR[0][2] + qx * dR[1][0] + qz * dR[1][2] - qw * dR[2][0] +
                  qz * dR[2][1] - 2 * qy * dR[2][2]);
    dqn[3] = 2 * (-2 * qz * dR[0][0] - qw * dR[0][1] + qx * dR[0][2] + qw * dR[1][0] - 2 * qz * dR[1][1] +
                  qy * dR[1][2] + qx * dR[2][0] + qy * dR[2][1]);
    const double qn[4] = {qw, qx, qy, qz};
    double dot = 0;
    for (int k = 0; k < 4; ++k) dot += qn[k] * dqn[k];
    double dq[4];
    for (int k = 0; k < 4; ++k) dq[k] = (dqn[k] - qn[k] * dot) / nq;
    // SH colour: rgb = max(0, sum_k Y_k h_k + 0.5); dir = (mu - campos)/|mu - campos|
    double d[3] = {mu[0] - cam.campos[0], mu[1] - cam.campos[1], mu[2] - cam.campos[2]};
    double len = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double dir[3] = {d[0] / len, d[1] / len, d[2] / len};
    double Y[16], dY[16][3];
    sh_basis<double>(dir[0], dir[1], dir[2], Y);
    sh_basis_grad(dir[0], dir[1], dir[2], dY);
    const int nc = (s.sh_degree + 1) * (s.sh_degree + 1);
    double ddir[3] = {0, 0, 0};
    for (int ch = 0; ch < 3; ++ch) {
        double raw = 0.5;
        for (int k = 0; k < nc; ++k) raw += Y[k] * double(s.sh[(k * 3 + ch) * n + i]);
        const double graw = raw >= 0.0 ? gr.rgb[ch] : 0.0;
        for (int k = 0; k < nc; ++k) {
            out[11 + 3 * k + ch] = Y[k] * graw;
            for (int j = 0; j < 3; ++j) ddir[j] += graw * dY[k][j] * double(s.sh[(k * 3 + ch) * n + i]);
        }
    }
    double dd = dir[0] * ddir[0] + dir[1] * ddir[1] + dir[2] * ddir[2];
    for (int k = 0; k < 3; ++k) dmu[k] += (ddir[k] - dir[k] * dd) / len;
    for (int k = 0; k < 3; ++k) out[k] = dmu[k];
    for (int k = 0; k < 3; ++k) out[3 + k] = ds[k];
    for (int k = 0; k < 4; ++k) out[6 + k] = dq[k];
    out[10] = gr.sigma;
}

void pack_proj(const Proj<double>& P, double* o) {
    o[0] = P.u; o[1] = P.v; o[2] = P.depth; o[3] = P.opacity;
    o[4] = P.a; o[5] = P.b; o[6] = P.c; o[7] = P.t;
    o[8] = P.rgb[0]; o[9] = P.rgb[1]; o[10] = P.rgb[2];
    o[11] = P.cov[0]; o[12] = P.cov[1]; o[13] = P.cov[2];
    o[14] = P.radius; o[15] = P.valid ? 1.0 : 0.0;
}
void pack_proj(const Proj<float>& P, double* o) {
    o[0] = P.u; o[1] = P.v; o[2] = P.depth; o[3] = P.opacity;
    o[4] = P.a; o[5] = P.b; o[6] = P.c; o[7] = P.t;
    o[8] = P.rgb[0]; o[9] = P.rgb[1]; o[10] = P.rgb[2];
    o[11] = P.cov[0]; o[12] = P.cov[1]; o[13] = P.cov[2];
    o[14] = P.radius; o[15] = P.valid ? 1.0 : 0.0;
}

template <typename R> Proj<R> proj_from(const double* e) {
    // e: u v a b c t [radius]; a hand-specified 2D Gaussian for tile-set tests
    Proj<R> P;
    P.valid = true;
    P.u = R(e[0]); P.v = R(e[1]); P.a = R(e[2]); P.b = R(e[3]); P.c = R(e[4]); P.t = R(e[5]);
    P.radius = static_cast<int32_t>(e[6]);
    P.opacity = R(1);
    return P;
}

}  // namespace

// ============================================================== C interface
extern "C" {

int oracle_version() { return 1; }

void oracle_log_f32(const float* x, float* y, int64_t n) {
    for (int64_t i = 0; i < n; ++i) y[i] = log_f32(x[i]);
}
void oracle_exp_f32(const float* x, float* y, int64_t n) {
    for (int64_t i = 0; i < n; ++i) y[i] = exp_f32(x[i]);
}

// SH basis at unit directions dirs[n][3]; out[n][16].
void oracle_sh_basis(int prec64, const double* dirs, double* out, int64_t n) {
    for (int64_t i = 0; i < n; ++i) {
        if (prec64) {
            double Y[16];
            sh_basis<double>(dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2], Y);
            for (int k = 0; k < 16; ++k) out[16 * i + k] = Y[k];
        } else {
            float Y[16];
            sh_basis<float>(float(dirs[3 * i]), float(dirs[3 * i + 1]), float(dirs[3 * i + 2]), Y);
            for (int k = 0; k < 16; ++k) out[16 * i + k] = Y[k];
        }
    }
}

// Per-Gaussian preprocess.  out[n][16] = u v depth opacity a b c t r g b
// cov_xx cov_xy cov_yy radius valid; counts[n] = tile count in `mode`.
void oracle_preprocess(int prec64, int64_t n, const float* means, const float* scales, const float* rots,
                       const float* opac, const float* sh, int sh_degree, int width, int height, const float* camf,
                       int tile, int mode, double* out, int64_t* counts) {
    SceneIn s{n, sh_degree, means, scales, rots, opac, sh};
    Grid g = make_grid(width, height, tile);
    auto noop = [](int, int) {};
    if (prec64) {
        Cam<double> cam = make_cam<double>(width, height, camf);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            Proj<double> P = preprocess_one<double>(s, i, cam);
            pack_proj(P, out + 16 * i);
            counts[i] = mode_tiles<double>(mode, P, g, noop);
        }
    } else {
        Cam<float> cam = make_cam<float>(width, height, camf);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            Proj<float> P = preprocess_one<float>(s, i, cam);
            pack_proj(P, out + 16 * i);
            counts[i] = mode_tiles<float>(mode, P, g, noop);
        }
    }
}

// Tile set of one hand-specified 2D Gaussian.  e = u v a b c t radius.
// mode 0/1/2 as the library; dir used by AccuTile only (0 auto, 1 rows,
// 2 columns).  out[cap][2] = (tx, ty) in emission order; returns the count.
int64_t oracle_ellipse_tiles(int prec64, int mode, int dir, const double* e, int tile, int gx, int gy, int32_t* out,
                             int64_t cap) {
    Grid g{tile, gx, gy};
    int64_t k = 0;
    auto emit = [&](int tx, int ty) {
        if (k < cap) {
            out[2 * k] = tx;
            out[2 * k + 1] = ty;
        }
        ++k;
    };
    if (prec64) {
        Proj<double> P = proj_from<double>(e);
        if (mode == 2) return accutile_tiles<double>(P, g, dir, emit);
        return mode_tiles<double>(mode, P, g, emit);
    }
    Proj<float> P = proj_from<float>(e);
    if (mode == 2) return accutile_tiles<float>(P, g, dir, emit);
    return mode_tiles<float>(mode, P, g, emit);
}

// SnugBox of a hand-specified 2D Gaussian: out = x0 x1 y0 y1 tx0 tx1 ty0 ty1; returns 1 if non-empty.
int oracle_snugbox(int prec64, const double* e, int tile, int gx, int gy, double* out) {
    Grid g{tile, gx, gy};
    if (prec64) {
        Snug<double> S = snugbox(proj_from<double>(e), g);
        out[0] = S.x0; out[1] = S.x1; out[2] = S.y0; out[3] = S.y1;
        out[4] = S.tx0; out[5] = S.tx1; out[6] = S.ty0; out[7] = S.ty1;
        return S.ok;
    }
    Snug<float> S = snugbox(proj_from<float>(e), g);
    out[0] = S.x0; out[1] = S.x1; out[2] = S.y0; out[3] = S.y1;
    out[4] = S.tx0; out[5] = S.tx1; out[6] = S.ty0; out[7] = S.ty1;
    return S.ok;
}

// Brute-force continuous-exact tile set (FP64), as a gx*gy mask.
void oracle_exact_tile_mask(const double* e, int tile, int gx, int gy, uint8_t* mask) {
    const double T = tile;
    for (int ty = 0; ty < gy; ++ty)
        for (int tx = 0; tx < gx; ++tx) {
            double m = min_q_on_box(e[0], e[1], e[2], e[3], e[4], tx * T, (tx + 1) * T, ty * T, (ty + 1) * T);
            mask[ty * gx + tx] = (e[5] > 0.0 && m <= e[5]) ? 1 : 0;
        }
}

// Full forward pipeline for one mode.  Returns 0, or 3 if K > key_cap
// (num_keys then holds the required K and nothing else is written).
int oracle_render(int prec64, int64_t n, const float* means, const float* scales, const float* rots,
                  const float* opac, const float* sh, int sh_degree, int width, int height, const float* camf,
                  int tile, int mode, const float* bg, int64_t key_cap, uint64_t* keys_unsorted,
                  uint32_t* vals_unsorted, uint64_t* keys_sorted, uint32_t* vals_sorted, int64_t* num_keys,
                  uint32_t* ranges, double* image, double* final_T, uint32_t* last, int64_t* pair_counts) {
    SceneIn s{n, sh_degree, means, scales, rots, opac, sh};
    if (prec64)
        return render_impl<double>(s, width, height, camf, tile, mode, bg, key_cap, keys_unsorted, vals_unsorted,
                                   keys_sorted, vals_sorted, num_keys, ranges, image, final_T, last, pair_counts);
    return render_impl<float>(s, width, height, camf, tile, mode, bg, key_cap, keys_unsorted, vals_unsorted,
                              keys_sorted, vals_sorted, num_keys, ranges, image, final_T, last, pair_counts);
}

void oracle_render_notile(int prec64, int64_t n, const float* means, const float* scales, const float* rots,
                          const float* opac, const float* sh, int sh_degree, int width, int height,
                          const float* camf, const float* bg, double* image, double* final_T, int literal_exp,
                          int64_t* decisions_differ) {
    SceneIn s{n, sh_degree, means, scales, rots, opac, sh};
    if (prec64)
        render_notile_impl<double>(s, width, height, camf, bg, image, final_T, literal_exp, decisions_differ);
    else
        render_notile_impl<float>(s, width, height, camf, bg, image, final_T, literal_exp, decisions_differ);
}

// Blend of one pixel over an explicit list of 2D Gaussians (closed-form tests).
// g[m][10] = u v a b c t opacity r g b; out = C0 C1 C2 T last.
void oracle_blend_pixel(int prec64, const double* gs, int64_t m, double px, double py, const float* bg, double* out) {
    auto run = [&](auto tag) {
        using R = decltype(tag);
        Pixel<R> pix;
        for (int64_t k = 0; k < m; ++k) {
            Proj<R> P;
            const double* e = gs + 10 * k;
            P.valid = true;
            P.u = R(e[0]); P.v = R(e[1]); P.a = R(e[2]); P.b = R(e[3]); P.c = R(e[4]); P.t = R(e[5]);
            P.opacity = R(e[6]);
            P.rgb[0] = R(e[7]); P.rgb[1] = R(e[8]); P.rgb[2] = R(e[9]);
            if (!blend_step<R>(pix, P, R(px), R(py), uint32_t(k + 1))) break;
        }
        for (int ch = 0; ch < 3; ++ch) out[ch] = double(std::fma(pix.T, R(bg[ch]), pix.C[ch]));
        out[3] = double(pix.T);
        out[4] = double(pix.last);
    };
    if (prec64) run(double(0));
    else run(float(0));
}

// Backward of one tile mode (FP64).  dL_dimage [3][H][W]; grads [59][n]
// planar (dmu 3, ds 3, dq 4, dsigma 1, dh 48 as [k][ch]); g2d [10][n] =
// du dv da db dc dsigma dr dg db score (the blend's per-Gaussian sums).
void oracle_backward(int64_t n, const float* means, const float* scales, const float* rots, const float* opac,
                     const float* sh, int sh_degree, int width, int height, const float* camf, int tile, int mode,
                     const float* bg, const double* dL_dimage, double* grads, double* g2d) {
    SceneIn s{n, sh_degree, means, scales, rots, opac, sh};
    Cam<double> cam = make_cam<double>(width, height, camf);
    Grid g = make_grid(width, height, tile);
    std::vector<Proj<double>> P = preprocess_all<double>(s, cam);
    std::vector<uint64_t> keys;
    std::vector<uint32_t> vals;
    for (int64_t i = 0; i < n; ++i) {
        float depth_f = static_cast<float>(P[i].depth);
        uint32_t dbits;
        std::memcpy(&dbits, &depth_f, 4);
        mode_tiles<double>(mode, P[i], g, [&](int tx, int ty) {
            keys.push_back(((uint64_t(ty) * uint64_t(g.gx) + uint64_t(tx)) << 32) | uint64_t(dbits));
            vals.push_back(static_cast<uint32_t>(i));
        });
    }
    std::vector<int64_t> order(keys.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return keys[a] < keys[b]; });
    const int64_t G = int64_t(g.gx) * g.gy;
    std::vector<std::vector<uint32_t>> lists(static_cast<size_t>(G));
    for (int64_t k : order) lists[keys[k] >> 32].push_back(vals[k]);
    std::vector<Grad2D> acc(static_cast<size_t>(n));
    const int64_t HW = int64_t(width) * height;
    for (int py = 0; py < height; ++py)
        for (int px = 0; px < width; ++px) {
            const auto& L = lists[int64_t(py / tile) * g.gx + px / tile];
            const int64_t o = int64_t(py) * width + px;
            double Gp[3] = {dL_dimage[o], dL_dimage[HW + o], dL_dimage[2 * HW + o]};
            blend_backward_pixel(P, L.data(), uint32_t(L.size()), px, py, Gp, bg, acc);
        }
    for (int64_t i = 0; i < n; ++i) {
        double out[59];
        if (P[i].valid) preprocess_backward_one(s, i, cam, acc[i], out);
        else for (double& v : out) v = 0.0;
        for (int k = 0; k < 59; ++k) grads[k * n + i] = out[k];
        const Grad2D& a = acc[i];
        const double v2[10] = {a.u, a.v, a.a, a.b, a.c, a.sigma, a.rgb[0], a.rgb[1], a.rgb[2], a.score};
        for (int k = 0; k < 10; ++k) g2d[k * n + i] = v2[k];
    }
}

// SH basis gradient at unit directions dirs[n][3]; out[n][16][3].
// PUP sensitivity of one view, added to hess[21][n] (FP64).
void oracle_pup(int64_t n, const float* means, const float* scales, const float* rots, const float* opac,
                const float* sh, int sh_degree, int width, int height, const float* camf, int tile, int mode,
                const float* bg, double* hess) {
    SceneIn s{n, sh_degree, means, scales, rots, opac, sh};
    pup_view(s, width, height, camf, tile, mode, bg, hess);
}

void oracle_sh_basis_grad(const double* dirs, double* out, int64_t n) {
    for (int64_t i = 0; i < n; ++i) {
        double dY[16][3];
        sh_basis_grad(dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2], dY);
        for (int k = 0; k < 16; ++k)
            for (int j = 0; j < 3; ++j) out[48 * i + 3 * k + j] = dY[k][j];
    }
}

}  // extern "C"
