"""Pins of the CPU oracle against things other than itself.

Each test checks the oracle against a closed form, a library routine (numpy,
scipy), brute force, or a hand-derived fixture, chosen so that a dropped
term, a wrong sign or index, or a transposed operand fails at least one of
them.  Nothing here needs a GPU.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation
from scipy.special import sph_harm_y

import oracle
from paper_2412_00578_gb300 import synth

SNUG, ACCU, SIG3 = 1, 2, 0


def f32_ulp_err(y, ref):
    y = np.asarray(y, np.float64)
    sp = np.spacing(np.abs(np.asarray(ref, np.float32))).astype(np.float64)
    return np.abs(y - ref) / sp


# ---------------------------------------------------------------- elementary
def test_log_f32_against_libm():
    rng = np.random.default_rng(1)
    x = np.exp(rng.uniform(-80, 80, 200_000)).astype(np.float32)
    x = np.concatenate([x, np.float32([1.0, 2.0, 0.5, 255.0, 1 / 255.0, 1.0000001, 0.9999999])])
    y = oracle.log_f32(x)
    ref = np.log(x.astype(np.float64))
    err = f32_ulp_err(y, ref)
    assert err.max() <= 3.0, err.max()
    assert oracle.log_f32(np.float32([1.0]))[0] == 0.0
    assert np.isneginf(oracle.log_f32(np.float32([0.0]))[0])


def test_exp_f32_against_libm():
    rng = np.random.default_rng(2)
    x = rng.uniform(-87, 88, 200_000).astype(np.float32)
    x = np.concatenate([x, rng.uniform(-6, 0, 100_000).astype(np.float32), np.float32([0.0, -0.5, -5.53])])
    y = oracle.exp_f32(x)
    ref = np.exp(x.astype(np.float64))
    assert f32_ulp_err(y, ref).max() <= 2.0
    assert oracle.exp_f32(np.float32([0.0]))[0] == 1.0


# ---------------------------------------------------------------- SH colour
def real_sh_scipy(d):
    """Real SH built from scipy's complex SH (Condon-Shortley phase kept):
    m<0: sqrt2 Im Y_l^|m|, m=0: Y_l^0, m>0: sqrt2 Re Y_l^m."""
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    cols = []
    for l in range(4):
        for m in range(-l, l + 1):
            if m < 0:
                cols.append(np.sqrt(2) * np.imag(sph_harm_y(l, -m, theta, phi)))
            elif m == 0:
                cols.append(np.real(sph_harm_y(l, 0, theta, phi)))
            else:
                cols.append(np.sqrt(2) * np.real(sph_harm_y(l, m, theta, phi)))
    return np.stack(cols, 1)


def test_sh_basis_against_scipy():
    rng = np.random.default_rng(3)
    d = rng.normal(size=(2000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    ref = real_sh_scipy(d)
    np.testing.assert_allclose(oracle.sh_basis(d, prec64=True), ref, atol=1e-13)
    np.testing.assert_allclose(oracle.sh_basis(d, prec64=False), ref, atol=3e-6)


def _one(mean, scale=(0.1, 0.1, 0.1), quat=(1, 0, 0, 0), opacity=0.8, sh=None, deg=3):
    sc = synth.Scene.__new__(synth.Scene)
    sc.means = np.asarray(mean, np.float32).reshape(3, -1)
    n = sc.means.shape[1]
    sc.scales = np.asarray(scale, np.float32).reshape(3, -1) * np.ones((1, n), np.float32)
    sc.rotations = np.asarray(quat, np.float32).reshape(4, -1) * np.ones((1, n), np.float32)
    sc.opacities = np.full(n, opacity, np.float32)
    sc.sh = np.zeros((16, 3, n), np.float32) if sh is None else np.asarray(sh, np.float32).reshape(16, 3, n)
    sc.sh_degree = deg
    return sc


def test_colour_against_scipy_basis():
    scene, cam = synth.small_box_workload()
    st, _ = oracle.preprocess(scene, cam, 16, ACCU, prec64=True)
    m = scene.means.numpy().astype(np.float64)
    d = (m - cam.campos.astype(np.float64)[:, None]).T
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = real_sh_scipy(d)
    sh = scene.sh.numpy().astype(np.float64)  # (16, 3, N)
    col = np.maximum(np.einsum("nk,kcn->nc", Y, sh) + 0.5, 0.0)
    v = st[:, 15] > 0
    np.testing.assert_allclose(st[v][:, 8:11], col[v], atol=1e-12)
    # degree 0: colour = C0 h0 + 0.5
    one = _one([0.3, -0.2, 4.0], sh=np.r_[np.full(3, 0.7), np.zeros(45)].reshape(16, 3, 1), deg=0)
    st0, _ = oracle.preprocess(one, cam, 16, ACCU, prec64=True)
    assert st0[0, 8] == pytest.approx(0.5 / math.sqrt(math.pi) * float(np.float32(0.7)) + 0.5, abs=1e-15)


# ---------------------------------------------------------------- projection
def test_isotropic_on_axis_closed_form():
    """An isotropic Gaussian on the optical axis projects to
    Sigma2D = ((f s / z)^2 + 0.3) I centred at the principal point."""
    _, cam = synth.small_box_workload()
    for z, s in [(3.0, 0.01), (5.0, 0.05), (7.5, 0.2)]:
        one = _one([0.0, 0.0, z - 5.0], scale=(s, s, s), quat=(0.3, 0.5, -0.2, 0.7))
        st, _ = oracle.preprocess(one, cam, 16, ACCU, prec64=True)
        f = cam.fx
        s = float(np.float32(s))  # inputs are stored in float32
        z = float(np.float32(z - 5.0)) + 5.0
        var = (f * s / z) ** 2 + 0.3
        assert st[0, 0] == pytest.approx(cam.cx, abs=1e-12)
        assert st[0, 1] == pytest.approx(cam.cy, abs=1e-12)
        assert st[0, 2] == pytest.approx(z, rel=1e-12)
        np.testing.assert_allclose(st[0, 11:14], [var, 0.0, var], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(st[0, 4:7], [1 / var, 0.0, 1 / var], rtol=1e-12, atol=1e-15)
        assert st[0, 7] == pytest.approx(2 * math.log(255 * float(np.float32(0.8))), rel=1e-14)


def pinhole(p, cam):
    return np.array([cam.fx * p[0] / p[2] + cam.cx, cam.fy * p[1] / p[2] + cam.cy])


def test_projection_against_numeric_jacobian_and_scipy_rotation():
    """Sigma2D = J W Sigma3D W^T J^T + 0.3 I with J from central finite
    differences of the pinhole map (at the clamped point) and R from scipy."""
    rng = np.random.default_rng(4)
    cam = synth.look_at(320, 240, 60.0, (3.0, -2.0, -6.0), (0.2, 0.1, 0.3))
    n = 300
    means = rng.uniform(-3, 3, (3, n))
    scales = np.exp(rng.normal(-2.5, 0.6, (3, n)))
    q = rng.normal(size=(4, n))
    q /= np.linalg.norm(q, axis=0)
    sc = _one(means, scales, q, 0.6)
    st, _ = oracle.preprocess(sc, cam, 16, ACCU, prec64=True)
    V = cam.viewmat.astype(np.float64)
    W = V[:, :3]
    limx, limy = 1.3 * cam.tan_fovx, 1.3 * cam.tan_fovy
    checked = 0
    for i in range(n):
        if st[i, 15] == 0:
            continue
        p = W @ sc.means[:, i].astype(np.float64) + V[:, 3]
        pc = np.array([np.clip(p[0] / p[2], -limx, limx) * p[2], np.clip(p[1] / p[2], -limy, limy) * p[2], p[2]])
        h = 1e-5 * max(1.0, abs(p[2]))
        J = np.stack([(pinhole(pc + h * e, cam) - pinhole(pc - h * e, cam)) / (2 * h) for e in np.eye(3)], 1)
        R = Rotation.from_quat(sc.rotations[:, i].astype(np.float64), scalar_first=True).as_matrix()
        S3 = R @ np.diag(sc.scales[:, i].astype(np.float64) ** 2) @ R.T
        S2 = J @ W @ S3 @ W.T @ J.T + 0.3 * np.eye(2)
        np.testing.assert_allclose(st[i, [11, 12, 13]], [S2[0, 0], S2[0, 1], S2[1, 1]], rtol=1e-6, atol=1e-8)
        conic = np.linalg.inv(S2)
        np.testing.assert_allclose(st[i, [4, 5, 6]], [conic[0, 0], conic[0, 1], conic[1, 1]], rtol=1e-6, atol=1e-9)
        uv = pinhole(p, cam)
        np.testing.assert_allclose(st[i, :2], uv, rtol=1e-12, atol=1e-9)
        lam = np.linalg.eigvalsh(S2).max()
        mid = 0.5 * (S2[0, 0] + S2[1, 1])
        if mid * mid - np.linalg.det(S2) > 0.1 + 1e-6:
            assert st[i, 14] == math.ceil(3 * math.sqrt(lam)) or abs(3 * math.sqrt(lam) - round(3 * math.sqrt(lam))) < 1e-6
        checked += 1
    assert checked > 100


def test_culling():
    _, cam = synth.small_box_workload()
    # behind the near plane (view z = 0.1 < 0.2), non-finite, zero quaternion
    sc = _one(np.array([[0, 0, 0, 0], [0, 0, 0, 0], [-4.9, 1.0, np.nan, 1.0]]),
              quat=np.array([[1, 1, 1, 0], [0, 0, 0, 0], [0, 0, 0, 0], [0, 0, 0, 0]]))
    st, cnt = oracle.preprocess(sc, cam, 16, ACCU, prec64=True)
    assert list(st[:, 15]) == [0, 1, 0, 0]
    assert cnt[0] == 0 and cnt[2] == 0 and cnt[3] == 0


# ---------------------------------------------------------------- tile sets
def random_ellipses(rng, n, gx, gy, T):
    out = []
    for _ in range(n):
        sx = np.exp(rng.uniform(np.log(0.5), np.log(6 * T)))
        sy = np.exp(rng.uniform(np.log(0.5), np.log(6 * T)))
        rho = rng.uniform(-0.999, 0.999) if rng.random() < 0.8 else 0.0
        cov = np.array([[sx * sx, rho * sx * sy], [rho * sx * sy, sy * sy]])
        a, b, _, c = np.linalg.inv(cov).ravel()
        sigma = rng.uniform(0.005, 1.0)
        t = 2 * math.log(255 * sigma)
        u = rng.uniform(-2 * T, (gx + 2) * T)
        v = rng.uniform(-2 * T, (gy + 2) * T)
        out.append((u, v, a, b, c, t))
    return out


def tile_set(arr):
    return {(int(x), int(y)) for x, y in arr}


def test_snugbox_closed_form_and_paper_equations():
    rng = np.random.default_rng(5)
    for (u, v, a, b, c, t) in random_ellipses(rng, 400, 20, 15, 16):
        if t <= 0:
            continue
        ok, box = oracle.snugbox((u, v, a, b, c, t), 16, 20, 15, prec64=True)
        cov = np.linalg.inv(np.array([[a, b], [b, c]]))
        hx, hy = math.sqrt(t * cov[0, 0]), math.sqrt(t * cov[1, 1])
        np.testing.assert_allclose(box[:4], [u - hx, u + hx, v - hy, v + hy], rtol=1e-9, atol=1e-9)
        # Eqs. ellipse_intersect and bbox_args taken literally give y_min/y_max.
        xa = math.sqrt(-b * b * t / ((b * b - a * c) * a)) if b != 0 else 0.0
        ys = []
        for x in (xa, -xa):
            disc = (b * b - a * c) * x * x + t * c
            r = math.sqrt(max(disc, 0.0))
            ys += [(-b * x + r) / c, (-b * x - r) / c]
        assert max(ys) == pytest.approx(hy, rel=1e-7, abs=1e-9)
        assert min(ys) == pytest.approx(-hy, rel=1e-7, abs=1e-9)
        # boundary samples lie inside the box; the box touches the ellipse
        th = np.linspace(0, 2 * np.pi, 721)
        L = np.linalg.cholesky(cov * t)
        pts = (L @ np.stack([np.cos(th), np.sin(th)]))
        assert pts[0].max() <= hx * (1 + 1e-9) and pts[0].min() >= -hx * (1 + 1e-9)
        assert pts[1].max() <= hy * (1 + 1e-9) and pts[1].min() >= -hy * (1 + 1e-9)
        xd, yd = hx, -(b / c) * hx
        assert a * xd * xd + 2 * b * xd * yd + c * yd * yd == pytest.approx(t, rel=1e-9)


@pytest.mark.parametrize("T,gx,gy", [(16, 20, 15), (8, 17, 11), (32, 6, 5)])
def test_accutile_equals_bruteforce_exact_set(T, gx, gy):
    """AccuTile (FP64) returns exactly the tiles whose closed square meets the
    ellipse q <= t (amb: continuous-exact set), except tiles that only touch
    the boundary within rounding."""
    rng = np.random.default_rng(6 + T)
    n_cmp = 0
    for e in random_ellipses(rng, 1500, gx, gy, T):
        got = oracle.ellipse_tiles(e, ACCU, T, gx, gy, prec64=True)
        assert len(got) == len(tile_set(got)), "a tile was emitted twice"
        mask = oracle.exact_tile_mask(e, T, gx, gy)
        want = {(x, y) for y, x in zip(*np.nonzero(mask))}
        diff = tile_set(got) ^ want
        for (x, y) in diff:  # only boundary-touching tiles may differ
            u, v, a, b, c, t = e
            tight = oracle.exact_tile_mask((u, v, a, b, c, t * (1 + 1e-7)), T, gx, gy)[y, x] != \
                oracle.exact_tile_mask((u, v, a, b, c, t * (1 - 1e-7)), T, gx, gy)[y, x]
            assert tight, (e, (x, y), (x, y) in want)
        n_cmp += 1
    assert n_cmp == 1500


def test_accutile_rows_equal_columns_and_nesting():
    rng = np.random.default_rng(7)
    T, gx, gy = 16, 20, 15
    for e in random_ellipses(rng, 1500, gx, gy, T):
        rows = tile_set(oracle.ellipse_tiles(e, ACCU, T, gx, gy, True, direction=1))
        cols = tile_set(oracle.ellipse_tiles(e, ACCU, T, gx, gy, True, direction=2))
        auto = tile_set(oracle.ellipse_tiles(e, ACCU, T, gx, gy, True))
        snug = tile_set(oracle.ellipse_tiles(e, SNUG, T, gx, gy, True))
        assert auto in (rows, cols)
        assert auto <= snug
        # rows vs columns agree except for rounding-level boundary tiles
        for (x, y) in rows ^ cols:
            u, v, a, b, c, t = e
            hi = oracle.exact_tile_mask((u, v, a, b, c, t * (1 + 1e-7)), T, gx, gy)[y, x]
            lo = oracle.exact_tile_mask((u, v, a, b, c, t * (1 - 1e-7)), T, gx, gy)[y, x]
            assert hi != lo
        # SnugBox is the rectangle of its box; 3-sigma contains it when t <= 9
        if e[5] <= 9.0 and snug:
            cov = np.linalg.inv(np.array([[e[2], e[3]], [e[3], e[4]]]))
            mid = 0.5 * (cov[0, 0] + cov[1, 1])
            lam = mid + math.sqrt(max(0.1, mid * mid - np.linalg.det(cov)))
            r = math.ceil(3 * math.sqrt(lam))
            sig = tile_set(oracle.ellipse_tiles(tuple(e) + (r,), SIG3, T, gx, gy, True))
            # The baseline's max bound trunc((mu + r + T - 1)/T) admits a tile only
            # once the square reaches >= 1 px into it: that 1-px slack is the
            # only way a SnugBox tile may be missing.
            for (x, y) in snug - sig:
                assert x * T > e[0] + r - 1 or y * T > e[1] + r - 1, (e, r, (x, y))


@pytest.mark.parametrize("prec64", [False, True])
def test_accutile_single_line_with_outer_boundaries_is_whole(prec64):
    """Sec. 4.1.2, Algorithm 1: when the SnugBox tile rectangle is one tile
    line thick on its shorter side and both boundaries of that line lie
    outside the SnugBox span, the line holds the whole ellipse, so AccuTile
    intersects no boundary and keeps the rectangle's whole span.  Checked on
    the oracle's sweep (tiles and their order) and, in FP64, against the
    brute-force set of tiles whose closed square meets the ellipse."""
    rng = np.random.default_rng(17 + prec64)
    T, gx, gy = 16, 20, 15
    whole = other = cut = 0
    for e in random_ellipses(rng, 3000, gx, gy, T):
        ok, sb = oracle.snugbox(e, T, gx, gy, prec64)
        if not ok:
            continue
        x0, x1, y0, y1 = sb[:4]
        tx0, tx1, ty0, ty1 = (int(z) for z in sb[4:])
        rows = (ty1 - ty0) <= (tx1 - tx0)
        k0, k1 = (ty0, ty1) if rows else (tx0, tx1)
        lo, hi = (y0, y1) if rows else (x0, x1)
        got = [tuple(map(int, p)) for p in oracle.ellipse_tiles(e, ACCU, T, gx, gy, prec64)]
        want = [(tx, ty) for ty in range(ty0, ty1 + 1) for tx in range(tx0, tx1 + 1)]
        if k0 != k1:
            other += 1
            continue
        if k0 * T >= lo or (k0 + 1) * T <= hi:
            # a boundary inside the span (the rectangle clipped at an image
            # edge across its line, or a box edge exactly on a tile edge):
            # the line's extent may be shorter
            cut += len(got) < len(want)
            continue
        assert got == want, (e, got, want)
        if prec64:
            mask = oracle.exact_tile_mask(e, T, gx, gy)
            exact = {(x, y) for y, x in zip(*np.nonzero(mask))}
            for (x, y) in exact ^ set(want):  # only tiles the ellipse just touches may differ
                u, v, a, b, c, t = e
                assert oracle.exact_tile_mask((u, v, a, b, c, t * (1 + 1e-7)), T, gx, gy)[y, x] != \
                    oracle.exact_tile_mask((u, v, a, b, c, t * (1 - 1e-7)), T, gx, gy)[y, x], (e, (x, y))
        whole += 1
    assert whole > 300 and other > 300 and cut > 20, (whole, other, cut)


def test_accutile_fp32_is_superset_of_fp32_pixels():
    """Every pixel whose FP32 blend test q <= t passes lies in a tile of the
    Gaussian's FP32 AccuTile set (the tile lists lose no contributing pixel);
    the surplus (tiles with no such pixel) is small."""
    scene, cam = synth.small_box_workload()
    st, cnt = oracle.preprocess(scene, cam, 16, ACCU, prec64=False)
    gx, gy = oracle.grid(cam.width, cam.height, 16)
    surplus = total = 0
    f = np.float32
    for i in np.nonzero(cnt)[0][:3000]:
        u, v, a, b, c, t = (f(st[i, k]) for k in (0, 1, 4, 5, 6, 7))
        tiles = tile_set(oracle.ellipse_tiles((u, v, a, b, c, t), ACCU, 16, gx, gy, prec64=False))
        ok, box = oracle.snugbox((u, v, a, b, c, t), 16, gx, gy, prec64=False)
        xs = np.arange(max(0, int(box[0]) - 2), min(cam.width, int(box[1]) + 3), dtype=np.float32)
        ys = np.arange(max(0, int(box[2]) - 2), min(cam.height, int(box[3]) + 3), dtype=np.float32)
        X, Y = np.meshgrid(xs, ys)
        dx = (X - u).astype(f)
        dy = (Y - v).astype(f)
        e_ = ((b + b) * dy).astype(f)
        f_ = ((c * dy).astype(f) * dy).astype(f)
        inner = (a * dx.astype(np.float64) + e_).astype(f)  # fma(a, dx, e), single rounding
        q = (dx.astype(np.float64) * inner + f_).astype(f)  # fma(dx, inner, f)
        hit = q <= t
        ptiles = {(int(x) // 16, int(y) // 16) for x, y in zip(X[hit], Y[hit])}
        assert ptiles <= tiles, i
        surplus += len(tiles - ptiles)
        total += len(tiles)
    assert surplus < 0.35 * total


def test_accutile_appendix_cases_golden():
    """Hand-built ellipses for the cases of App. A.1 (tests/golden/accutile_cases.txt):
    each fixture line lists the ellipse and the tile set derived by hand."""
    path = __file__.replace("test_oracle_pins.py", "golden/accutile_cases.txt")
    n = 0
    for line in open(path):
        line = line.split("#")[0].strip()
        if not line:
            continue
        name, rest = line.split(":", 1)
        nums, tiles = rest.split("|")
        u, v, a, b, c, t, T, gx, gy = (float(x) for x in nums.split())
        want = {tuple(int(k) for k in p.split(",")) for p in tiles.split()}
        for d in (0, 1, 2):
            got = tile_set(oracle.ellipse_tiles((u, v, a, b, c, t), ACCU, int(T), int(gx), int(gy), True, d))
            assert got == want, (name, d, sorted(got), sorted(want))
        n += 1
    assert n >= 7


# ---------------------------------------------------------------- blend
def test_blend_single_and_two_gaussian_closed_forms():
    rng = np.random.default_rng(8)
    for _ in range(200):
        g = [rng.uniform(0, 20), rng.uniform(0, 20), rng.uniform(0.05, 1), 0.0, rng.uniform(0.05, 1), 0.0,
             rng.uniform(0.05, 0.9), rng.uniform(0, 1), rng.uniform(0, 1), rng.uniform(0, 1)]
        g[3] = rng.uniform(-0.9, 0.9) * math.sqrt(g[2] * g[4])
        g[5] = 2 * math.log(255 * g[6])
        px, py = rng.integers(0, 21, 2)
        dx, dy = px - g[0], py - g[1]
        q = g[2] * dx * dx + 2 * g[3] * dx * dy + g[4] * dy * dy
        alpha = min(0.99, g[6] * math.exp(-q / 2)) if q <= g[5] else 0.0
        C, T, last = oracle.blend_pixel([g], px, py, bg=(0.25, 0.5, 0.75))
        np.testing.assert_allclose(C, np.array(g[7:10]) * alpha + (1 - alpha) * np.array([0.25, 0.5, 0.75]),
                                   rtol=1e-13, atol=1e-15)
        assert T == pytest.approx(1 - alpha, rel=1e-14)
        g2 = list(g)
        g2[7:10] = [0.9, 0.1, 0.4]
        C2, T2, _ = oracle.blend_pixel([g, g2], px, py)
        want = np.array(g[7:10]) * alpha + np.array(g2[7:10]) * alpha * (1 - alpha)
        if (1 - alpha) ** 2 >= 1e-4:
            np.testing.assert_allclose(C2, want, rtol=1e-13, atol=1e-15)


def test_blend_stop_rule():
    """Identical opaque splats with alpha = 0.95: T = 0.05, 0.0025, 1.25e-4,
    then the 4th would give 6.25e-6 < 1e-4, so exactly 3 contribute."""
    g = [5.0, 5.0, 1.0, 0.0, 1.0, 2 * math.log(255 * 0.95), 0.95, 1.0, 0.5, 0.25]
    for prec64 in (True, False):
        C, T, last = oracle.blend_pixel([g] * 8, 5, 5, prec64=prec64)
        assert last == 3
        assert T == pytest.approx(0.05 ** 3, rel=1e-6)
        np.testing.assert_allclose(C, np.array([1.0, 0.5, 0.25]) * (1 - 0.05 ** 3), rtol=1e-6)


def test_threshold_form_equals_literal_alpha_test():
    """q <= t decides exactly like sigma exp(-q/2) >= 1/255 (FP64)."""
    scene = synth.uniform_box_scene(600, seed=11)
    _, cam = synth.small_box_workload()
    small = synth.pinhole(96, 72, 60.0, np.eye(3), np.array([0.0, 0.0, 5.0]))
    out = oracle.render_notile(scene, small, prec64=True, literal_exp=True)
    assert out["decisions_differ"] == 0


# ---------------------------------------------------------------- pipeline
def small_case(n=1500, seed=12, w=100, h=75):
    scene = synth.uniform_box_scene(n, seed=seed, log_scale_mu=-3.0)
    cam = synth.pinhole(w, h, 60.0, np.eye(3), np.array([0.0, 0.0, 5.0]))
    return scene, cam


@pytest.mark.parametrize("tile", [8, 16, 32])
@pytest.mark.parametrize("prec64", [True, False])
def test_tiled_render_equals_tile_free_definition(tile, prec64):
    """SnugBox and AccuTile lists reproduce the tile-free image exactly."""
    scene, cam = small_case()
    ref = oracle.render_notile(scene, cam, prec64=prec64, bg=(0.1, 0.2, 0.3))
    for mode in (SNUG, ACCU):
        out = oracle.render(scene, cam, tile, mode, bg=(0.1, 0.2, 0.3), prec64=prec64)
        assert np.array_equal(out["image"], ref["image"])
        assert np.array_equal(out["final_T"], ref["final_T"])


def test_sort_and_ranges_against_numpy():
    scene, cam = small_case()
    for mode in (SIG3, SNUG, ACCU):
        out = oracle.render(scene, cam, 16, mode, prec64=False)
        ku, vu = out["keys_unsorted"], out["vals_unsorted"]
        order = np.lexsort((np.arange(len(ku)), ku))  # by key, ties by emission position
        assert np.array_equal(out["keys"], ku[order])
        assert np.array_equal(out["vals"], vu[order])
        gx, gy = out["grid"]
        tiles = (out["keys"] >> np.uint64(32)).astype(np.int64)
        counts = np.bincount(tiles, minlength=gx * gy)
        r = out["ranges"].astype(np.int64)
        assert np.array_equal(r[:, 1] - r[:, 0], counts)
        nz = counts > 0
        assert np.array_equal(r[nz, 0], np.cumsum(counts)[nz] - counts[nz])
        assert np.all(r[~nz] == 0)
        # emission is grouped by Gaussian id in ascending order
        assert np.all(np.diff(vu.astype(np.int64)) >= 0)


def test_modes_agree_and_3sigma_slack_is_one_pixel():
    """SnugBox and AccuTile render identical images.  With sigma <= 0.35
    (t < 9) the 3-sigma circle contains the ellipse, so the baseline differs
    only through its rectangle's max bound trunc((mu + r + T - 1)/T), which
    skips a tile that the square reaches less than one pixel into: every
    differing pixel is the first pixel row or column of a tile."""
    scene, cam = small_case(seed=13)
    scene.opacities = scene.opacities * 0.35
    imgs = [oracle.render(scene, cam, 16, m, prec64=True)["image"] for m in (SIG3, SNUG, ACCU)]
    assert np.array_equal(imgs[1], imgs[2])
    ys, xs = np.nonzero(np.abs(imgs[0] - imgs[1]).max(0) > 0)
    assert np.all((xs % 16 == 0) | (ys % 16 == 0))


def test_key_counts_decrease_with_precision_of_mode():
    scene, cam = synth.small_box_workload()
    k = [oracle.count_keys(scene, cam, 16, m) for m in (SIG3, SNUG, ACCU)]
    assert k[0] > k[1] > k[2] > 0


def test_blend_pair_counts():
    """The blend's pair counts (the work the roofline counts).  Faint splats
    never stop a pixel, so every pixel evaluates its whole tile list: the
    evaluated pairs equal the sum over tiles of entries x pixels of the tile
    inside the image.  AccuTile and SnugBox give the same images, hence the
    same contributing pairs, and SnugBox's lists are supersets of AccuTile's."""
    scene = synth.uniform_box_scene(2500, seed=71, log_scale_mu=-3.0)
    cam = synth.pinhole(97, 61, 60.0, np.eye(3), np.array([0.0, 0.0, 5.0]))
    faint = synth.uniform_box_scene(2500, seed=71, log_scale_mu=-3.0)
    faint.opacities[:] = 0.01
    for tile in (8, 16):
        r = oracle.render(faint, cam, tile, 2, prec64=False)
        gx, gy = r["grid"]
        rng = r["ranges"].reshape(-1, 2).astype(np.int64)
        n = rng[:, 1] - rng[:, 0]
        tx, ty = np.arange(gx * gy) % gx, np.arange(gx * gy) // gx
        pw = np.minimum(tile, cam.width - tx * tile)
        ph = np.minimum(tile, cam.height - ty * tile)
        assert np.all(r["final_T"] >= 1e-4)  # precondition: nothing stopped
        assert r["evaluated_pairs"] == int((n * pw * ph).sum())
        assert 0 < r["contributing_pairs"] < r["evaluated_pairs"]
    acc = oracle.render(scene, cam, 16, 2, prec64=False)
    snug = oracle.render(scene, cam, 16, 1, prec64=False)
    assert np.array_equal(acc["image"], snug["image"])
    assert acc["contributing_pairs"] == snug["contributing_pairs"]
    assert snug["evaluated_pairs"] >= acc["evaluated_pairs"]
    assert acc["evaluated_pairs"] > acc["contributing_pairs"] > 0


# ---------------------------------------------------------------- 3-sigma rectangle
def sigma3_golden():
    path = __file__.replace("test_oracle_pins.py", "golden/sigma3_cases.txt")
    cases = []
    for line in open(path):
        line = line.split("#")[0].strip()
        if not line:
            continue
        name, rest = line.split(":", 1)
        nums, rect = rest.split("|")
        u, v, r, T, gx, gy = (float(x) for x in nums.split())
        x0, x1, y0, y1 = (int(x) for x in rect.split())
        want = {(tx, ty) for ty in range(y0, y1) for tx in range(x0, x1)}
        cases.append((name, (u, v, 1.0, 0.0, 1.0, 1.0, r), int(T), int(gx), int(gy), want))
    return cases


def sigma3_failures(tiles_fn):
    bad = []
    for name, e, T, gx, gy, want in sigma3_golden():
        for prec64 in (True, False):
            got = tile_set(tiles_fn(e, SIG3, T, gx, gy, prec64))
            if got != want:
                bad.append((name, prec64, sorted(got), sorted(want)))
    return bad


def test_sigma3_rectangle_golden():
    """The 3-sigma square's tile rectangle (Sec. 4.1, Eq. radius, Fig. 2a:
    the 3D-GS rule) on hand-derived cases where its bounds land on, half a
    pixel before and one pixel past tile edges, near 0 and past the grid
    (tests/golden/sigma3_cases.txt derives each expected rectangle)."""
    assert len(sigma3_golden()) >= 20
    assert sigma3_failures(oracle.ellipse_tiles) == []


# Plausible slips in the rectangle: each planted into a copy of the oracle
# source (never into oracle.cpp itself) must fail the golden cases above.
SIGMA3_MUTANTS = {
    "max_plus_T": ("(P.u + r + (T - R(1))) / T", "(P.u + r + T) / T"),
    "max_floor_as_ceil": ("return static_cast<int>(x);  // truncation toward zero",
                          "return static_cast<int>(std::ceil(x));"),
    "min_plus_half": ("tr((P.u - r) / T, g.gx)", "tr((P.u - r + R(0.5)) / T, g.gx)"),
    "y_max_plus_T": ("(P.v + r + (T - R(1))) / T", "(P.v + r + T) / T"),
}


@pytest.mark.parametrize("mutant", sorted(SIGMA3_MUTANTS))
def test_sigma3_golden_catches_planted_mistakes(mutant, tmp_path):
    import ctypes
    import subprocess

    src = oracle._SRC.read_text()
    old, new = SIGMA3_MUTANTS[mutant]
    assert src.count(old) == 1, f"pattern for {mutant} not found exactly once"
    mut = tmp_path / "oracle_mutant.cpp"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "liboracle_mutant.so"
    subprocess.run(["g++", *oracle.CXXFLAGS, str(mut), "-o", str(so)], check=True)
    L = ctypes.CDLL(str(so))
    oracle._declare(L)

    def tiles(e, mode, T, gx, gy, prec64):
        ee = np.zeros(7, np.float64)
        ee[:len(e)] = e
        cap = gx * gy + 1
        out = np.zeros((cap, 2), np.int32)
        k = L.oracle_ellipse_tiles(int(prec64), mode, 0, oracle._ptr(ee), T, gx, gy, oracle._ptr(out), cap)
        return out[:k].copy()

    assert sigma3_failures(tiles), f"planted mistake {mutant} passed every golden case"


# ---------------------------------------------------------------- tile-based culling and pixel-exact tiles
TBC, PIX = 3, 4


def rotated_ellipses(rng, count, T, gx, gy):
    """Ellipses with random orientation, axis lengths from sub-pixel to a few
    tiles, centres over and around a gx x gy grid of T-pixel tiles."""
    out = []
    for _ in range(count):
        th = rng.uniform(0, np.pi)
        s1, s2 = np.exp(rng.uniform(np.log(0.4), np.log(2.5 * T), 2))
        Rm = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
        cov = Rm @ np.diag([s1 * s1, s2 * s2]) @ Rm.T + 0.3 * np.eye(2)
        con = np.linalg.inv(cov)
        u = rng.uniform(-T, (gx + 1) * T)
        v = rng.uniform(-T, (gy + 1) * T)
        t = rng.uniform(0.05, 11.0)
        out.append((u, v, con[0, 0], con[0, 1], con[1, 1], t))
    return out


def test_tbc_tile_test_against_numerical_minimum():
    """The tile-based culling test (App. A.4): a tile is kept iff the minimum
    of q over its closed square is <= t.  Checked against scipy's bounded
    quasi-Newton minimiser of the same quadratic on each candidate tile (ties
    within 1e-7 t excluded)."""
    from scipy.optimize import minimize

    rng = np.random.default_rng(91)
    T, gx, gy = 16, 6, 5
    checked = 0
    for e in rotated_ellipses(rng, 150, T, gx, gy):
        u, v, a, b, c, t = e
        ok, sb = oracle.snugbox(e, T, gx, gy, True)
        if not ok:
            continue
        got = tile_set(oracle.ellipse_tiles(e, TBC, T, gx, gy, True))
        q = lambda p: a * (p[0] - u) ** 2 + 2 * b * (p[0] - u) * (p[1] - v) + c * (p[1] - v) ** 2
        for ty in range(int(sb[6]), int(sb[7]) + 1):
            for tx in range(int(sb[4]), int(sb[5]) + 1):
                box = [(tx * T, (tx + 1) * T), (ty * T, (ty + 1) * T)]
                x0 = np.clip([u, v], [box[0][0], box[1][0]], [box[0][1], box[1][1]])
                res = minimize(q, x0, bounds=box, method="L-BFGS-B", options={"ftol": 1e-15, "gtol": 1e-12})
                m = min(float(res.fun), q(x0))
                if abs(m - t) <= 1e-7 * t:
                    continue
                assert ((tx, ty) in got) == (m <= t), (e, tx, ty, m)
                checked += 1
    assert checked > 300


def test_tbc_and_accutile_are_the_same_exact_set():
    """In FP64 the culled SnugBox (tile-based culling) and the AccuTile sweep
    are two algorithms for one set, the tiles whose closed square meets the
    ellipse: equal on random ellipses and on the App. A.1 fixtures."""
    rng = np.random.default_rng(92)
    for T, gx, gy in ((16, 6, 5), (8, 9, 7)):
        for e in rotated_ellipses(rng, 400, T, gx, gy):
            tbc = tile_set(oracle.ellipse_tiles(e, TBC, T, gx, gy, True))
            acc = tile_set(oracle.ellipse_tiles(e, ACCU, T, gx, gy, True))
            assert tbc == acc, e


def test_pixel_tiles_against_whole_image_brute_force():
    """Pixel-exact tiles: the tiles of the pixels inside the image whose q
    (in the blend's operation order) is <= t, found here by testing every
    pixel of the image (the oracle tests only the widened SnugBox), in FP64
    and FP32; the set nests inside AccuTile's (FP64)."""
    rng = np.random.default_rng(93)
    T, gx, gy = 8, 7, 6
    W, H = gx * T, gy * T
    X, Y = np.meshgrid(np.arange(W), np.arange(H))
    surplus = total = 0
    for e in rotated_ellipses(rng, 300, T, gx, gy):
        u, v, a, b, c, t = e
        for prec64, dt in ((True, np.float64), (False, np.float32)):
            uu, vv, aa, bb, cc, tt = (dt(x) for x in e)
            dx = X.astype(dt) - uu
            dy = Y.astype(dt) - vv
            if prec64:
                q = dx * (aa * dx + (bb + bb) * dy) + (cc * dy) * dy
            else:  # the FP32 order: fma(dx, fma(a, dx, (2b) dy), (c dy) dy), one rounding per fma
                inner = (aa.astype(np.float64) * dx + ((bb + bb) * dy).astype(np.float64)).astype(np.float32)
                q = (dx.astype(np.float64) * inner + ((cc * dy) * dy).astype(np.float64)).astype(np.float32)
            hit = q <= tt
            want = {(int(x) // T, int(y) // T) for x, y in zip(X[hit], Y[hit])}
            got = tile_set(oracle.ellipse_tiles(e, PIX, T, gx, gy, prec64))
            assert got == want, (e, prec64)
            if prec64:
                acc = tile_set(oracle.ellipse_tiles(e, ACCU, T, gx, gy, True))
                assert got <= acc, e
                surplus += len(acc - got)
                total += len(acc)
    assert 0 < surplus < total


@pytest.mark.parametrize("prec64", [False, True])
def test_full_rectangles_are_listed_row_major(prec64):
    """A tile set that fills its bounding rectangle is listed row by row,
    left to right, in SnugBox, tile-based culling (the SnugBox rectangle
    walked that way, App. A.4) and pixel-exact modes (tile row by tile row),
    and for AccuTile when it is a single line; so a key writer that knows the
    set is a whole rectangle may write it in that order.  AccuTile lists a
    multi-line rectangle line by line along its sweep (columns when they are
    the shorter side), so only its set is checked there."""
    rng = np.random.default_rng(94 + prec64)
    T, gx, gy = 8, 9, 7
    full = {m: 0 for m in (SNUG, ACCU, TBC, PIX)}
    for e in rotated_ellipses(rng, 400, T, gx, gy):
        for m in full:
            got = [tuple(map(int, p)) for p in oracle.ellipse_tiles(e, m, T, gx, gy, prec64)]
            if not got:
                continue
            xs = [p[0] for p in got]
            ys = [p[1] for p in got]
            rect = [(x, y) for y in range(min(ys), max(ys) + 1) for x in range(min(xs), max(xs) + 1)]
            if len(got) != len(rect):
                continue
            single = min(ys) == max(ys) or min(xs) == max(xs)
            if m == ACCU and not single:
                assert sorted(got) == sorted(rect)  # rows or columns, whichever is shorter
                continue
            assert got == rect, (m, e, got)
            full[m] += 1
    assert min(full.values()) > 50, full


def test_new_modes_render_the_definition_image():
    """Tile-based culling and pixel-exact tiles lose no contributing pixel:
    their tiled images equal the tile-free image bit for bit, in FP32 and
    FP64, and their key counts nest: pixel <= AccuTile = TBC <= SnugBox."""
    scene, cam = small_case(seed=17)
    for prec64 in (False, True):
        ref = oracle.render_notile(scene, cam, prec64=prec64)["image"]
        for mode in (TBC, PIX):
            img = oracle.render(scene, cam, 16, mode, prec64=prec64)["image"]
            assert np.array_equal(img, ref), (mode, prec64)
    k = {m: oracle.count_keys(scene, cam, 16, m, prec64=True) for m in (SNUG, ACCU, TBC, PIX)}
    assert k[PIX] <= k[ACCU] == k[TBC] <= k[SNUG]
    assert k[PIX] < k[ACCU]
