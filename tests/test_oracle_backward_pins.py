"""Pins of the oracle's analytic backward (FP64) against central finite
differences of the oracle's own FP64 forward (a different code path: the
forward never differentiates), the SH basis derivative against finite
differences of the basis, and the pruning score against its closed form."""
import numpy as np
import torch
import pytest

import oracle
from paper_2412_00578_gb300 import synth


def tiny_scene(n=40, seed=50, w=48, h=40):
    scene = synth.uniform_box_scene(n, seed=seed, half=1.0, log_scale_mu=-2.5, log_scale_sd=0.4)
    cam = synth.look_at(w, h, 60.0, (0.4, -0.3, -4.0), (0.0, 0.0, 0.0))
    return scene, cam


def as_np(scene):
    d = {k: np.array(getattr(scene, k).numpy(), copy=True) for k in ("means", "scales", "rotations", "opacities", "sh")}
    return d


class NpScene:
    def __init__(self, d, deg=3):
        for k, v in d.items():
            setattr(self, k, v)
        self.sh_degree = deg


def loss(d, cam, W, tile, mode, bg):
    img = oracle.render(NpScene(d), cam, tile, mode, bg=bg, prec64=True)["image"]
    return float((W * img).sum())


def fd_grad(d, cam, W, key, idx, tile, mode, bg, rel):
    x0 = d[key][idx]
    h = max(abs(float(x0)) * rel, 1e-4)
    vals = []
    for step in (h, h / 2):
        dp = {k: v.copy() for k, v in d.items()}
        dm = {k: v.copy() for k, v in d.items()}
        dp[key][idx] = np.float32(x0 + step)
        dm[key][idx] = np.float32(x0 - step)
        he = (float(dp[key][idx]) - float(dm[key][idx])) / 2
        vals.append((loss(dp, cam, W, tile, mode, bg) - loss(dm, cam, W, tile, mode, bg)) / (2 * he))
    return vals


@pytest.mark.parametrize("mode", [2, 0])
def test_backward_matches_finite_differences(mode):
    scene, cam = tiny_scene()
    d = as_np(scene)
    rng = np.random.default_rng(51)
    W = rng.normal(size=(3, cam.height, cam.width))
    bg = (0.2, 0.1, 0.3)
    grads, g2d = oracle.backward(scene, cam, W, 16, mode, bg)
    contributing = np.nonzero(np.abs(g2d[:6]).sum(0) > 0)[0]
    assert len(contributing) > 10
    scale = {k: np.sqrt(np.mean(np.square(v))) for k, v in grads.items()}
    checked = skipped = 0
    errs = []
    for trial in range(120):
        i = int(rng.choice(contributing))
        key = ["means", "scales", "rotations", "opacities", "sh"][trial % 5]
        if key == "means":
            idx = (int(rng.integers(3)), i)
        elif key == "scales":
            idx = (int(rng.integers(3)), i)
        elif key == "rotations":
            idx = (int(rng.integers(4)), i)
        elif key == "opacities":
            idx = (i,)
        else:
            idx = (int(rng.integers(16)), int(rng.integers(3)), i)
        f1, f2 = fd_grad(d, cam, W, key, idx, 16, mode, bg, 2e-3)
        if abs(f1 - f2) > 1e-3 * max(abs(f1), abs(f2), scale[key]):
            skipped += 1  # the perturbation crossed a threshold, clamp or stop decision
            continue
        # Richardson extrapolation of the two central differences (steps h and
        # h/2) cancels their h^2 error term, leaving O(h^4)
        fd = (4.0 * f2 - f1) / 3.0
        g = float(grads[key][idx])
        denom = max(abs(fd), 1e-3 * scale[key], 1e-12)
        errs.append(abs(g - fd) / denom)
        assert errs[-1] <= 1e-6, (key, idx, g, fd, errs[-1])
        checked += 1
    assert checked >= 64 and skipped <= 40, (checked, skipped)
    print(f"mode {mode}: {checked} parameters checked, {skipped} skipped, max rel err {max(errs):.2e}")


def test_sh_basis_gradient_against_finite_differences():
    rng = np.random.default_rng(52)
    d = rng.normal(size=(200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    G = oracle.sh_basis_grad(d)
    h = 1e-6
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        fd = (oracle.sh_basis(d + e) - oracle.sh_basis(d - e)) / (2 * h)  # derivative of the polynomial form
        np.testing.assert_allclose(G[:, :, j], fd, atol=1e-7)


def test_pruning_score_single_gaussian_closed_form():
    """One Gaussian, bg = 0, colour c: C = c alpha, dC/dg = sigma c wherever
    sigma g < 0.99 and q <= t, so score = sigma^2 |c|^2 #{such pixels}."""
    scene = synth.uniform_box_scene(1, seed=53)
    scene.means[:] = 0.0
    scene.scales[:] = 0.02
    scene.opacities[:] = 0.6
    scene.sh[:] = 0.0
    scene.sh[0] = 1.0  # colour = C0 + 0.5 per channel
    cam = synth.pinhole(32, 32, 60.0, np.eye(3), np.array([0.0, 0.0, 3.0]))
    W = np.zeros((3, 32, 32))
    _, g2d = oracle.backward(scene, cam, W, 16, 2)
    st, _ = oracle.preprocess(scene, cam, 16, 2, prec64=True)
    u, v, a, b, c, t = st[0, [0, 1, 4, 5, 6, 7]]
    col = st[0, 8:11]
    X, Y = np.meshgrid(np.arange(32.0), np.arange(32.0))
    dx, dy = X - u, Y - v
    q = a * dx * dx + 2 * b * dx * dy + c * dy * dy
    sig = float(np.float32(0.6))
    inside = (q <= t) & (sig * np.exp(-q / 2) < 0.99)
    assert inside.sum() > 5
    assert g2d[9, 0] == pytest.approx(sig * sig * float((col ** 2).sum()) * inside.sum(), rel=1e-12)


# ---------------------------------------------------------------- PUP sensitivity
def pup_fd(d, cam, keys=("means", "scales"), rel=1e-3):
    """grad_{mu,s} of every pixel and channel of the FP64 tile-free image, by
    Richardson-extrapolated central differences, for every Gaussian:
    returns [n, 6, 3 H W]."""
    n = d["means"].shape[1]
    out = np.zeros((n, 6, 3 * cam.height * cam.width))
    for i in range(n):
        j = 0
        for key in keys:
            for k in range(3):
                x0 = d[key][k, i]
                h = max(abs(float(x0)) * rel, 1e-5)
                est = []
                for step in (h, h / 2):
                    dp = {kk: vv.copy() for kk, vv in d.items()}
                    dm = {kk: vv.copy() for kk, vv in d.items()}
                    dp[key][k, i] = np.float32(x0 + step)
                    dm[key][k, i] = np.float32(x0 - step)
                    he = float(dp[key][k, i]) - float(dm[key][k, i])
                    ip = oracle.render_notile(NpScene(dp, 0), cam, prec64=True)["image"].ravel()
                    im = oracle.render_notile(NpScene(dm, 0), cam, prec64=True)["image"].ravel()
                    est.append((ip - im) / he)
                out[i, j] = (4.0 * est[1] - est[0]) / 3.0
                j += 1
    return out


def test_pup_sensitivity_against_finite_differences_of_the_image():
    """PUP's H_i = sum_p sum_ch grad_{mu,s} C grad_{mu,s} C^T (Sec. 4.2, Eq.
    pup_score), from the oracle's construction (back-to-front dC/dg, the
    projection Jacobian by differences of the projection alone, analytic
    dg/d(u, v, a, b, c)), against the same sum built from central
    differences of the whole FP64 tile-free image, for three overlapping
    Gaussians with view-independent colour (SH degree 0) whose ellipses have
    no pixel near their threshold (so no inclusion decision moves)."""
    cam = synth.look_at(40, 32, 60.0, (0.3, -0.2, -4.0), (0.0, 0.0, 0.0))
    rng = np.random.default_rng(60)
    for attempt in range(2000):
        scene = synth.uniform_box_scene(3, seed=int(rng.integers(1 << 30)), half=0.25, log_scale_mu=-1.6,
                                        log_scale_sd=0.3, sh_degree=0)
        scene.opacities[:] = torch.tensor([0.6, 0.45, 0.8])
        st, _ = oracle.preprocess(scene, cam, 16, 2, prec64=True)
        X, Y = np.meshgrid(np.arange(cam.width), np.arange(cam.height))
        margin = np.inf
        for i in range(3):
            u, v, a, b, c, t = st[i, [0, 1, 4, 5, 6, 7]]
            dx, dy = X - u, Y - v
            q = a * dx * dx + 2 * b * dx * dy + c * dy * dy
            margin = min(margin, np.abs(q - t).min() / t)
        if margin > 0.004 and st[:, 15].all():
            break
    else:
        pytest.fail("no configuration without near-threshold pixels")
    d = {k: np.array(getattr(scene, k).numpy(), copy=True) for k in ("means", "scales", "rotations", "opacities", "sh")}
    D = pup_fd(d, cam, rel=1e-4)
    H_fd = np.einsum("iap,ibp->iab", D, D)
    H = oracle.pup_full(oracle.pup(NpScene(d, 0), [cam], 16, 2))
    for i in range(3):
        rel = np.linalg.norm(H[i] - H_fd[i]) / np.linalg.norm(H_fd[i])
        assert rel <= 1e-6, (i, rel)
    # one view gives a rank-deficient 6 x 6 block (the image sees only the 5
    # parameters of the 2D Gaussian); a second view makes it definite
    assert np.linalg.matrix_rank(H[0], tol=1e-9 * np.abs(H[0]).max()) <= 5
    cam2 = synth.look_at(40, 32, 60.0, (-2.5, 1.0, -3.0), (0.0, 0.0, 0.0))
    H2 = oracle.pup_full(oracle.pup(NpScene(d, 0), [cam, cam2], 16, 2))
    assert np.all(np.linalg.eigvalsh(H2) > 0)
