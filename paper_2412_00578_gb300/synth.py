"""Seeded synthetic scenes and cameras.

This module holds input generation only: it draws Gaussian parameter sets and
pinhole cameras, and contains none of the rasterizer's arithmetic.  Both the
CPU oracle (in tests) and the CUDA path consume what it produces.

Parameter set (Sec. 3.1): per Gaussian a mean mu (3), a scale s (3), a
rotation quaternion r (4, order w x y z), spherical-harmonic colour
coefficients h (16 x 3) and an opacity sigma.  Scales and opacities are stored
*activated* (exp / sigmoid already applied); quaternions are stored
normalised.

Memory layout (planar structure of arrays, float32, C-contiguous):
    means     (3, N)       x plane, y plane, z plane
    scales    (3, N)
    rotations (4, N)       w, x, y, z planes
    opacities (N,)
    sh        (16, 3, N)   coefficient k, channel c at sh[k, c, i]

Every draw uses ``torch.Generator().manual_seed(seed)`` on the CPU in float32,
in the fixed order: means -> log-scales -> quaternions -> opacity logits -> SH.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

SH_COEFFS = 16  # degree 3


@dataclass
class Scene:
    means: torch.Tensor      # (3, N) float32
    scales: torch.Tensor     # (3, N) float32, activated
    rotations: torch.Tensor  # (4, N) float32, w x y z, unit norm
    opacities: torch.Tensor  # (N,)  float32, activated
    sh: torch.Tensor         # (16, 3, N) float32
    sh_degree: int = 3

    @property
    def n(self) -> int:
        return int(self.means.shape[1])

    def to(self, device) -> "Scene":
        return Scene(self.means.to(device), self.scales.to(device), self.rotations.to(device),
                     self.opacities.to(device), self.sh.to(device), self.sh_degree)

    def contiguous(self) -> "Scene":
        return Scene(self.means.contiguous(), self.scales.contiguous(), self.rotations.contiguous(),
                     self.opacities.contiguous(), self.sh.contiguous(), self.sh_degree)

    def subset(self, idx: torch.Tensor) -> "Scene":
        return Scene(self.means[:, idx], self.scales[:, idx], self.rotations[:, idx],
                     self.opacities[idx], self.sh[:, :, idx], self.sh_degree).contiguous()

    def nbytes(self) -> int:
        nc = (self.sh_degree + 1) ** 2
        return self.n * 4 * (3 + 3 + 4 + 1 + 3 * nc)

    def numpy(self) -> dict:
        return {k: getattr(self, k).detach().cpu().numpy() for k in
                ("means", "scales", "rotations", "opacities", "sh")}


@dataclass
class Camera:
    """Pinhole camera, OpenCV axes (x right, y down, z forward).

    ``viewmat`` is the row-major 3x4 world-to-camera transform [R | t];
    ``campos`` the camera centre in world coordinates.  Pixel (i, j) sits at
    the point (i, j); the principal point is ((W-1)/2, (H-1)/2).
    """
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    tan_fovx: float
    tan_fovy: float
    viewmat: np.ndarray   # (3, 4) float32
    campos: np.ndarray    # (3,) float32
    near_z: float = 0.2

    def as_floats(self) -> np.ndarray:
        """Flat float32 vector: fx fy cx cy tan_fovx tan_fovy near_z viewmat[12] campos[3]."""
        v = [self.fx, self.fy, self.cx, self.cy, self.tan_fovx, self.tan_fovy, self.near_z]
        return np.concatenate([np.asarray(v, np.float32), self.viewmat.astype(np.float32).ravel(),
                               self.campos.astype(np.float32)]).astype(np.float32)


def _f32(x) -> float:
    return float(np.float32(x))


def pinhole(width: int, height: int, fov_y_deg: float, R: np.ndarray, t: np.ndarray) -> Camera:
    """Camera with square pixels and vertical field of view ``fov_y_deg``.

    ``R`` (3x3) and ``t`` (3,) map world to camera: p_cam = R p_world + t.
    """
    tan_y = math.tan(math.radians(fov_y_deg) / 2.0)
    fy = height / (2.0 * tan_y)
    fx = fy
    tan_x = width / (2.0 * fx)
    vm = np.zeros((3, 4), np.float64)
    vm[:, :3] = R
    vm[:, 3] = t
    campos = -R.T @ t
    return Camera(width, height, _f32(fx), _f32(fy), _f32((width - 1) / 2.0), _f32((height - 1) / 2.0),
                  _f32(tan_x), _f32(tan_y), vm.astype(np.float32), campos.astype(np.float32))


def look_at(width: int, height: int, fov_y_deg: float, pos, target=(0.0, 0.0, 0.0)) -> Camera:
    """Camera at ``pos`` looking at ``target``; world -y is 'up' (camera y points down)."""
    pos = np.asarray(pos, np.float64)
    z = np.asarray(target, np.float64) - pos
    z /= np.linalg.norm(z)
    down = np.array([0.0, 1.0, 0.0])
    x = np.cross(down, z)
    if np.linalg.norm(x) < 1e-9:
        x = np.array([1.0, 0.0, 0.0])
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z])
    t = -R @ pos
    return pinhole(width, height, fov_y_deg, R, t)


def orbit_camera(gen: torch.Generator, width: int, height: int, fov_y_deg: float = 60.0) -> Camera:
    """Pose on the orbit used for multi-view and serving: radius U(20,30),
    elevation U(-15, 30) degrees, azimuth uniform, looking at the origin."""
    u = torch.rand(3, generator=gen, dtype=torch.float64)
    radius = 20.0 + 10.0 * float(u[0])
    elev = math.radians(-15.0 + 45.0 * float(u[1]))
    az = 2.0 * math.pi * float(u[2])
    pos = (radius * math.cos(elev) * math.sin(az), -radius * math.sin(elev), -radius * math.cos(elev) * math.cos(az))
    return look_at(width, height, fov_y_deg, pos)


def _quats(gen: torch.Generator, n: int) -> torch.Tensor:
    q = torch.randn(4, n, generator=gen, dtype=torch.float32)
    return q / q.norm(dim=0, keepdim=True).clamp_min(1e-12)


def _finish(gen, means, log_scale_mu, log_scale_sd, sh_degree=3) -> Scene:
    n = means.shape[1]
    log_s = log_scale_mu + log_scale_sd * torch.randn(3, n, generator=gen, dtype=torch.float32)
    rots = _quats(gen, n)
    logit = 1.5 * torch.randn(n, generator=gen, dtype=torch.float32)
    nc = (sh_degree + 1) ** 2
    sh = torch.zeros(SH_COEFFS, 3, n, dtype=torch.float32)
    sh[0] = 0.5 + 0.2 * torch.randn(3, n, generator=gen, dtype=torch.float32)
    if nc > 1:
        sh[1:nc] = 0.3 * torch.randn(nc - 1, 3, n, generator=gen, dtype=torch.float32)
    return Scene(means.contiguous(), torch.exp(log_s).contiguous(), rots.contiguous(),
                 torch.sigmoid(logit).contiguous(), sh.contiguous(), sh_degree)


def uniform_box_scene(n: int, seed: int = 0, half: float = 2.0, log_scale_mu: float = -4.0,
                      log_scale_sd: float = 0.5, sh_degree: int = 3) -> Scene:
    """Means uniform in [-half, half]^3 (the 16,384-Gaussian plain forward workload)."""
    gen = torch.Generator().manual_seed(seed)
    means = (torch.rand(3, n, generator=gen, dtype=torch.float32) * 2.0 - 1.0) * half
    return _finish(gen, means, log_scale_mu, log_scale_sd, sh_degree)


def blob_scene(n: int, seed: int = 0, n_blobs: int = 200, shell_frac: float = 0.1,
               log_scale_mu: float = -4.5, log_scale_sd: float = 0.8, sh_degree: int = 3) -> Scene:
    """Outdoor-like scene: (1 - shell_frac) of the means from ``n_blobs`` anisotropic
    Gaussian blobs (centres U([-20,20]x[-3,3]x[-20,20]), random rotation, axis
    std exp(N(0.5,0.5)), weights ~ Gamma(1)), the rest on a shell of radius U(60,80)."""
    gen = torch.Generator().manual_seed(seed)
    n_shell = int(round(n * shell_frac))
    n_blob = n - n_shell
    lo = torch.tensor([-20.0, -3.0, -20.0])
    hi = torch.tensor([20.0, 3.0, 20.0])
    centres = lo[:, None] + (hi - lo)[:, None] * torch.rand(3, n_blobs, generator=gen, dtype=torch.float32)
    # random blob orientations: Q factor of a Gaussian matrix, signs fixed so det = +1
    A = torch.randn(n_blobs, 3, 3, generator=gen, dtype=torch.float64)
    Q, Rr = torch.linalg.qr(A)
    Q = Q * torch.sign(torch.diagonal(Rr, dim1=-2, dim2=-1))[:, None, :]
    Q[torch.linalg.det(Q) < 0, :, 0] *= -1.0
    Rb = Q.permute(1, 2, 0).to(torch.float32)  # (3, 3, n_blobs)
    axis_sd = torch.exp(0.5 + 0.5 * torch.randn(3, n_blobs, generator=gen, dtype=torch.float32))
    weights = -torch.log(torch.rand(n_blobs, generator=gen, dtype=torch.float64).clamp_min(1e-300))  # Gamma(1)
    assign = torch.multinomial(weights / weights.sum(), n_blob, replacement=True, generator=gen)
    local = torch.randn(3, n_blob, generator=gen, dtype=torch.float32) * axis_sd[:, assign]
    blob_pts = torch.einsum("ijn,jn->in", Rb[:, :, assign], local) + centres[:, assign]
    d = torch.randn(3, n_shell, generator=gen, dtype=torch.float32)
    d = d / d.norm(dim=0, keepdim=True).clamp_min(1e-12)
    r = 60.0 + 20.0 * torch.rand(n_shell, generator=gen, dtype=torch.float32)
    shell_pts = d * r
    means = torch.cat([blob_pts, shell_pts], dim=1)
    return _finish(gen, means, log_scale_mu, log_scale_sd, sh_degree)


def prune_random(scene: Scene, keep: int, seed: int = 1) -> Scene:
    gen = torch.Generator().manual_seed(seed)
    idx = torch.randperm(scene.n, generator=gen)[:keep]
    return scene.subset(idx)


# ---- named workloads ---------------------------------------------------------

def small_box_workload(seed: int = 0):
    """16,384 Gaussians, means uniform in [-2,2]^3, 320x240, fov_y 60 deg, camera
    at (0,0,-5) looking down +z."""
    scene = uniform_box_scene(16384, seed)
    cam = pinhole(320, 240, 60.0, np.eye(3), np.array([0.0, 0.0, 5.0]))
    return scene, cam


def outdoor_workload(n: int = 3_000_000, seed: int = 0, width: int = 1280, height: int = 840):
    """Blob-mixture outdoor-like scene viewed from (0,0,-25) toward the origin."""
    scene = blob_scene(n, seed)
    cam = pinhole(width, height, 60.0, np.eye(3), np.array([0.0, 0.0, 25.0]))
    return scene, cam


RESOLUTIONS = [(640, 480), (980, 545), (1332, 876), (1920, 1080)]


def multiview_cameras(count: int = 64, seed: int = 6):
    gen = torch.Generator().manual_seed(seed)
    cams = []
    for _ in range(count):
        k = int(torch.randint(len(RESOLUTIONS), (1,), generator=gen))
        w, h = RESOLUTIONS[k]
        cams.append(orbit_camera(gen, w, h))
    return cams
