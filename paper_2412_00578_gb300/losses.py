"""Image losses of the 3D-GS objective (Eq. gs_loss): L1 and D-SSIM, in plain
PyTorch (autograd supplies dL/dimage for the rasterizer's backward).

SSIM uses the usual 11x11 Gaussian window with sigma 1.5 and constants
C1 = 0.01^2, C2 = 0.03^2 on images in [0, 1]; D-SSIM = 1 - SSIM.  The
combination (1 - lam) L1 + lam D-SSIM with lam = 0.2 is the 3D-GS weighting.
"""
from __future__ import annotations

import torch
import torch.nn.functional as F


def _window(size: int = 11, sigma: float = 1.5, device=None) -> torch.Tensor:
    x = torch.arange(size, dtype=torch.float32, device=device) - (size - 1) / 2
    g = torch.exp(-(x * x) / (2 * sigma * sigma))
    g = g / g.sum()
    return (g[:, None] * g[None, :]).expand(3, 1, size, size).contiguous()


def ssim(img: torch.Tensor, ref: torch.Tensor) -> torch.Tensor:
    """Mean SSIM of two (3, H, W) images."""
    w = _window(device=img.device)
    a = img[None]
    b = ref[None]
    pad = w.shape[-1] // 2
    mu_a = F.conv2d(a, w, padding=pad, groups=3)
    mu_b = F.conv2d(b, w, padding=pad, groups=3)
    s_aa = F.conv2d(a * a, w, padding=pad, groups=3) - mu_a * mu_a
    s_bb = F.conv2d(b * b, w, padding=pad, groups=3) - mu_b * mu_b
    s_ab = F.conv2d(a * b, w, padding=pad, groups=3) - mu_a * mu_b
    c1, c2 = 0.01 ** 2, 0.03 ** 2
    m = ((2 * mu_a * mu_b + c1) * (2 * s_ab + c2)) / ((mu_a * mu_a + mu_b * mu_b + c1) * (s_aa + s_bb + c2))
    return m.mean()


def gs_loss(img: torch.Tensor, ref: torch.Tensor, lam: float = 0.2) -> torch.Tensor:
    return (1.0 - lam) * (img - ref).abs().mean() + lam * (1.0 - ssim(img, ref))
