"""Soft and Hard Pruning (Sec. 4.2.2, 4.2.3) on a synthetic fitting task,
and the post-hoc comparison of the efficient pruning score with PUP's
(the shape of Table 4).

The rasterizer's differentiable render (``raster.DiffRenderer``) fits a
Gaussian model to seeded multi-view target images with the 3D-GS objective
(L1 + D-SSIM, Adam).  The loop follows the 3D-GS training recipe the paper
builds on, with every iteration count scaled by ``scale`` (1.0 = the paper's
30,000 iterations):
  * densification (clone small / split large Gaussians whose view-space
    positional gradient is large, drop transparent ones) from 500 to 15,000
    every 100 iterations, opacity reset every 3,000 until 15,000;
  * Soft Pruning: the ``soft_ratio`` lowest-scoring Gaussians are removed
    immediately before the opacity resets at 6,000, 9,000 and 12,000;
  * Hard Pruning: ``hard_ratio`` of them every 3,000 iterations from 15,000.
The score is the efficient pruning score of Sec. 4.2.1, summed over all
training views at pruning time (``gs_render_backward``'s score output), or
PUP's log det of the (mu, s) Hessian block (``raster.pup_scores``).

This is evaluation code around the hot path, not part of it: it runs the
CUDA rasterizer for every render, gradient and score.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np
import torch

from . import losses, raster, synth

KEYS = ("means", "scales", "rotations", "opacities", "sh")


@dataclass
class Schedule:
    scale: float = 0.1            # iteration counts relative to the paper's 30,000
    iterations: int = 30_000
    densify_from: int = 500
    densify_until: int = 15_000
    densify_every: int = 100
    reset_every: int = 3_000
    soft_at: tuple = (6_000, 9_000, 12_000)
    hard_from: int = 15_000
    hard_every: int = 3_000
    soft_ratio: float = 0.8
    hard_ratio: float = 0.3
    grad_threshold: float = 2e-4  # view-space positional gradient, normalised image coordinates
    dense_percent: float = 0.01   # a Gaussian is "small" below this fraction of the scene extent

    def at(self, it: int) -> int:
        return int(round(it * self.scale))

    def events(self, total: int, prune: bool = True):
        """Iterations of the Soft Prunes, the opacity resets and the Hard
        Prunes of a run of `total` iterations (scaled counts)."""
        soft = {self.at(x) for x in self.soft_at} if prune else set()
        resets = set(range(self.at(self.reset_every), self.at(self.densify_until), max(self.at(self.reset_every), 1)))
        hard = set(range(self.at(self.hard_from), total + 1, max(self.at(self.hard_every), 1))) if prune else set()
        return soft, resets, hard


class Model:
    """Raw (pre-activation) Gaussian parameters and their Adam optimiser."""

    def __init__(self, scene: synth.Scene, device, extent: float):
        d = torch.device(device)
        self.extent = extent
        self.means = scene.means.to(d).clone().requires_grad_(True)
        self.log_scales = torch.log(scene.scales.to(d)).clone().requires_grad_(True)
        self.quats = scene.rotations.to(d).clone().requires_grad_(True)
        op = scene.opacities.to(d).clamp(1e-4, 1 - 1e-4)
        self.logits = torch.log(op / (1 - op)).clone().requires_grad_(True)
        self.sh = scene.sh.to(d).clone().requires_grad_(True)
        self.sh_degree = scene.sh_degree
        self.make_optimizer()

    def params(self):
        return [self.means, self.log_scales, self.quats, self.logits, self.sh]

    def make_optimizer(self, states=None):
        lr = [1.6e-4 * self.extent, 5e-3, 1e-3, 5e-2, 2.5e-3]
        self.opt = torch.optim.Adam([{"params": [p], "lr": r} for p, r in zip(self.params(), lr)], eps=1e-15)
        if states is not None:
            for p, st in zip(self.params(), states):
                if st:
                    self.opt.state[p] = st

    @property
    def n(self) -> int:
        return int(self.means.shape[1])

    def activated(self):
        q = self.quats / self.quats.norm(dim=0, keepdim=True).clamp_min(1e-12)
        return (self.means, torch.exp(self.log_scales), q, torch.sigmoid(self.logits), self.sh)

    def scene(self) -> synth.Scene:
        with torch.no_grad():
            m, s, q, o, h = self.activated()
            return synth.Scene(m.detach().contiguous(), s.detach().contiguous(), q.detach().contiguous(),
                               o.detach().contiguous(), h.detach().contiguous(), self.sh_degree)

    def _replace(self, tensors, state_fn):
        """New parameter tensors; Adam moments carried over through state_fn."""
        states = []
        for p in self.params():
            st = self.opt.state.get(p, {})
            states.append({k: (state_fn(v) if torch.is_tensor(v) and v.dim() > 0 else v) for k, v in st.items()})
        self.means, self.log_scales, self.quats, self.logits, self.sh = [t.detach().contiguous().requires_grad_(True)
                                                                         for t in tensors]
        self.make_optimizer(states)

    def keep(self, mask: torch.Tensor):
        idx = torch.nonzero(mask).squeeze(1)
        self._replace([p.detach()[..., idx] for p in self.params()], lambda v: v[..., idx].contiguous())

    def append(self, parts):
        k = parts[0].shape[-1]
        self._replace([torch.cat([p.detach(), x], dim=-1) for p, x in zip(self.params(), parts)],
                      lambda v: torch.cat([v, torch.zeros(*v.shape[:-1], k, dtype=v.dtype, device=v.device)], -1))

    def reset_opacity(self):
        with torch.no_grad():
            self.logits.copy_(torch.minimum(self.logits, torch.full_like(self.logits, math.log(0.01 / 0.99))))
        st = self.opt.state.get(self.logits)
        if st:
            st["exp_avg"].zero_()
            st["exp_avg_sq"].zero_()


def densify(model: Model, grad_acc: torch.Tensor, counts: torch.Tensor, sch: Schedule, gen: torch.Generator):
    """3D-GS adaptive density control: clone small and split large Gaussians
    whose mean view-space positional gradient exceeds the threshold; drop
    nearly transparent ones."""
    with torch.no_grad():
        g = grad_acc / counts.clamp_min(1)
        big = g >= sch.grad_threshold
        smax = torch.exp(model.log_scales).max(0).values
        small = smax <= sch.dense_percent * model.extent
        clone = big & small
        split = big & ~small
        parts = []
        if clone.any():
            parts.append([p.detach()[..., clone] for p in model.params()])
        if split.any():
            idx = torch.nonzero(split).squeeze(1)
            s = torch.exp(model.log_scales[:, idx])
            q = model.quats[:, idx] / model.quats[:, idx].norm(dim=0, keepdim=True)
            w, x, y, z = q
            R = torch.stack([torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)]),
                             torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)]),
                             torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)])])
            for _ in range(2):
                off = torch.randn(3, len(idx), generator=gen).to(s.device) * s
                mu = model.means[:, idx] + torch.einsum("ijn,jn->in", R, off)
                parts.append([mu, model.log_scales[:, idx] - math.log(1.6), model.quats[:, idx],
                              model.logits[idx], model.sh[..., idx]])
        keep = ~split & (torch.sigmoid(model.logits) > 0.005)
    if parts:
        cat = [torch.cat([pp[k] for pp in parts], dim=-1).detach() for k in range(5)]
        model.keep(keep)
        model.append(cat)
    else:
        model.keep(keep)


def efficient_scores(model: Model, views, renderer: raster.Renderer, mode="accutile", tile=16):
    """Sec. 4.2.1: sum over the views, pixels and channels of (dC/dg_i)^2."""
    scene = model.scene()
    n = scene.n
    dev = scene.means.device
    score = torch.zeros(n, device=dev)
    grads = {k: torch.empty_like(getattr(scene, k)) for k in KEYS}
    grads["score"] = score
    work = torch.empty(max(raster.backward_work_bytes(n) // 4, 4), device=dev)
    cfg = raster.cfg_struct(tile, mode)
    for cam in views:
        out = renderer.render(scene, cam, mode, tile)
        zero = torch.zeros(3, cam.height, cam.width, device=dev)
        renderer.rast.gs_render_backward(scene, cam, cfg, out.frame, zero, grads, work)
    return score


def pup_scores(model: Model, views, renderer: raster.Renderer, mode="accutile", tile=16):
    return raster.pup_scores(renderer, model.scene(), views, mode, tile)[1]


def psnr(model: Model, views, targets, renderer: raster.Renderer, mode="accutile", tile=16) -> float:
    scene = model.scene()
    vals = []
    for cam, tgt in zip(views, targets):
        img = renderer.render(scene, cam, mode, tile).image.clamp(0, 1)
        mse = float(((img - tgt) ** 2).mean())
        vals.append(10 * math.log10(1.0 / max(mse, 1e-12)))
    return float(np.mean(vals))


def render_ms(model: Model, views, renderer: raster.Renderer, mode="accutile", tile=16, reps=5) -> float:
    """ms per view of the forward render of the model (CUDA events)."""
    scene = model.scene()
    rast = renderer.rast
    cfg = raster.cfg_struct(tile, mode)
    frames = [renderer.render(scene, c, mode, tile).frame for c in views]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(rast.stream)
    for _ in range(reps):
        for c, f in zip(views, frames):
            rast.gs_forward(scene, c, cfg, f)
    e1.record(rast.stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / (reps * len(views))


def prune_by(model: Model, score: torch.Tensor, ratio: float):
    """Remove the ``ratio`` lowest-scoring Gaussians (NaN and -inf count lowest)."""
    n = model.n
    k = int(math.floor(ratio * n))
    if k <= 0:
        return
    s = torch.nan_to_num(score.float(), nan=-float("inf"))
    order = torch.argsort(s, stable=True)
    keep = torch.ones(n, dtype=torch.bool, device=s.device)
    keep[order[:k]] = False
    model.keep(keep)


@dataclass
class Task:
    """Seeded multi-view fitting task: a ground-truth scene, its training and
    test views and their target images, and an over-complete initial model."""
    gt: synth.Scene
    train: list
    test: list
    train_img: list
    test_img: list
    init: synth.Scene
    extent: float


def make_task(device, n_gt=20_000, n_extra=20_000, train_views=16, test_views=4, res=(256, 192), seed=30) -> Task:
    gen = torch.Generator().manual_seed(seed)
    gt = synth.uniform_box_scene(n_gt, seed=seed, half=2.0, log_scale_mu=-3.3, log_scale_sd=0.4)

    def ring(k, count, radius, phase):
        a = 2 * math.pi * (k + phase) / count
        el = 0.35 * math.sin(3 * a)
        return synth.look_at(res[0], res[1], 50.0, (radius * math.cos(el) * math.sin(a), -radius * math.sin(el),
                                                    -radius * math.cos(el) * math.cos(a)))

    train = [ring(k, train_views, 7.0, 0.0) for k in range(train_views)]
    test = [ring(k, test_views, 7.5, 0.37) for k in range(test_views)]
    r = raster.Renderer(device)
    gd = gt.to(device)
    train_img = [r.render(gd, c, "accutile", 16).image.clone() for c in train]
    test_img = [r.render(gd, c, "accutile", 16).image.clone() for c in test]
    # over-complete start: the ground truth's Gaussians displaced, with
    # flattened colours and half opacity, plus extra random ones
    jit = synth.Scene(gt.means + 0.05 * torch.randn(gt.means.shape, generator=gen),
                      gt.scales * torch.exp(0.3 * torch.randn(gt.scales.shape, generator=gen)),
                      gt.rotations, torch.full_like(gt.opacities, 0.5),
                      gt.sh * 0.5 + 0.05 * torch.randn(gt.sh.shape, generator=gen), gt.sh_degree)
    extra = synth.uniform_box_scene(n_extra, seed=seed + 1, half=2.2, log_scale_mu=-3.3, log_scale_sd=0.4)
    extra.opacities[:] = 0.1
    init = synth.Scene(*[torch.cat([getattr(jit, k), getattr(extra, k)], dim=-1).contiguous() for k in KEYS], 3)
    return Task(gt, train, test, train_img, test_img, init, extent=2.0 * math.sqrt(3.0))


def fit(task: Task, device, sch: Schedule, prune: bool = True, score: str = "efficient", start=None, log=None,
        iterations=None, densify_on: bool = True, seed: int = 31):
    """Train from ``start`` (default: the task's initial model).  Returns the
    model and a list of events (iteration, what, Gaussians)."""
    dev = torch.device(device)
    model = start if start is not None else Model(task.init, dev, task.extent)
    diff = raster.DiffRenderer(dev)
    renderer = diff.renderer
    gen = torch.Generator().manual_seed(seed)
    total = sch.at(sch.iterations) if iterations is None else iterations
    grad_acc = torch.zeros(model.n, device=dev)
    seen = torch.zeros(model.n, device=dev)
    events = []
    order = torch.randperm(len(task.train), generator=gen).tolist()
    soft, resets, hard = sch.events(total, prune)
    lr0 = model.opt.param_groups[0]["lr"]
    t0 = time.perf_counter()
    for it in range(1, total + 1):
        if not order:
            order = torch.randperm(len(task.train), generator=gen).tolist()
        v = order.pop()
        cam, tgt = task.train[v], task.train_img[v]
        # position learning rate: exponential decay to 1% over the run
        model.opt.param_groups[0]["lr"] = lr0 * (0.01 ** (it / total))
        img = diff.render(*model.activated(), cam)
        loss = losses.gs_loss(img, tgt)
        model.opt.zero_grad(set_to_none=True)
        loss.backward()
        model.opt.step()
        if densify_on and it < sch.at(sch.densify_until) and diff.means2d_grad is not None:
            g2 = diff.means2d_grad
            # gradient in normalised image coordinates, as 3D-GS thresholds it
            gn = torch.sqrt((g2[0] * cam.width * 0.5) ** 2 + (g2[1] * cam.height * 0.5) ** 2)
            grad_acc += gn
            seen += (gn > 0).float()
            if it >= sch.at(sch.densify_from) and it % max(sch.at(sch.densify_every), 1) == 0:
                densify(model, grad_acc, seen, sch, gen)
                grad_acc = torch.zeros(model.n, device=dev)
                seen = torch.zeros(model.n, device=dev)
        if prune and it in soft:
            s = efficient_scores(model, task.train, renderer) if score == "efficient" else \
                pup_scores(model, task.train, renderer)
            prune_by(model, s, sch.soft_ratio)
            events.append((it, "soft", model.n))
            grad_acc = torch.zeros(model.n, device=dev)
            seen = torch.zeros(model.n, device=dev)
        if it in resets:
            model.reset_opacity()
            events.append((it, "reset", model.n))
        if prune and it in hard:
            s = efficient_scores(model, task.train, renderer) if score == "efficient" else \
                pup_scores(model, task.train, renderer)
            prune_by(model, s, sch.hard_ratio)
            events.append((it, "hard", model.n))
        if log and it % max(total // 10, 1) == 0:
            log(f"it {it}: n {model.n}, loss {float(loss):.4f}, {time.perf_counter() - t0:.1f} s")
    return model, events


def run_schedule(device, sch: Schedule | None = None, task: Task | None = None, log=None) -> dict:
    """The baseline fit (densification, no pruning) against the same fit with
    Soft + Hard Pruning by the efficient score: Gaussians, test PSNR, render
    ms per view and training time (the shape of Tables 1 and 2)."""
    sch = sch or Schedule()
    task = task or make_task(device)
    r = raster.Renderer(device)
    out = {"schedule": {k: getattr(sch, k) for k in ("scale", "soft_ratio", "hard_ratio")},
           "iterations": sch.at(sch.iterations), "train_views": len(task.train), "test_views": len(task.test),
           "resolution": f"{task.train[0].width}x{task.train[0].height}", "gt_gaussians": task.gt.n,
           "init_gaussians": task.init.n}
    # an untimed 20-iteration fit first, so neither timed fit carries the
    # process's first-use set-up (library handles, allocator growth)
    fit(task, device, sch, prune=False, iterations=20)
    torch.cuda.synchronize()
    for name, prune in (("baseline", False), ("soft_hard", True)):
        t0 = time.perf_counter()
        model, events = fit(task, device, sch, prune=prune, log=log)
        torch.cuda.synchronize()
        out[name] = {"gaussians": model.n, "test_psnr": psnr(model, task.test, task.test_img, r),
                     "render_ms_per_view": render_ms(model, task.test, r), "train_s": time.perf_counter() - t0,
                     "events": events}
    b, p = out["baseline"], out["soft_hard"]
    out["compression"] = b["gaussians"] / max(p["gaussians"], 1)
    out["render_speedup"] = b["render_ms_per_view"] / p["render_ms_per_view"]
    return out


def run_pup_vs_efficient(device, sch: Schedule | None = None, task: Task | None = None, rounds=2, ratio=0.66,
                         refine=None, log=None) -> dict:
    """Table 4's protocol on the synthetic task: from one fitted baseline,
    ``rounds`` of (prune ``ratio`` of the Gaussians by a score, fine-tune
    ``refine`` iterations), with the efficient score and with PUP's; plus
    each score's memory per Gaussian and time over the training views."""
    sch = sch or Schedule()
    task = task or make_task(device)
    r = raster.Renderer(device)
    base, _ = fit(task, device, sch, prune=False, log=log)
    refine = refine if refine is not None else sch.at(5_000)
    snap = [p.detach().clone() for p in base.params()]
    out = {"baseline": {"gaussians": base.n, "test_psnr": psnr(base, task.test, task.test_img, r),
                        "render_ms_per_view": render_ms(base, task.test, r)},
           "rounds": rounds, "ratio_per_round": ratio, "refine_iterations": refine}
    for name in ("efficient", "pup"):
        m = Model(base.scene(), torch.device(device), task.extent)
        with torch.no_grad():
            for p, s in zip(m.params(), snap):
                p.copy_(s)
        t_score = 0.0
        for _ in range(rounds):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s = efficient_scores(m, task.train, r) if name == "efficient" else pup_scores(m, task.train, r)
            torch.cuda.synchronize()
            t_score += time.perf_counter() - t0
            prune_by(m, s, ratio)
            m, _ = fit(task, device, sch, prune=False, start=m, iterations=refine, densify_on=False)
        out[name] = {"gaussians": m.n, "test_psnr": psnr(m, task.test, task.test_img, r),
                     "render_ms_per_view": render_ms(m, task.test, r), "score_s_per_round": t_score / rounds,
                     "score_floats_per_gaussian": 1 if name == "efficient" else 21}
    return out
