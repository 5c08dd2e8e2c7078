"""Python binding of the C ABI in ``include/gs.h`` (argument marshalling only).

Every stage runs in the CUDA library ``_build/libgs.so``; this module only
allocates the caller-owned device buffers with PyTorch, fills the C structs
and checks status codes.  Importing it raises if the library has not been
built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
from ctypes import POINTER, c_float, c_int32, c_int64, c_uint32, c_void_p
from dataclasses import dataclass

import torch

from . import build as _build

MODES = {"3sigma": 0, "snugbox": 1, "accutile": 2, "tbc": 3, "pixel": 4}
MODE_NAMES = {v: k for k, v in MODES.items()}
FLAG_CAPACITY = 1
FLAG_TIMEOUT = 2
FLAG_KEYRANGE = 8
STATUS_NAMES = {0: "GS_OK", 1: "GS_ERR_INVALID", 2: "GS_ERR_OOM", 3: "GS_ERR_CAPACITY", 4: "GS_ERR_CUDA",
                5: "GS_ERR_TIMEOUT"}
MAX_KEYS = (1 << 30) - 1


class GsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class GsScene(ctypes.Structure):
    _fields_ = [("n", c_int64), ("sh_degree", c_int32), ("means", c_void_p), ("scales", c_void_p),
                ("rotations", c_void_p), ("opacities", c_void_p), ("sh", c_void_p)]


class GsCamera(ctypes.Structure):
    _fields_ = [("width", c_int32), ("height", c_int32), ("fx", c_float), ("fy", c_float), ("cx", c_float),
                ("cy", c_float), ("tan_fovx", c_float), ("tan_fovy", c_float), ("near_z", c_float),
                ("viewmat", c_float * 12), ("campos", c_float * 3)]


class GsRasterCfg(ctypes.Structure):
    _fields_ = [("tile", c_int32), ("mode", c_int32), ("bg", c_float * 3), ("sort_digit_bits", c_int32)]


class GsFrame(ctypes.Structure):
    _fields_ = [("n_capacity", c_int64), ("key_capacity", c_int64), ("width", c_int32), ("height", c_int32),
                ("tile", c_int32), ("proj", c_void_p), ("counts", c_void_p), ("keys", c_void_p),
                ("vals", c_void_p), ("ranges", c_void_p), ("image", c_void_p), ("final_T", c_void_p),
                ("last", c_void_p), ("scratch", c_void_p)]


class GsBatchFrame(ctypes.Structure):
    _fields_ = [("n_capacity", c_int64), ("key_capacity", c_int64), ("tile_capacity", c_int64),
                ("pixel_capacity", c_int64), ("max_cams", c_int32), ("tile", c_int32), ("proj", c_void_p),
                ("counts", c_void_p), ("keys", c_void_p), ("vals", c_void_p), ("ranges", c_void_p),
                ("image", c_void_p), ("final_T", c_void_p), ("last", c_void_p), ("scratch", c_void_p)]


class GsGrads(ctypes.Structure):
    _fields_ = [(k, c_void_p) for k in ("means", "scales", "rotations", "opacities", "sh", "means2d", "score",
                                        "work")]


class GsFrameBytes(ctypes.Structure):
    _fields_ = [(k, c_int64) for k in ("proj", "counts", "keys", "vals", "ranges", "image", "final_T", "last",
                                       "scratch")]


EXPORTS = ["gs_create", "gs_destroy", "gs_set_stream", "gs_last_error", "gs_launch_count", "gs_frame_sizes",
           "gs_preprocess", "gs_intersect", "gs_sort", "gs_tile_ranges", "gs_render", "gs_render_stats",
           "gs_forward", "gs_read_status", "gs_backward_work_bytes", "gs_render_backward", "gs_intersect_noalloc",
           "gs_batch_sizes", "gs_forward_batch", "gs_batch_status", "gs_read_culled", "gs_set_sort_wait",
           "gs_pup_work_bytes", "gs_pup_accumulate", "gs_pup_score", "gs_read_sort_plan", "gs_sort_plan_for"]

_lib = None


def load(path=None) -> ctypes.CDLL:
    """Load libgs.so; raises if it is missing (build it with ``build.build()``)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or _build.LIB
    if not p.exists():
        raise RuntimeError(f"CUDA library {p} is not built; run paper_2412_00578_gb300.build.build() "
                           "(there is no CPU fallback)")
    L = ctypes.CDLL(str(p))
    P = c_void_p
    L.gs_create.argtypes = [ctypes.c_int, P, POINTER(c_void_p)]
    L.gs_destroy.argtypes = [P]
    L.gs_destroy.restype = None
    L.gs_set_stream.argtypes = [P, P]
    L.gs_last_error.argtypes = [P]
    L.gs_last_error.restype = ctypes.c_char_p
    L.gs_launch_count.argtypes = [P]
    L.gs_launch_count.restype = c_int64
    L.gs_frame_sizes.argtypes = [c_int64, c_int32, c_int32, c_int32, c_int64, POINTER(GsFrameBytes)]
    L.gs_preprocess.argtypes = [P, POINTER(GsScene), POINTER(GsCamera), POINTER(GsRasterCfg), POINTER(GsFrame)]
    L.gs_intersect.argtypes = [P, POINTER(GsCamera), POINTER(GsRasterCfg), POINTER(GsFrame), POINTER(c_int64)]
    for name in ("gs_sort", "gs_tile_ranges", "gs_render"):
        getattr(L, name).argtypes = [P, POINTER(GsCamera), POINTER(GsRasterCfg), POINTER(GsFrame)]
    L.gs_forward.argtypes = [P, POINTER(GsScene), POINTER(GsCamera), POINTER(GsRasterCfg), POINTER(GsFrame)]
    L.gs_read_status.argtypes = [P, POINTER(GsFrame), POINTER(c_int64), POINTER(c_uint32)]
    L.gs_read_sort_plan.argtypes = [P, POINTER(GsRasterCfg), POINTER(GsFrame), POINTER(c_int32), POINTER(c_int32),
                                    POINTER(c_int32)]
    L.gs_sort_plan_for.argtypes = [c_int64, c_uint32, c_uint32, c_int32, c_int32, POINTER(c_int32), POINTER(c_int32),
                                   POINTER(c_int32), POINTER(c_int32)]
    L.gs_render_stats.argtypes = [P, POINTER(GsCamera), POINTER(GsRasterCfg), POINTER(GsFrame),
                                  POINTER(ctypes.c_uint64), POINTER(ctypes.c_uint64), POINTER(ctypes.c_uint64)]
    L.gs_backward_work_bytes.argtypes = [c_int64]
    L.gs_batch_sizes.argtypes = [c_int64, c_int32, c_int32, c_int64, c_int64, c_int64, POINTER(GsFrameBytes)]
    L.gs_forward_batch.argtypes = [P, POINTER(GsScene), P, c_int32, POINTER(GsRasterCfg), POINTER(GsBatchFrame)]
    L.gs_batch_status.argtypes = [P, POINTER(GsBatchFrame), POINTER(c_int64), POINTER(c_uint32)]
    L.gs_intersect_noalloc.argtypes = [P, POINTER(GsCamera), POINTER(GsRasterCfg), POINTER(GsFrame),
                                       POINTER(c_int64)]
    L.gs_read_culled.argtypes = [P, POINTER(GsFrame), POINTER(c_int64)]
    L.gs_pup_work_bytes.argtypes = [c_int64]
    L.gs_pup_accumulate.argtypes = [P, POINTER(GsScene), POINTER(GsCamera), POINTER(GsRasterCfg), POINTER(GsFrame), P, P]
    L.gs_pup_score.argtypes = [P, P, c_int64, P]
    L.gs_set_sort_wait.argtypes = [P, c_uint32, c_int64]
    L.gs_render_backward.argtypes = [P, POINTER(GsScene), POINTER(GsCamera), POINTER(GsRasterCfg), POINTER(GsFrame),
                                     P, POINTER(GsGrads)]
    for name in EXPORTS:
        getattr(L, name).restype = ctypes.c_int
    L.gs_backward_work_bytes.restype = c_int64
    L.gs_pup_work_bytes.restype = c_int64
    L.gs_destroy.restype = None
    L.gs_last_error.restype = ctypes.c_char_p
    L.gs_launch_count.restype = c_int64
    if path is None:
        _lib = L
    return L


# ---------------------------------------------------------------- marshalling
def camera_struct(cam) -> GsCamera:
    c = GsCamera()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.tan_fovx, c.tan_fovy = float(cam.tan_fovx), float(cam.tan_fovy)
    c.near_z = float(getattr(cam, "near_z", 0.2))
    vm = [float(x) for x in cam.viewmat.reshape(-1)]
    c.viewmat[:] = vm
    c.campos[:] = [float(x) for x in cam.campos.reshape(-1)]
    return c


def scene_struct(scene) -> GsScene:
    for k in ("means", "scales", "rotations", "opacities", "sh"):
        t = getattr(scene, k)
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise ValueError(f"scene.{k} must be a contiguous float32 CUDA tensor")
    s = GsScene()
    s.n = int(scene.means.shape[1])
    s.sh_degree = int(scene.sh_degree)
    s.means, s.scales = scene.means.data_ptr(), scene.scales.data_ptr()
    s.rotations, s.opacities, s.sh = scene.rotations.data_ptr(), scene.opacities.data_ptr(), scene.sh.data_ptr()
    return s


def cfg_struct(tile: int, mode, bg=(0.0, 0.0, 0.0), sort_digit_bits: int = 0) -> GsRasterCfg:
    c = GsRasterCfg()
    c.tile = int(tile)
    c.mode = MODES[mode] if isinstance(mode, str) else int(mode)
    c.bg[:] = [float(x) for x in bg]
    c.sort_digit_bits = int(sort_digit_bits)
    return c


def frame_sizes(n: int, width: int, height: int, tile: int, key_capacity: int) -> GsFrameBytes:
    out = GsFrameBytes()
    st = load().gs_frame_sizes(int(n), int(width), int(height), int(tile), int(key_capacity), ctypes.byref(out))
    if st != 0:
        raise GsError(st, f"gs_frame_sizes(n={n}, {width}x{height}, tile={tile}, keys={key_capacity})")
    return out


class Frame:
    """Caller-owned device buffers of one raster (gs_frame), allocated by torch."""

    def __init__(self, n: int, width: int, height: int, tile: int, key_capacity: int, device=None):
        device = torch.device(device or "cuda")
        sz = frame_sizes(n, width, height, tile, key_capacity)
        self.n, self.width, self.height, self.tile, self.key_capacity = n, width, height, tile, key_capacity
        self.gx, self.gy = (width + tile - 1) // tile, (height + tile - 1) // tile
        e = lambda nbytes, dt, es: torch.empty(max(nbytes // es, 1), dtype=dt, device=device)
        self.proj = e(sz.proj, torch.float32, 4)
        self.counts = e(sz.counts, torch.int32, 4)
        self.keys = e(sz.keys, torch.int64, 8)
        self.vals = e(sz.vals, torch.int32, 4)
        self.ranges = e(sz.ranges, torch.int32, 4)
        self.image = torch.empty(3, height, width, dtype=torch.float32, device=device)
        self.final_T = torch.empty(height, width, dtype=torch.float32, device=device)
        self.last = torch.empty(height, width, dtype=torch.int32, device=device)
        self.scratch = torch.zeros(max(sz.scratch, 1), dtype=torch.uint8, device=device)
        self.bytes = sz
        f = GsFrame()
        f.n_capacity, f.key_capacity = n, key_capacity
        f.width, f.height, f.tile = width, height, tile
        f.proj, f.counts, f.keys, f.vals = (self.proj.data_ptr(), self.counts.data_ptr(), self.keys.data_ptr(),
                                            self.vals.data_ptr())
        f.ranges, f.image, f.final_T, f.last = (self.ranges.data_ptr(), self.image.data_ptr(),
                                                self.final_T.data_ptr(), self.last.data_ptr())
        f.scratch = self.scratch.data_ptr()
        self.struct = f

    # views (valid after the corresponding stage has run)
    def proj_planes(self):
        return self.proj[: 3 * self.n * 4].view(3, self.n, 4)

    def sorted_pairs(self, K: int):
        return self.keys[:K], self.vals[:K]

    def unsorted_pairs(self, K: int):
        return self.keys[:K], self.vals[:K]

    generation = 0  # bumped by every forward render into this frame

    def tile_ranges(self):
        return self.ranges[: self.gx * self.gy * 2].view(self.gx * self.gy, 2)

    def nbytes(self) -> int:
        s = self.bytes
        return s.proj + s.counts + s.keys + s.vals + s.ranges + s.image + s.final_T + s.last + s.scratch


class Rasterizer:
    """A gs_context bound to one device and stream, with the six stage calls."""

    def __init__(self, device=None, stream=None):
        self.lib = load()
        self.device = torch.device(device or "cuda")
        idx = self.device.index if self.device.index is not None else torch.cuda.current_device()
        self.device = torch.device("cuda", idx)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        ctx = c_void_p()
        st = self.lib.gs_create(idx, c_void_p(s.cuda_stream), ctypes.byref(ctx))
        if st != 0:
            raise GsError(st, "gs_create failed")
        self.ctx = ctx
        self.stream = s

    def __del__(self):
        ctx = getattr(self, "ctx", None)
        if ctx and getattr(self, "lib", None) is not None:
            self.lib.gs_destroy(ctx)
            self.ctx = None

    def set_stream(self, stream):
        self.stream = stream
        self._check(self.lib.gs_set_stream(self.ctx, c_void_p(stream.cuda_stream)), "gs_set_stream")

    def _check(self, st: int, what: str):
        if st != 0:
            raise GsError(st, f"{what}: {self.lib.gs_last_error(self.ctx).decode(errors='replace')}")

    def launch_count(self) -> int:
        return int(self.lib.gs_launch_count(self.ctx))

    # ---- stages (names follow gs.h)
    def gs_preprocess(self, scene, cam, cfg, frame: Frame):
        s, c = scene_struct(scene), camera_struct(cam)
        self._check(self.lib.gs_preprocess(self.ctx, ctypes.byref(s), ctypes.byref(c), ctypes.byref(cfg),
                                           ctypes.byref(frame.struct)), "gs_preprocess")

    def gs_intersect(self, cam, cfg, frame: Frame, sync: bool = False):
        c = camera_struct(cam)
        if sync:
            k = c_int64(0)
            st = self.lib.gs_intersect(self.ctx, ctypes.byref(c), ctypes.byref(cfg), ctypes.byref(frame.struct),
                                       ctypes.byref(k))
            if st == 3:
                return int(k.value)
            self._check(st, "gs_intersect")
            return int(k.value)
        self._check(self.lib.gs_intersect(self.ctx, ctypes.byref(c), ctypes.byref(cfg), ctypes.byref(frame.struct),
                                          None), "gs_intersect")
        return None

    def gs_intersect_noalloc(self, cam, cfg, frame_struct: GsFrame) -> int:
        """gs_intersect without caller scratch (frame_struct.scratch may be None);
        synchronises and returns the key total K."""
        c = camera_struct(cam)
        k = c_int64(0)
        self._check(self.lib.gs_intersect_noalloc(self.ctx, ctypes.byref(c), ctypes.byref(cfg),
                                                  ctypes.byref(frame_struct), ctypes.byref(k)), "gs_intersect_noalloc")
        return int(k.value)

    def gs_sort(self, cam, cfg, frame: Frame):
        c = camera_struct(cam)
        self._check(self.lib.gs_sort(self.ctx, ctypes.byref(c), ctypes.byref(cfg), ctypes.byref(frame.struct)),
                    "gs_sort")

    def gs_tile_ranges(self, cam, cfg, frame: Frame):
        c = camera_struct(cam)
        self._check(self.lib.gs_tile_ranges(self.ctx, ctypes.byref(c), ctypes.byref(cfg),
                                             ctypes.byref(frame.struct)), "gs_tile_ranges")

    def gs_render(self, cam, cfg, frame: Frame):
        c = camera_struct(cam)
        self._check(self.lib.gs_render(self.ctx, ctypes.byref(c), ctypes.byref(cfg), ctypes.byref(frame.struct)),
                    "gs_render")

    def gs_render_stats(self, cam, cfg, frame: Frame):
        """Instrumented blend: (pairs the definition evaluates, contributing pairs, pairs executed)."""
        c = camera_struct(cam)
        ev, co, ex = ctypes.c_uint64(0), ctypes.c_uint64(0), ctypes.c_uint64(0)
        self._check(self.lib.gs_render_stats(self.ctx, ctypes.byref(c), ctypes.byref(cfg), ctypes.byref(frame.struct),
                                             ctypes.byref(ev), ctypes.byref(co), ctypes.byref(ex)), "gs_render_stats")
        return int(ev.value), int(co.value), int(ex.value)

    def gs_render_backward(self, scene, cam, cfg, frame: Frame, dL_dimage: torch.Tensor, grads: dict,
                           work: torch.Tensor):
        """grads: dict of CUDA float32 tensors shaped like the scene arrays
        (means, scales, rotations, opacities, sh), optional means2d (2, n)
        and score (n,) (added to)."""
        s, c = scene_struct(scene), camera_struct(cam)
        if not (dL_dimage.is_cuda and dL_dimage.dtype == torch.float32 and dL_dimage.is_contiguous()):
            raise ValueError("dL_dimage must be a contiguous float32 CUDA tensor of shape (3, H, W)")
        g = GsGrads()
        for k in ("means", "scales", "rotations", "opacities", "sh", "means2d", "score"):
            t = grads.get(k)
            setattr(g, k, t.data_ptr() if t is not None else None)
        g.work = work.data_ptr()
        self._check(self.lib.gs_render_backward(self.ctx, ctypes.byref(s), ctypes.byref(c), ctypes.byref(cfg),
                                                ctypes.byref(frame.struct), c_void_p(dL_dimage.data_ptr()),
                                                ctypes.byref(g)), "gs_render_backward")

    def gs_pup_accumulate(self, scene, cam, cfg, frame: Frame, hessian: torch.Tensor, work: torch.Tensor):
        """Adds one view's PUP sensitivity terms to hessian ([21, n] float32,
        device) for the frame's completed forward render."""
        s, c = scene_struct(scene), camera_struct(cam)
        self._check(self.lib.gs_pup_accumulate(self.ctx, ctypes.byref(s), ctypes.byref(c), ctypes.byref(cfg),
                                               ctypes.byref(frame.struct), c_void_p(hessian.data_ptr()),
                                               c_void_p(work.data_ptr())), "gs_pup_accumulate")

    def gs_pup_score(self, hessian: torch.Tensor, n: int, score: torch.Tensor):
        self._check(self.lib.gs_pup_score(self.ctx, c_void_p(hessian.data_ptr()), int(n), c_void_p(score.data_ptr())),
                    "gs_pup_score")

    def gs_forward(self, scene, cam, cfg, frame: Frame):
        s, c = scene_struct(scene), camera_struct(cam)
        self._check(self.lib.gs_forward(self.ctx, ctypes.byref(s), ctypes.byref(c), ctypes.byref(cfg),
                                        ctypes.byref(frame.struct)), "gs_forward")

    def gs_forward_batch(self, scene, cams_dev: torch.Tensor, num_cams: int, cfg, frame: "BatchFrame"):
        """cams_dev: device tensor holding num_cams packed gs_camera structs."""
        s = scene_struct(scene)
        self._check(self.lib.gs_forward_batch(self.ctx, ctypes.byref(s), c_void_p(cams_dev.data_ptr()),
                                              int(num_cams), ctypes.byref(cfg), ctypes.byref(frame.struct)),
                    "gs_forward_batch")

    def gs_batch_status(self, frame: "BatchFrame", raise_on_error: bool = True):
        k = c_int64(0)
        fl = c_uint32(0)
        st = self.lib.gs_batch_status(self.ctx, ctypes.byref(frame.struct), ctypes.byref(k), ctypes.byref(fl))
        if st != 0 and (raise_on_error or st not in (1, 3, 5) or not fl.value):
            self._check(st, "gs_batch_status")  # CUDA errors always raise
        return int(k.value), int(fl.value)

    def gs_read_culled(self, frame: Frame) -> int:
        k = c_int64(0)
        self._check(self.lib.gs_read_culled(self.ctx, ctypes.byref(frame.struct), ctypes.byref(k)), "gs_read_culled")
        return int(k.value)

    def gs_set_sort_wait(self, max_polls: int = 0, withhold_partition: int = -1):
        self._check(self.lib.gs_set_sort_wait(self.ctx, int(max_polls), int(withhold_partition)), "gs_set_sort_wait")

    def gs_read_sort_plan(self, cfg, frame: Frame):
        """(passes, digit_bits, depth_bits) of gs_sort for the frame's last emitted keys."""
        p, d, w = c_int32(0), c_int32(0), c_int32(0)
        self._check(self.lib.gs_read_sort_plan(self.ctx, ctypes.byref(cfg), ctypes.byref(frame.struct),
                                               ctypes.byref(p), ctypes.byref(d), ctypes.byref(w)), "gs_read_sort_plan")
        return int(p.value), int(d.value), int(w.value)

    def gs_read_status(self, frame: Frame, raise_on_error: bool = True):
        k = c_int64(0)
        fl = c_uint32(0)
        st = self.lib.gs_read_status(self.ctx, ctypes.byref(frame.struct), ctypes.byref(k), ctypes.byref(fl))
        if st != 0 and (raise_on_error or st not in (1, 3, 5) or not fl.value):
            self._check(st, "gs_read_status")  # CUDA errors always raise
        return int(k.value), int(fl.value)


@dataclass
class RenderOutput:
    image: torch.Tensor
    final_T: torch.Tensor
    last: torch.Tensor
    num_keys: int
    frame: Frame


class Renderer:
    """Forward renderer that owns frames and grows the key capacity on demand.

    ``render`` runs gs_forward (the five stages, with preprocess, scan and
    key emission fused) asynchronously, then reads the frame status (one
    synchronisation); if the keys did not fit it grows the capacity to
    ``headroom`` x K and renders the frame again.
    """

    def __init__(self, device=None, stream=None, headroom: float = 1.25):
        self.rast = Rasterizer(device, stream)
        self.headroom = headroom
        self.frames = {}

    def frame(self, n, width, height, tile, min_keys=0) -> Frame:
        key = (n, width, height, tile)
        f = self.frames.get(key)
        if f is None or f.key_capacity < min_keys:
            cap = min(MAX_KEYS, max(int(min_keys), 1 << 16, f.key_capacity if f else 0))
            f = Frame(n, width, height, tile, cap, self.rast.device)
            self.frames[key] = f
        return f

    def render(self, scene, cam, mode="accutile", tile: int = 16, bg=(0.0, 0.0, 0.0)) -> RenderOutput:
        cfg = cfg_struct(tile, mode, bg)
        n = int(scene.means.shape[1])
        f = self.frame(n, cam.width, cam.height, tile)
        r = self.rast
        f.generation += 1
        r.gs_forward(scene, cam, cfg, f)
        K, flags = r.gs_read_status(f, raise_on_error=False)
        if flags & FLAG_CAPACITY:
            if K > MAX_KEYS:
                raise GsError(3, f"{K} keys exceed the library maximum {MAX_KEYS}")
            f = self.frame(n, cam.width, cam.height, tile, min_keys=int(K * self.headroom) + 1)
            f.generation += 1
            r.gs_forward(scene, cam, cfg, f)
            K, flags = r.gs_read_status(f, raise_on_error=False)
        if flags:
            r.gs_read_status(f, raise_on_error=True)
        return RenderOutput(f.image, f.final_T, f.last, K, f)


def backward_work_bytes(n: int) -> int:
    return int(load().gs_backward_work_bytes(int(n)))


def sort_plan_for(tiles: int, least: int, greatest: int, sort_digit_bits: int = 0, fused: bool = True):
    """(passes, digit_bits, depth_bits, start_buffer) of the sort plan for keys
    whose depth bits lie in [least, greatest] (least > greatest: none recorded)."""
    out = [c_int32(0) for _ in range(4)]
    st = load().gs_sort_plan_for(int(tiles), int(least), int(greatest), int(sort_digit_bits), int(bool(fused)),
                                 *[ctypes.byref(o) for o in out])
    if st:
        raise GsError(st, f"gs_sort_plan_for(tiles={tiles}, digits={sort_digit_bits})")
    return tuple(int(o.value) for o in out)


def pup_work_bytes(n: int) -> int:
    return int(load().gs_pup_work_bytes(int(n)))


def pup_scores(renderer: "Renderer", scene, cams, mode="accutile", tile=16, bg=(0.0, 0.0, 0.0)):
    """PUP sensitivity over the views ``cams``: returns (hessian [21, n],
    score [n] = log det H_i) as device tensors."""
    n = int(scene.means.shape[1])
    dev = scene.means.device
    H = torch.zeros(21, n, dtype=torch.float32, device=dev)
    work = torch.empty(max(pup_work_bytes(n) // 4, 4), dtype=torch.float32, device=dev)
    cfg = cfg_struct(tile, mode, bg)
    for cam in cams:
        out = renderer.render(scene, cam, mode, tile, bg)
        renderer.rast.gs_pup_accumulate(scene, cam, cfg, out.frame, H, work)
    score = torch.empty(n, dtype=torch.float32, device=dev)
    renderer.rast.gs_pup_score(H, n, score)
    return H, score


class SceneView:
    """Scene arrays as a plain object (the layout of synth.Scene)."""

    def __init__(self, means, scales, rotations, opacities, sh, sh_degree=3):
        self.means, self.scales, self.rotations, self.opacities, self.sh = means, scales, rotations, opacities, sh
        self.sh_degree = sh_degree


class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, scales, rotations, opacities, sh, diff, cam, mode, tile, bg, sh_degree):
        scene = SceneView(means.detach().contiguous(), scales.detach().contiguous(), rotations.detach().contiguous(),
                          opacities.detach().contiguous(), sh.detach().contiguous(), sh_degree)
        out = diff.renderer.render(scene, cam, mode, tile, bg)
        ctx.diff, ctx.cam, ctx.cfg = diff, cam, cfg_struct(tile, mode, bg)
        ctx.frame, ctx.generation, ctx.scene = out.frame, out.frame.generation, scene
        return out.image.clone()

    @staticmethod
    def backward(ctx, grad_image):
        f = ctx.frame
        if f.generation != ctx.generation:
            raise RuntimeError("the frame was re-rendered before backward; call backward before the next forward "
                               "of the same size")
        sc = ctx.scene
        n = sc.means.shape[1]
        diff = ctx.diff
        grads = {k: torch.empty_like(getattr(sc, k)) for k in ("means", "scales", "rotations", "opacities", "sh")}
        grads["means2d"] = torch.empty(2, n, dtype=torch.float32, device=sc.means.device)
        if diff.score is not None:
            grads["score"] = diff.score
        work = diff.work(f.n, sc.means.device)
        diff.renderer.rast.gs_render_backward(sc, ctx.cam, ctx.cfg, f, grad_image.contiguous().float(), grads, work)
        diff.means2d_grad = grads["means2d"]
        return (grads["means"], grads["scales"], grads["rotations"], grads["opacities"], grads["sh"], None, None, None,
                None, None, None)


class DiffRenderer:
    """Differentiable forward render (torch.autograd) over the CUDA library.

    ``render(means, scales, rotations, opacities, sh, cam)`` returns the
    (3, H, W) image; its backward runs gs_render_backward.  If ``score`` is a
    (N,) tensor, each backward adds the efficient pruning score to it.  The
    frame is reused per raster size, so call backward before the next forward
    of the same size (checked).
    """

    def __init__(self, device=None, mode="accutile", tile=16, bg=(0.0, 0.0, 0.0)):
        self.renderer = Renderer(device)
        self.mode, self.tile, self.bg = mode, tile, bg
        self.score = None
        self.means2d_grad = None
        self._work = None

    def work(self, n, device):
        need = backward_work_bytes(n) // 4
        if self._work is None or self._work.numel() < need:
            self._work = torch.empty(need, dtype=torch.float32, device=device)
        return self._work

    def render(self, means, scales, rotations, opacities, sh, cam, sh_degree=3):
        return _RenderFn.apply(means, scales, rotations, opacities, sh, self, cam, self.mode, self.tile, self.bg,
                               sh_degree)


# ---------------------------------------------------------------- multi-view
FLAG_BATCH = 4
CAMERA_BYTES = ctypes.sizeof(GsCamera)


def pack_cameras(cams) -> torch.Tensor:
    """Packed gs_camera structs as a uint8 CPU tensor (pinned) of len(cams) * CAMERA_BYTES."""
    arr = (GsCamera * len(cams))(*[camera_struct(c) for c in cams])
    host = torch.empty(len(cams) * CAMERA_BYTES, dtype=torch.uint8).pin_memory()
    ctypes.memmove(host.data_ptr(), ctypes.addressof(arr), len(cams) * CAMERA_BYTES)
    return host


def batch_layout(cams, tile):
    """Per-camera (tile offset, pixel offset) and totals, in camera order."""
    toff, poff, t, p = [], [], 0, 0
    for c in cams:
        toff.append(t)
        poff.append(p)
        t += ((c.width + tile - 1) // tile) * ((c.height + tile - 1) // tile)
        p += c.width * c.height
    return toff, poff, t, p


class BatchFrame:
    """Caller-owned buffers of a multi-view batch (gs_batch_frame)."""

    def __init__(self, n, max_cams, tile, tile_capacity, pixel_capacity, key_capacity, device=None):
        device = torch.device(device or "cuda")
        sz = GsFrameBytes()
        st = load().gs_batch_sizes(int(n), int(max_cams), int(tile), int(tile_capacity), int(pixel_capacity),
                                   int(key_capacity), ctypes.byref(sz))
        if st != 0:
            raise GsError(st, "gs_batch_sizes")
        self.n, self.max_cams, self.tile = n, max_cams, tile
        self.tile_capacity, self.pixel_capacity, self.key_capacity = tile_capacity, pixel_capacity, key_capacity
        e = lambda nbytes, dt, es: torch.empty(max(nbytes // es, 1), dtype=dt, device=device)
        self.proj = e(sz.proj, torch.float32, 4)
        self.counts = e(sz.counts, torch.int32, 4)
        self.keys = e(sz.keys, torch.int64, 8)
        self.vals = e(sz.vals, torch.int32, 4)
        self.ranges = e(sz.ranges, torch.int32, 4)
        self.image = e(sz.image, torch.float32, 4)
        self.final_T = e(sz.final_T, torch.float32, 4)
        self.last = e(sz.last, torch.int32, 4)
        self.scratch = torch.zeros(max(sz.scratch, 1), dtype=torch.uint8, device=device)
        self.cams_dev = torch.empty(max_cams * CAMERA_BYTES, dtype=torch.uint8, device=device)
        f = GsBatchFrame()
        f.n_capacity, f.key_capacity = n, key_capacity
        f.tile_capacity, f.pixel_capacity = tile_capacity, pixel_capacity
        f.max_cams, f.tile = max_cams, tile
        for k in ("proj", "counts", "keys", "vals", "ranges", "image", "final_T", "last", "scratch"):
            setattr(f, k, getattr(self, k).data_ptr())
        self.struct = f

    def images(self, cams):
        """Views (3, H, W) of each camera's image in the packed buffer."""
        _, poff, _, _ = batch_layout(cams, self.tile)
        return [self.image[3 * p: 3 * p + 3 * c.width * c.height].view(3, c.height, c.width)
                for c, p in zip(cams, poff)]

    def nbytes(self) -> int:
        return sum(t.numel() * t.element_size() for t in (self.proj, self.counts, self.keys, self.vals, self.ranges,
                                                          self.image, self.final_T, self.last, self.scratch))


class BatchRenderer:
    """Renders many cameras of one scene per call (gs_forward_batch), growing
    capacities on demand; ``capture``/``replay`` run the batch as a CUDA graph
    whose camera poses are rewritten before each replay."""

    def __init__(self, device=None, tile=16, mode="accutile", bg=(0.0, 0.0, 0.0), sort_digit_bits=0,
                 headroom=1.25):
        self.rast = Rasterizer(device)
        self.device = self.rast.device
        self.tile, self.mode, self.bg = tile, mode, bg
        self.sort_digit_bits = sort_digit_bits
        self.headroom = headroom
        self.frame = None
        self.graph = None

    def cfg(self):
        return cfg_struct(self.tile, self.mode, self.bg, self.sort_digit_bits)

    def ensure(self, n, cams, min_keys=0):
        _, _, T, P = batch_layout(cams, self.tile)
        f = self.frame
        if (f is None or f.n < n or f.max_cams < len(cams) or f.tile_capacity < T or f.pixel_capacity < P
                or f.key_capacity < min_keys or f.tile != self.tile):
            keys = max(int(min_keys), 1 << 20, f.key_capacity if f is not None else 0)
            self.frame = BatchFrame(n, max(len(cams), f.max_cams if f else 0), self.tile,
                                    max(T, f.tile_capacity if f else 0), max(P, f.pixel_capacity if f else 0),
                                    min(keys, MAX_KEYS), self.device)
            self.graph = None
        return self.frame

    def _launch(self, scene, cams):
        f = self.frame
        host = pack_cameras(cams)
        f.cams_dev[: host.numel()].copy_(host, non_blocking=True)
        self.rast.gs_forward_batch(scene, f.cams_dev, len(cams), self.cfg(), f)

    def render(self, scene, cams):
        """Returns the list of (3, H, W) images (views into the frame) and K."""
        n = int(scene.means.shape[1])
        self.ensure(n, cams)
        self._launch(scene, cams)
        K, flags = self.rast.gs_batch_status(self.frame, raise_on_error=False)
        if flags & FLAG_CAPACITY:
            self.ensure(n, cams, min_keys=int(K * self.headroom) + 1)
            self._launch(scene, cams)
            K, flags = self.rast.gs_batch_status(self.frame, raise_on_error=False)
        if flags:
            self.rast.gs_batch_status(self.frame, raise_on_error=True)
        return self.frame.images(cams), K

    def capture(self, scene, cams):
        """Capture one batch as a CUDA graph (after a sizing render)."""
        self.render(scene, cams)
        f = self.frame
        self._graph_scene = scene
        self._graph_ncams = len(cams)
        stream = torch.cuda.Stream(self.device)
        stream.wait_stream(torch.cuda.current_stream(self.device))
        g = torch.cuda.CUDAGraph()
        old = self.rast.stream
        with torch.cuda.stream(stream):
            self.rast.set_stream(stream)
            self.rast.gs_forward_batch(scene, f.cams_dev, len(cams), self.cfg(), f)  # warm on the side stream
            stream.synchronize()
            with torch.cuda.graph(g, stream=stream):
                self.rast.gs_forward_batch(scene, f.cams_dev, len(cams), self.cfg(), f)
        self.rast.set_stream(old)
        torch.cuda.current_stream(self.device).wait_stream(stream)
        self.graph = g
        return g

    def replay(self, cams=None):
        """Replay the captured batch, optionally with new poses (same or fewer
        tiles and pixels in total, same camera count)."""
        if self.graph is None:
            raise RuntimeError("capture() first")
        f = self.frame
        if cams is not None:
            if len(cams) != self._graph_ncams:
                raise ValueError("a replay keeps the captured camera count")
            host = pack_cameras(cams)
            f.cams_dev[: host.numel()].copy_(host, non_blocking=True)
        self.graph.replay()
