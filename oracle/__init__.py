"""CPU oracle for the Speedy-Splat tile rasterizer — TEST INFRASTRUCTURE ONLY.

A plain, slow, sequential implementation (``oracle.cpp``) of what the
rasterizer computes, written from the paper's definitions (Sec. 3.2, Sec. 4.1,
Algorithm 1), in FP64 (reference of record) or FP32 (the documented
single-precision operation order).  Only the tests, the package's smoke check
and the benchmark's CPU-baseline leg may import this module.  It imports
nothing from the CUDA library and the library imports nothing from it.

Parity status: every routine is pinned by ``tests/test_oracle_pins.py``
against closed forms, library routines (numpy, scipy) or brute force, except
the Fig. 2c walk-through of Algorithm 1, for which the paper prints no
numbers (parity unpinned for that example; the algorithm itself is pinned by
brute force).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "oracle.cpp"
_OUT = _HERE / "_build" / "liboracle.so"
_OUT_OMP = _HERE / "_build" / "liboracle_omp.so"
CXXFLAGS = ["-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]

MODES = {"3sigma": 0, "snugbox": 1, "accutile": 2, "tbc": 3, "pixel": 4}


def build(force: bool = False, omp: bool = False) -> Path:
    """Compile ``oracle.cpp`` into ``_build/liboracle.so`` with g++ (FP
    contraction off); with ``omp`` also into ``_build/liboracle_omp.so``
    (-fopenmp: the same code with its independent loops on all host cores)."""
    out = _OUT_OMP if omp else _OUT
    if not force and out.exists() and out.stat().st_mtime >= _SRC.stat().st_mtime:
        return out
    out.parent.mkdir(parents=True, exist_ok=True)
    tmp = out.with_suffix(f".{os.getpid()}.tmp")
    cmd = [os.environ.get("CXX", "g++"), *CXXFLAGS, *(["-fopenmp"] if omp else []), str(_SRC), "-o", str(tmp)]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


_lib = None
_lib_omp = None


def lib(omp: bool = False) -> ctypes.CDLL:
    global _lib, _lib_omp
    if omp:
        if _lib_omp is None:
            _lib_omp = ctypes.CDLL(str(build(omp=True)))
            _declare(_lib_omp)
        return _lib_omp
    if _lib is None:
        _lib = ctypes.CDLL(str(build()))
        _declare(_lib)
    return _lib


P = ctypes.c_void_p
I64 = ctypes.c_int64
I32 = ctypes.c_int


def _declare(L):
    L.oracle_log_f32.argtypes = [P, P, I64]
    L.oracle_exp_f32.argtypes = [P, P, I64]
    L.oracle_sh_basis.argtypes = [I32, P, P, I64]
    L.oracle_preprocess.argtypes = [I32, I64, P, P, P, P, P, I32, I32, I32, P, I32, I32, P, P]
    L.oracle_ellipse_tiles.argtypes = [I32, I32, I32, P, I32, I32, I32, P, I64]
    L.oracle_ellipse_tiles.restype = I64
    L.oracle_snugbox.argtypes = [I32, P, I32, I32, I32, P]
    L.oracle_snugbox.restype = I32
    L.oracle_exact_tile_mask.argtypes = [P, I32, I32, I32, P]
    L.oracle_render.argtypes = [I32, I64, P, P, P, P, P, I32, I32, I32, P, I32, I32, P, I64, P, P, P, P, P, P, P, P,
                                P, P]
    L.oracle_render.restype = I32
    L.oracle_render_notile.argtypes = [I32, I64, P, P, P, P, P, I32, I32, I32, P, P, P, P, I32, P]
    L.oracle_blend_pixel.argtypes = [I32, P, I64, ctypes.c_double, ctypes.c_double, P, P]
    L.oracle_backward.argtypes = [I64, P, P, P, P, P, I32, I32, I32, P, I32, I32, P, P, P, P]
    L.oracle_sh_basis_grad.argtypes = [P, P, I64]
    L.oracle_pup.argtypes = [I64, P, P, P, P, P, I32, I32, I32, P, I32, I32, P, P]


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _np(x, dtype=np.float32) -> np.ndarray:
    if hasattr(x, "detach"):
        x = x.detach().cpu().numpy()
    return np.ascontiguousarray(np.asarray(x), dtype=dtype)


def _scene_arrays(scene):
    """Accepts any object with attributes means, scales, rotations, opacities,
    sh (numpy arrays or CPU tensors, planar layout) and sh_degree."""
    arrs = [_np(getattr(scene, k)) for k in ("means", "scales", "rotations", "opacities", "sh")]
    n = arrs[0].shape[1] if arrs[0].ndim == 2 else 0
    return n, arrs, int(getattr(scene, "sh_degree", 3))


def _cam(cam):
    return int(cam.width), int(cam.height), np.ascontiguousarray(cam.as_floats(), dtype=np.float32)


def grid(width: int, height: int, tile: int):
    return (width + tile - 1) // tile, (height + tile - 1) // tile


# ------------------------------------------------------------------ elementary
def log_f32(x) -> np.ndarray:
    x = _np(x)
    y = np.empty_like(x)
    lib().oracle_log_f32(_ptr(x), _ptr(y), x.size)
    return y


def exp_f32(x) -> np.ndarray:
    x = _np(x)
    y = np.empty_like(x)
    lib().oracle_exp_f32(_ptr(x), _ptr(y), x.size)
    return y


def sh_basis(dirs, prec64: bool = True) -> np.ndarray:
    d = _np(dirs, np.float64).reshape(-1, 3)
    out = np.empty((d.shape[0], 16), np.float64)
    lib().oracle_sh_basis(int(prec64), _ptr(d), _ptr(out), d.shape[0])
    return out


# ------------------------------------------------------------------ per Gaussian
PROJ_FIELDS = ["u", "v", "depth", "opacity", "a", "b", "c", "t", "r", "g", "b_", "cov_xx", "cov_xy", "cov_yy",
               "radius", "valid"]


def preprocess(scene, cam, tile: int = 16, mode: int = 2, prec64: bool = True, omp: bool = False):
    """Returns (state[n,16] in PROJ_FIELDS order, counts[n] int64)."""
    n, (m, s, r, o, sh), deg = _scene_arrays(scene)
    w, h, cf = _cam(cam)
    out = np.zeros((n, 16), np.float64)
    counts = np.zeros(n, np.int64)
    lib(omp).oracle_preprocess(int(prec64), n, _ptr(m), _ptr(s), _ptr(r), _ptr(o), _ptr(sh), deg, w, h, _ptr(cf),
                            tile, mode, _ptr(out), _ptr(counts))
    return out, counts


def ellipse_tiles(e, mode: int, tile: int, gx: int, gy: int, prec64: bool = True, direction: int = 0):
    """Tile list (k, 2) of (tx, ty) for one 2D Gaussian e = (u, v, a, b, c, t[, radius])."""
    ee = np.zeros(7, np.float64)
    ee[:len(e)] = e
    cap = gx * gy + 1
    out = np.zeros((cap, 2), np.int32)
    k = lib().oracle_ellipse_tiles(int(prec64), mode, direction, _ptr(ee), tile, gx, gy, _ptr(out), cap)
    return out[:k].copy()


def snugbox(e, tile: int, gx: int, gy: int, prec64: bool = True):
    ee = np.zeros(7, np.float64)
    ee[:len(e)] = e
    out = np.zeros(8, np.float64)
    ok = lib().oracle_snugbox(int(prec64), _ptr(ee), tile, gx, gy, _ptr(out))
    return bool(ok), out


def exact_tile_mask(e, tile: int, gx: int, gy: int) -> np.ndarray:
    ee = np.zeros(7, np.float64)
    ee[:len(e)] = e
    mask = np.zeros((gy, gx), np.uint8)
    lib().oracle_exact_tile_mask(_ptr(ee), tile, gx, gy, _ptr(mask))
    return mask.astype(bool)


# ------------------------------------------------------------------ pipelines
def count_keys(scene, cam, tile: int, mode: int, prec64: bool = False, omp: bool = False) -> int:
    return int(preprocess(scene, cam, tile, mode, prec64, omp)[1].sum())


def render(scene, cam, tile: int = 16, mode: int = 2, bg=(0.0, 0.0, 0.0), prec64: bool = False, key_cap=None,
           omp: bool = False):
    """Full forward pipeline of one tile mode.  Returns a dict with the
    unsorted and sorted (key, id) lists, tile ranges, image (3,H,W), final T
    and last-contributor index, all as numpy arrays, and the blend's pair
    counts (evaluated: every tile-list entry a pixel walks, up to and
    including the one that stops it; contributing: those that add colour)."""
    n, (m, s, r, o, sh), deg = _scene_arrays(scene)
    w, h, cf = _cam(cam)
    gx, gy = grid(w, h, tile)
    bgv = np.asarray(bg, np.float32)
    if key_cap is None:
        key_cap = count_keys(scene, cam, tile, mode, prec64, omp)
    key_cap = max(int(key_cap), 1)
    ku = np.zeros(key_cap, np.uint64)
    vu = np.zeros(key_cap, np.uint32)
    ks = np.zeros(key_cap, np.uint64)
    vs = np.zeros(key_cap, np.uint32)
    nk = np.zeros(1, np.int64)
    ranges = np.zeros((gx * gy, 2), np.uint32)
    img = np.zeros((3, h, w), np.float64)
    T = np.zeros((h, w), np.float64)
    last = np.zeros((h, w), np.uint32)
    pairs = np.zeros(2, np.int64)
    rc = lib(omp).oracle_render(int(prec64), n, _ptr(m), _ptr(s), _ptr(r), _ptr(o), _ptr(sh), deg, w, h, _ptr(cf), tile,
                             mode, _ptr(bgv), key_cap, _ptr(ku), _ptr(vu), _ptr(ks), _ptr(vs), _ptr(nk),
                             _ptr(ranges), _ptr(img), _ptr(T), _ptr(last), _ptr(pairs))
    K = int(nk[0])
    if rc != 0:
        raise RuntimeError(f"oracle_render: key capacity {key_cap} < required {K}")
    return {"num_keys": K, "evaluated_pairs": int(pairs[0]), "contributing_pairs": int(pairs[1]),
            "keys_unsorted": ku[:K], "vals_unsorted": vu[:K], "keys": ks[:K], "vals": vs[:K],
            "ranges": ranges, "image": img, "final_T": T, "last": last, "grid": (gx, gy)}


def render_notile(scene, cam, bg=(0.0, 0.0, 0.0), prec64: bool = True, literal_exp: bool = False):
    n, (m, s, r, o, sh), deg = _scene_arrays(scene)
    w, h, cf = _cam(cam)
    bgv = np.asarray(bg, np.float32)
    img = np.zeros((3, h, w), np.float64)
    T = np.zeros((h, w), np.float64)
    differ = np.zeros(1, np.int64)
    lib().oracle_render_notile(int(prec64), n, _ptr(m), _ptr(s), _ptr(r), _ptr(o), _ptr(sh), deg, w, h, _ptr(cf),
                               _ptr(bgv), _ptr(img), _ptr(T), int(literal_exp), _ptr(differ))
    return {"image": img, "final_T": T, "decisions_differ": int(differ[0])}


def blend_pixel(gaussians, px: float, py: float, bg=(0.0, 0.0, 0.0), prec64: bool = True):
    """Composite one pixel over an ordered list of 2D Gaussians
    (rows: u v a b c t opacity r g b).  Returns (C[3], T, last)."""
    g = _np(gaussians, np.float64).reshape(-1, 10)
    bgv = np.asarray(bg, np.float32)
    out = np.zeros(5, np.float64)
    lib().oracle_blend_pixel(int(prec64), _ptr(g), g.shape[0], float(px), float(py), _ptr(bgv), _ptr(out))
    return out[:3].copy(), float(out[3]), int(out[4])


# ------------------------------------------------------------------ backward
GRAD_SLICES = {"means": (0, 3), "scales": (3, 6), "rotations": (6, 10), "opacities": (10, 11), "sh": (11, 59)}
G2D_FIELDS = ["u", "v", "a", "b", "c", "sigma", "r", "g", "b_", "score"]


def backward(scene, cam, dL_dimage, tile: int = 16, mode: int = 2, bg=(0.0, 0.0, 0.0)):
    """FP64 gradients of L = sum(dL_dimage * image) for one tile mode.
    Returns (grads, g2d): grads maps each scene array name to an array shaped
    like it; g2d is [10, n] (du dv da db dc dsigma dr dg db score)."""
    n, (m, s, r, o, sh), deg = _scene_arrays(scene)
    w, h, cf = _cam(cam)
    G = np.ascontiguousarray(np.asarray(dL_dimage, np.float64).reshape(3, h, w))
    bgv = np.asarray(bg, np.float32)
    grads = np.zeros((59, n), np.float64)
    g2d = np.zeros((10, n), np.float64)
    lib().oracle_backward(n, _ptr(m), _ptr(s), _ptr(r), _ptr(o), _ptr(sh), deg, w, h, _ptr(cf), tile, mode, _ptr(bgv),
                          _ptr(G), _ptr(grads), _ptr(g2d))
    out = {k: grads[a:b] for k, (a, b) in GRAD_SLICES.items()}
    out["sh"] = out["sh"].reshape(16, 3, n)
    out["opacities"] = out["opacities"].reshape(n)
    return out, g2d


def pup(scene, cams, tile: int = 16, mode: int = 2, bg=(0.0, 0.0, 0.0)) -> np.ndarray:
    """PUP sensitivity H (FP64): [21, n], the upper triangle (row-major,
    order mu_x mu_y mu_z s_0 s_1 s_2) of sum over the views ``cams``, pixels
    and channels of grad_{mu,s} C grad_{mu,s} C^T through g_i (Sec. 4.2,
    Eq. pup_score)."""
    n, (m, s, r, o, sh), deg = _scene_arrays(scene)
    bgv = np.asarray(bg, np.float32)
    H = np.zeros((21, n), np.float64)
    for cam in cams:
        w, h, cf = _cam(cam)
        lib().oracle_pup(n, _ptr(m), _ptr(s), _ptr(r), _ptr(o), _ptr(sh), deg, w, h, _ptr(cf), tile, mode, _ptr(bgv),
                         _ptr(H))
    return H


def pup_full(H: np.ndarray) -> np.ndarray:
    """[n, 6, 6] symmetric matrices from the [21, n] upper triangles."""
    n = H.shape[1]
    M = np.zeros((n, 6, 6))
    e = 0
    for a in range(6):
        for b in range(a, 6):
            M[:, a, b] = M[:, b, a] = H[e]
            e += 1
    return M


def sh_basis_grad(dirs) -> np.ndarray:
    d = _np(dirs, np.float64).reshape(-1, 3)
    out = np.empty((d.shape[0], 16, 3), np.float64)
    lib().oracle_sh_basis_grad(_ptr(d), _ptr(out), d.shape[0])
    return out
