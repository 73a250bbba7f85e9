"""FP64 CPU oracle of Three-Filters-to-Normal -- TEST INFRASTRUCTURE ONLY.

This package is the plain, slow reference that the CUDA path is checked
against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import it; the product package never does.  It shares no
code with the CUDA library (``tfn_oracle.c`` is self-contained).

The method follows Fan et al., "Three-Filters-to-Normal" (RA-L 2021):
Sec. III, Eq. (intrinsic matrix), Eq. (nx2_ny2_nz2) for depth input and
Eqs. (z_d), (nx2_ny2_nz3) for disparity input.  The readings taken where the
paper is silent are listed at the top of ``tfn_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tfn_oracle.c")
_LIB = os.path.join(_HERE, "libtfn_oracle.so")

DEPTH_F32, DEPTH_F16, DISP_U16, DISP_F32, DEPTH_F64 = 0, 1, 2, 3, 100
FD, SOBEL, SCHARR, PREWITT, WEIGHTED, SEP5, FD5, SOBEL5, PREWITT5 = 0, 1, 2, 3, 4, 5, 6, 7, 8
MEAN, MEDIAN = 0, 1
LITERAL, ALGEBRAIC = 0, 1

_GRADS = {"fd": FD, "sobel": SOBEL, "scharr": SCHARR, "prewitt": PREWITT, "weighted": WEIGHTED, "sep5": SEP5,
          "fd5": FD5, "sobel5": SOBEL5, "prewitt5": PREWITT5}
_PHIS = {"mean": MEAN, "median": MEDIAN}


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/libtfn_oracle.so`` (plain C11, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        compile_to(_SRC, _LIB + ".tmp")
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def compile_to(src: str, out: str) -> str:
    """Compile an oracle source file into a shared library at ``out``."""
    subprocess.check_call(["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o",
                           out, src, "-lm", "-lpthread"])
    return out


def open_library(path: str):
    """Load a compiled oracle and declare its entry points."""
    lib = ctypes.CDLL(path)
    d, i, i64, p = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
    lib.tfn_oracle_normals.argtypes = [p, i64, i, i, i, d, d, d, d, d, d, i, i, i, p, p, p, p]
    lib.tfn_oracle_normals.restype = i
    lib.tfn_oracle_normals_batch.argtypes = [p, i64, i, i, i, i, d, d, d, d, d, d, i, i, i, p, p, i]
    lib.tfn_oracle_normals_batch.restype = i
    lib.tfn_oracle_points.argtypes = [p, i64, i, i, i, d, d, d, d, d, d, p]
    lib.tfn_oracle_normals_weighted.argtypes = [p, i64, i, i, i, d, d, d, d, d, d, i, p, i, i, p, p, p, p]
    lib.tfn_oracle_normals_weighted.restype = i
    lib.tfn_oracle_points.restype = i
    return lib


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = open_library(build())
    return _lib


def _input_type(img: np.ndarray, disparity: bool) -> int:
    if disparity:
        if img.dtype == np.uint16:
            return DISP_U16
        if img.dtype == np.float32:
            return DISP_F32
    else:
        if img.dtype == np.float32:
            return DEPTH_F32
        if img.dtype == np.float16:
            return DEPTH_F16
        if img.dtype == np.float64:
            return DEPTH_F64
    raise TypeError(f"unsupported input dtype {img.dtype} (disparity={disparity})")


def _code(table, v):
    return table[v] if isinstance(v, str) else int(v)


def normals(img, fx, fy, u0, v0, *, grad="fd", phi="mean", disparity=False, baseline=1.0,
            disp_scale=1.0 / 16, form=LITERAL, diagnostics=False, weights=None, lib=None):
    """Normals of one H x W image.

    Returns ``(n, mask)`` with ``n`` of shape (3, H, W) float64 and ``mask``
    (H, W) uint8; with ``diagnostics=True`` also ``cands`` (8, H, W; NaN where
    a neighbour gives no candidate, neighbour raster order) and ``nprime``
    (3, H, W), the unnormalised (nx, ny, n_z) of Eq. (nx2_ny2_nz2).
    ``grad="weighted"`` takes the row weights (w0, w1, w2) in ``weights``; ``grad="sep5"`` takes the
    5x5 separable profiles (d1, d2, s0, s1, s2) (reading R15); "fd5", "sobel5" and "prewitt5" are its
    named members.
    """
    img = np.ascontiguousarray(img)
    H, W = img.shape
    t = _input_type(img, disparity)
    n = np.empty((3, H, W), np.float64)
    m = np.empty((H, W), np.uint8)
    cands = np.empty((8, H, W), np.float64) if diagnostics else None
    npr = np.empty((3, H, W), np.float64) if diagnostics else None
    w = (ctypes.c_double * len(weights))(*weights) if weights is not None else None
    st = (lib or _load()).tfn_oracle_normals_weighted(
        img.ctypes.data, img.strides[0], H, W, t, disp_scale, fx, fy, u0, v0, baseline,
        _code(_GRADS, grad), w, _code(_PHIS, phi), form, n.ctypes.data, m.ctypes.data,
        cands.ctypes.data if diagnostics else None, npr.ctypes.data if diagnostics else None)
    if st:
        raise ValueError(f"oracle rejected its arguments (status {st})")
    return (n, m, cands, npr) if diagnostics else (n, m)


def normals_batch(imgs, fx, fy, u0, v0, *, grad="fd", phi="mean", disparity=False, baseline=1.0,
                  disp_scale=1.0 / 16, form=LITERAL, threads=1):
    """Normals of a stack of same-shaped images (N, H, W) -> ((N, 3, H, W), (N, H, W))."""
    imgs = np.ascontiguousarray(imgs)
    N, H, W = imgs.shape
    t = _input_type(imgs[0], disparity)
    n = np.empty((N, 3, H, W), np.float64)
    m = np.empty((N, H, W), np.uint8)
    st = _load().tfn_oracle_normals_batch(
        imgs.ctypes.data, imgs.strides[1], N, H, W, t, disp_scale, fx, fy, u0, v0, baseline,
        _code(_GRADS, grad), _code(_PHIS, phi), form, n.ctypes.data, m.ctypes.data, threads)
    if st:
        raise ValueError(f"oracle rejected its arguments (status {st})")
    return n, m


def points(img, fx, fy, u0, v0, *, disparity=False, baseline=1.0, disp_scale=1.0 / 16, lib=None):
    """Back-projected points of every valid sample of one H x W image, (3, H, W) float64 (X, Y, Z);
    holes give (0, 0, 0).  Sec. III, Eq. (intrinsic matrix); disparity input through Eq. (z_d)."""
    img = np.ascontiguousarray(img)
    H, W = img.shape
    out = np.empty((3, H, W), np.float64)
    st = (lib or _load()).tfn_oracle_points(img.ctypes.data, img.strides[0], H, W, _input_type(img, disparity),
                                            disp_scale, fx, fy, u0, v0, baseline, out.ctypes.data)
    if st:
        raise ValueError(f"oracle rejected its arguments (status {st})")
    return out


from .pca import planepca  # noqa: E402  (Sec. II item 2, Eq. planepca; uses points() above)


def oct_encode(n):
    """Octahedral map of vectors (3, ...) onto the square [-1, 1]^2 (Cigolle et al., "A Survey of
    Efficient Representations for Independent Unit Vectors", JCGT 3(2), 2014, the "oct" mapping):
    p = (x, y) / (|x| + |y| + |z|), and for z < 0 the lower hemisphere is folded over the square's
    corners, p <- ((1 - |p_y|) sgn p_x, (1 - |p_x|) sgn p_y) with sgn(0) = +1.  Zero vectors map to
    (0, 0)."""
    n = np.asarray(n, np.float64)
    s = np.abs(n[0]) + np.abs(n[1]) + np.abs(n[2])
    safe = np.where(s > 0, s, 1.0)
    px = np.where(s > 0, n[0] / safe, 0.0)
    py = np.where(s > 0, n[1] / safe, 0.0)
    sx = np.where(px >= 0, 1.0, -1.0)
    sy = np.where(py >= 0, 1.0, -1.0)
    low = n[2] < 0
    qx = np.where(low, (1 - np.abs(py)) * sx, px)
    qy = np.where(low, (1 - np.abs(px)) * sy, py)
    return np.stack([qx, qy])


def oct_quantize(p):
    """Signed 16-bit code of an octahedral point: round-to-nearest-even of p * 32767."""
    return np.rint(np.clip(np.asarray(p, np.float64), -1.0, 1.0) * 32767.0).astype(np.int16)


def oct_decode(q):
    """Unit vectors (3, ...) of octahedral points (2, ...) (floats in [-1, 1], or int16 codes / 32767):
    v = (p_x, p_y, 1 - |p_x| - |p_y|), unfolded where v_z < 0, normalised."""
    q = np.asarray(q)
    p = q.astype(np.float64) / 32767.0 if q.dtype == np.int16 else q.astype(np.float64)
    vx, vy = p[0], p[1]
    vz = 1.0 - np.abs(vx) - np.abs(vy)
    sx = np.where(vx >= 0, 1.0, -1.0)
    sy = np.where(vy >= 0, 1.0, -1.0)
    low = vz < 0
    ux = np.where(low, (1 - np.abs(vy)) * sx, vx)
    uy = np.where(low, (1 - np.abs(vx)) * sy, vy)
    v = np.stack([ux, uy, vz])
    return v / np.sqrt((v * v).sum(0))


def angle_deg(a, b):
    """Per-pixel angle in degrees between two (3, ...) vector fields.

    Sec. IV-A, Eq. (ea_ep): psi = arccos(<n, n_hat> / (|n| |n_hat|)), evaluated
    as atan2(|n x n_hat|, n . n_hat), the same angle without arccos' loss of
    accuracy near zero.
    """
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    cr = np.cross(a, b, axis=0)
    return np.degrees(np.arctan2(np.sqrt((cr * cr).sum(0)), (a * b).sum(0)))
