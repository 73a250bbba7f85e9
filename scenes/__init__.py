"""Seeded synthetic range images shared by the tests and the benchmark.

The paper's datasets (480x640 depth images rendered from meshes) are not
available; these scenes stand in for them: 6 planes and 3 spheres ray-cast
through a pinhole camera, optional Gaussian depth noise (sigma = k Z^2) and iid
holes, optionally quantised to 16-bit fixed-point stereo disparity.  Nothing
here computes normals from depth; the analytic ground-truth normals come from
the primitives themselves.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tfn_scenes.c")
_LIB = os.path.join(_HERE, "libtfn_scenes.so")


def build(force: bool = False) -> str:
    """Compile the generator into ``scenes/libtfn_scenes.so``."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", _LIB + ".tmp",
               _SRC, "-lm", "-lpthread"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Recipe(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int),
                ("fx", ctypes.c_double), ("fy", ctypes.c_double),
                ("u0", ctypes.c_double), ("v0", ctypes.c_double),
                ("zmin", ctypes.c_double), ("zmax", ctypes.c_double),
                ("n_planes", ctypes.c_int), ("n_spheres", ctypes.c_int),
                ("plane_z0", ctypes.c_double), ("plane_z1", ctypes.c_double),
                ("max_tilt_deg", ctypes.c_double),
                ("sphere_z0", ctypes.c_double), ("sphere_z1", ctypes.c_double),
                ("radius0", ctypes.c_double), ("radius1", ctypes.c_double),
                ("noise_k", ctypes.c_double), ("hole_frac", ctypes.c_double)]


@dataclasses.dataclass
class Recipe:
    """Scene recipe; the defaults are the 480x640 indoor-range scene."""
    H: int = 480
    W: int = 640
    fx: float = 481.2
    fy: float = 481.2
    u0: float = 319.5
    v0: float = 239.5
    zmin: float = 0.5
    zmax: float = 10.0
    n_planes: int = 6
    n_spheres: int = 3
    plane_z0: float = 0.5
    plane_z1: float = 10.0
    max_tilt_deg: float = 75.0
    sphere_z0: float = 1.5
    sphere_z1: float = 9.0
    radius0: float = 0.2
    radius1: float = 1.0
    noise_k: float = 0.0
    hole_frac: float = 0.0

    def _c(self):
        return _Recipe(*[getattr(self, f.name) for f in dataclasses.fields(self)])

    @property
    def camera(self):
        return dict(fx=self.fx, fy=self.fy, u0=self.u0, v0=self.v0)


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        p = ctypes.c_void_p
        lib.tfn_scene_recipe_size.restype = ctypes.c_int
        assert lib.tfn_scene_recipe_size() == ctypes.sizeof(_Recipe)
        lib.tfn_scene_render.argtypes = [p, ctypes.c_uint64, p, p, p, p]
        lib.tfn_scene_render_batch.argtypes = [p, ctypes.c_uint64, ctypes.c_int, p, p, p, ctypes.c_int]
        lib.tfn_scene_disparity_u16.argtypes = [p, ctypes.c_int64, ctypes.c_double, ctypes.c_int,
                                                ctypes.c_double, ctypes.c_uint64, p]
        _lib = lib
    return _lib


def render(seed: int, recipe: Recipe | None = None, *, with_truth: bool = False):
    """One depth frame (H, W) float32, 0 = hole.

    With ``with_truth``: also the exact FP64 ray-cast depth before noise (0 where
    nothing in range was hit), the primitive index per pixel (-1 none) and the
    analytic unit normal facing the camera (3, H, W) float32.
    """
    r = recipe or Recipe()
    rc = r._c()
    depth = np.empty((r.H, r.W), np.float32)
    if not with_truth:
        _load().tfn_scene_render(ctypes.byref(rc), seed, depth.ctypes.data, None, None, None)
        return depth
    d64 = np.empty((r.H, r.W), np.float64)
    prim = np.empty((r.H, r.W), np.int32)
    gt = np.empty((3, r.H, r.W), np.float32)
    _load().tfn_scene_render(ctypes.byref(rc), seed, depth.ctypes.data, d64.ctypes.data,
                             prim.ctypes.data, gt.ctypes.data)
    return depth, d64, prim, gt


def render_batch(seed0: int, n: int, recipe: Recipe | None = None, threads: int | None = None,
                 out: np.ndarray | None = None):
    """n frames (n, H, W) float32; frame k uses seed ``seed0 + k``."""
    r = recipe or Recipe()
    rc = r._c()
    depth = out if out is not None else np.empty((n, r.H, r.W), np.float32)
    assert depth.shape == (n, r.H, r.W) and depth.dtype == np.float32 and depth.flags.c_contiguous
    threads = threads or min(32, os.cpu_count() or 1)
    _load().tfn_scene_render_batch(ctypes.byref(rc), seed0, n, depth.ctypes.data, None, None, threads)
    return depth


def disparity_u16(depth: np.ndarray, f_tc: float, *, frac_bits: int = 4, hole_frac: float = 0.0,
                  seed: int = 0) -> np.ndarray:
    """Stereo disparity f*t_c/Z in u16 fixed point (``frac_bits`` fractional bits)."""
    depth = np.ascontiguousarray(depth, np.float32)
    out = np.empty(depth.shape, np.uint16)
    _load().tfn_scene_disparity_u16(depth.ctypes.data, depth.size, f_tc, frac_bits, hole_frac, seed,
                                    out.ctypes.data)
    return out


# --- the paper-shaped workloads (480x640, Sec. IV-A) -----------------------------------------

CAMERA = dict(fx=481.2, fy=481.2, u0=319.5, v0=239.5)
STEREO = dict(f=615.0, baseline=0.1, u0=319.5, v0=239.5)


def single_frame():
    """One clean 480x640 FP32 depth frame (seed 1): 6 planes + 3 spheres at 0.5-10 m."""
    return render(1)


def noisy_batch(n: int = 256, seed0: int = 1000, threads=None):
    """n FP32 480x640 frames with sigma = 0.0012 Z^2 depth noise and 3% holes."""
    return render_batch(seed0, n, Recipe(noise_k=0.0012, hole_frac=0.03), threads)


def disparity_recipe() -> Recipe:
    """Scenes placed at 0.640625-61.5 m so that d = 61.5/Z spans 1-96 px."""
    return Recipe(fx=615.0, fy=615.0, zmin=0.640625, zmax=61.5, plane_z0=0.640625, plane_z1=61.5,
                  sphere_z0=2.0, sphere_z1=50.0, radius0=0.5, radius1=5.0)


def disparity_batch(n: int = 256, seed0: int = 2000, threads=None):
    """n u16 disparity images (1/16 px fixed point, 1-96 px, 5% zeros)."""
    st = STEREO
    depth = render_batch(seed0, n, disparity_recipe(), threads)
    out = np.empty(depth.shape, np.uint16)
    for k in range(n):
        out[k] = disparity_u16(depth[k], st["f"] * st["baseline"], frac_bits=4, hole_frac=0.05,
                               seed=seed0 + 7919 * (k + 1))
    return out


def fp16_batch(n: int = 1024, seed0: int = 3000, threads=None):
    """n clean 480x640 frames rounded to FP16 depth."""
    return render_batch(seed0, n, Recipe(), threads).astype(np.float16)
