"""CPU oracle for RICI generation and CRSS search.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU-baseline leg
may import this package; the product path (``paper_2007_02306_gb300``) never does.  It
shares no code with the GPU library.

The arithmetic lives in ``rici_oracle.c`` (FP64 brute force, int64 distances), compiled
with contraction disabled; this module only builds it with gcc and marshals numpy arrays.
``oracle.exact`` is an independent exact-rational restatement for tiny inputs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rici_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle_rici.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, FP contraction off, OpenMP when available)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-shared", "-fPIC"]
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    try:
        subprocess.run(base + ["-fopenmp", _SRC, "-o", tmp, "-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [_SRC, "-o", tmp, "-lm"], check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64, i32, f32 = ctypes.c_int64, ctypes.c_int32, ctypes.c_float
            lib.oracle_rici_fp64.argtypes = [P, P, i64, P, i64, P, i64, f32, i32, P, i32, P]
            lib.oracle_rici_fp64.restype = ctypes.c_int
            lib.oracle_crss.argtypes = [P, P, i32]
            lib.oracle_crss.restype = i64
            lib.oracle_crss_search.argtypes = [P, i64, P, i64, i32, P, P, P, P, P, i32]
            lib.oracle_crss_search.restype = ctypes.c_int
            lib.oracle_max_threads.restype = ctypes.c_int
            lib.oracle_project_fp64.argtypes = [P, i64, P, P, P]
            lib.oracle_project_fp64.restype = None
            lib.oracle_project_fp32.argtypes = [P, i64, P, P, P]
            lib.oracle_project_fp32.restype = None
            lib.oracle_rici_fp32.argtypes = [P, P, i64, P, i64, P, i64, f32, i32, P, i32, P]
            lib.oracle_rici_fp32.restype = ctypes.c_int
            lib.oracle_clutter_areas.argtypes = [P, P, i64, P, i64, P, i64, f32, i64, P, P, i32]
            lib.oracle_clutter_areas.restype = ctypes.c_int
            lib.oracle_spin_samples.argtypes = [P, i64, P, i64, i32, P]
            lib.oracle_spin_samples.restype = ctypes.c_int
            lib.oracle_spin_images_fp32.argtypes = [P, P, i64, P, i64, P, i64, f32, i32, i32, P,
                                                    i32]
            lib.oracle_spin_images_fp32.restype = ctypes.c_int
            lib.oracle_spin_images_fp64.argtypes = [P, P, i64, P, i64, P, i64, f32, i32, i32, P,
                                                    P, i32]
            lib.oracle_spin_images_fp64.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def rici_fp64(vertices, normals, triangles, origins, support_radius: float, resolution: int,
              num_threads: int = 0, return_counters: bool = False):
    """RICI images (uint16 [O, N, N]) by FP64 brute force over every triangle."""
    lib = _load()
    v = np.ascontiguousarray(vertices, dtype=np.float32).reshape(-1, 3)
    n = np.ascontiguousarray(normals, dtype=np.float32).reshape(-1, 3)
    t = np.ascontiguousarray(triangles, dtype=np.int32).reshape(-1, 3)
    o = np.ascontiguousarray(origins, dtype=np.int32).reshape(-1)
    if n.shape != v.shape:
        raise ValueError("normals must match vertices")
    N = int(resolution)
    out = np.zeros((o.size, N, N), dtype=np.uint16)
    cnt = np.zeros(4, dtype=np.int64)
    rc = lib.oracle_rici_fp64(_ptr(v), _ptr(n), v.shape[0], _ptr(t), t.shape[0], _ptr(o), o.size,
                              float(support_radius), N, _ptr(out), int(num_threads), _ptr(cnt))
    if rc != 0:
        raise ValueError(f"oracle_rici_fp64 failed with status {rc}")
    if return_counters:
        return out, {"pairs_crossing": int(cnt[0]), "layer_crossings": int(cnt[1]),
                     "pairs_contributing": int(cnt[2]), "crossings_contributing": int(cnt[3])}
    return out


def project_fp64(points, spin_vertex, spin_normal):
    """(Tx, Ty, Tz) float64 [n, 3] of FP32 points in the frame of one FP32 oriented point."""
    lib = _load()
    p = np.ascontiguousarray(points, dtype=np.float32).reshape(-1, 3)
    s = np.ascontiguousarray(spin_vertex, dtype=np.float32).reshape(3)
    n = np.ascontiguousarray(spin_normal, dtype=np.float32).reshape(3)
    out = np.zeros((p.shape[0], 3), np.float64)
    lib.oracle_project_fp64(_ptr(p), p.shape[0], _ptr(s), _ptr(n), _ptr(out))
    return out


def project_fp32(points, spin_vertex, spin_normal):
    """(Tx, Ty, Tz) float32 [n, 3] in the FP32 same-operation-order mode (frame in FP64, rounded
    to float; projection in float with explicit fmaf)."""
    lib = _load()
    p = np.ascontiguousarray(points, dtype=np.float32).reshape(-1, 3)
    s = np.ascontiguousarray(spin_vertex, dtype=np.float32).reshape(3)
    n = np.ascontiguousarray(spin_normal, dtype=np.float32).reshape(3)
    out = np.zeros((p.shape[0], 3), np.float32)
    lib.oracle_project_fp32(_ptr(p), p.shape[0], _ptr(s), _ptr(n), _ptr(out))
    return out


def rici_fp32(vertices, normals, triangles, origins, support_radius: float, resolution: int,
              num_threads: int = 0):
    """Images of the FP32 same-operation-order mode and its counters: FP32 crossings and the
    (origin, triangle, layer) items whose counts differ from the FP64 definition."""
    lib = _load()
    v = np.ascontiguousarray(vertices, dtype=np.float32).reshape(-1, 3)
    n = np.ascontiguousarray(normals, dtype=np.float32).reshape(-1, 3)
    t = np.ascontiguousarray(triangles, dtype=np.int32).reshape(-1, 3)
    o = np.ascontiguousarray(origins, dtype=np.int32).reshape(-1)
    if n.shape != v.shape:
        raise ValueError("normals must match vertices")
    N = int(resolution)
    out = np.zeros((o.size, N, N), dtype=np.uint16)
    cnt = np.zeros(4, dtype=np.int64)
    rc = lib.oracle_rici_fp32(_ptr(v), _ptr(n), v.shape[0], _ptr(t), t.shape[0], _ptr(o), o.size,
                              float(support_radius), N, _ptr(out), int(num_threads), _ptr(cnt))
    if rc != 0:
        raise ValueError(f"oracle_rici_fp32 failed with status {rc}")
    return out, {"crossings": int(cnt[0]), "items_differing_from_fp64": int(cnt[1])}


def crss(needle, haystack) -> int:
    """Clutter-resistant distance of one needle image against one haystack image."""
    a = np.ascontiguousarray(needle, dtype=np.uint16)
    b = np.ascontiguousarray(haystack, dtype=np.uint16)
    if a.shape != b.shape or a.ndim != 2 or a.shape[0] != a.shape[1]:
        raise ValueError("expected two N x N images")
    return int(_load().oracle_crss(_ptr(a), _ptr(b), a.shape[0]))


def crss_search(needles, haystack, true_match=None, return_distances: bool = False,
                num_threads: int = 0):
    """Per needle: rank of its true match, true distance, top-1 index (and optionally all distances)."""
    lib = _load()
    q = np.ascontiguousarray(needles, dtype=np.uint16)
    h = np.ascontiguousarray(haystack, dtype=np.uint16)
    N = int(q.shape[-1])
    Q, H = int(q.shape[0]), int(h.shape[0])
    m = None if true_match is None else np.ascontiguousarray(true_match, dtype=np.int64).reshape(-1)
    rank = np.zeros(Q, np.int32)
    dt = np.zeros(Q, np.int64)
    top1 = np.zeros(Q, np.int32)
    dist = np.zeros((Q, H), np.int64) if return_distances else None
    rc = lib.oracle_crss_search(_ptr(q), Q, _ptr(h), H, N, _ptr(m), _ptr(rank), _ptr(dt),
                                _ptr(top1), _ptr(dist), int(num_threads))
    if rc != 0:
        raise ValueError(f"oracle_crss_search failed with status {rc}")
    out = {"rank": rank, "true_distance": dt, "top1": top1}
    if dist is not None:
        out["distances"] = dist
    return out


def clutter_areas(vertices, normals, triangles, origins, support_radius: float,
                  object_vertices: int, num_threads: int = 0):
    """Eq. clutter inputs per oriented point, FP64 brute force over every triangle: the surface
    area inside the support volume (radius R around the normal axis, |beta| <= R/2) and the part
    of it on triangles whose first vertex index is below ``object_vertices``.

    Returns (area_all, area_object), float64 [O] each."""
    lib = _load()
    v = np.ascontiguousarray(vertices, dtype=np.float32).reshape(-1, 3)
    n = np.ascontiguousarray(normals, dtype=np.float32).reshape(-1, 3)
    t = np.ascontiguousarray(triangles, dtype=np.int32).reshape(-1, 3)
    o = np.ascontiguousarray(origins, dtype=np.int32).reshape(-1)
    a_all = np.zeros(o.shape[0], np.float64)
    a_obj = np.zeros(o.shape[0], np.float64)
    rc = lib.oracle_clutter_areas(_ptr(v), _ptr(n), v.shape[0], _ptr(t), t.shape[0], _ptr(o),
                                  o.shape[0], float(support_radius), int(object_vertices),
                                  _ptr(a_all), _ptr(a_obj), int(num_threads))
    if rc != 0:
        raise ValueError(f"oracle_clutter_areas failed with status {rc}")
    return a_all, a_obj


def clutter(vertices, normals, triangles, origins, support_radius: float, object_vertices: int):
    """Eq. clutter per oriented point: (A_all - A_object) / A_all (NaN where A_all = 0)."""
    a_all, a_obj = clutter_areas(vertices, normals, triangles, origins, support_radius,
                                 object_vertices)
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(a_all > 0, (a_all - a_obj) / np.where(a_all > 0, a_all, 1.0), np.nan)


def spin_samples(vertices, triangles, m: int):
    """The m^2 point samples of every triangle used by ``spin_images``: float32 [T, m^2, 3]."""
    lib = _load()
    v = np.ascontiguousarray(vertices, dtype=np.float32).reshape(-1, 3)
    t = np.ascontiguousarray(triangles, dtype=np.int32).reshape(-1, 3)
    out = np.zeros((t.shape[0], m * m, 3), np.float32)
    rc = lib.oracle_spin_samples(_ptr(v), v.shape[0], _ptr(t), t.shape[0], int(m), _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle_spin_samples failed with status {rc}")
    return out


def _spin_args(vertices, normals, triangles, origins):
    v = np.ascontiguousarray(vertices, dtype=np.float32).reshape(-1, 3)
    n = np.ascontiguousarray(normals, dtype=np.float32).reshape(-1, 3)
    t = np.ascontiguousarray(triangles, dtype=np.int32).reshape(-1, 3)
    o = np.ascontiguousarray(origins, dtype=np.int32).reshape(-1)
    return v, n, t, o


def spin_images(vertices, normals, triangles, origins, support_radius: float, resolution: int,
                m: int = 3, num_threads: int = 0, return_bound: bool = False):
    """Spin images (Section 2.1) of the oriented points from m^2 samples per triangle: sample
    positions, projection and bilinear weights around the bin centres in FP64, summed in FP64
    and rounded once to float32 [O, N, N] (row = beta bin, column = alpha bin).

    With ``return_bound`` also a float64 [O, N, N] bound on how far a single-precision
    evaluation of the same definition may lie from each bin (derivation in rici_oracle.c)."""
    lib = _load()
    v, n, t, o = _spin_args(vertices, normals, triangles, origins)
    N = int(resolution)
    out = np.zeros((o.shape[0], N, N), np.float32)
    bound = np.zeros((o.shape[0], N, N), np.float64) if return_bound else None
    rc = lib.oracle_spin_images_fp64(_ptr(v), _ptr(n), v.shape[0], _ptr(t), t.shape[0], _ptr(o),
                                     o.shape[0], float(support_radius), N, int(m), _ptr(out),
                                     _ptr(bound), int(num_threads))
    if rc != 0:
        raise ValueError(f"oracle_spin_images_fp64 failed with status {rc}")
    return (out, bound) if return_bound else out


def spin_images_fp32(vertices, normals, triangles, origins, support_radius: float,
                     resolution: int, m: int = 3, num_threads: int = 0):
    """Single-precision same-operation-order mode of ``spin_images``: every operation in FP32 in
    one fixed order, weights summed exactly as integers in units of 2^-24, float32 [O, N, N]."""
    lib = _load()
    v, n, t, o = _spin_args(vertices, normals, triangles, origins)
    N = int(resolution)
    out = np.zeros((o.shape[0], N, N), np.float32)
    rc = lib.oracle_spin_images_fp32(_ptr(v), _ptr(n), v.shape[0], _ptr(t), t.shape[0], _ptr(o),
                                     o.shape[0], float(support_radius), N, int(m), _ptr(out),
                                     int(num_threads))
    if rc != 0:
        raise ValueError(f"oracle_spin_images_fp32 failed with status {rc}")
    return out
