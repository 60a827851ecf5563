"""ctypes binding of librici (argument marshalling only).

Every step of generation and search runs in the CUDA library; this module checks tensor
dtypes/devices, allocates outputs and a cached workspace with PyTorch, and passes raw device
pointers plus the current CUDA stream through the C ABI declared in include/rici.h.  There
is no CPU fallback: if the library is missing or cannot be loaded the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

GEN_DEFAULT = 0
GEN_FP64 = 1
SEARCH_DEFAULT = 0
SEARCH_CUDA_CORE = 1
SEARCH_EXACT_SLOW = 2
SEARCH_TENSOR = 3
SEARCH_SPARSE = 4
SEARCH_INT8_TC = 5
SEARCH_AUTO = 6
SEARCH_TEST_WITHHOLD_LOAD = 0x100  # test hook (see include/rici.h)

ERR_INVALID_ARGUMENT = 1
ERR_INDEX_OUT_OF_RANGE = 2
ERR_NONFINITE_INPUT = 4
ERR_OUT_TOO_LARGE = 8
ERR_CUDA = 16
ERR_WORKSPACE = 32
ERR_TIMEOUT = 64

MAX_RESOLUTION = 128

_lock = threading.Lock()
_lib = None
_workspaces: dict = {}


class _GenScene(ctypes.Structure):
    _fields_ = [("vertices", ctypes.c_void_p), ("normals", ctypes.c_void_p),
                ("num_vertices", ctypes.c_int64), ("triangles", ctypes.c_void_p),
                ("num_triangles", ctypes.c_int64), ("origins", ctypes.c_void_p),
                ("num_origins", ctypes.c_int64), ("out_images", ctypes.c_void_p)]


class _SearchScene(ctypes.Structure):
    _fields_ = [("needles", ctypes.c_void_p), ("num_needles", ctypes.c_int64),
                ("haystack", ctypes.c_void_p), ("num_haystack", ctypes.c_int64),
                ("true_match", ctypes.c_void_p), ("out_rank", ctypes.c_void_p),
                ("out_true_distance", ctypes.c_void_p), ("out_top1", ctypes.c_void_p)]


class _BatchScene(ctypes.Structure):
    _fields_ = [("vertices", ctypes.c_void_p), ("normals", ctypes.c_void_p),
                ("num_vertices", ctypes.c_int64), ("triangles", ctypes.c_void_p),
                ("num_triangles", ctypes.c_int64), ("target_triangles", ctypes.c_int64),
                ("needle_origins", ctypes.c_void_p), ("num_needles", ctypes.c_int64),
                ("haystack_origins", ctypes.c_void_p), ("num_haystack", ctypes.c_int64),
                ("true_match", ctypes.c_void_p), ("needle_images", ctypes.c_void_p),
                ("haystack_images", ctypes.c_void_p), ("out_rank", ctypes.c_void_p),
                ("out_true_distance", ctypes.c_void_p), ("out_top1", ctypes.c_void_p)]


class RiciError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"librici error {code}: {message}")
        self.code = code


def library_path() -> str:
    return _build.LIB


def load_library(path: str | None = None):
    """Load librici.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or library_path()
        if not os.path.exists(p):
            raise RuntimeError(f"librici.so not found at {p}; build it with "
                               "paper_2007_02306_gb300.build.build() (nvcc, sm_103a)")
        lib = ctypes.CDLL(p)
        P, i64, i32, f32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_float
        lib.rici_generate_workspace_size.argtypes = [i64, i64, i64, i32]
        lib.rici_generate_workspace_size.restype = i64
        lib.rici_generate.argtypes = [P, P, i64, P, i64, P, i64, f32, i32, P, P, i64, P]
        lib.rici_generate.restype = ctypes.c_int
        lib.rici_generate_ex.argtypes = [P, P, i64, P, i64, P, i64, f32, i32, P, i32, P, P, i64, P]
        lib.rici_generate_ex.restype = ctypes.c_int
        lib.crss_search_workspace_size.argtypes = [i64, i64, i32, i32]
        lib.crss_search_workspace_size.restype = i64
        lib.crss_search.argtypes = [P, i64, P, i64, i32, P, P, P, P, P, i32, P, i64, P]
        lib.crss_search.restype = ctypes.c_int
        lib.crss_search_ex.argtypes = [P, i64, P, i64, i32, P, P, P, P, P, i32, P, P, i64, P]
        lib.crss_search_ex.restype = ctypes.c_int
        lib.rici_generate_noalloc.argtypes = [P, P, i64, P, i64, P, i64, f32, i32, P, P]
        lib.rici_generate_noalloc.restype = ctypes.c_int
        lib.rici_generate_batch_workspace_size.argtypes = [P, i32, i32]
        lib.rici_generate_batch_workspace_size.restype = i64
        lib.rici_generate_batch.argtypes = [P, i32, f32, i32, P, i64, P]
        lib.rici_generate_batch.restype = ctypes.c_int
        lib.crss_search_batch_workspace_size.argtypes = [P, i32, i32, i32]
        lib.crss_search_batch_workspace_size.restype = i64
        lib.crss_search_batch.argtypes = [P, i32, i32, i32, P, i64, P]
        lib.crss_search_batch.restype = ctypes.c_int
        lib.rici_batch_run_workspace_size.argtypes = [P, i32, i32, i32]
        lib.rici_batch_run_workspace_size.restype = i64
        lib.rici_batch_run.argtypes = [P, i32, f32, i32, i32, P, i64, P]
        lib.rici_batch_run.restype = ctypes.c_int
        lib.rici_batch_run_ex.argtypes = [P, i32, f32, i32, i32, P, P, i64, P]
        lib.rici_batch_run_ex.restype = ctypes.c_int
        lib.rici_sync_status.argtypes = [P, ctypes.POINTER(i32)]
        lib.rici_sync_status.restype = ctypes.c_int
        lib.rici_release_workspace.argtypes = []
        lib.rici_release_workspace.restype = ctypes.c_int
        lib.rici_last_error_string.argtypes = []
        lib.rici_last_error_string.restype = ctypes.c_char_p
        lib.rici_kernel_launches.argtypes = []
        lib.rici_kernel_launches.restype = i64
        lib.rici_clutter_workspace_size.argtypes = [i64]
        lib.rici_clutter_workspace_size.restype = i64
        lib.rici_clutter.argtypes = [P, P, i64, P, i64, P, i64, f32, i64, P, P, P, P, i64, P]
        lib.rici_clutter.restype = ctypes.c_int
        lib.rici_spin_images.argtypes = [P, P, i64, P, i64, P, i64, f32, i32, i32, P, P, i64, P]
        lib.rici_spin_images.restype = ctypes.c_int
        lib.rici_project_fp32.argtypes = [P, i64, P, P, P, P]
        lib.rici_project_fp32.restype = ctypes.c_int
        lib.rici_set_tuning.argtypes = [P]
        lib.rici_set_tuning.restype = ctypes.c_int
        lib.rici_get_tuning.argtypes = [P]
        lib.rici_get_tuning.restype = ctypes.c_int
        lib.rici_autotune_generate_batch.argtypes = [P, i32, f32, i32, P, i64, P, i32, P, P]
        lib.rici_autotune_generate_batch.restype = ctypes.c_int
        lib.rici_autotune_search_batch.argtypes = [P, i32, i32, P, i64, P, i32, P, P]
        lib.rici_autotune_search_batch.restype = ctypes.c_int
        lib.rici_measure_dp4a_rate.argtypes = [P, ctypes.POINTER(ctypes.c_double)]
        lib.rici_measure_dp4a_rate.restype = ctypes.c_int
        lib.rici_measure_mma_s8_rate.argtypes = [P, ctypes.POINTER(ctypes.c_double)]
        lib.rici_measure_mma_s8_rate.restype = ctypes.c_int
        lib.rici_version.argtypes = []
        lib.rici_version.restype = ctypes.c_char_p
        _lib = lib
        return lib


def _check(rc: int):
    if rc != 0:
        msg = load_library().rici_last_error_string().decode(errors="replace")
        raise RiciError(rc, msg)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _need(t, dtype, name, shape_tail=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape_tail is not None and tuple(t.shape[1:]) != tuple(shape_tail):
        raise ValueError(f"{name} must have shape [*, {', '.join(map(str, shape_tail))}]")
    return t


def workspace(device, nbytes: int) -> torch.Tensor:
    """Cached per-device scratch buffer (uint8, 256-byte aligned), grown on demand."""
    dev = torch.device(device)
    key = dev.index if dev.index is not None else torch.cuda.current_device()
    buf = _workspaces.get(key)
    if buf is None or buf.numel() < nbytes:
        _workspaces.pop(key, None)
        buf = torch.empty(max(int(nbytes), 256) + 256, dtype=torch.uint8, device=dev)
        _workspaces[key] = buf
    off = (-buf.data_ptr()) % 256
    return buf[off:]


def release_workspaces() -> None:
    """Drop the cached scratch buffers of every device (their memory returns to torch's
    allocator once no call still holds them)."""
    _workspaces.clear()


def rici_generate(vertices, normals, triangles, origins, support_radius: float, resolution: int,
                  *, out=None, mode: int = GEN_DEFAULT, counters=None, stream=None):
    """uint16 [O, N, N] RICI images of the oriented points (vertices[origins], normals[origins])."""
    lib = load_library()
    v = _need(vertices, torch.float32, "vertices", (3,))
    n = _need(normals, torch.float32, "normals", (3,))
    t = _need(triangles, torch.int32, "triangles", (3,))
    o = _need(origins, torch.int32, "origins")
    if n.shape != v.shape:
        raise ValueError("normals must have the same shape as vertices")
    N = int(resolution)
    if out is None:
        out = torch.empty((o.numel(), N, N), dtype=torch.uint16, device=v.device)
    else:
        _need(out, torch.uint16, "out", (N, N))
        if out.shape[0] != o.numel():
            raise ValueError("out must have one image per origin")
    if counters is not None:
        _need(counters, torch.int64, "counters")
        if counters.numel() < 4:
            raise ValueError("counters needs 4 int64 entries")
    nb = lib.rici_generate_workspace_size(v.shape[0], t.shape[0], o.numel(), N)
    if nb < 0:
        raise ValueError("invalid sizes")
    ws = workspace(v.device, nb)
    with torch.cuda.device(v.device):
        _check(lib.rici_generate_ex(_ptr(v), _ptr(n), v.shape[0], _ptr(t), t.shape[0], _ptr(o),
                                    o.numel(), float(support_radius), N, _ptr(out), int(mode),
                                    _ptr(counters), _ptr(ws), ws.numel(), _stream_handle(stream)))
    return out


def clutter_areas(vertices, normals, triangles, origins, support_radius: float,
                  object_vertices: int, *, with_clutter: bool = False, stream=None):
    """Eq. clutter inputs per oriented point: float64 [O] tensors (A_all, A_object), the surface
    area inside the support volume and its part on triangles whose first vertex index is below
    ``object_vertices``; with ``with_clutter`` also Eq. clutter itself, (A_all - A_object) /
    A_all computed by the library (NaN where A_all = 0)."""
    lib = load_library()
    v = _need(vertices, torch.float32, "vertices", (3,))
    n = _need(normals, torch.float32, "normals", (3,))
    t = _need(triangles, torch.int32, "triangles", (3,))
    o = _need(origins, torch.int32, "origins")
    if n.shape != v.shape:
        raise ValueError("normals must have the same shape as vertices")
    a_all = torch.empty(o.numel(), dtype=torch.float64, device=v.device)
    a_obj = torch.empty(o.numel(), dtype=torch.float64, device=v.device)
    clu = torch.empty(o.numel(), dtype=torch.float64, device=v.device) if with_clutter else None
    nb = lib.rici_clutter_workspace_size(t.shape[0])
    if nb < 0:
        raise ValueError("invalid sizes")
    ws = workspace(v.device, nb)
    with torch.cuda.device(v.device):
        _check(lib.rici_clutter(_ptr(v), _ptr(n), v.shape[0], _ptr(t), t.shape[0], _ptr(o),
                                o.numel(), float(support_radius), int(object_vertices),
                                _ptr(a_all), _ptr(a_obj), _ptr(clu), _ptr(ws), ws.numel(),
                                _stream_handle(stream)))
    return (a_all, a_obj, clu) if with_clutter else (a_all, a_obj)


def spin_images(vertices, normals, triangles, origins, support_radius: float, resolution: int,
                samples_side: int = 3, *, out=None, stream=None):
    """float32 [O, N, N] spin images (Section 2.1) of the oriented points from samples_side^2
    point samples per triangle (see include/rici.h for the sampling and binning)."""
    lib = load_library()
    v = _need(vertices, torch.float32, "vertices", (3,))
    n = _need(normals, torch.float32, "normals", (3,))
    t = _need(triangles, torch.int32, "triangles", (3,))
    o = _need(origins, torch.int32, "origins")
    if n.shape != v.shape:
        raise ValueError("normals must have the same shape as vertices")
    N = int(resolution)
    if out is None:
        out = torch.empty((o.numel(), N, N), dtype=torch.float32, device=v.device)
    else:
        _need(out, torch.float32, "out", (N, N))
        if out.shape[0] != o.numel():
            raise ValueError("out must have one image per origin")
    nb = lib.rici_clutter_workspace_size(t.shape[0])
    if nb < 0:
        raise ValueError("invalid sizes")
    ws = workspace(v.device, nb)
    with torch.cuda.device(v.device):
        _check(lib.rici_spin_images(_ptr(v), _ptr(n), v.shape[0], _ptr(t), t.shape[0], _ptr(o),
                                    o.numel(), float(support_radius), N, int(samples_side),
                                    _ptr(out), _ptr(ws), ws.numel(), _stream_handle(stream)))
    return out


def crss_search(needles, haystack, true_match=None, *, mode: int = SEARCH_DEFAULT,
                return_distances: bool = False, counters=None, stream=None):
    """Rank of each needle's true match, its true distance and the top-1 haystack index."""
    lib = load_library()
    q = _need(needles, torch.uint16, "needles")
    h = _need(haystack, torch.uint16, "haystack")
    if q.dim() != 3 or h.dim() != 3 or q.shape[1] != q.shape[2] or tuple(h.shape[1:]) != tuple(q.shape[1:]):
        raise ValueError("needles and haystack must be [*, N, N] with the same N")
    N = int(q.shape[-1])
    Q, H = int(q.shape[0]), int(h.shape[0])
    dev = q.device
    m = None
    if true_match is not None:
        m = _need(true_match, torch.int64, "true_match")
        if m.numel() != Q:
            raise ValueError("true_match needs one entry per needle")
    rank = torch.empty(Q, dtype=torch.int32, device=dev)
    dt = torch.empty(Q, dtype=torch.int64, device=dev)
    top1 = torch.empty(Q, dtype=torch.int32, device=dev)
    dist = torch.empty((Q, H), dtype=torch.int64, device=dev) if return_distances else None
    if counters is not None:
        _need(counters, torch.int64, "counters")
        if counters.numel() < 4:
            raise ValueError("counters needs 4 int64 entries")
    nb = lib.crss_search_workspace_size(Q, H, N, int(mode))
    if nb < 0:
        raise ValueError("invalid sizes")
    ws = workspace(dev, nb)
    with torch.cuda.device(dev):
        _check(lib.crss_search_ex(_ptr(q), Q, _ptr(h), H, N, _ptr(m), _ptr(rank), _ptr(dt),
                                  _ptr(top1), _ptr(dist), int(mode), _ptr(counters), _ptr(ws),
                                  ws.numel(), _stream_handle(stream)))
    out = {"rank": rank, "true_distance": dt, "top1": top1}
    if dist is not None:
        out["distances"] = dist
    return out


def _ptr0(t):
    return None if t is None else t.data_ptr()


def rici_generate_batch(scenes, support_radius: float, resolution: int, *, workspace_tensor=None,
                        stream=None):
    """Generation for several scenes in one set of launches.

    scenes: list of dicts with CUDA tensors "vertices" [V,3] f32, "normals" [V,3] f32,
    "triangles" [T,3] i32, "origins" [O] i32 and optionally "out" uint16 [O,N,N].
    Returns the list of output tensors.  workspace_tensor: optional uint8 CUDA tensor (kept by
    the caller, e.g. for CUDA-graph replay); otherwise the cached per-device workspace is used.
    """
    lib = load_library()
    N = int(resolution)
    arr, outs = _gen_scene_array(scenes, N)
    nb = lib.rici_generate_batch_workspace_size(arr, len(scenes), N)
    if nb < 0:
        _check(1)
    dev = outs[0].device if outs else torch.device("cuda")
    ws = workspace_tensor if workspace_tensor is not None else workspace(dev, nb)
    if ws.numel() < nb:
        raise ValueError(f"workspace_tensor needs {nb} bytes")
    with torch.cuda.device(dev):
        _check(lib.rici_generate_batch(arr, len(scenes), float(support_radius), N, _ptr(ws),
                                       ws.numel(), _stream_handle(stream)))
    return outs


def _gen_scene_array(scenes, N):
    arr = (_GenScene * max(1, len(scenes)))()
    outs = []
    for k, sc in enumerate(scenes):
        v = _need(sc["vertices"], torch.float32, "vertices", (3,))
        n = _need(sc["normals"], torch.float32, "normals", (3,))
        t = _need(sc["triangles"], torch.int32, "triangles", (3,))
        o = _need(sc["origins"], torch.int32, "origins")
        out = sc.get("out")
        if out is None:
            out = torch.empty((o.numel(), N, N), dtype=torch.uint16, device=v.device)
        _need(out, torch.uint16, "out", (N, N))
        outs.append(out)
        arr[k] = _GenScene(_ptr0(v), _ptr0(n), v.shape[0], _ptr0(t), t.shape[0], _ptr0(o), o.numel(),
                           _ptr0(out))
    return arr, outs


def generate_batch_workspace_bytes(scenes, resolution: int) -> int:
    lib = load_library()
    arr = (_GenScene * max(1, len(scenes)))()
    for k, sc in enumerate(scenes):
        arr[k] = _GenScene(_ptr0(sc["vertices"]), _ptr0(sc["normals"]), sc["vertices"].shape[0],
                           _ptr0(sc["triangles"]), sc["triangles"].shape[0], _ptr0(sc["origins"]),
                           sc["origins"].numel(), 1)
    return int(lib.rici_generate_batch_workspace_size(arr, len(scenes), int(resolution)))


def batch_run(scenes, support_radius: float, resolution: int, *, mode: int = SEARCH_TENSOR,
              workspace_tensor=None, outputs=None, tuning=None, stream=None):
    """The whole path for several scenes in one call (rici_batch_run).

    scenes: list of dicts with CUDA tensors "vertices" [V,3] f32, "normals" [V,3] f32,
    "triangles" [T,3] i32 (the target mesh first), "needle_origins" [Q] i32, "haystack_origins"
    [H] i32, optional "true_match" [Q] i64, and the int "target_triangles".  outputs: optional
    list of dicts of preallocated "needle_images", "haystack_images", "rank", "true_distance",
    "top1" (needed to replay a captured graph).  tuning: a dict of RiciTuning fields in force for
    this call only (rici_batch_run_ex), or None for the process-wide setting.  Returns the list of
    output dicts.
    """
    lib = load_library()
    N = int(resolution)
    arr = (_BatchScene * max(1, len(scenes)))()
    res = []
    for k, sc in enumerate(scenes):
        v = _need(sc["vertices"], torch.float32, "vertices", (3,))
        n = _need(sc["normals"], torch.float32, "normals", (3,))
        t = _need(sc["triangles"], torch.int32, "triangles", (3,))
        on = _need(sc["needle_origins"], torch.int32, "needle_origins")
        oh = _need(sc["haystack_origins"], torch.int32, "haystack_origins")
        m = sc.get("true_match")
        if m is not None:
            _need(m, torch.int64, "true_match")
        Q, H = on.numel(), oh.numel()
        if outputs is not None:
            r = outputs[k]
        else:
            r = {"needle_images": torch.empty((Q, N, N), dtype=torch.uint16, device=v.device),
                 "haystack_images": torch.empty((H, N, N), dtype=torch.uint16, device=v.device),
                 "rank": torch.empty(Q, dtype=torch.int32, device=v.device),
                 "true_distance": torch.empty(Q, dtype=torch.int64, device=v.device),
                 "top1": torch.empty(Q, dtype=torch.int32, device=v.device)}
        res.append(r)
        arr[k] = _BatchScene(_ptr0(v), _ptr0(n), v.shape[0], _ptr0(t), t.shape[0],
                             int(sc["target_triangles"]), _ptr0(on), Q, _ptr0(oh), H, _ptr0(m),
                             _ptr0(r["needle_images"]), _ptr0(r["haystack_images"]),
                             _ptr0(r["rank"]), _ptr0(r["true_distance"]), _ptr0(r["top1"]))
    nb = lib.rici_batch_run_workspace_size(arr, len(scenes), N, int(mode))
    if nb < 0:
        _check(1)
    dev = scenes[0]["vertices"].device if scenes else torch.device("cuda")
    ws = workspace_tensor if workspace_tensor is not None else workspace(dev, nb)
    if ws.numel() < nb:
        raise ValueError(f"workspace_tensor needs {nb} bytes")
    tun = None
    if tuning is not None:
        tun = _Tuning(**{k: tuning[k] for k in TUNING_FIELDS})
    with torch.cuda.device(dev):
        _check(lib.rici_batch_run_ex(arr, len(scenes), float(support_radius), N, int(mode),
                                     None if tun is None else ctypes.byref(tun), _ptr(ws),
                                     ws.numel(), _stream_handle(stream)))
    return res


def batch_run_workspace_bytes(scenes, resolution: int, outputs, mode: int = SEARCH_TENSOR) -> int:
    """Workspace bytes ``batch_run`` needs for these scenes and preallocated ``outputs`` (to
    size a caller workspace for graph capture)."""
    lib = load_library()
    N = int(resolution)
    arr = (_BatchScene * max(1, len(scenes)))()
    for k, (sc, r) in enumerate(zip(scenes, outputs)):
        arr[k] = _BatchScene(_ptr0(sc["vertices"]), _ptr0(sc["normals"]), int(sc["vertices"].shape[0]),
                             _ptr0(sc["triangles"]), int(sc["triangles"].shape[0]),
                             int(sc["target_triangles"]), _ptr0(sc["needle_origins"]),
                             int(sc["needle_origins"].numel()), _ptr0(sc["haystack_origins"]),
                             int(sc["haystack_origins"].numel()), _ptr0(sc.get("true_match")),
                             _ptr0(r["needle_images"]), _ptr0(r["haystack_images"]),
                             _ptr0(r["rank"]), _ptr0(r.get("true_distance")), _ptr0(r.get("top1")))
    nb = lib.rici_batch_run_workspace_size(arr, len(scenes), N, int(mode))
    if nb < 0:
        _check(1)
    return nb


def crss_search_batch(scenes, resolution: int, *, mode: int = SEARCH_TENSOR, workspace_tensor=None,
                      outputs=None, stream=None):
    """Search several scenes in one set of launches; each needle only against its scene.

    scenes: list of dicts with "needles" uint16 [Q,N,N], "haystack" uint16 [H,N,N] and optional
    "true_match" int64 [Q] (scene-local).  outputs: optional list of dicts of preallocated
    "rank" / "true_distance" / "top1" tensors (needed to replay a captured graph).
    """
    lib = load_library()
    N = int(resolution)
    arr, res = _search_scene_array(scenes, outputs)
    nb = lib.crss_search_batch_workspace_size(arr, len(scenes), N, int(mode))
    if nb < 0:
        _check(1)
    dev = scenes[0]["needles"].device if scenes else torch.device("cuda")
    ws = workspace_tensor if workspace_tensor is not None else workspace(dev, nb)
    if ws.numel() < nb:
        raise ValueError(f"workspace_tensor needs {nb} bytes")
    with torch.cuda.device(dev):
        _check(lib.crss_search_batch(arr, len(scenes), N, int(mode), _ptr(ws), ws.numel(),
                                     _stream_handle(stream)))
    return res


def _search_scene_array(scenes, outputs=None):
    arr = (_SearchScene * max(1, len(scenes)))()
    res = []
    for k, sc in enumerate(scenes):
        q = _need(sc["needles"], torch.uint16, "needles")
        h = _need(sc["haystack"], torch.uint16, "haystack")
        m = sc.get("true_match")
        if m is not None:
            _need(m, torch.int64, "true_match")
        if outputs is not None:
            r = outputs[k]
        else:
            Q = q.shape[0]
            r = {"rank": torch.empty(Q, dtype=torch.int32, device=q.device),
                 "true_distance": torch.empty(Q, dtype=torch.int64, device=q.device),
                 "top1": torch.empty(Q, dtype=torch.int32, device=q.device)}
        res.append(r)
        arr[k] = _SearchScene(_ptr0(q), q.shape[0], _ptr0(h), h.shape[0], _ptr0(m),
                              _ptr0(r["rank"]), _ptr0(r["true_distance"]), _ptr0(r["top1"]))
    return arr, res


def search_batch_workspace_bytes(scenes, resolution: int, mode: int = SEARCH_TENSOR) -> int:
    lib = load_library()
    arr = (_SearchScene * max(1, len(scenes)))()
    for k, sc in enumerate(scenes):
        arr[k] = _SearchScene(_ptr0(sc["needles"]), sc["needles"].shape[0], _ptr0(sc["haystack"]),
                              sc["haystack"].shape[0], None, 1, None, None)
    return int(lib.crss_search_batch_workspace_size(arr, len(scenes), int(resolution), int(mode)))


def sync_status(stream=None) -> int:
    """Synchronise the stream and return (and clear) the device status word."""
    lib = load_library()
    v = ctypes.c_int32(0)
    _check(lib.rici_sync_status(_stream_handle(stream), ctypes.byref(v)))
    return int(v.value)


def kernel_launches() -> int:
    """Kernels the library has enqueued in this process so far."""
    return int(load_library().rici_kernel_launches())


def version() -> str:
    return load_library().rici_version().decode()


def measure_dp4a_rate(stream=None) -> float:
    """Whole-device dp4a instructions per second (the search kernel's multiply pipe)."""
    lib = load_library()
    out = ctypes.c_double(0.0)
    _check(lib.rici_measure_dp4a_rate(_stream_handle(stream), ctypes.byref(out)))
    return float(out.value)


def measure_mma_s8_rate(stream=None) -> float:
    """Whole-device int8 multiply-adds per second through mma.sync s8 (the int8 tensor-core
    search's instruction)."""
    lib = load_library()
    out = ctypes.c_double(0.0)
    _check(lib.rici_measure_mma_s8_rate(_stream_handle(stream), ctypes.byref(out)))
    return float(out.value)


class _Tuning(ctypes.Structure):
    _fields_ = [("gen_cells_per_reach", ctypes.c_int32), ("gen_big_radius", ctypes.c_float),
                ("gen_warps", ctypes.c_int32), ("tc_group_m", ctypes.c_int32)]


TUNING_FIELDS = tuple(f for f, _ in _Tuning._fields_)


def _tuning_dict(t: _Tuning) -> dict:
    return {f: (float(getattr(t, f)) if f == "gen_big_radius" else int(getattr(t, f)))
            for f in TUNING_FIELDS}


def get_tuning() -> dict:
    """The process-wide launch tuning in force (see RiciTuning in include/rici.h)."""
    t = _Tuning()
    _check(load_library().rici_get_tuning(ctypes.byref(t)))
    return _tuning_dict(t)


def set_tuning(tuning=None) -> None:
    """Set the launch tuning (a dict with every field of RiciTuning); None restores defaults."""
    lib = load_library()
    if tuning is None:
        _check(lib.rici_set_tuning(None))
        return
    missing = [f for f in TUNING_FIELDS if f not in tuning]
    if missing:
        raise ValueError(f"tuning lacks {missing}")
    t = _Tuning(*(tuning[f] for f in TUNING_FIELDS))
    _check(lib.rici_set_tuning(ctypes.byref(t)))


def autotune_generate_batch(scenes, support_radius: float, resolution: int, *, repeats: int = 1,
                            stream=None):
    """Time every candidate generation tuning on these scenes; returns (best tuning, ms)."""
    lib = load_library()
    N = int(resolution)
    arr, outs = _gen_scene_array(scenes, N)
    nb = lib.rici_generate_batch_workspace_size(arr, len(scenes), N)
    if nb < 0:
        _check(1)
    dev = outs[0].device if outs else torch.device("cuda")
    ws = workspace(dev, nb)
    best, ms = _Tuning(), ctypes.c_float(0.0)
    with torch.cuda.device(dev):
        _check(lib.rici_autotune_generate_batch(arr, len(scenes), float(support_radius), N, _ptr(ws),
                                                ws.numel(), _stream_handle(stream), int(repeats),
                                                ctypes.byref(best), ctypes.byref(ms)))
    return _tuning_dict(best), float(ms.value)


def autotune_search_batch(scenes, resolution: int, *, repeats: int = 1, stream=None):
    """Time every candidate tensor-core search tuning on these scenes; returns (best, ms)."""
    lib = load_library()
    N = int(resolution)
    arr, _ = _search_scene_array(scenes)
    nb = lib.crss_search_batch_workspace_size(arr, len(scenes), N, SEARCH_TENSOR)
    if nb < 0:
        _check(1)
    dev = scenes[0]["needles"].device if scenes else torch.device("cuda")
    ws = workspace(dev, nb)
    best, ms = _Tuning(), ctypes.c_float(0.0)
    with torch.cuda.device(dev):
        _check(lib.rici_autotune_search_batch(arr, len(scenes), N, _ptr(ws), ws.numel(),
                                              _stream_handle(stream), int(repeats),
                                              ctypes.byref(best), ctypes.byref(ms)))
    return _tuning_dict(best), float(ms.value)


def project_fp32(points, spin_vertex, spin_normal, stream=None):
    """The generation kernel's FP32 projection of points [n, 3] into one oriented point's frame."""
    lib = load_library()
    pts = _need(points, torch.float32, "points")
    sv = _need(spin_vertex, torch.float32, "spin_vertex")
    sn = _need(spin_normal, torch.float32, "spin_normal")
    if pts.dim() != 2 or pts.shape[1] != 3 or sv.numel() != 3 or sn.numel() != 3:
        raise ValueError("points must be [n, 3]; spin_vertex and spin_normal 3 floats")
    out = torch.empty_like(pts)
    with torch.cuda.device(pts.device):
        _check(lib.rici_project_fp32(_ptr(pts), pts.shape[0], _ptr(sv), _ptr(sn), _ptr(out),
                                     _stream_handle(stream)))
    return out
