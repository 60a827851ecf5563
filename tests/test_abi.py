"""The C-ABI library builds, loads and exports every symbol include/*.h declares (CPU only).

No compute call is made here: argument checks that fail on the host return before any CUDA
call, so they run without a GPU.
"""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2007_02306_gb300 import build, binding

    build.build()
    return binding.load_library()


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"RICI_API\s+[\w\s\*]+?\b(\w+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("rici_generate", "crss_search", "rici_sync_status", "rici_last_error_string"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_library_exports_nothing_undeclared(lib):
    import subprocess

    from paper_2007_02306_gb300 import binding

    out = subprocess.run(["nm", "-D", "--defined-only", binding.library_path()],
                         capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert exported == set(declared_functions())


def test_version_and_workspace_queries(lib):
    assert b"sm_103a" in lib.rici_version()
    assert lib.rici_generate_workspace_size(10, 100, 5, 64) > 100 * 64
    assert lib.rici_generate_workspace_size(10, -1, 5, 64) == -1
    assert lib.crss_search_workspace_size(10, 100, 64, 0) >= 110 * 64 * 64
    # sparse-needle form: a slab of N^2/4 16-byte entries per needle on top of the packed deltas
    assert (lib.crss_search_workspace_size(10, 100, 64, 4)
            >= lib.crss_search_workspace_size(10, 100, 64, 1) - 10 * 64 * 4 + 10 * 64 * 64 * 4)
    assert lib.crss_search_workspace_size(10, 100, 0, 0) == -1


@pytest.mark.parametrize("N,R", [(0, 0.3), (129, 0.3), (64, 0.0), (64, -1.0), (64, float("nan")),
                                 (64, float("inf"))])
def test_generate_rejects_bad_arguments_on_host(lib, N, R):
    dummy = ctypes.c_void_p(16)
    rc = lib.rici_generate(dummy, dummy, 3, dummy, 1, dummy, 1, R, N, dummy, None, 0, None)
    assert rc == 1
    assert lib.rici_last_error_string()


def test_generate_rejects_null_and_negative(lib):
    dummy = ctypes.c_void_p(16)
    assert lib.rici_generate(dummy, dummy, -1, dummy, 1, dummy, 1, 0.3, 64, dummy, None, 0, None) == 1
    assert lib.rici_generate(None, dummy, 3, dummy, 1, dummy, 1, 0.3, 64, dummy, None, 0, None) == 1
    assert lib.rici_generate_ex(dummy, dummy, 3, dummy, 1, dummy, 1, 0.3, 64, dummy, 7, None, None,
                                0, None) == 1


def test_search_rejects_bad_arguments_on_host(lib):
    dummy = ctypes.c_void_p(16)
    # empty haystack with needles, bad resolution, bad mode, oversized distance matrix
    assert lib.crss_search(dummy, 1, dummy, 0, 64, None, dummy, None, None, None, 0, None, 0, None) == 1
    assert lib.crss_search(dummy, 1, dummy, 1, 1, None, dummy, None, None, None, 0, None, 0, None) == 1
    assert lib.crss_search(dummy, 1, dummy, 1, 64, None, dummy, None, None, None, 9, None, 0, None) == 1
    assert lib.crss_search(dummy, 1, dummy, 1, 64, None, dummy, None, None, None, 7, None, 0, None) == 1
    # the withheld-load hook is a tensor-core test bit: rejected with the sparse-needle form
    assert lib.crss_search(dummy, 1, dummy, 1, 64, None, dummy, None, None, None, 0x104, None, 0,
                           None) == 1
    # the withheld-load test bit is only accepted with the tensor-core form; other high bits never
    assert lib.crss_search(dummy, 1, dummy, 1, 64, None, dummy, None, None, None, 0x101, None, 0,
                           None) == 1
    assert lib.crss_search(dummy, 1, dummy, 1, 64, None, dummy, None, None, None, 0x203, None, 0,
                           None) == 1
    assert lib.crss_search(dummy, 1 << 15, dummy, 1 << 14, 64, None, dummy, None, None, dummy, 0,
                           None, 0, None) == 8


def test_zero_work_calls_are_no_ops(lib):
    dummy = ctypes.c_void_p(16)
    assert lib.rici_generate(dummy, dummy, 3, dummy, 1, dummy, 0, 0.3, 64, dummy, None, 0, None) == 0
    assert lib.crss_search(dummy, 0, dummy, 5, 64, None, dummy, None, None, None, 0, None, 0, None) == 0


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2007_02306_gb300 import binding

    saved = binding._lib
    binding._lib = None
    try:
        with pytest.raises(RuntimeError):
            binding.load_library(str(tmp_path / "missing.so"))
    finally:
        binding._lib = saved


def test_projection_and_tuning_reject_bad_arguments_on_host(lib):
    dummy = ctypes.c_void_p(16)
    assert lib.rici_project_fp32(dummy, -1, dummy, dummy, dummy, None) == 1
    assert lib.rici_project_fp32(None, 4, dummy, dummy, dummy, None) == 1
    assert lib.rici_project_fp32(dummy, 0, None, None, None, None) == 0
    assert lib.rici_get_tuning(None) == 1
    assert lib.rici_measure_dp4a_rate(None, None) == 1
    assert lib.rici_measure_mma_s8_rate(None, None) == 1


def test_clutter_rejects_bad_arguments_on_host(lib):
    dummy = ctypes.c_void_p(16)
    # bad support radius, negative object vertex count, null outputs
    assert lib.rici_clutter(dummy, dummy, 3, dummy, 1, dummy, 1, 0.0, 0, dummy, dummy, None, None,
                            0, None) == 1
    assert lib.rici_clutter(dummy, dummy, 3, dummy, 1, dummy, 1, 0.3, -1, dummy, dummy, None, None,
                            0, None) == 1
    assert lib.rici_clutter(dummy, dummy, 3, dummy, 1, dummy, 1, 0.3, 0, None, dummy, None, None,
                            0, None) == 1
    assert lib.rici_clutter(dummy, dummy, 3, dummy, 1, dummy, 1, 0.3, 0, dummy, None, None, None,
                            0, None) == 1
    # no oriented points: a valid no-op; the workspace is the generation grid's
    assert lib.rici_clutter(dummy, dummy, 3, dummy, 1, dummy, 0, 0.3, 0, None, None, None, None,
                            0, None) == 0
    assert lib.rici_clutter_workspace_size(100) == lib.rici_generate_workspace_size(3, 100, 1, 64)
    assert lib.rici_clutter_workspace_size(-1) == -1


def test_spin_images_reject_bad_arguments_on_host(lib):
    dummy = ctypes.c_void_p(16)
    # samples per side outside [1, 16], bad resolution, null output
    for m in (0, 17):
        assert lib.rici_spin_images(dummy, dummy, 3, dummy, 1, dummy, 1, 0.3, 64, m, dummy, None,
                                    0, None) == 1
    assert lib.rici_spin_images(dummy, dummy, 3, dummy, 1, dummy, 1, 0.3, 0, 3, dummy, None, 0,
                                None) == 1
    assert lib.rici_spin_images(dummy, dummy, 3, dummy, 1, dummy, 1, 0.3, 64, 3, None, None, 0,
                                None) == 1
    assert lib.rici_spin_images(dummy, dummy, 3, dummy, 1, dummy, 0, 0.3, 64, 3, None, None, 0,
                                None) == 0


def test_batch_run_rejects_bad_scenes_on_host(lib):
    from paper_2007_02306_gb300 import binding

    arr = (binding._BatchScene * 1)()
    arr[0] = binding._BatchScene(16, 16, 3, 16, 1, 2, 16, 1, 16, 1, None, 16, 16, 16, None, None)
    # target_triangles larger than the scene's triangle count
    assert lib.rici_batch_run(arr, 1, 0.3, 64, 3, None, 0, None) == 1
    assert lib.rici_batch_run_workspace_size(arr, 1, 64, 3) == -1
    # null scene array with scenes, negative scene count
    assert lib.rici_batch_run(None, 1, 0.3, 64, 3, None, 0, None) == 1
    assert lib.rici_batch_run(arr, -1, 0.3, 64, 3, None, 0, None) == 1
    # bad resolution and support radius reach the generation checks
    arr[0] = binding._BatchScene(16, 16, 3, 16, 1, 1, 16, 1, 16, 1, None, 16, 16, 16, None, None)
    assert lib.rici_batch_run(arr, 1, 0.3, 0, 3, None, 0, None) == 1
    assert lib.rici_batch_run(arr, 1, -1.0, 64, 3, None, 0, None) == 1
    assert lib.rici_batch_run(arr, 0, 0.3, 64, 3, None, 0, None) == 0


def test_noalloc_rejects_on_host_with_error_text(lib):
    dummy = ctypes.c_void_p(16)
    lib.rici_last_error_string.restype = ctypes.c_char_p
    # one triangle beyond the largest accepted mesh
    assert lib.rici_generate_noalloc(dummy, dummy, 3, dummy, 262145, dummy, 1, ctypes.c_float(0.3),
                                     64, dummy, None) == 8
    assert b"262144" in lib.rici_last_error_string()
    # the checks of rici_generate: radius, resolution, null output
    for R, N, out in ((float("inf"), 64, dummy), (0.3, 0, dummy), (0.3, 64, None)):
        assert lib.rici_generate_noalloc(dummy, dummy, 3, dummy, 1, dummy, 1, ctypes.c_float(R),
                                         N, out, None) == 1
        assert lib.rici_last_error_string() != b""
    # a finite radius near FLT_MAX is valid: no origins makes the call a no-op
    assert lib.rici_generate_noalloc(dummy, dummy, 3, dummy, 1, dummy, 0,
                                     ctypes.c_float(3.4028e38), 64, None, None) == 0
    assert lib.rici_last_error_string() == b""


def test_batch_run_ex_rejects_a_bad_tuning_on_host(lib):
    class T(ctypes.Structure):
        _fields_ = [("gen_cells_per_reach", ctypes.c_int32), ("gen_big_radius", ctypes.c_float),
                    ("gen_warps", ctypes.c_int32), ("tc_group_m", ctypes.c_int32)]

    lib.rici_last_error_string.restype = ctypes.c_char_p
    bad = T(5, 0.25, 4, 8)
    assert lib.rici_batch_run_ex(None, 0, ctypes.c_float(0.3), 64, 3, ctypes.byref(bad), None, 0,
                                 None) == 1
    assert b"tuning" in lib.rici_last_error_string()
    # a valid tuning for an empty batch: a no-op that leaves the process-wide tuning alone
    before = T()
    assert lib.rici_get_tuning(ctypes.byref(before)) == 0
    good = T(4, 1.0, 8, 16)
    assert lib.rici_batch_run_ex(None, 0, ctypes.c_float(0.3), 64, 3, ctypes.byref(good), None, 0,
                                 None) == 0
    after = T()
    assert lib.rici_get_tuning(ctypes.byref(after)) == 0
    assert (after.gen_cells_per_reach, after.tc_group_m) == (before.gen_cells_per_reach,
                                                            before.tc_group_m)
