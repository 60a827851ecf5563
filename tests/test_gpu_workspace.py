"""Caller workspaces that are too small or misaligned are rejected on the host with
RICI_ERR_WORKSPACE before anything is launched, and the library keeps working afterwards."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rici():
    import torch

    import paper_2007_02306_gb300 as p
    from paper_2007_02306_gb300 import build

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    p.load_library()
    return p


def test_small_or_misaligned_workspace_is_rejected(rici):
    import torch

    lib = rici.binding.load_library()
    err = rici.binding.ERR_WORKSPACE
    s = synth.tiny_scene()
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    v, n, t = d(s.vertices), d(s.normals), d(s.triangles)
    o = torch.arange(s.num_vertices, dtype=torch.int32, device="cuda")
    out = torch.empty((s.num_vertices, 32, 32), dtype=torch.uint16, device="cuda")
    need = lib.rici_generate_workspace_size(s.num_vertices, s.num_triangles, s.num_vertices, 32)
    ws = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
    base = ws.data_ptr() + ((-ws.data_ptr()) % 256)
    P = ctypes.c_void_p
    args = (P(v.data_ptr()), P(n.data_ptr()), s.num_vertices, P(t.data_ptr()), s.num_triangles,
            P(o.data_ptr()), s.num_vertices, ctypes.c_float(0.3), 32, P(out.data_ptr()))
    small = lib.rici_generate(*args, P(base), need - 1, None)
    unaligned = lib.rici_generate(*args, P(base + 16), need, None)
    for rc in (small, unaligned):
        assert rc == err
        assert b"workspace" in lib.rici_last_error_string()
    # a correct workspace still works, and gives the same images as the library's own
    assert lib.rici_generate(*args, P(base), need, None) == 0
    ref = rici.rici_generate(v, n, t, o, 0.3, 32)
    torch.cuda.synchronize()
    assert rici.sync_status() == 0
    assert torch.equal(out.view(torch.int16), ref.view(torch.int16))
