"""Launch tuning: the C-ABI setter/getter and the autotune cache (CPU only).

rici_set_tuning / rici_get_tuning touch no device, so they run here.  The cache logic of
paper_2007_02306_gb300.autotune is exercised with stand-in tuners that record their calls: the
first batch of a workload class is measured and stored, later batches of the same class reuse the
entry, another class or a damaged cache is measured again, and the merged tuning is applied.
"""
import json

import pytest
import torch


@pytest.fixture(scope="module")
def binding():
    from paper_2007_02306_gb300 import binding as b
    from paper_2007_02306_gb300 import build

    build.build()
    b.load_library()
    yield b
    b.set_tuning(None)


DEFAULT = {"gen_cells_per_reach": 2, "gen_big_radius": 0.25, "gen_warps": 4, "tc_group_m": 8}


def test_defaults_and_roundtrip(binding):
    binding.set_tuning(None)
    assert binding.get_tuning() == DEFAULT
    t = {"gen_cells_per_reach": 3, "gen_big_radius": 0.125, "gen_warps": 8, "tc_group_m": 16}
    binding.set_tuning(t)
    assert binding.get_tuning() == t
    binding.set_tuning(None)
    assert binding.get_tuning() == DEFAULT


@pytest.mark.parametrize("field,value", [("gen_cells_per_reach", 1), ("gen_cells_per_reach", 5),
                                         ("gen_big_radius", 0.01), ("gen_big_radius", 1.5),
                                         ("gen_warps", 6), ("tc_group_m", 0),
                                         ("tc_group_m", 65)])
def test_out_of_range_is_rejected_and_changes_nothing(binding, field, value):
    binding.set_tuning(None)
    bad = dict(DEFAULT, **{field: value})
    with pytest.raises(binding.RiciError):
        binding.set_tuning(bad)
    assert binding.get_tuning() == DEFAULT


def gen_scene(t, o):
    return {"triangles": torch.zeros((t, 3), dtype=torch.int32),
            "origins": torch.zeros(o, dtype=torch.int32)}


def search_scene(q, h):
    return {"needles": torch.zeros((q, 2, 2), dtype=torch.int16),
            "haystack": torch.zeros((h, 2, 2), dtype=torch.int16)}


class Recorder:
    def __init__(self, best):
        self.best = best
        self.calls = []

    def __call__(self, scenes, *args, **kw):
        self.calls.append(len(scenes))
        return dict(self.best), 1.5


def test_cache_measures_once_per_class(binding, tmp_path):
    from paper_2007_02306_gb300 import autotune

    path = str(tmp_path / "tuning.json")
    g = Recorder({"gen_cells_per_reach": 3, "gen_big_radius": 0.5, "gen_warps": 8, "tc_group_m": 8})
    s = Recorder({"gen_cells_per_reach": 2, "gen_big_radius": 0.25, "gen_warps": 4, "tc_group_m": 32})
    gens = [gen_scene(100_000, 50_000) for _ in range(6)]
    srch = [search_scene(256, 50_000) for _ in range(6)]
    binding.set_tuning(None)
    t = autotune.tune_batch(gens, srch, 0.3, 64, gpu_name="GPU-X", sample=4, path=path,
                            gen_tuner=g, search_tuner=s)
    assert g.calls == [4] and s.calls == [4]
    want = {"gen_cells_per_reach": 3, "gen_big_radius": 0.5, "gen_warps": 8, "tc_group_m": 32}
    assert t == want and binding.get_tuning() == want
    data = json.load(open(path))
    assert len(data) == 2 and all(k.startswith("GPU-X|") for k in data)
    # same classes (sizes within the same power of two): served from the cache
    binding.set_tuning(None)
    t2 = autotune.tune_batch([gen_scene(110_000, 52_000)], [search_scene(250, 48_000)], 0.3, 64,
                             gpu_name="GPU-X", path=path, gen_tuner=g, search_tuner=s)
    assert t2 == want and g.calls == [4] and s.calls == [4]
    # another GPU, resolution or size class is measured again
    autotune.tune_batch(gens, [], 0.3, 64, gpu_name="GPU-Y", path=path, gen_tuner=g)
    autotune.tune_batch(gens, [], 0.3, 32, gpu_name="GPU-X", path=path, gen_tuner=g)
    autotune.tune_batch([gen_scene(10_000, 5_000)], [], 0.3, 64, gpu_name="GPU-X", path=path,
                        gen_tuner=g)
    assert g.calls == [4, 4, 4, 1] and len(json.load(open(path))) == 5
    binding.set_tuning(None)


def test_damaged_cache_is_measured_again(binding, tmp_path):
    from paper_2007_02306_gb300 import autotune

    path = tmp_path / "tuning.json"
    path.write_text("{not json")
    g = Recorder(dict(DEFAULT, gen_warps=8))
    autotune.tune_batch([gen_scene(1000, 100)], [], 0.3, 64, gpu_name="G", path=str(path),
                        gen_tuner=g)
    assert g.calls == [1]
    key = next(iter(json.load(open(path))))
    data = json.load(open(path))
    data[key] = {"tuning": {"gen_warps": 4}}  # incomplete entry
    path.write_text(json.dumps(data))
    autotune.tune_batch([gen_scene(1000, 100)], [], 0.3, 64, gpu_name="G", path=str(path),
                        gen_tuner=g)
    assert g.calls == [1, 1]
    binding.set_tuning(None)


def test_classes_name_their_shape():
    from paper_2007_02306_gb300 import autotune

    c = autotune.generation_class([gen_scene(1 << 20, 1 << 19)], 64)
    assert c == "generate|N=64|tri=2^20|origins=2^19"
    c = autotune.search_class([search_scene(256, 1 << 16)], 32)
    assert c == "search|N=32|needles=2^8|haystack=2^16"
