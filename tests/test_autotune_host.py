"""Host logic of the launch-shape autotuner (paper_2606_06720_gb300/autotune.py),
on the CPU with a stand-in solver. The stand-in's kernel times are a known
function of the launch shapes, so the choice the tuner must make is known.
Covered: the candidate limits; the weighted coordinate search; skipping shapes
the library rejects; the on-disk cache (hit, corrupted file, stale entry);
3D grids keeping their fixed shapes."""
import importlib.util
import json
import math
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture()
def tuner(tmp_path, monkeypatch):
    # load the module by path: importing the package would load the CUDA library
    spec = importlib.util.spec_from_file_location(
        "hc_autotune", os.path.join(ROOT, "paper_2606_06720_gb300", "autotune.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    monkeypatch.setenv("HC_TUNING_CACHE", str(tmp_path / "tuning.json"))
    monkeypatch.setattr(mod, "_key", lambda s: f"gpu|{s.n[0]}x{s.n[1]}|{s.precision}|test")
    return mod


COL = {"cg_grad", "cg_div", "split_grad", "split_heat"}
ROW = {"cg_apply", "split_row", "split_c2r"}


class Stand:
    """Times: the FP32 column kernels are fastest at col_tile 4 with the pipelined pass,
    the FP32 row kernels at row_rows 2 without it, the FP64 column kernels at col_tile 2
    with the plain pass and the FP64 row kernel at row_rows 1."""

    def __init__(self, n=(256, 128), precision="fp32_refined", dim=2, reject=None):
        self.n, self.precision, self.dim, self.device = n, precision, dim, "cpu"
        self.t = {"col_tile": [1, 1], "row_rows": [1, 1], "col_pipe": [0, 0], "row_pipe": [0, 0]}
        self.reject = reject or (lambda t: False)
        self.timings = 0

    def get_tuning(self):
        return {k: list(v) for k, v in self.t.items()}

    def set_tuning(self, col, row, cpipe=None, rpipe=None):
        t = {"col_tile": list(col), "row_rows": list(row),
             "col_pipe": list(cpipe if cpipe is not None else self.t["col_pipe"]),
             "row_pipe": list(rpipe if rpipe is not None else self.t["row_pipe"])}
        if self.reject(t):
            raise RuntimeError("rejected launch shape")
        self.t = t

    def time_kernel(self, name, reps):
        self.timings += 1
        t = self.t
        if name in COL:
            return 1 + abs(math.log2(t["col_tile"][0]) - 2) + (0 if t["col_pipe"][0] else 0.5)
        if name in ROW:
            return 1 + abs(math.log2(t["row_rows"][0]) - 1) + (0.25 if t["row_pipe"][0] else 0)
        if name in ("res_grad", "res_div"):
            return 1 + abs(math.log2(t["col_tile"][1]) - 1) + (0.5 if t["col_pipe"][1] else 0)
        return 1 + abs(math.log2(t["row_rows"][1]))


def test_candidates_respect_the_thread_limits(tuner):
    s = Stand(n=(256, 128))
    assert tuner._candidates(s, "col_tile") == [1, 2, 4, 8, 16, 32]   # v <= nx/2, v*ny/8 <= 512
    assert tuner._candidates(s, "row_rows") == [1, 2, 4, 8, 16]       # v <= ny, v*nx/8 <= 512
    s = Stand(n=(2048, 2048))
    assert tuner._candidates(s, "col_tile") == [1, 2]
    assert tuner._candidates(s, "col_tile", 0) == [1, 2, 4]            # FP32: v*ny/8 <= 1024
    assert tuner._candidates(s, "row_rows") == [1, 2]
    s = Stand(n=(4096, 8))
    assert tuner._candidates(s, "col_tile") == [1, 2, 4, 8, 16, 32]
    assert tuner._candidates(s, "row_rows") == [1]


def test_search_finds_the_fastest_shapes(tuner):
    s = Stand()
    report = {}
    best = tuner.autotune(s, reps=1, report=report)
    assert best == {"col_tile": [4, 2], "row_rows": [2, 1], "col_pipe": [1, 0], "row_pipe": [0, 0]}
    assert s.get_tuning() == best
    assert set(report["us"]) == {"col_tile[0]", "row_rows[0]", "col_tile[1]", "row_rows[1]"}
    assert report["us"]["col_tile[0]"]["4p"] == min(report["us"]["col_tile[0]"].values())


def test_rejected_shapes_are_skipped(tuner):
    s = Stand(reject=lambda t: t["col_tile"][0] == 4)
    best = tuner.autotune(s, reps=1)
    assert best["col_tile"][0] in (2, 8) and best["col_pipe"][0] == 1


def test_cache_hit_measures_nothing(tuner, tmp_path):
    first = tuner.autotune(Stand(), reps=1)
    s = Stand()
    report = {}
    assert tuner.autotune(s, reps=1, report=report) == first
    assert s.timings == 0 and report.get("cached") is True
    cache = json.loads((tmp_path / "tuning.json").read_text())
    assert cache["gpu|256x128|fp32_refined|test"] == first


def test_corrupted_cache_or_stale_entry_retunes(tuner, tmp_path):
    path = tmp_path / "tuning.json"
    path.write_text("{ not json")
    s = Stand()
    best = tuner.autotune(s, reps=1)
    assert s.timings > 0 and best["col_tile"][0] == 4
    # an entry the library now rejects is measured again and replaced
    path.write_text(json.dumps({"gpu|256x128|fp32_refined|test": {
        "col_tile": [64, 1], "row_rows": [1, 1], "col_pipe": [0, 0], "row_pipe": [0, 0]}}))
    s = Stand(reject=lambda t: t["col_tile"][0] > 32)
    assert tuner.autotune(s, reps=1)["col_tile"][0] == 4 and s.timings > 0
    assert json.loads(path.read_text())["gpu|256x128|fp32_refined|test"]["col_tile"][0] == 4


def test_fp64_searches_only_its_own_families(tuner):
    s = Stand(precision="fp64")
    best = tuner.autotune(s, reps=1, use_cache=False)
    assert best["col_tile"][0] == 1 and best["row_rows"][0] == 1   # the FP32 slots untouched


def test_3d_grids_keep_their_shapes(tuner):
    s = Stand(n=(64, 64, 64), dim=3)
    before = s.get_tuning()
    assert tuner.autotune(s, reps=1) == before and s.timings == 0
