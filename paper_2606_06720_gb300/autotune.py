"""Launch-shape autotuner of the FFT passes.

For a Solver it measures, with ``hc_time_kernel`` on the solver's own data,
every admissible column-tile width and rows-per-CTA count of the FP32 and
FP64 kernel families and keeps the fastest.  Results are cached on disk per
(GPU name, grid, precision) so later processes reuse them; the cache lives in
``$HC_TUNING_CACHE`` or ``~/.cache/hucai_gb300/tuning.json``.
"""
from __future__ import annotations

import json
import os

# kernels that share each launch-shape knob, per precision mode
_FAMILIES = {
    "fp32_refined": {
        ("col_tile", 0): ["cg_grad", "cg_div", "split_grad", "split_heat"],
        ("row_rows", 0): ["cg_apply", "split_row", "split_c2r"],
        ("col_tile", 1): ["res_grad", "res_div"],
        ("row_rows", 1): ["res_apply"],
    },
    "fp64": {
        ("col_tile", 1): ["cg_grad", "cg_div", "split_grad", "split_heat", "res_grad"],
        ("row_rows", 1): ["cg_apply", "split_row", "split_c2r", "res_apply"],
    },
}


def _cache_path() -> str:
    return os.environ.get("HC_TUNING_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "hucai_gb300", "tuning.json"))


# Launches per step of each kernel relative to the once-per-step ones: the CG
# kernels run every iteration (about 20 per step on the large grids), so a
# shared knob is chosen by the weighted sum of the kernels' times.
_WEIGHT = {"cg_grad": 20, "cg_apply": 20, "cg_div": 20}

# Bumped whenever the kernels' launch-shape trade-offs change, so cached
# choices made for older kernels are not reused.
_KERNELS_VERSION = 7


def _key(solver) -> str:
    import torch
    name = torch.cuda.get_device_name(solver.device)
    return f"{name}|{solver.n[0]}x{solver.n[1]}|{solver.precision}|k{_KERNELS_VERSION}"


def _candidates(solver, knob: str, idx: int = 1):
    """Admissible values of a launch-shape knob: FP32 column passes ([0]) take
    CTAs of up to 1024 threads, the FP64 ones and the row passes up to 512."""
    nx, ny = solver.n
    out = []
    v = 1
    while v <= 32:
        if knob == "col_tile":
            ok = v <= nx // 2 and v * (ny // 8) <= (1024 if idx == 0 else 512)
        else:
            ok = v <= ny and v * (nx // 8) <= 512
        if ok:
            out.append(v)
        v *= 2
    return out


def autotune(solver, reps: int = 20, use_cache: bool = True, verbose: bool = False,
             report: dict | None = None) -> dict:
    """Pick the fastest launch shapes for this solver and apply them; returns
    the tuning.  If `report` is a dict it receives the cache key and the
    measured microseconds per candidate, weighted by launches per step
    (empty when the cache answered).
    3D grids have fixed launch shapes: their tuning is returned unchanged."""
    if getattr(solver, "dim", 2) != 2:
        return solver.get_tuning()
    path = _cache_path()
    key = _key(solver)
    if report is not None:
        report["key"] = key
        report["us"] = {}
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except Exception:
            cache = {}
    if use_cache and key in cache:
        t = cache[key]
        try:
            solver.set_tuning(t["col_tile"], t["row_rows"], t.get("col_pipe", [0, 0]),
                              t.get("row_pipe", [0, 0]))
            if report is not None:
                report["cached"] = True
            return solver.get_tuning()
        except Exception:
            pass
    prec = "fp64" if solver.precision.startswith("fp64") else "fp32_refined"
    best = solver.get_tuning()
    measured = {}
    for (knob, idx), kernels in _FAMILIES[prec].items():
        times = {}
        for v in _candidates(solver, knob, idx):
            # the knob's pipelined variants: col_pipe 0/1 for the column
            # passes, row_pipe 0/1 for the FP32 apply row pass
            if knob == "col_tile":
                pipes, pkey = (0, 1), "col_pipe"
            else:
                pipes, pkey = ((0, 1) if idx == 0 else (None,)), "row_pipe"
            for pipe in pipes:
                trial = {k: list(best[k]) for k in ("col_tile", "row_rows", "col_pipe", "row_pipe")}
                trial[knob][idx] = v
                if pipe is not None:
                    trial[pkey][idx] = pipe
                try:
                    solver.set_tuning(trial["col_tile"], trial["row_rows"], trial["col_pipe"],
                                      trial["row_pipe"])
                except Exception:
                    continue
                label = f"{v}" if pipe is None else f"{v}{['', 'p', 'q'][pipe]}"
                times[label] = (sum(_WEIGHT.get(k, 1) * solver.time_kernel(k, reps)
                                    for k in kernels), v, pipe, pkey)
        if times:
            lab = min(times, key=lambda k: times[k][0])
            _, v, pipe, pkey = times[lab]
            best[knob][idx] = v
            if pipe is not None:
                best[pkey][idx] = pipe
            measured[f"{knob}[{idx}]"] = {k: round(t[0] * 1e3, 2) for k, t in times.items()}
    solver.set_tuning(best["col_tile"], best["row_rows"], best["col_pipe"], best["row_pipe"])
    if report is not None:
        report["us"] = measured
    if verbose:
        print(json.dumps({"autotune": key, "us": measured, "best": best}))
    if use_cache:
        cache[key] = best
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            tmp = path + f".{os.getpid()}.tmp"
            with open(tmp, "w") as f:
                json.dump(cache, f, indent=1)
            os.replace(tmp, path)
        except OSError:
            pass
    return best
