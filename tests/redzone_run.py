"""Runs the library's paths under the bounds-checked build and scans every
guard zone after each, then plants a damaged byte in chosen zones to show the
scan reports it (a host-issued memset inside the workspace, no kernel).

tests/test_gpu_check_build.py starts this in a subprocess with
HC_GB300_CHECK=1, so the package loads libhc_gb300_check.so. It prints one
JSON object on its last line."""
import json
import os
import sys
import traceback

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402
import paper_2606_06720_gb300 as P  # noqa: E402

results, errors, pokes = [], [], []


def scan(s, what):
    z = s.check_redzones()
    results.append(dict(what=what, **z))


def solver(n, L, precision, **kw):
    args = dict(c=10.0, D=0.05, gamma=0.75, dt=1e-3, precision=precision, cg_rtol=1e-8,
                cg_maxit=3000)
    args.update(kw)
    s = P.Solver(n, L, **args)
    shape = tuple(reversed(n))
    rng = np.random.default_rng(len(results))
    s.set_r(0.1 + 0.05 * rng.uniform(0, 1, shape))
    s.set_source(W.minus_mean(rng.standard_normal(shape)))
    s.set_m(rng.uniform(0, 0.5, (len(n),) + shape))
    return s


def guarded(what, fn):
    try:
        fn()
    except Exception:
        errors.append({"what": what, "error": traceback.format_exc()[-1500:]})


def paths_2d(precision, n, L):
    tag = f"{precision} {n}"
    with solver(n, L, precision, diagnostics=True) as s:
        scan(s, f"create {tag}")
        s.step(3)
        scan(s, f"graph steps {tag}")
        s.set_params(use_graph=0)
        s.step(2)
        scan(s, f"host-loop steps {tag}")
        s.set_params(use_graph=1)
        f = np.random.default_rng(5).standard_normal(s.shape)
        s.gradient()
        s.apply_operator(f)
        s.spectrum(f)
        s.split_step()
        scan(s, f"components {tag}")
        s.run(4, eps=0.0, stop_on_energy=False)
        scan(s, f"run {tag}")
        if precision != "fp32_refined_df":
            lam = np.random.default_rng(6).standard_normal((2,) + s.shape)
            # hc_adjoint scans its own workspace's zones: damage would raise HC_EBOUNDS here
            out = s.adjoint(3, lam, every=2)
            results.append({"what": f"adjoint workspace {tag}", "rc": 0 if out["rc"] in (0, -4)
                            else out["rc"], "zones": -1, "zone": -1, "owner_bytes": 0})
            scan(s, f"adjoint {tag}")


def paths_3d(precision):
    n, L = (16, 16, 16), (1.0, 1.0, 1.0)
    tag = f"{precision} {n}"
    with solver(n, L, precision, diagnostics=True) as s:
        scan(s, f"create {tag}")
        s.step(2)
        scan(s, f"graph steps {tag}")
        s.set_params(use_graph=0)
        s.step(1)
        s.set_params(use_graph=1)
        s.gradient()
        s.split_step()
        s.run(3, eps=0.0, stop_on_energy=False)
        scan(s, f"run {tag}")


def tunings():
    n, L = (256, 256), (1.0, 1.0)
    for precision in ("fp64", "fp32_refined"):
        with solver(n, L, precision) as s:
            t = s.get_tuning()
            for col, row, pipe in [((1, 1), (1, 1), (0, 0)), ((4, 2), (2, 1), (0, 0)),
                                   ((8, 4), (1, 2), (0, 0)), ((2, 1), (1, 1), (1, 1))]:
                s.set_tuning(list(col), list(row), list(pipe))
                s.step(2)
                scan(s, f"tuning {precision} {col} {row} {pipe}")
            if precision != "fp32_refined":
                continue
            for rows, rpipe in ((2, 0), (4, 0), (1, 1), (4, 1)):   # FP32 row-pass variants
                s.set_tuning(t["col_tile"], [rows, t["row_rows"][1]], t["col_pipe"], [rpipe, 0])
                s.step(2)
                scan(s, f"row tuning {precision} rows {rows} pipe {rpipe}")


def batch():
    sizes = [((128, 128), (1.0, 1.0)), ((256, 128), (1.0, 0.5)), ((64, 64), (1.0, 1.0))]
    solvers = [solver(n, L, "fp32_refined") for n, L in sizes]
    try:
        b = P.Batch(solvers)
        b.step(3)
        b.close()
        for k, s in enumerate(solvers):
            scan(s, f"batch member {k}")
    finally:
        for s in solvers:
            s.close()


def poke():
    """Damage zones last-to-first: each scan then reports the zone just hit."""
    with solver((64, 32), (1.0, 0.5), "fp32_refined") as s:
        nz = s.check_redzones()["zones"]
        for k in sorted({nz - 1, nz // 2, 0}, reverse=True):
            rc = P._binding.hc_check_poke(s.ctx, k)
            z = s.check_redzones()
            pokes.append({"poked": k, "poke_rc": rc, **z})


assert P.CHECKED and P.library_path().endswith("libhc_gb300_check.so"), P.library_path()
for precision in ("fp64", "fp32_refined", "fp32_refined_df"):
    for n, L in (((64, 32), (1.0, 0.5)), ((8, 8), (1.0, 1.0)), ((4096, 8), (1.0, 1.0)),
                 ((8, 4096), (1.0, 1.0)), ((256, 256), (1.0, 1.0))):
        guarded(f"2d {precision} {n}", lambda: paths_2d(precision, n, L))
    guarded(f"3d {precision}", lambda: paths_3d(precision))
guarded("tunings", tunings)
guarded("batch", batch)
guarded("poke", poke)
print(json.dumps({"library": os.path.basename(P.library_path()), "results": results,
                  "errors": errors, "pokes": pokes}))
