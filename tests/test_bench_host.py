"""Host logic of the benchmark: the labels that tell the passes of one solve
apart (each label carries its own algorithmic bytes per point in the roofline
arithmetic) and the reference arm's JSON line, which runs the CPU oracle only
and so needs no GPU."""
import importlib.util
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _solve(first_in, sweep_ins, outs):
    """Launch names of one refinement solve: three FP32 solves (x, y, z, y,
    x) with the residual stages between them."""
    names = []
    for s, (xin, xout) in enumerate(zip([first_in] + sweep_ins, outs)):
        if s > 0:
            names.append(xin)
        names += ["x_fwd", "y_fwd", "z_solve", "y_inv", xout]
    return [(n, 1.0) for n in names]


def test_fast_solve_passes_get_their_own_labels():
    B = _bench()
    prof = _solve(None, ["residual", "residual_update"], ["x_inv", "x_inv_acc", "x_inv_acc"])
    keys = B.kernel_keys(prof)
    assert keys == ["x_fwd", "y_fwd", "z_solve", "y_inv", "x_inv",
                    "residual", "x_fwd_sweep", "y_fwd", "z_solve", "y_inv", "x_inv_acc_d",
                    "residual_update", "x_fwd_sweep", "y_fwd", "z_solve", "y_inv", "x_inv_acc"]
    # FP64 f in (12 B), FP32 residual in (8 B), the pair update that also
    # stores the correction (24 B), the final FP64 write (20 B)
    assert [B.KERNEL_BYTES_PER_POINT[k] for k in ("x_fwd", "x_fwd_sweep", "x_inv_acc_d", "x_inv_acc")] == \
        [12.0, 8.0, 24.0, 20.0]


def test_fused_update_keeps_the_correction_storing_pair_update():
    B = _bench()
    prof = [("x_inv_acc", 1.0), ("x_fwd_ru", 1.0), ("y_fwd", 1.0)]
    assert B.kernel_keys(prof) == ["x_inv_acc_d", "x_fwd_ru", "y_fwd"]
    assert B.KERNEL_BYTES_PER_POINT["x_fwd_ru"] == 12.0


def test_exact_mode_passes_are_labelled():
    B = _bench()
    prof = _solve(None, ["residual", "residual"], ["x_inv", "x_inv_acc", "x_inv_acc"])
    keys = B.kernel_keys(prof)
    assert keys.count("x_fwd_sweep") == 2 and "x_inv_acc_d" not in keys
    assert all(k in B.KERNEL_BYTES_PER_POINT for k in keys)


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "Gpoints/s"
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "duct_poisson_1536x512x512"
