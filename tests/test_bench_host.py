"""Host logic of bench.py on the CPU: the flop model of the reported metric, the seeded
erasure plans of the timed workloads, the BLAS-3 CPU baseline and the reference arm's line."""
import os

import numpy as np
import pytest

import bench
from oracle import oracle as O
from paper_2311_11943_gb300 import synth


@pytest.mark.parametrize("m,n,p_r,p_c,f,b,protect_r", [
    (4096, 4096, 8, 8, 2, 128, True), (16384, 16384, 16, 16, 4, 256, True),
    (1000, 480, 8, 4, 2, 100, True), (333, 96, 5, 4, 1, 40, False), (256, 256, 4, 4, 0, 32, True)])
def test_flop_model_is_the_per_panel_work(m, n, p_r, p_c, f, b, protect_r):
    # F_coded = 2 (m+c) n (n+2d) is the sum over panels k (width b_k, trailing width w_k) of
    # the panel at one pass, 2 M b_k^2, and the two trailing GEMMs, 4 M b_k w_k (Algorithm
    # PBMGS), with M and N from the oracle's geometry (m padded to a multiple of p_r)
    g = O.geom(m, n, p_r, p_c, f, protect_r)
    total, kb = 0, 0
    while kb < n:
        bk = min(b, n - kb)
        wk = g.N - kb - bk
        total += 2 * g.M * bk * bk + 4 * g.M * bk * wk
        kb += bk
    assert bench.coded_flops(m, n, p_r, p_c, f, b, protect_r) == total
    assert total == 2 * g.M * n * (n + 2 * g.d)


def _check_plan(plan, T, grid_rows, grid_cols, f):
    assert all(0 <= t < T and 0 <= i < grid_rows and 0 <= j < grid_cols for (t, i, j) in plan)
    for t in {t for (t, _, _) in plan}:
        tiles = [(i, j) for (tt, i, j) in plan if tt == t]
        assert len(set(tiles)) == len(tiles)
        assert max(np.bincount([i for i, _ in tiles])) <= f
        assert max(np.bincount([j for _, j in tiles])) <= f


@pytest.mark.parametrize("name", ["c1", "c2", "c3"])
def test_erasure_plans_are_recoverable_and_reproducible(name):
    cfg = bench.CONFIGS[name]
    T = -(-cfg["n"] // cfg["b"])
    plan = bench.erasure_plan(cfg)
    assert plan == bench.erasure_plan(cfg)
    assert len(plan) == cfg["erasure_panels"] * cfg["per_panel"]
    assert len({t for (t, _, _) in plan}) == cfg["erasure_panels"]
    _check_plan(plan, T, cfg["p_r"] + cfg["f"], cfg["p_c"] + cfg["f"], cfg["f"])


def test_every_panel_plan_of_the_overhead_sweep():
    cfg = bench.EXTRA["ovh"]
    T = -(-cfg["n"] // cfg["b"])
    for (p, f, protect_r, every) in bench.OVH_ROWS:
        if not every:
            continue
        gc = p + (f if protect_r else 0)
        plan = [(t, i, j) for t in range(T)
                for (i, j) in synth.random_erasures(p + f, gc, f, 1, cfg["seed"] + t)]
        assert len(plan) == T
        _check_plan(plan, T, p + f, gc, f)


def test_both_arms_describe_the_same_workload():
    cfg = bench.CONFIGS["c2"]
    a = bench.step_config(cfg, "3xtf32", True, 1)
    assert a == bench.step_config(dict(cfg), "3xtf32", True, 1)
    assert a["erasures"] == [list(p) for p in bench.erasure_plan(cfg)]
    assert "4096x4096" in a["workload"] and "f=2" in a["workload"]


@pytest.mark.parametrize("m,n,p_r,p_c,f,b,rb", [(256, 256, 4, 4, 1, 32, False),
                                                (256, 256, 4, 4, 1, 32, True),
                                                (203, 96, 8, 4, 2, 20, True)])
def test_blas3_baseline_computes_the_oracles_step(m, n, p_r, p_c, f, b, rb):
    # the torch CPU baseline timed beside the oracle runs the same algorithm: its R, G_0 Q_1
    # and x agree with the oracle's in FP64 to the n u kappa forward-error scale
    torch = pytest.importorskip("torch")
    kappa = 1e2
    A = synth.kappa_matrix(m, n, kappa, seed=5)
    y = synth.rhs(m, 1, 5)
    ref = O.run(A, p_r, p_c, f, b, seed=3, y=y if m == n else None, reorth_block=rb)
    Qo, R, x = bench.blas3_step(A, y, ref["Gt"], ref["Gh"], p_r, p_c, f, b, torch.float64,
                                reorth_block=rb)
    tol = n * np.finfo(np.float64).eps * kappa
    assert np.abs(R.numpy() - ref["R"]).max() < tol * np.abs(ref["R"]).max()
    assert np.abs(Qo.numpy().T - ref["Qo"]).max() < tol
    if m == n:
        assert np.abs(x.numpy() - ref["x"]).max() < tol * kappa * np.abs(ref["x"]).max()


def _bench_line(*args):
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py")] + list(args),
                         capture_output=True, text=True, timeout=600, cwd=root,
                         env=dict(os.environ, RANK="0", WORLD_SIZE="1"))
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_reference_arm_prints_the_contract_line():
    # the oracle arm (CPU): one JSON line with the GPU arm's metric, unit and config (on the
    # 4096^2 workload here: the default 16384^2 input is drawn on a GPU)
    line = _bench_line("--impl", "reference", "--config", "c2", "--steps", "1", "--warmup", "0")
    cfg = bench.CONFIGS["c2"]
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == "TFLOP/s" and line["higher_is_better"] is True
    assert line["config"] == bench.step_config(cfg, "3xtf32", True, 1)
    assert line["steps"] == 1 and line["warmup"] == 0 and line["value"] > 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "TFLOP/s",
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_of_the_other_legs_says_unavailable():
    line = _bench_line("--impl", "reference", "--config", "c4")
    assert line["impl"] == "reference" and "unavailable" in line


def test_reference_step_sample_is_panel_zero_of_the_workload():
    # the bounded step of the reference arm on the largest workload: encode + panel 0 with its
    # trailing update over the next `cols` columns; its R block equals the full problem's
    # panel-0 R entries over those columns (the update of a column does not depend on the
    # columns to its right)
    cfg = dict(m=96, n=96, p_r=4, p_c=4, f=1, b=16, seed=2)
    A = synth.gaussian(96, 96, 9)
    v, cores, sample, dt = bench.oracle_panel_sample(cfg, A, 40)
    assert v > 0 and cores >= 1 and "next 40 columns" in sample
    g = O.geom(96, 96, 4, 4, 1)
    Gt, Gh = O.generator(1, 4, 4, 2)
    Q = O.encode(g, Gt, Gh, A)
    R = np.zeros((g.N, g.N), order="F")
    O.factor(Q, R, 96, 16, 0, 1)
    Qs = O.encode(g, Gt, Gh, A)[:, :56]
    Rs = np.zeros((56, 56), order="F")
    O.factor(Qs, Rs, 56, 16, 0, 1)
    assert np.allclose(Rs[:16, :56], R[:16, :56], rtol=0, atol=1e-13)
    assert np.allclose(Qs, Q[:, :56], rtol=0, atol=1e-13)


def test_default_workload_is_the_largest_configuration():
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--help"],
                         capture_output=True, text=True, timeout=120, cwd=root)
    assert out.returncode == 0
    cfg = bench.CONFIGS["c3"]
    assert (cfg["m"], cfg["n"], cfg["p_r"], cfg["f"], cfg["b"]) == (16384, 16384, 16, 4, 256)
    assert cfg["device_input"] and cfg["erasure_panels"] * cfg["per_panel"] == 4
    src = open(os.path.join(root, "bench.py")).read()
    assert 'ap.add_argument("--config", default="c3"' in src
