#!/usr/bin/env python
"""Benchmark: coded block Gram-Schmidt QR (arXiv 2311.11943) on GB300.

One step = the whole hot path on one synthetic problem: generator + checksum encode, PBMGS
with ICGS panels on the encoded matrix (erasures injected at the start of seeded panels and
recovered before they run), post-orthogonalisation and the solve.  Reported: coded GS-QR
TFLOP/s (F_coded = 2 (m+c) n (n+2d) per step), the coding overhead against the uncoded GPU
QR of the same matrix, and the errors ||A - Q_1 R|| / ||A||, ||I - Qo^T Qo||.  The default
workload is the largest single-GPU configuration: 16384^2, kappa 1e4, grid 16 x 16, f = 4,
b = 256, four simultaneous erasures, FP32 storage with 3xTF32 tensor-core products; beside
it the line carries the same workload in the other precisions and the 4096^2 workload in
FP64 on the GPU against the mixed-precision step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config c3] [--mode 3xtf32|tf32|f32|f64]
  python bench.py --impl reference ...     (the FP64 CPU oracle on the host cores)
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

CONFIGS = {
    # 4096 x 4096 = U diag(sigma) V^T, kappa 1e2; grid 8 x 8, f = 2, b = 128; two nodes erased at
    # two seeded panels
    "c2": dict(m=4096, n=4096, p_r=8, p_c=8, f=2, b=128, kappa=1e2, seed=2, erasure_panels=2,
               per_panel=1),
    "c2k6": dict(m=4096, n=4096, p_r=8, p_c=8, f=2, b=128, kappa=1e6, seed=2, erasure_panels=2,
                 per_panel=1),
    # 16384 x 16384, kappa 1e4; grid 16 x 16, f = 4, b = 256; four simultaneous erasures (the
    # input drawn on the device: the host construction takes minutes at this size); the
    # reference arm's step is the oracle's encode + panel 0 over the next ref_cols columns
    "c3": dict(m=16384, n=16384, p_r=16, p_c=16, f=4, b=256, kappa=1e4, seed=3, erasure_panels=1,
               per_panel=4, device_input=True, ref_cols=2048),
    "c1": dict(m=256, n=256, p_r=4, p_c=4, f=1, b=32, kappa=0, seed=1, erasure_panels=1,
               per_panel=1),
}
# Configurations with their own bench legs (not the single-problem step above):
#   ovh: coding overhead at n = 16384 (b = 256, N(0,1)) over the grid, the checksum count and
#        the vertical-only code, and the cost of one erasure recovered at every panel
#   c4: 512 independent coded QRs, m ~ U[256, 8192], n ~ U[32, 256] (multiples of p_c, m >= 4 n),
#       N(0,1), grid 8 x 4, f = 2 per instance, up to two erased tiles per instance at one
#       seeded panel; one persistent factor launch per phase, recorded into a CUDA graph
#   c5: differentiable least squares, 16 x A 8192 x 1024 with kappa 1e3, y ~ N(0,1); grid 8 x 8,
#       f = 1, b = 128, one node erased at the middle panel; forward + hand-written adjoint
EXTRA = {
    "c4": dict(count=512, p_r=8, p_c=4, f=2, seed=4),
    "c5": dict(batch=16, m=8192, n=1024, p_r=8, p_c=8, f=1, b=128, kappa=1e3, seed=5),
    "e1": dict(),
    "f3": dict(),
    "ovh": dict(m=16384, n=16384, b=256, seed=3),
}
MODES = {"f64": ("f64", "simt"), "f32": ("f32", "simt"), "tf32": ("f32", "tf32"),
         "3xtf32": ("f32", "3xtf32"), "bf16": ("f32", "bf16"), "bf16x3": ("f32", "bf16x3")}
L2_BYTES = 126 * 1024 * 1024
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of a dominant kernel from
# one ncu capture of the current kernel, keyed by (config, mode, profile class):
# profiles/k_panel_c3.md for the 20480 x 256 panel of the 16384^2 workload (captured on a
# 16384 x 8192 problem with the same panel shape and grid).  Absent (the 4096^2 register panel
# has changed since its capture): reported as null.
NCU_TRAFFIC = {("c3", "3xtf32", "panel_icgs"): 21.079552e6 + 0.007680e6}


def coded_flops(m, n, p_r, p_c, f, b, protect_r=True):
    mb = -(-m // p_r)
    c = f * mb
    d = f * (n // p_c) if protect_r and f > 0 else 0
    return 2.0 * (mb * p_r + c) * n * (n + 2 * d)


def workload_name(cfg, mode, reorth_block=True):
    k = ("kappa=%g" % cfg["kappa"]) if cfg["kappa"] else "N(0,1)"
    return ("coded PBMGS/ICGS %dx%d %s, grid %dx%d, f=%d, b=%d, %d erasure(s) at %d seeded "
            "panel(s), %s%s" % (cfg["m"], cfg["n"], k, cfg["p_r"], cfg["p_c"], cfg["f"], cfg["b"],
                                cfg["erasure_panels"] * cfg["per_panel"], cfg["erasure_panels"],
                                mode, ", block reorthogonalisation" if reorth_block else ""))


METRIC = ("coded GS-QR TFLOP/s (F_coded = 2(m+c)n(n+2d) per step) + coding overhead vs uncoded, "
          "at the stated QR/orthogonality error")


def step_config(cfg, mode, rb, world):
    """The `config` object of both arms' lines for a single-problem workload."""
    return {"workload": workload_name(cfg, mode, rb), "m": cfg["m"], "n": cfg["n"],
            "p_r": cfg["p_r"], "p_c": cfg["p_c"], "f": cfg["f"], "b": cfg["b"],
            "kappa": cfg["kappa"], "erasures": [list(p) for p in erasure_plan(cfg)],
            "reorth_block": rb,
            "l2": "L2 flushed between timed steps (256 MB write outside the events)",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def make_inputs(cfg, torch=None, device=None):
    """Seeded synthetic A (m x n, FP64) and y (m x 1)."""
    from paper_2311_11943_gb300 import synth
    m, n = cfg["m"], cfg["n"]
    if not cfg["kappa"]:
        A = synth.gaussian(m, n, cfg["seed"])
    else:
        A = synth.kappa_matrix(m, n, cfg["kappa"], cfg["seed"])
    y = synth.rhs(m, 1, cfg["seed"])
    return A, y


def erasure_plan(cfg):
    from paper_2311_11943_gb300 import synth
    T = -(-cfg["n"] // cfg["b"])
    panels = synth.random_panels(T, cfg["erasure_panels"], cfg["seed"])
    gr = cfg["p_r"] + cfg["f"]
    gc = cfg["p_c"] + cfg["f"]
    plan = []
    for t in panels:
        for (i, j) in synth.random_erasures(gr, gc, cfg["f"], cfg["per_panel"], cfg["seed"] + t):
            plan.append((t, i, j))
    return plan


def coded_factor(q, Ad, plan):
    """The factorisation part of one step: encode, then factor(t, t1) over the segments between
    erasure panels, with the panel's erasures injected and recovered before it runs."""
    q.encode(Ad)
    T = q.geo["panels"]
    t = 0
    while t < T:
        tiles = [(i, j) for (tt, i, j) in plan if tt == t]
        if tiles:
            q.inject(tiles)
            q.recover()
        t1 = t + 1
        while t1 < T and not any(tt == t1 for (tt, _, _) in plan):
            t1 += 1
        q.factor(t, t1)
        t = t1


def coded_step(q, Ad, yd, xd, plan):
    """One timed step: the asynchronous verbs of the C ABI in the order of coded_qr_run
    (factorisation, post-orthogonalisation of Q_1 inside the handle, the solve)."""
    coded_factor(q, Ad, plan)
    q.post_orth()
    q.solve(yd, xd)


class ClockSampler:
    """nvidia-smi SM clocks and throttle reasons sampled while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons, pw = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                pw.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [s for s, p in zip(sm, pw) if p > 200.0] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ------------------------------------------------------------------------ CPU oracle legs
def blas3_step(A, y, Gt, Gh, p_r, p_c, f, b, dtype, reorth_block=True, tau=1.0 / np.sqrt(2.0)):
    """A BLAS-3 CPU baseline of the same step in torch on the host cores (context beside the
    plain oracle, not a fallback: nothing in the library calls it).  Encode (Section 4.2), PBMGS
    with the right-looking ICGS panel, the optional block reorthogonalisation pass, the
    trailing GEMMs (Algorithm PBMGS), post-orthogonalisation G_0 Q_1 and the square solve
    (Section 4.1), without erasures.  Q~ is held transposed (row j = column j) so that every
    column operation is contiguous.  Gt (f x p_r) and Gh (p_c x f) are the generator.
    Returns (Qt, R, x) with Qt the post-orthogonalised factor, N x M."""
    import torch
    m, n = A.shape
    mb = -(-m // p_r)
    m_pad, nb = mb * p_r, n // p_c
    c, d = f * mb, f * nb
    M, N = m_pad + c, n + d
    Gt_t = torch.as_tensor(np.asarray(Gt), dtype=dtype)
    Gh_t = torch.as_tensor(np.asarray(Gh), dtype=dtype)
    Qt = torch.zeros(N, M, dtype=dtype)
    Qt[:n, :m] = torch.as_tensor(np.ascontiguousarray(A.T), dtype=dtype)
    if f > 0:
        Qt[:n, m_pad:] = torch.einsum("nts,it->nis", Qt[:n, :m_pad].view(n, p_r, mb),
                                      Gt_t).reshape(n, c)
        Qt[n:] = torch.einsum("jsm,jl->lsm", Qt[:n].view(p_c, nb, M), Gh_t).reshape(d, M)
    R = torch.zeros(N, N, dtype=dtype)
    for kb in range(0, n, b):
        bk = min(b, n - kb)
        P = Qt[kb:kb + bk]
        if reorth_block and kb > 0:
            S = Qt[:kb] @ P.T
            P -= S.T @ Qt[:kb]
            R[:kb, kb:kb + bk] += S
        eta = (P * P).sum(1)
        for j in range(bk):
            q = P[j]
            v = P[j:] @ q
            if j > 0 and v[0] < tau * tau * eta[j]:
                sv = P[:j] @ q
                q -= sv @ P[:j]
                R[kb:kb + j, kb + j] += sv
                v = P[j:] @ q
            rjj = torch.sqrt(v[0])
            if not rjj > 0:
                raise RuntimeError("breakdown at column %d" % (kb + j))
            R[kb + j, kb + j] = rjj
            q /= rjj
            r = v[1:] / rjj
            R[kb + j, kb + j + 1:kb + bk] = r
            P[j + 1:].addr_(r, q, alpha=-1.0)
        if kb + bk < N:
            Rbar = P @ Qt[kb + bk:].T
            R[kb:kb + bk, kb + bk:] = Rbar
            Qt[kb + bk:] -= Rbar.T @ P
    # G_0 = [[I + G~_1, V], [V^T, -I]] on tile rows (Theorem G_0), applied to Q_1 and [y; 0]
    G0 = -torch.eye(p_r, dtype=dtype)
    if f > 0:
        G0[:f, :f] = torch.eye(f, dtype=dtype) + Gt_t[:, :f]
        G0[:f, f:] = Gt_t[:, f:]
        G0[f:, :f] = Gt_t[:, f:].T
    Qo = torch.einsum("nts,it->nis", Qt[:n, :m_pad].view(n, p_r, mb), G0).reshape(n, m_pad)
    yp = torch.zeros(m_pad, dtype=dtype)
    yp[:m] = torch.as_tensor(np.asarray(y).reshape(-1), dtype=dtype)
    yo = torch.einsum("ts,it->is", yp.view(p_r, mb), G0).reshape(m_pad)
    x = torch.linalg.solve_triangular(R[:n, :n], (Qo @ yo).reshape(n, 1), upper=True)
    return Qo, R, x


def blas3_baseline(cfg, A, y, rb):
    """Times blas3_step on the whole workload in FP64 and FP32 on all host cores."""
    import torch
    from oracle import oracle as O
    threads = os.cpu_count() or 1
    torch.set_num_threads(threads)
    Gt, Gh = O.generator(cfg["f"], cfg["p_r"], cfg["p_c"], cfg["seed"])
    F = coded_flops(cfg["m"], cfg["n"], cfg["p_r"], cfg["p_c"], cfg["f"], cfg["b"])
    out = []
    for name, dt in (("f64", torch.float64), ("f32", torch.float32)):
        t0 = time.perf_counter()
        blas3_step(A, y, Gt, Gh, cfg["p_r"], cfg["p_c"], cfg["f"], cfg["b"], dt, reorth_block=rb)
        sec = time.perf_counter() - t0
        out.append({"dtype": name, "value": F / sec / 1e12, "unit": "TFLOP/s",
                    "ms_per_step": sec * 1e3, "cores": threads,
                    "kind": "torch CPU BLAS-3, same algorithm",
                    "sample": "the whole step (encode, factor%s, post-orth, solve), no erasure"
                    % (" with block reorthogonalisation" if rb else "")})
    return out


def oracle_sample(cfg, A, budget_s, max_panels=None):
    """Time the FP64 oracle on a bounded sample of the workload: encode plus as many PBMGS
    panels (full trailing updates) as fit in budget_s.  Returns (TFLOP/s, cores, sample)."""
    from oracle import oracle as O
    m, n, p_r, p_c, f, b = (cfg[k] for k in ("m", "n", "p_r", "p_c", "f", "b"))
    g = O.geom(m, n, p_r, p_c, f)
    Gt, Gh = O.generator(f, p_r, p_c, cfg["seed"])
    t0 = time.perf_counter()
    Q = O.encode(g, Gt, Gh, A)
    R = np.zeros((g.N, g.N), order="F")
    flops = 0.0
    panels = 0
    T = -(-n // b)
    while panels < T and (time.perf_counter() - t0) < budget_s:
        if max_panels is not None and panels >= max_panels:
            break
        kb = panels * b
        bk = min(b, n - kb)
        w = g.N - kb - bk
        O.factor(Q, R, n, b, panels, panels + 1)
        flops += 4.0 * g.M * bk * w + 4.0 * g.M * bk * bk
        panels += 1
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = ("FP64 oracle: encode + panels 0..%d of %d (%.1f GFLOP of trailing update and panel "
              "work) of the %dx%d coded problem, %.1f s" % (panels - 1, T, flops / 1e9, m, n, dt))
    return flops / dt / 1e12, cores, sample, dt


def oracle_panel_sample(cfg, A, cols):
    """One bounded step of the FP64 oracle: encode of the whole matrix, then panel 0 (ICGS)
    with its trailing update restricted to the first `cols` columns right of it (the coded
    matrix's leading b + cols columns, factored as a problem of their own).  Returns
    (TFLOP/s, cores, sample, seconds)."""
    from oracle import oracle as O
    m, n, p_r, p_c, f, b = (cfg[k] for k in ("m", "n", "p_r", "p_c", "f", "b"))
    g = O.geom(m, n, p_r, p_c, f)
    Gt, Gh = O.generator(f, p_r, p_c, cfg["seed"])
    t0 = time.perf_counter()
    Q = O.encode(g, Gt, Gh, A)
    k = min(b + cols, g.N)
    Qs = Q[:, :k]                       # leading columns of a Fortran array: contiguous
    Rs = np.zeros((k, k), order="F")
    O.factor(Qs, Rs, k, b, 0, 1)
    dt = time.perf_counter() - t0
    flops = 4.0 * g.M * b * (k - b) + 4.0 * g.M * b * b
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = ("FP64 oracle: encode of the %dx%d coded problem + panel 0 with its trailing update "
              "over the next %d columns (%.1f GFLOP), %.1f s" % (m, n, k - b, flops / 1e9, dt))
    return flops / dt / 1e12, cores, sample, dt


def host_inputs(cfg, seed):
    """(A FP64 Fortran-ordered, y) on the host for workloads without a device generator."""
    return make_inputs(dict(cfg, seed=seed))


def device_inputs(cfg, seed, torch):
    """A (FP32, column-major, on the current device) from the seeded device generator, and its
    FP64 host copy (the bytes the oracle and the host-buffer path see)."""
    from paper_2311_11943_gb300 import synth
    A32 = synth.kappa_matrix_torch(cfg["m"], cfg["n"], cfg["kappa"], seed)
    A_np = A32.double().cpu().numpy()
    assert A_np.flags.f_contiguous
    return A32, A_np


def run_reference(args, cfg):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
    if cfg.get("device_input"):
        # input generation only (not timed): the seeded device generator of the GPU arm, on the
        # GPU when there is one; the oracle itself runs on the host cores
        import torch
        if torch.cuda.is_available():
            A32, A = device_inputs(cfg, cfg["seed"], torch)
            del A32
            torch.cuda.empty_cache()
        else:
            from paper_2311_11943_gb300 import synth
            A = synth.kappa_matrix_torch(cfg["m"], cfg["n"], cfg["kappa"], cfg["seed"],
                                         device="cpu").double().numpy()
    else:
        A, _ = make_inputs(cfg)
    vals = []
    sample = ""
    cores = 1
    for it in range(args.warmup + args.steps):
        if cfg.get("ref_cols"):
            v, cores, sample, dt = oracle_panel_sample(cfg, A, cfg["ref_cols"])
        else:
            v, cores, sample, dt = oracle_sample(cfg, A, budget_s=1e9, max_panels=1)
        if it >= args.warmup:
            vals.append((v, dt))
    value = statistics.mean(v for v, _ in vals)
    ms = statistics.mean(dt for _, dt in vals) * 1e3
    # the same metric and config as the GPU arm's line; each step times a bounded sample of
    # the workload, described in cpu_baseline.sample
    line = {"metric": METRIC, "value": value,
            "unit": "TFLOP/s", "impl": "reference", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": step_config(cfg, args.mode, not args.no_reorth_block,
                                  int(os.environ.get("WORLD_SIZE", "1"))),
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                             "sample": sample + "; each step of this arm is that sample"},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------------ GPU leg
def measure_peaks_here(torch):
    """TF32 and FP64 dense matmul rates of this GPU, measured in the run by the same torch
    method as the measured BF16 peaks file: torch.matmul, best of 10 (burst) and back to back
    for about two seconds (sustained, TF32 only), CUDA events."""
    out = {}
    prev = torch.backends.cuda.matmul.allow_tf32
    try:
        for name, dt, n, tf32 in (("tf32", torch.float32, 8192, True),
                                  ("fp64", torch.float64, 4096, False)):
            torch.backends.cuda.matmul.allow_tf32 = tf32
            a = torch.randn(n, n, device="cuda", dtype=dt)
            b = torch.randn(n, n, device="cuda", dtype=dt)
            c = torch.empty(n, n, device="cuda", dtype=dt)
            for _ in range(3):
                torch.matmul(a, b, out=c)
            best = float("inf")
            for _ in range(10):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b, out=c)
                e1.record()
                e1.synchronize()
                best = min(best, e0.elapsed_time(e1))
            out[name + "_tflops"] = 2.0 * n ** 3 / (best * 1e-3) / 1e12
            if tf32:
                reps = max(1, int(2000.0 / best))
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    torch.matmul(a, b, out=c)
                e1.record()
                e1.synchronize()
                out[name + "_tflops_sustained"] = 2.0 * n ** 3 * reps / (e0.elapsed_time(e1) * 1e-3) / 1e12
            del a, b, c
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    out["how"] = ("torch.matmul 8192^3 TF32 (allow_tf32) and 4096^3 FP64: best of 10 (burst); TF32 "
                  "also back to back for ~2 s (sustained); CUDA events; this run")
    return out


def sampled_errors(A64, Qt, Rt, Qo, m, n, cols=1024, seed=0):
    """Backward error and orthogonality estimated on a seeded sample of `cols` columns (for the
    legs beside the headline, where the full FP64 Gram matrices would take seconds each):
    |A[:,S] - Q_1 R_1[:,S]|_F / |A[:,S]|_F, max |I - Q[:,S]^T Q[:,S]| for the coded Q and the
    post-orthogonalised Q."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    S = torch.randperm(n, generator=g)[:min(cols, n)].sort().values.to(A64.device)
    As = A64[:, S]
    back = (torch.linalg.norm(As - Qt[:m, :n].double() @ Rt[:n, :n].double()[:, S]) /
            torch.linalg.norm(As)).item()
    eye = torch.eye(S.numel(), device=A64.device, dtype=torch.float64)
    Qs = Qt[:, S].double()
    oc = (Qs.T @ Qs - eye).abs().max().item()
    Qos = Qo[:, S].double()
    oo = (Qos.T @ Qos - eye).abs().max().item()
    return {"backward_rel_fro": back, "orth_max_coded_Q": oc, "orth_max_post_orth": oo,
            "how": "sampled: %d seeded columns" % S.numel()}


def run_ours(args, cfg):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2311_11943_gb300 import binding as B
    from paper_2311_11943_gb300 import replicas

    dtype, mma = MODES[args.mode]
    td = torch.float64 if dtype == "f64" else torch.float32
    es = 8 if dtype == "f64" else 4
    m, n, p_r, p_c, f, b = (cfg[k] for k in ("m", "n", "p_r", "p_c", "f", "b"))
    # every rank factorises its own draw of the recipe (replicas of one coded QR)
    seed_r = replicas.rank_seed(cfg["seed"], rank)
    if cfg.get("device_input"):
        A_dev, A_np = device_inputs(cfg, seed_r, torch)
        Ad = B.colmajor_empty(m, n, td)
        Ad.copy_(A_dev)
        del A_dev
    else:
        A_np, _ = host_inputs(cfg, seed_r)
        Ad = B.colmajor_empty(m, n, td)
        Ad.copy_(torch.from_numpy(np.ascontiguousarray(A_np)))
    from paper_2311_11943_gb300 import synth
    y_np = synth.rhs(m, 1, seed_r)
    yd = B.colmajor_empty(m, 1, td)
    yd.copy_(torch.from_numpy(np.ascontiguousarray(y_np)))
    xd = B.colmajor_empty(n, 1, td)
    plan = erasure_plan(cfg)
    stream = torch.cuda.current_stream()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    def timed(q, with_plan, steps, warmup, profile=False, sync_ranks=True):
        pl = plan if with_plan else []
        for _ in range(warmup):
            coded_step(q, Ad, yd, xd, pl)
        torch.cuda.synchronize()
        if profile:
            q.profile(True)
            q.profile_read(reset=True)
        times = []
        if world > 1 and sync_ranks:
            dist.barrier()
        torch.cuda.synchronize()
        for _ in range(steps):
            flush.fill_(1.0)  # L2 flush between timed steps (outside the events)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            coded_step(q, Ad, yd, xd, pl)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        prof = q.profile_read(reset=True) if profile else None
        if profile:
            q.profile(False)
        st = q.sync_status()
        if st != 0:
            raise RuntimeError("device status %d (%s)" % (st, B.errstr(st)))
        return times, prof

    def factor_untimed(q):
        """One more (untimed) factorisation with the plan, one panel per call; returns the
        coded factors before post-orthogonalisation."""
        q.encode(Ad)
        T = q.geo["panels"]
        for t in range(T):
            tiles = [(i, j) for (tt, i, j) in plan if tt == t]
            if tiles:
                q.inject(tiles)
                q.recover()
            q.factor(t, t + 1)
        return q.factors()

    rb = not args.no_reorth_block
    q = B.CodedQR(m, n, p_r, p_c, f, b, dtype=dtype, mma=mma, seed=cfg["seed"], stream=stream,
                  reorth_block=rb)
    clocks = ClockSampler(local)
    clocks.start()
    t_coded, _ = timed(q, True, args.steps, args.warmup)
    clk = clocks.stop()
    # the per-kernel breakdown (and the roofline's launch durations) from the same number of
    # steps run again with the library's event-pair profile on; the headline steps above run
    # without those events
    t_prof, prof = timed(q, True, args.steps, 0, profile=True)
    stats = q.stats()

    # uncoded GPU QR of the same matrix (f = 0, no checksums, no erasures)
    q0 = B.CodedQR(m, n, p_r, p_c, 0, b, dtype=dtype, mma=mma, seed=cfg["seed"], stream=stream,
                   reorth_block=rb)
    t_unc, _ = timed(q0, False, args.steps, max(1, args.warmup))
    q0.close()

    # errors of one more (untimed) run, in FP64 over the whole factors
    Qc, Rc = factor_untimed(q)
    A64 = torch.from_numpy(A_np).to(dev)
    M = q.geo["M"]
    Q1 = Qc[:m, :n].double()
    R1 = Rc[:n, :n].double()
    berr = (torch.linalg.norm(A64 - Q1 @ R1) / torch.linalg.norm(A64)).item()
    del Q1, R1
    Qt64 = Qc[:M, :n].double()
    orth_coded = (Qt64.T @ Qt64 - torch.eye(n, device=dev, dtype=torch.float64)).abs().max().item()
    Gt_np, _ = q.generator()
    Gv = torch.kron(torch.from_numpy(Gt_np), torch.eye(q.geo["mb"], dtype=torch.float64)).to(dev)
    drift = (Qt64[q.geo["m_pad"]:M] - Gv @ Qt64[:q.geo["m_pad"]]).abs().max().item()
    del Qt64, Gv
    Qo = B.colmajor_empty(q.geo["m_pad"], n, td)
    q.post_orth(Qo)
    Qo64 = Qo.double()
    orth = (Qo64.T @ Qo64 - torch.eye(n, device=dev, dtype=torch.float64)).abs().max().item()
    del Qo64, Qo
    q.solve(yd, xd)
    x64 = xd.double()
    y64 = torch.from_numpy(y_np).to(dev)
    resid = (torch.linalg.norm(A64 @ x64 - y64) / torch.linalg.norm(y64)).item()
    del A64
    torch.cuda.empty_cache()

    # end to end through the public one-call API with host buffers (pinned)
    A_pin = torch.empty((n, m), dtype=td, pin_memory=True)
    A_pin.copy_(torch.from_numpy(np.ascontiguousarray(A_np.T)))
    A_host = A_pin.numpy().T
    y_pin = torch.empty((1, m), dtype=td, pin_memory=True)
    y_pin.copy_(torch.from_numpy(np.ascontiguousarray(y_np.T)))
    y_host = y_pin.numpy().T
    x_pin = torch.empty((1, n), dtype=td, pin_memory=True)
    x_host = x_pin.numpy().T
    for _ in range(max(1, args.warmup)):
        q.run(A_host, y_host, x_host, plan=plan, host=True)
    e2e_times = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        q.run(A_host, y_host, x_host, plan=plan, host=True)
        e2e_times.append((time.perf_counter() - t0) * 1e3)
    geo = dict(q.geo)
    q.close()
    del A_pin

    F = coded_flops(m, n, p_r, p_c, f, b)
    ms = statistics.mean(t_coded)
    ms_unc = statistics.mean(t_unc)
    ms_e2e = statistics.mean(e2e_times)
    ms, ms_unc, ms_e2e = replicas.max_over_ranks([ms, ms_unc, ms_e2e], dist if world > 1 else None,
                                                 device=dev)
    value = replicas.job_throughput(F, world, ms)
    e2e_value = replicas.job_throughput(F, world, ms_e2e)
    launches = int(sum(v[1] for v in prof.values()) / args.steps)

    peaks_here = None
    legs = None
    cpu = None
    blas3 = None
    if rank == 0:
        peaks_here = measure_peaks_here(torch)
        if not args.no_legs:
            legs = extra_legs(args, cfg, torch, B, Ad, A_np, yd, xd, flush, stream)
    rl = roofline(args, cfg, prof, geo, dtype, mma, es, peaks_here)

    if rank == 0 and not args.no_cpu_baseline:
        os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
        v, cores, sample, _ = oracle_sample(cfg, A_np, budget_s=args.cpu_budget)
        cpu = {"value": v, "unit": "TFLOP/s", "cores": cores, "kind": "oracle", "sample": sample}
        if not args.no_blas3 and F <= 1e12:
            try:
                blas3 = blas3_baseline(cfg, A_np, y_np, rb)
            except Exception as e:  # context only: recorded in the line, not fatal to it
                blas3 = {"error": "%s: %s" % (type(e).__name__, e)}
        elif not args.no_blas3:
            blas3 = {"skipped": "the BLAS-3 CPU baseline runs whole steps; at %.2g flops per step "
                     "it would take minutes on the host cores" % F}

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE_NAMES[args.mode],
            "data": ("synthetic (seeded U diag(sigma) V^T drawn on the device in FP32, seed %d + "
                     "7919 x rank)" % cfg["seed"]) if cfg.get("device_input") else
                    "synthetic (seeded U diag(sigma) V^T / N(0,1), generated on the host)",
            "config": step_config(cfg, args.mode, rb, world),
            "coded_flops_per_step": F,
            "uncoded": {"ms_per_step": ms_unc, "tflops_uncoded_equiv": 2.0 * m * n * n /
                        (ms_unc * 1e-3) / 1e12},
            "coding_overhead": ms / ms_unc - 1.0,
            "flop_model_overhead_floor": F / (2.0 * m * n * n) - 1.0,
            "errors": {"backward_rel_fro": berr, "orth_max_coded_Q": orth_coded,
                       "orth_max_post_orth": orth, "checksum_drift_max": drift,
                       "solve_rel_residual": resid, "how": "FP64 over the whole factors"},
            "reorth_per_step": stats["n_reorth"] / max(1, (2 * args.steps + args.warmup)),
            "recovered_tiles_per_step": len(plan),
            "kernel_ms_per_step": {k: v[0] / args.steps for k, v in prof.items() if v[1] or v[0] > 0},
            "ms_per_step_profiled": statistics.mean(t_prof),
            "gpu_launches": launches,
            "clocks": clk,
            "roofline": rl,
            "peaks_measured_here": peaks_here,
            "legs": legs,
            "cpu_baseline": cpu,
            "cpu_blas3": blas3,
            "e2e": {"value": e2e_value, "unit": "TFLOP/s", "ms_per_step": ms_e2e,
                    "h2d_bytes_per_step": m * n * es + m * es, "d2h_bytes_per_step": n * es},
        }
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


DTYPE_NAMES = {"f64": "f64", "f32": "f32", "tf32": "f32 storage, tf32 tensor-core GEMMs",
               "3xtf32": "f32 storage, 3xtf32 tensor-core GEMMs",
               "bf16": "f32 storage, bf16 tensor-core GEMMs",
               "bf16x3": "f32 storage, bf16x3 tensor-core GEMMs"}


def roofline(args, cfg, prof, geo, dtype, mma, es, peaks_here):
    """Roofline of the dominant kernel class (largest share of device time in the profiled
    steps): algorithmic work per launch / average launch duration, against the measured peak
    of its bound."""
    peaks, peak_src = measured_peaks()
    m, n, b = cfg["m"], cfg["n"], cfg["b"]
    dom = max(prof.items(), key=lambda kv: kv[1][0])
    dom_name, (dom_ms, dom_launches) = dom[0], dom[1]
    M, N, T = geo["M"], geo["N"], geo["panels"]
    widths = [(min(b, n - t * b), N - t * b - min(b, n - t * b)) for t in range(T)]
    gemm_flops = sum(2.0 * M * bk * w for bk, w in widths if w > 0)
    reorth_flops = sum(4.0 * M * (t * b) * bk for t, (bk, _) in enumerate(widths))
    panel_bytes = sum(2.0 * M * bk * es for bk, _ in widths)
    per_step = {"tc_update": gemm_flops, "tc_rbar": gemm_flops, "gemm_rbar_simt": gemm_flops,
                "gemm_update_simt": gemm_flops, "block_reorth": reorth_flops}
    if dom_name in per_step:
        algo = per_step[dom_name] * args.steps / dom_launches
        achieved = algo / (dom_ms / dom_launches * 1e-3) / 1e12
        tf32 = (peaks_here or {}).get("tf32_tflops_sustained")
        if dtype == "f64":
            fp64 = (peaks_here or {}).get("fp64_tflops")
            peak = fp64 or 152 * 2 * 2 * 2.07e9 / 1e12
            rl = {"bound": "alu", "unit": "TFLOP/s", "peak_source":
                  "FP64 torch.matmul measured in this run" if fp64 else
                  "FP64 CUDA-core: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz"}
        elif mma == "simt":
            peak = 152 * 128 * 2 * 2.07e9 / 1e12
            rl = {"bound": "alu", "unit": "TFLOP/s", "peak_source": "FP32 CUDA-core: 152 SMs x "
                  "128 FFMA/clk x 2 flop x 2.07 GHz"}
        elif mma in ("bf16", "bf16x3"):
            k = 3.0 if mma == "bf16x3" else 1.0
            peak = peaks["bf16_tflops_sustained"] / k
            rl = {"bound": "tensor", "unit": "TFLOP/s", "peak_source": "%s bf16 sustained%s"
                  % (peak_src, " / 3 (three bf16 MMAs per FP32-accurate product)" if k > 1 else "")}
        else:
            k = 3.0 if mma == "3xtf32" else 1.0
            if tf32:
                peak = tf32 / k
                src = "tf32 sustained measured in this run"
            else:
                peak = peaks["bf16_tflops_sustained"] * 1.1 / 2.25 / k
                src = "%s bf16 sustained x nominal tf32/bf16 ratio 1.1/2.25" % peak_src
            rl = {"bound": "tensor", "unit": "TFLOP/s", "peak_source": src + (
                  " / 3 (three tf32 MMAs per FP32-accurate product)" if k > 1 else "")}
            rl["tensor_pipe_frac"] = achieved * k / (peak * k)
        rl.update(achieved=achieved, peak=peak, frac=achieved / peak)
    else:
        algo = panel_bytes * args.steps / dom_launches if dom_name == "panel_icgs" else None
        dur = dom_ms / dom_launches * 1e-3
        achieved = (algo / dur / 1e9) if algo else None
        peak = peaks["hbm_gbs"]
        rl = {"bound": "hbm", "unit": "GB/s", "achieved": achieved, "peak": peak,
              "frac": (achieved / peak) if achieved else None,
              "peak_source": "%s copy bandwidth" % peak_src}
    rl.update(kernel=dom_name, launches_per_step=dom_launches / args.steps,
              avg_launch_ms=dom_ms / dom_launches,
              traffic=NCU_TRAFFIC.get((args.config, args.mode, dom_name)))
    return rl


def extra_legs(args, cfg, torch, B, Ad, A_np, yd, xd, flush, stream):
    """Legs beside the headline, on rank 0 (untimed for `value`):
    modes: the same workload with the other tensor-core precisions of the configuration
           (TF32 and BF16 with one product, BF16x3), errors on sampled columns;
    fp64_vs_mixed: the C2 workload (4096^2, kappa 1e2) in FP64 on the GPU (the paper's
           arithmetic) and in FP32 with 3xTF32 products, same step, full FP64 errors."""
    out = {}
    steps = max(1, min(args.steps, 5))
    warm = max(1, min(args.warmup, 3))
    m, n, p_r, p_c, f, b = (cfg[k] for k in ("m", "n", "p_r", "p_c", "f", "b"))
    plan = erasure_plan(cfg)
    rb = not args.no_reorth_block

    def time_q(q, Ad_, yd_, xd_, pl, st, wu):
        for _ in range(wu):
            coded_step(q, Ad_, yd_, xd_, pl)
        torch.cuda.synchronize()
        ts = []
        for _ in range(st):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            coded_step(q, Ad_, yd_, xd_, pl)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        s = q.sync_status()
        if s != 0:
            raise RuntimeError("device status %d (%s)" % (s, B.errstr(s)))
        return statistics.mean(ts)

    def factored(q, Ad_, pl):
        q.encode(Ad_)
        for t in range(q.geo["panels"]):
            tiles = [(i, j) for (tt, i, j) in pl if tt == t]
            if tiles:
                q.inject(tiles)
                q.recover()
            q.factor(t, t + 1)
        Qc, Rc = q.factors()
        Qo = B.colmajor_empty(q.geo["m_pad"], q.geo["n"], Qc.dtype)
        q.post_orth(Qo)
        return Qc, Rc, Qo

    F = coded_flops(m, n, p_r, p_c, f, b)
    if args.mode in ("3xtf32", "tf32", "bf16", "bf16x3"):
        A64 = torch.from_numpy(A_np).cuda()
        rows = {}
        for mode in ("tf32", "bf16", "bf16x3"):
            if mode == args.mode:
                continue
            try:
                q = B.CodedQR(m, n, p_r, p_c, f, b, dtype="f32", mma=MODES[mode][1],
                              seed=cfg["seed"], stream=stream, reorth_block=rb)
                ms = time_q(q, Ad, yd, xd, plan, steps, warm)
                Qc, Rc, Qo = factored(q, Ad, plan)
                err = sampled_errors(A64, Qc[:q.geo["M"]], Rc, Qo, m, n)
                q.close()
                rows[mode] = {"ms_per_step": ms, "tflops": F / (ms * 1e-3) / 1e12,
                              "errors": err, "steps": steps}
            except Exception as e:  # recorded, not fatal to the headline
                rows[mode] = {"error": "%s: %s" % (type(e).__name__, e)}
        del A64
        torch.cuda.empty_cache()
        out["modes"] = rows
    # FP64 on the GPU against the mixed-precision step on the C2 workload
    c2 = CONFIGS["c2"]
    A2, y2 = make_inputs(c2)
    plan2 = erasure_plan(c2)
    F2 = coded_flops(c2["m"], c2["n"], c2["p_r"], c2["p_c"], c2["f"], c2["b"])
    rows = {}
    for label, mode, rb2 in (("f64", "f64", False), ("f64_block_reorth", "f64", True),
                             ("3xtf32_block_reorth", "3xtf32", True)):
        dt_, mma_ = MODES[mode]
        tdd = torch.float64 if dt_ == "f64" else torch.float32
        try:
            A2d = B.colmajor_empty(c2["m"], c2["n"], tdd)
            A2d.copy_(torch.from_numpy(np.ascontiguousarray(A2)))
            y2d = B.colmajor_empty(c2["m"], 1, tdd)
            y2d.copy_(torch.from_numpy(np.ascontiguousarray(y2)))
            x2d = B.colmajor_empty(c2["n"], 1, tdd)
            q = B.CodedQR(c2["m"], c2["n"], c2["p_r"], c2["p_c"], c2["f"], c2["b"], dtype=dt_,
                          mma=mma_, seed=c2["seed"], stream=stream, reorth_block=rb2)
            st_ = steps if dt_ == "f64" else max(steps, 10)
            ms = time_q(q, A2d, y2d, x2d, plan2, st_, warm)
            Qc, Rc, Qo = factored(q, A2d, plan2)
            A64 = torch.from_numpy(A2).cuda()
            nn = c2["n"]
            Qt = Qc[:q.geo["M"], :nn].double()
            eye = torch.eye(nn, device="cuda", dtype=torch.float64)
            err = {"backward_rel_fro": (torch.linalg.norm(A64 - Qc[:c2["m"], :nn].double() @
                                                          Rc[:nn, :nn].double()) /
                                        torch.linalg.norm(A64)).item(),
                   "orth_max_coded_Q": (Qt.T @ Qt - eye).abs().max().item(),
                   "orth_max_post_orth": (Qo.double().T @ Qo.double() - eye).abs().max().item()}
            q.close()
            rows[label] = {"ms_per_step": ms, "tflops": F2 / (ms * 1e-3) / 1e12, "errors": err,
                           "steps": st_}
        except Exception as e:
            rows[label] = {"error": "%s: %s" % (type(e).__name__, e)}
    if "ms_per_step" in rows.get("3xtf32_block_reorth", {}):
        best64 = min((rows[k]["ms_per_step"] for k in ("f64", "f64_block_reorth")
                      if "ms_per_step" in rows.get(k, {})), default=None)
        if best64:
            rows["mixed_speedup_vs_fastest_f64"] = best64 / rows["3xtf32_block_reorth"]["ms_per_step"]
    out["fp64_vs_mixed_c2"] = {"workload": workload_name(c2, "f64 / 3xtf32"), "rows": rows}
    return out


# ------------------------------------------------------------------------ c4: batched
def batch_erasures(geos, f, seed):
    """Up to two tiles (<= f per grid row / column) per instance, lost at one seeded panel."""
    from paper_2311_11943_gb300 import synth
    rng = np.random.default_rng(seed)
    quads = []
    for i, g in enumerate(geos):
        k = int(rng.integers(0, 3))
        if k == 0:
            continue
        t = int(rng.integers(0, g["panels"]))
        for (r, c) in synth.random_erasures(g["grid_rows"], g["grid_cols"], f, k, seed + 7 * i):
            quads.append((i, t, r, c))
    return quads


def oracle_batch_sample(shapes, cfg, budget_s):
    """FP64 oracle on a bounded sample of the batch: whole instances (encode + every panel, no
    erasure), smallest first, until budget_s.  Returns (TFLOP/s, cores, sample)."""
    from oracle import oracle as O
    from paper_2311_11943_gb300 import synth
    order = sorted(range(len(shapes)), key=lambda i: shapes[i][0] * shapes[i][1] ** 2)
    t0 = time.perf_counter()
    flops, done = 0.0, 0
    for i in order[::max(1, len(order) // 64)]:
        if time.perf_counter() - t0 > budget_s:
            break
        m, n = shapes[i]
        A = synth.gaussian(m, n, 4000 + i)
        b = 32 if n >= 96 else 16
        O.run(A, cfg["p_r"], cfg["p_c"], cfg["f"], b, seed=cfg["seed"])
        flops += coded_flops(m, n, cfg["p_r"], cfg["p_c"], cfg["f"], b)
        done += 1
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return flops / dt / 1e12, cores, ("FP64 oracle: %d whole instances of the batch (every %d-th "
                                      "by size), %.1f GFLOP, %.1f s" %
                                      (done, max(1, len(order) // 64), flops / 1e9, dt))


def run_batched(args):
    import torch
    from paper_2311_11943_gb300 import binding as B
    from paper_2311_11943_gb300 import synth
    cfg = EXTRA["c4"]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    # weak scaling over replicas: every rank factorises its own batch of the same recipe
    from paper_2311_11943_gb300 import replicas
    shapes = synth.batched_shapes(cfg["count"], replicas.rank_seed(cfg["seed"], rank))
    gen = torch.Generator(device="cuda").manual_seed(replicas.rank_seed(1000 * cfg["seed"], rank))
    As = [torch.randn(n, m, device="cuda", dtype=torch.float32, generator=gen).t()
          for (m, n) in shapes]
    bt = B.CodedQRBatch(shapes, cfg["p_r"], cfg["p_c"], cfg["f"], b=0, seed=cfg["seed"])
    quads = batch_erasures(bt.geo, cfg["f"], cfg["seed"])
    t0 = time.perf_counter()
    G = bt.autotune(As, quads, reps=1)
    tune_s = time.perf_counter() - t0
    quads = batch_erasures(bt.geo, cfg["f"], cfg["seed"])   # panels of the tuned widths
    F = sum(coded_flops(g["m"], g["n"], cfg["p_r"], cfg["p_c"], cfg["f"], 1) for g in bt.geo)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        bt.run(As, quads, graph=True)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    times = []
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bt.run(As, quads, graph=True)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    st, bad, nre = bt.sync_status()
    if st != 0:
        raise RuntimeError("instance %d: device status %d" % (bad, st))
    # the dominant kernel alone: the persistent factor launch over the whole batch
    fac = []
    for _ in range(max(2, args.steps)):
        bt.encode(As)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bt.factor()
        e1.record(stream)
        e1.synchronize()
        fac.append(e0.elapsed_time(e1))
    t_fac = statistics.median(fac)
    # end to end through the library with host buffers: every instance's A copied from
    # pinned host memory inside coded_qr_batched_run each step, status words read back
    hosts = [torch.empty((n, m), dtype=torch.float32, pin_memory=True) for (m, n) in shapes]
    for h, a in zip(hosts, As):
        h.copy_(a.t())
    host_views = [h.numpy().T for h in hosts]
    e2e = []
    for it in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bt.run(host_views, quads, graph=True, host=True)
        bt.sync_status()
        if it >= args.warmup:
            e2e.append((time.perf_counter() - t0) * 1e3)
    ms = statistics.mean(times)
    ms_e2e = statistics.mean(e2e)
    ms, ms_e2e = replicas.max_over_ranks([ms, ms_e2e], dist if world > 1 else None, device="cuda")
    peak = 152 * 128 * 2 * 2.07e9 / 1e12
    rl = {"bound": "alu", "unit": "TFLOP/s", "kernel": "k_b_factor", "achieved": F / (t_fac * 1e-3) / 1e12,
          "peak": peak, "frac": F / (t_fac * 1e-3) / 1e12 / peak, "traffic": None,
          "avg_launch_ms": t_fac, "peak_source": "FP32 CUDA-core: 152 SMs x 128 FFMA/clk x 2 flop "
          "x 2.07 GHz (the batched factor runs on the CUDA cores)"}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
        v, cores, sample = oracle_batch_sample(shapes, cfg, args.cpu_budget)
        cpu = {"value": v, "unit": "TFLOP/s", "cores": cores, "kind": "oracle", "sample": sample}
    h2d = sum(m * n * 4 for (m, n) in shapes)
    if rank == 0:
        cl, widths = bt.tuning()
        line = {
            "metric": "coded GS-QR TFLOP/s (sum over the batch of F_coded = 2(m+c)n(n+2d))",
            "value": replicas.job_throughput(F, world, ms), "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded N(0,1) drawn on the device)",
            "config": {"workload": "batched: %d coded QRs, m~U[256,8192], n~U[32,256] (m>=4n), "
                       "grid %dx%d, f=%d, %d erased tiles in %d instances" %
                       (cfg["count"], cfg["p_r"], cfg["p_c"], cfg["f"], len(quads),
                        len(set(q[0] for q in quads))),
                       "cluster": cl, "widths": sorted(set(widths)), "autotune_s": tune_s,
                       "l2": "inputs (%.1f GB) larger than L2" % (h2d / 1e9),
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "graph": "the whole run recorded once into a CUDA graph and replayed"},
            "coded_flops_per_step": F, "factor_kernel_ms": t_fac, "reorth": nre,
            "gpu_launches": 6, "clocks": clk, "roofline": rl, "cpu_baseline": cpu,
            "e2e": {"value": replicas.job_throughput(F, world, ms_e2e), "unit": "TFLOP/s",
                    "ms_per_step": ms_e2e, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": 16 * cfg["count"]},
        }
        print(json.dumps(line))
    bt.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------------ f3: panel variants
def run_panels(args):
    """NEXT f3: panel latency vs orthogonality on the C2 shape for the paper's ICGS and the
    MGS / CGS1 / CGS2 variants (FP32, 3xTF32 trailing updates, block reorthogonalisation on,
    so that the loss between panels is removed and the panel sets the orthogonality),
    kappa 1e2 and 1e4."""
    import torch
    from paper_2311_11943_gb300 import binding as B
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    rows = []
    for kappa in (1e2, 1e4):
        cfg = dict(CONFIGS["c2"], kappa=kappa)
        A_np, _ = make_inputs(cfg)
        Ad = B.colmajor_empty(cfg["m"], cfg["n"], torch.float32)
        Ad.copy_(torch.from_numpy(np.ascontiguousarray(A_np)))
        A64 = torch.from_numpy(A_np).cuda()
        for panel, reg in (("icgs", "1"), ("icgs", "0"), ("mgs", "0"), ("cgs1", "0"), ("cgs2", "0")):
            os.environ["CQR_PANEL_REG"] = reg
            q = B.CodedQR(cfg["m"], cfg["n"], cfg["p_r"], cfg["p_c"], cfg["f"], cfg["b"],
                          dtype="f32", mma="3xtf32", seed=cfg["seed"], panel=panel,
                          reorth_block=True)
            q.profile(True)
            for it in range(args.warmup + args.steps):
                if it == args.warmup:
                    q.profile_read(reset=True)
                q.encode(Ad)
                q.factor(0, -1)
            prof = q.profile_read(reset=True)
            st = q.sync_status()
            Qc, Rc = q.factors()
            M, n = q.geo["M"], cfg["n"]
            Qt = Qc[:M, :n].double()
            orth = (torch.eye(n, device="cuda", dtype=torch.float64) - Qt.T @ Qt).abs().max().item()
            back = (torch.linalg.norm(A64 - Qc[:cfg["m"], :n].double() @ Rc[:n, :n].double()) /
                    torch.linalg.norm(A64)).item()
            q.close()
            pm = prof["panel_icgs"][0] / args.steps
            rows.append({"kappa": kappa, "panel": panel,
                         "kernel": "register" if (panel == "icgs" and reg == "1") else "shared-memory",
                         "panel_ms_per_factorisation": pm, "us_per_column": pm * 1e3 / n,
                         "orth_coded_Q": orth, "backward_rel_fro": back, "status": st})
    os.environ.pop("CQR_PANEL_REG", None)
    best = min(r["panel_ms_per_factorisation"] for r in rows)
    line = {"metric": "panel factorisation time per C2 factorisation (NEXT f3 comparison)",
            "value": best, "unit": "ms", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": best, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 storage, 3xtf32 trailing updates",
            "data": "synthetic (seeded U diag(sigma) V^T)",
            "config": {"workload": "C2 shape 4096x4096, grid 8x8, f=2, b=128; ICGS / MGS / CGS1 / "
                       "CGS2 panels, block reorthogonalisation, kappa 1e2 and 1e4, no erasure"},
            "variants": rows, "cpu_baseline": None, "e2e": None}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------------ ovh: overhead sweep
# (p, f, protect_r, one erasure at every panel)
OVH_ROWS = [(16, 4, True, False), (16, 4, False, False), (32, 1, True, False),
            (32, 1, False, False), (64, 1, True, False), (32, 1, True, True)]


def run_overhead(args):
    """Coding overhead t_coded / t_uncoded - 1 of the whole step (encode, factor, post-orth,
    solve) at n = 16384 over the grid p x p, the checksum count f and the code (two-way or
    vertical only), against the flop-model floor (1 + f/p)(1 + 2f/p) - 1 (vertical only:
    f/p); plus one row with one erased tile recovered at the start of every panel (the
    every-iteration failure experiment on one GPU).  FP32 storage, 3xTF32 updates, block
    reorthogonalisation.  The matrix is N(0,1): the step's time depends on the values only
    through the ICGS criterion, whose reorthogonalisation counts are reported."""
    import torch
    from paper_2311_11943_gb300 import binding as B
    from paper_2311_11943_gb300 import synth
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    cfg = EXTRA["ovh"]
    m, n, b = cfg["m"], cfg["n"], cfg["b"]
    A_np = synth.gaussian(m, n, cfg["seed"])
    y_np = synth.rhs(m, 1, cfg["seed"])
    stream = torch.cuda.current_stream()
    Ad = B.colmajor_empty(m, n, torch.float32)
    Ad.copy_(torch.from_numpy(np.ascontiguousarray(A_np)))
    yd = B.colmajor_empty(m, 1, torch.float32)
    yd.copy_(torch.from_numpy(np.ascontiguousarray(y_np)))
    xd = B.colmajor_empty(n, 1, torch.float32)
    del A_np

    def time_steps(p, f, protect_r, plan):
        q = B.CodedQR(m, n, p, p, f, b, dtype="f32", mma="3xtf32", seed=cfg["seed"],
                      protect_r=protect_r, stream=stream, reorth_block=True)
        for _ in range(args.warmup):
            coded_step(q, Ad, yd, xd, plan)
        torch.cuda.synchronize()
        times = []
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            coded_step(q, Ad, yd, xd, plan)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        st = q.sync_status()
        stats = q.stats()
        q.close()
        if st != 0:
            raise RuntimeError("device status %d (%s)" % (st, B.errstr(st)))
        return statistics.mean(times), stats

    t_unc, _ = time_steps(16, 0, True, [])
    rows = []
    for (p, f, protect_r, every) in OVH_ROWS:
        plan = []
        if every:
            T = -(-n // b)
            for t in range(T):
                for (i, j) in synth.random_erasures(p + f, p + (f if protect_r else 0), f, 1,
                                                    cfg["seed"] + t):
                    plan.append((t, i, j))
        ms, stats = time_steps(p, f, protect_r, plan)
        F = coded_flops(m, n, p, p, f, b, protect_r)
        floor = (1.0 + f / p) * (1.0 + (2.0 * f / p if protect_r else 0.0)) - 1.0
        rows.append({"p": p, "f": f, "code": "two-way" if protect_r else "vertical only",
                     "erasures": "one tile at every panel" if every else "none",
                     "ms_per_step": ms, "tflops_coded": F / (ms * 1e-3) / 1e12,
                     "overhead_vs_uncoded": ms / t_unc - 1.0, "flop_model_floor": floor,
                     "recovered_tiles_per_step": len(plan),
                     "reorth_per_step": stats["n_reorth"] / (args.warmup + args.steps)})
    free = [r for r in rows if r["erasures"] == "none"]
    best = min(free, key=lambda r: r["overhead_vs_uncoded"])
    line = {"metric": "coding overhead vs uncoded GPU QR at n = 16384 (whole step)",
            "value": best["overhead_vs_uncoded"], "unit": "fraction", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": best["ms_per_step"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 storage, 3xtf32 tensor-core GEMMs",
            "data": "synthetic (seeded N(0,1), generated on the host)",
            "config": {"workload": "16384x16384 N(0,1), b=256, block reorthogonalisation; grids "
                       "16x16 f=4, 32x32 f=1, 64x64 f=1; two-way and vertical-only codes; "
                       "no erasure, and one erasure at every panel",
                       "l2": "inputs (1 GB) larger than L2"},
            "uncoded_ms_per_step": t_unc, "rows": rows, "cpu_baseline": None, "e2e": None}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------------ e1: MDS statistics
def run_mds(args):
    """E1: least |det| and largest condition number over all square submatrices of the
    structured generator G~ = [-V V^T / 2, V] and of the completely random G~' = [G1', V]
    (G1' i.i.d. Unif(0,1)), f = 2..6, p_r = 16, 32, 64, mean of log10 over seeded trials."""
    import torch
    from paper_2311_11943_gb300 import binding as B
    from paper_2311_11943_gb300 import synth
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    trials = max(1, args.steps)
    table = []
    total_sub, total_ms = 0, 0.0
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    for p_r in (16, 32, 64):
        for f in range(2, 7):
            acc = {"det": [], "cond": [], "det_rand": [], "cond_rand": []}
            for t in range(trials):
                q = B.CodedQR(p_r, 1, p_r, 1, f, 1, dtype="f64", protect_r=False, seed=100 + t)
                q.encode(torch.zeros((1, p_r), dtype=torch.float64, device="cuda").t())
                Gt, _ = q.generator()      # computed on the device by encode
                q.close()
                Gr = Gt.copy()
                Gr[:, :f] = synth.unif01(f, f, 100 + t)
                for G, kd, kc in ((Gt, "det", "cond"), (Gr, "det_rand", "cond_rand")):
                    t0 = time.perf_counter()
                    md, mc, cnt = B.coded_qr_mds_stats(G)
                    total_ms += (time.perf_counter() - t0) * 1e3
                    total_sub += cnt
                    acc[kd].append(np.log10(md[0]))
                    acc[kc].append(np.log10(mc[0]))
            table.append({"p_r": p_r, "f": f, **{k: float(np.mean(v)) for k, v in acc.items()}})
    clk = clocks.stop()
    # CPU oracle on a bounded sample: the smallest case, structured generator
    cpu = None
    if not args.no_cpu_baseline:
        from oracle import oracle as O
        q = B.CodedQR(16, 1, 16, 1, 3, 1, dtype="f64", protect_r=False, seed=100)
        q.encode(torch.zeros((1, 16), dtype=torch.float64, device="cuda").t())
        Gt, _ = q.generator()
        q.close()
        t0 = time.perf_counter()
        O.mds_stats(Gt)
        dt = time.perf_counter() - t0
        n3 = 3 * 16 + 3 * 120 + 560
        cpu = {"value": n3 / dt, "unit": "submatrices/s", "cores": 1, "kind": "oracle",
               "sample": "numpy brute force, f = 3, p_r = 16 (%d submatrices), %.2f s" % (n3, dt)}
    line = {"metric": "E1 MDS statistics: square submatrices (|det| and 2-norm condition) per second",
            "value": total_sub / (total_ms * 1e-3), "unit": "submatrices/s", "n_gpus": 1,
            "steps": trials, "warmup": 0, "ms_per_step": total_ms / trials,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (the library's seeded generator; G1' from a seeded Unif(0,1))",
            "config": {"workload": "E1: f = 2..6, p_r = 16/32/64, structured vs completely "
                       "random generator, %d trial(s) each" % trials},
            "log10_table": table, "submatrices": total_sub, "clocks": clk, "cpu_baseline": cpu,
            "e2e": None}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------------ c5: autograd
def run_autograd(args):
    import torch
    from paper_2311_11943_gb300 import binding as B
    from paper_2311_11943_gb300.autograd import coded_lstsq
    cfg = EXTRA["c5"]
    local = int(os.environ.get("LOCAL_RANK", "0"))
    rank = int(os.environ.get("RANK", "0"))
    torch.cuda.set_device(local)
    bs, m, n = cfg["batch"], cfg["m"], cfg["n"]
    from paper_2311_11943_gb300 import replicas
    # every rank draws its own problems of the recipe (rank 0: the seed itself)
    gen = torch.Generator(device="cuda").manual_seed(replicas.rank_seed(cfg["seed"], rank))
    # A = U diag(sigma) V^T with Haar U (m x n), V (n x n), sigma geometric to kappa (data
    # generation on the device, not timed)
    A = torch.empty((bs, m, n), device="cuda", dtype=torch.float32)
    sig = cfg["kappa"] ** (-torch.arange(n, device="cuda", dtype=torch.float64) / (n - 1))
    for i in range(bs):
        U, Ru = torch.linalg.qr(torch.randn(m, n, device="cuda", dtype=torch.float64, generator=gen))
        U = U * torch.sign(torch.diagonal(Ru))
        V, Rv = torch.linalg.qr(torch.randn(n, n, device="cuda", dtype=torch.float64, generator=gen))
        V = V * torch.sign(torch.diagonal(Rv))
        A[i] = ((U * sig) @ V.T).float()
    y = torch.randn(bs, m, device="cuda", dtype=torch.float32, generator=gen)
    W = [torch.randn(s, device="cuda", dtype=torch.float32, generator=gen)
         for s in ((bs, m, n), (bs, n, n), (bs, n))]
    opts = dict(p_r=cfg["p_r"], p_c=cfg["p_c"], f=cfg["f"], b=cfg["b"], seed=cfg["seed"],
                erasures={(n // cfg["b"]) // 2: [(3, 6)]})
    stream = torch.cuda.current_stream()

    def step():
        Ad = A.detach().requires_grad_(True)
        yd = y.detach().requires_grad_(True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e2 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Q, R, x = coded_lstsq(Ad, yd, **opts)
        L = (W[0] * Q).sum() + (W[1] * torch.triu(R)).sum() + (W[2] * x).sum()
        e1.record(stream)
        L.backward()
        e2.record(stream)
        e2.synchronize()
        return e0.elapsed_time(e1), e1.elapsed_time(e2), Ad.grad

    for _ in range(args.warmup):
        step()
    clocks = ClockSampler(local)
    clocks.start()
    fw, bw = [], []
    for _ in range(args.steps):
        a, b_, grad = step()
        fw.append(a)
        bw.append(b_)
    clk = clocks.stop()
    F = bs * coded_flops(m, n, cfg["p_r"], cfg["p_c"], cfg["f"], cfg["b"])
    ms = statistics.mean(f_ + b_ for f_, b_ in zip(fw, bw))
    # gradient check of the last step against a CPU FP64 reference on problem 0
    from oracle import oracle as O
    g = O.geom(m, n, cfg["p_r"], cfg["p_c"], cfg["f"], True)
    Gt, _ = O.generator(cfg["f"], cfg["p_r"], cfg["p_c"], cfg["seed"])
    G0 = torch.tensor(O.build_G0(g, Gt), dtype=torch.float64)
    A0 = A[0].double().cpu().requires_grad_(True)
    y0 = y[0].double().cpu()
    Qr, Rr = torch.linalg.qr(G0 @ A0)
    d = torch.sign(torch.diagonal(Rr))
    x0 = torch.linalg.solve(A0.T @ A0, A0.T @ y0)
    L0 = ((W[0][0].double().cpu() * (Qr * d)).sum() + (W[1][0].double().cpu() *
          torch.triu(d[:, None] * Rr)).sum() + (W[2][0].double().cpu() * x0).sum())
    L0.backward()
    gref = A0.grad
    gerr = (torch.linalg.norm(grad[0].double().cpu() - gref) / torch.linalg.norm(gref)).item()
    # dominant kernel of the forward: one problem with the same options, profiled
    q = B.CodedQR(m, n, cfg["p_r"], cfg["p_c"], cfg["f"], cfg["b"], dtype="f32", mma="3xtf32",
                  seed=cfg["seed"])
    Ac = B.colmajor_empty(m, n, torch.float32)
    Ac.copy_(A[0])
    q.profile(True)
    q.profile_read(reset=True)
    for _ in range(2):
        q.encode(Ac)
        q.factor(0, -1)
    prof = q.profile_read(reset=True)
    q.close()
    dom = max(prof.items(), key=lambda kv: kv[1][0])
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
        c5 = dict(m=m, n=n, p_r=cfg["p_r"], p_c=cfg["p_c"], f=cfg["f"], b=cfg["b"], seed=cfg["seed"])
        v, cores, sample, _ = oracle_sample(c5, A[0].double().cpu().numpy(), budget_s=args.cpu_budget)
        cpu = {"value": v, "unit": "TFLOP/s", "cores": cores, "kind": "oracle", "sample": sample}
    line = {
        "metric": "coded GS-QR TFLOP/s of forward + adjoint (F_coded per problem x batch)",
        "value": F / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 storage, 3xtf32 tensor-core GEMMs, FP64 CG",
        "data": "synthetic (seeded U diag(sigma) V^T, kappa 1e3, drawn on the device)",
        "config": {"workload": "differentiable least squares: %d x A %dx%d kappa=%g, grid %dx%d, "
                   "f=%d, b=%d, one erasure at panel %d; loss <W_Q,Q>+<W_R,R>+<W_x,x>" %
                   (bs, m, n, cfg["kappa"], cfg["p_r"], cfg["p_c"], cfg["f"], cfg["b"],
                    (n // cfg["b"]) // 2)},
        "forward_ms": statistics.mean(fw), "backward_ms": statistics.mean(bw),
        "grad_rel_err_vs_cpu_fp64": gerr,
        "forward_kernel_ms_per_problem": {k: v[0] / 2 for k, v in prof.items() if v[1]},
        "clocks": clk,
        "roofline": {"kernel": dom[0], "note": "see forward_kernel_ms_per_problem; the C2 line "
                     "carries the kernel roofline"},
        "cpu_baseline": cpu,
        "e2e": None,
    }
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c3", choices=sorted(CONFIGS) + sorted(EXTRA))
    ap.add_argument("--mode", default=os.environ.get("CQR_BENCH_MODE", "3xtf32"),
                    choices=sorted(MODES))
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-blas3", action="store_true",
                    help="skip the torch CPU BLAS-3 baseline beside the oracle")
    ap.add_argument("--no-legs", action="store_true",
                    help="skip the legs beside the headline (other precisions, FP64 vs mixed)")
    ap.add_argument("--no-reorth-block", action="store_true",
                    help="skip the block reorthogonalisation pass (faster, orthogonality ~ u kappa)")
    args = ap.parse_args()
    if args.config in EXTRA:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the reference arm times the "
                              "oracle on the single-problem workloads (c1, c2, c2k6, c3) only"}))
            return 0
        if args.config == "e1":
            return run_mds(args)
        if args.config == "ovh":
            return run_overhead(args)
        if args.config == "f3":
            return run_panels(args)
        return run_batched(args) if args.config == "c4" else run_autograd(args)
    cfg = CONFIGS[args.config]
    if args.impl == "reference":
        return run_reference(args, cfg)
    return run_ours(args, cfg)


if __name__ == "__main__":
    sys.exit(main())
