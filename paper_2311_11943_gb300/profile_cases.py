"""Small fixed workloads for capturing single kernels under a profiler (ncu), through the
library's public API.  Each case runs twice (the first run warms up the handle).

  python -m paper_2311_11943_gb300.profile_cases tc_c2      # C2 shape, FP32 3xTF32: 2 panels
  python -m paper_2311_11943_gb300.profile_cases panel_c2   # same handle (register panel)
  python -m paper_2311_11943_gb300.profile_cases bfactor64  # 64 batched instances, no erasure
  python -m paper_2311_11943_gb300.profile_cases adjoint    # 8192 x 1024: forward + both adjoints
  python -m paper_2311_11943_gb300.profile_cases bandwidth8192  # encode / decode / post-orth
  python -m paper_2311_11943_gb300.profile_cases c3_tall    # the 16384^2 workload's panel shape
  python -m paper_2311_11943_gb300.profile_cases exchange_floor  # per-column exchange floor
  python -m paper_2311_11943_gb300.profile_cases bfactor_phases  # batched factor phase clocks

Launch order per run (for ncu's --launch-skip; filter by kernel name with -k, as the commands
in profiles/ do, since two streams interleave):
  tc_c2 / panel_c2: generator, encode (2), then per panel: block reorthogonalisation (split,
                    GEMM1, reduce, GEMM2 and, when split over K, a subtraction), panel, split,
                    the next panel's columns (GEMM1, reduce, GEMM2); the rest of the trailing
                    update (GEMM1, reduce, GEMM2) on the low-priority stream
  bfactor64:        encode (2), one k_b_factor
  bandwidth8192:    encode (vertical, horizontal), panels 0-15, poison, decode (Q, R),
                    panels 16-31, post-orthogonalisation
  c3_tall:          generator, encode (2), then per panel in one stream: block
                    reorthogonalisation (from panel 1), panel, split, GEMM1, reduce, GEMM2
"""
import sys

import numpy as np


def _cm(torch, B, X):
    d = B.colmajor_empty(X.shape[0], X.shape[1], torch.float32)
    d.copy_(torch.as_tensor(np.ascontiguousarray(X), dtype=torch.float32))
    return d


def case_c2(panels=2):
    import torch
    from . import binding as B
    from . import synth
    A = _cm(torch, B, synth.gaussian(4096, 4096, 2))
    q = B.CodedQR(4096, 4096, 8, 8, 2, 128, dtype="f32", mma="3xtf32", seed=2)
    for _ in range(2):
        q.encode(A)
        q.factor(0, panels)
    torch.cuda.synchronize()
    assert q.sync_status() == 0
    q.close()


def case_bfactor(count=64):
    import torch
    from . import binding as B
    from . import synth
    shapes = synth.batched_shapes(count, 4)
    As = [_cm(torch, B, synth.gaussian(m, n, 4000 + i, dtype=np.float32))
          for i, (m, n) in enumerate(shapes)]
    bt = B.CodedQRBatch(shapes, 8, 4, 2, b=0, seed=4)
    bt.set_tuning(2)
    for _ in range(2):
        bt.run(As, [], graph=False)
    torch.cuda.synchronize()
    assert bt.sync_status()[0] == 0
    bt.close()


def case_adjoint():
    import torch
    from . import binding as B
    from . import synth
    m, n = 8192, 1024
    A = synth.kappa_matrix(m, n, 1e3, 31)
    y = synth.rhs(m, 1, 81)
    q = B.CodedQR(m, n, 8, 8, 1, 128, dtype="f32", mma="3xtf32", seed=5)
    Ac, yc = _cm(torch, B, A), _cm(torch, B, y)
    rng = np.random.default_rng(3)
    Qb = _cm(torch, B, rng.standard_normal((q.geo["m_pad"], n)))
    Rb = _cm(torch, B, np.triu(rng.standard_normal((n, n))))
    xb = _cm(torch, B, rng.standard_normal((n, 1)))
    for _ in range(2):
        q.encode(Ac)
        q.factor(0, -1)
        Qo = B.colmajor_empty(q.geo["m_pad"], n, torch.float32)
        q.post_orth(Qo)
        x = B.colmajor_empty(n, 1, torch.float32)
        q.solve(yc, x)
        Ab = B.colmajor_empty(m, n, torch.float32)
        Ab.zero_()
        yb = B.colmajor_empty(m, 1, torch.float32)
        yb.zero_()
        q.adjoint_qr(Qo, Qb, Rb, Ab)
        q.adjoint_lstsq(Ac, yc, x, xb, Ab, yb)
    torch.cuda.synchronize()
    assert q.sync_status() == 0
    q.close()


def case_bandwidth():
    """The bandwidth kernels on inputs larger than L2: 8192 x 8192 N(0,1), grid 16 x 16, f = 4,
    b = 256, FP32 3xTF32; encode, four tiles erased at the start of panel 16 and recovered,
    the rest of the factorisation, post-orthogonalisation into a separate buffer; twice."""
    import torch
    from . import binding as B
    from . import synth
    n = 8192
    A = _cm(torch, B, synth.gaussian(n, n, 3, dtype=np.float32))
    q = B.CodedQR(n, n, 16, 16, 4, 256, dtype="f32", mma="3xtf32", seed=3)
    tiles = synth.random_erasures(20, 20, 4, 4, 3)
    Qo = B.colmajor_empty(n, n, torch.float32)
    for _ in range(2):
        q.encode(A)
        q.factor(0, 16)
        q.inject(tiles)
        q.recover()
        q.factor(16, -1)
        q.post_orth(Qo)
    torch.cuda.synchronize()
    assert q.sync_status() == 0
    q.close()


def case_c3_tall(panels=2):
    """Panels 0 and 1 of a 16384 x 8192 N(0,1) problem on the 16384^2 workload's grid (16 x 16,
    f = 4, b = 256): the panel is the same 20480 x 256 block as in the full problem, GEMM1 has
    156 output tiles (the full problem: 316), about 2 GB on the device; FP32 3xTF32 with
    block reorthogonalisation; twice."""
    import torch
    from . import binding as B
    from . import synth
    A = _cm(torch, B, synth.gaussian(16384, 8192, 3, dtype=np.float32))
    q = B.CodedQR(16384, 8192, 16, 16, 4, 256, dtype="f32", mma="3xtf32", seed=3,
                  reorth_block=True)
    for _ in range(2):
        q.encode(A)
        q.factor(0, panels)
    torch.cuda.synchronize()
    assert q.sync_status() == 0
    q.close()


def case_exchange_floor(reps=8):
    """The latency floor of the panel's per-column reduction (coded_qr_probe_exchange) beside
    the panel's own time per column, for the panels of the 4096^2 workload (5120 x 128, the
    register panel in one cluster) and of the 16384^2 workload (20480 x 256, the shared-memory
    panel with the two-level exchange).  The panel time comes from the handle's event profile
    over factor(0, 4), after a warm-up run; one JSON line per panel."""
    import json

    import torch
    from . import binding as B
    from . import synth
    rows = []
    for (m, n, p, f, b, kind, name) in [(4096, 4096, 8, 2, 128, 0, "5120x128 register panel"),
                                        (16384, 8192, 16, 4, 256, 1,
                                         "20480x256 two-level shared-memory panel")]:
        M = m + f * (m // p)
        floor = B.probe_exchange(kind, M, b, reps)
        A = _cm(torch, B, synth.gaussian(m, n, 3, dtype=np.float32))
        q = B.CodedQR(m, n, p, p, f, b, dtype="f32", mma="3xtf32", seed=3, reorth_block=True)
        q.encode(A)
        q.factor(0, 4)
        q.profile(True)
        q.profile_read(reset=True)
        q.encode(A)
        q.factor(0, 4)
        torch.cuda.synchronize()
        ms, launches = q.profile_read(reset=True)["panel_icgs"]
        assert q.sync_status() == 0
        q.close()
        per_col = 1000.0 * ms / max(1, launches * b)
        rows.append({"panel": name, "rows": M, "columns": b,
                     "exchange_floor_us_per_column": floor,
                     "panel_us_per_column": per_col,
                     "panel_launches": launches,
                     "floor_share": floor / per_col if per_col > 0 else None})
    for r in rows:
        print(json.dumps(r))


def case_bfactor_phases(count=512):
    """Phase clocks (coded_qr_batched_profile) of the persistent batched factor on the batch
    recipe of 512 instances: m ~ U[256, 8192], n ~ U[32, 256] (m >= 4 n), grid 8 x 4, f = 2,
    shapes from seed 4, N(0,1) entries drawn on the device, cluster size and widths picked by
    the autotuner.  Two launch kinds, each timed with CUDA events after a warm-up: the factor
    launch alone (encode, then factor, no erasure), and the whole run with one tile of every
    instance lost at its middle panel and recovered inside the launch.  One JSON line each:
    kernel (or run) ms, SM cycles per CTA in each phase and the phases' shares."""
    import json

    import torch
    from . import binding as B
    from . import synth
    shapes = synth.batched_shapes(count, 4)
    gen = torch.Generator(device="cuda").manual_seed(4000)
    As = [torch.randn(n, m, device="cuda", dtype=torch.float32, generator=gen).t()
          for (m, n) in shapes]
    bt = B.CodedQRBatch(shapes, 8, 4, 2, b=0, seed=4)
    bt.autotune(As, [], reps=1)
    quads = []
    for i, g in enumerate(bt.geo):
        (r, c), = synth.random_erasures(g["grid_rows"], g["grid_cols"], 2, 1, 11 + i)
        quads.append((i, g["panels"] // 2, r, c))
    stream = torch.cuda.current_stream()

    def timed(prep, fn, warm=True):
        if warm:
            prep()
            fn()
        prep()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1)

    kinds = [("factor launch alone, no erasure (encode outside the events)",
              lambda: bt.encode(As), lambda: bt.factor()),
             ("whole run (encode, factor with one tile per instance recovered in the launch)",
              lambda: None, lambda: bt.run(As, quads, graph=False))]
    runs = [(name, prep, fn) for (name, prep, fn) in kinds]
    # the factor launch again at the widest cluster (8 CTAs per instance, an eighth of the rows
    # each, widths by the shape rule)
    runs.append(("factor launch alone at clusters of 8, no erasure", "cluster8",
                 lambda: bt.factor()))
    for name, prep, fn in runs:
        if prep == "cluster8":
            bt.set_tuning(8)
            prep = lambda: bt.encode(As)  # noqa: E731
        cl, widths = bt.tuning()
        ms_plain = timed(prep, fn)
        bt.profile(True)
        prep()
        fn()
        bt.phases(reset=True)
        ms_prof = timed(prep, fn, warm=False)
        ph, ctas = bt.phases(reset=True)
        bt.profile(False)
        assert bt.sync_status()[0] == 0
        tot = sum(ph.values())
        per_cta = {k: v / max(1, ctas) for k, v in ph.items()}
        print(json.dumps({"launch": name, "instances": count, "cluster": cl,
                          "widths": sorted(set(widths)), "ms": ms_plain, "ms_clocked": ms_prof,
                          "ctas": ctas, "cycles_per_cta": per_cta,
                          "share": {k: v / tot for k, v in ph.items()} if tot else None}))
    bt.close()


CASES = {"tc_c2": case_c2, "panel_c2": case_c2, "bfactor64": case_bfactor, "adjoint": case_adjoint,
         "bandwidth8192": case_bandwidth, "c3_tall": case_c3_tall,
         "exchange_floor": case_exchange_floor, "bfactor_phases": case_bfactor_phases}

if __name__ == "__main__":
    CASES[sys.argv[1]]()
    print("ok", sys.argv[1])
