"""Child process of tests/test_gpu_debug_bounds.py: runs the hot path through the bounds-checked
build (CQR_LIBRARY=debug) on small odd shapes and prints one JSON line of results."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

from oracle import oracle as O  # noqa: E402
from paper_2311_11943_gb300 import binding as B  # noqa: E402
from paper_2311_11943_gb300 import synth  # noqa: E402

assert B.LIB_PATH.endswith("libcoded_qr_debug.so"), B.LIB_PATH

# (m, n, p_r, p_c, f, b, dtype, mma, erasures {panel: tiles}, post_orth form): ragged rows, a
# partial last panel, several checksum counts, the tensor-core and CUDA-core paths, both
# post-orthogonalisation forms, a tall problem (least squares)
CASES = [
    (203, 96, 8, 4, 2, 20, "f64", "simt", {2: [(3, 1), (9, 5)]}, "g0"),
    (203, 96, 8, 4, 2, 20, "f32", "3xtf32", {2: [(3, 1), (9, 5)]}, "projected"),
    (256, 256, 4, 4, 1, 32, "f32", "tf32", {3: [(2, 3)]}, "projected"),
    (330, 330, 6, 6, 3, 44, "f64", "simt", {1: [(7, 0), (0, 8), (4, 4)]}, "projected"),
    (1003, 192, 8, 4, 1, 48, "f32", "3xtf32", {1: [(2, 1)]}, "auto"),
]


def run_case(m, n, p_r, p_c, f, b, dtype, mma, er, form):
    td = torch.float64 if dtype == "f64" else torch.float32
    A = synth.kappa_matrix(m, n, 10.0, seed=m + n)
    y = synth.rhs(m, 1, m)
    q = B.CodedQR(m, n, p_r, p_c, f, b, dtype=dtype, mma=mma, seed=3, post_orth=form)
    Ad = B.colmajor_empty(m, n, td)
    Ad.copy_(torch.from_numpy(A))
    q.encode(Ad)
    for t in range(q.geo["panels"]):
        if er.get(t):
            q.inject(er[t])
            q.recover()
        q.factor(t, t + 1)
    _, Rc = q.factors()
    R = Rc.double().cpu().numpy()
    yd = B.colmajor_empty(m, 1, td)
    yd.copy_(torch.from_numpy(y))
    x = B.colmajor_empty(n, 1, td)
    if m == n:
        Qo = B.colmajor_empty(q.geo["m_pad"], n, td)
        q.post_orth(Qo)
    q.solve_ls(yd, x)
    torch.cuda.synchronize()
    st = q.sync_status()
    q.close()
    ref = O.run(A, p_r, p_c, f, b, seed=3, erasures=er)
    u = np.finfo(np.float64 if dtype == "f64" else np.float32).eps
    tol = n * u * 10.0 * (1e4 if mma == "tf32" else (8 if mma == "3xtf32" else 1))
    err = float(np.abs(R - ref["R"]).max() / np.abs(ref["R"]).max())
    bst, site = B.debug_bounds()
    return {"status": int(st), "bounds": int(bst), "site": int(site), "err": err, "tol": float(tol)}


out = {"cases": [run_case(*c) for c in CASES]}
torch.cuda.synchronize()
assert B.debug_bounds_selftest(0) == 0
torch.cuda.synchronize()
out["selftest"] = B.debug_bounds()
out["after"] = B.debug_bounds()
print(json.dumps(out))
