"""Differentiable least squares through the coded QR (torch.autograd.Function).

Forward, per problem of the batch and all in the CUDA library: encode A, PBMGS/ICGS panels with
the listed erasures injected and recovered, the post-orthogonalised factor Q = G_0 Q_1, the
coded R, and x = argmin |A x - y| through the coded factors.  G_0 A = Q R with Q^T Q = I
(post-orthogonalisation theorem, Section 4.3), so (Q, R) is the thin QR of G_0 A (rows of
the zero-padded A beyond m give the last m_pad - m rows of Q).

Backward: the hand-written adjoint kernels of the library (coded_qr_adjoint_qr for the (Q, R)
outputs, coded_qr_adjoint_lstsq for x).  Only tall problems (m > n) are accepted: for square
ones the solve post-orthogonalises in place and the least-squares adjoint needs Q_1.

The problems of a batch run concurrently, each on its own CUDA stream (joined to the caller's
stream at the end): one problem's panel factorisation occupies at most one thread-block
cluster, so several of them share the GPU.
"""
import torch

from . import binding as B


def _cm(t, rows=None):
    """Column-major device copy of a 2-D tensor (rows zero-padded up to `rows`)."""
    r, c = t.shape
    rows = rows or r
    out = B.colmajor_empty(rows, c, t.dtype)
    if rows > r:
        out.zero_()
    out[:r].copy_(t)
    return out


class CodedLstsqFunction(torch.autograd.Function):
    """(Q, R, x) = coded_lstsq(A, y); A (batch, m, n), y (batch, m, k)."""

    @staticmethod
    def forward(ctx, A, y, opts):
        batch, m, n = A.shape
        k = y.shape[2]
        if m <= n:
            raise ValueError("coded least squares needs m > n (got %d x %d)" % (m, n))
        dt = "f64" if A.dtype == torch.float64 else "f32"
        mma = opts.get("mma", "simt" if dt == "f64" else "3xtf32")
        erasures = opts.get("erasures") or {}
        cur = torch.cuda.current_stream()
        streams = [torch.cuda.Stream() for _ in range(min(batch, opts.get("streams", 16)))]
        Q = torch.empty((batch, m, n), dtype=A.dtype, device=A.device)
        R = torch.empty((batch, n, n), dtype=A.dtype, device=A.device)
        X = torch.empty((batch, n, k), dtype=A.dtype, device=A.device)
        for s in streams:
            s.wait_stream(cur)
        saved = []
        for i in range(batch):
            s = streams[i % len(streams)]
            with torch.cuda.stream(s):
                q = B.CodedQR(m, n, opts["p_r"], opts["p_c"], opts["f"], opts["b"], dtype=dt,
                              mma=mma, nrhs_max=k, seed=opts.get("seed", 1),
                              tau=opts.get("tau", 0.0), stream=s)
                Ac = _cm(A[i])
                yc = _cm(y[i])
                q.encode(Ac)
                T = q.geo["panels"]
                t = 0
                while t < T:
                    if erasures.get(t):
                        q.inject(erasures[t])
                        q.recover()
                    nxt = t + 1
                    while nxt < T and not erasures.get(nxt):
                        nxt += 1
                    q.factor(t, nxt)
                    t = nxt
                Qo = B.colmajor_empty(q.geo["m_pad"], n, A.dtype)
                q.post_orth(Qo)
                xc = B.colmajor_empty(n, k, A.dtype)
                q.solve(yc, xc)
                _, Rc = q.factors()
                Q[i].copy_(Qo[:m])
                R[i].copy_(torch.triu(Rc[:n, :n]))
                X[i].copy_(xc)
            saved.append((q, Ac, yc, Qo, xc, s))
        for s in streams:
            cur.wait_stream(s)
        for (_, Ac, yc, Qo, xc, s) in saved:
            for t_ in (Ac, yc, Qo, xc):
                t_.record_stream(cur)
        ctx.saved = saved
        ctx.shape = (batch, m, n, k)
        return Q, R, X

    @staticmethod
    def backward(ctx, Qbar, Rbar, xbar):
        batch, m, n, k = ctx.shape
        cur = torch.cuda.current_stream()
        Abar = torch.zeros((batch, m, n), dtype=ctx.saved[0][1].dtype, device="cuda")
        ybar = torch.zeros((batch, m, k), dtype=Abar.dtype, device="cuda")
        streams = []
        for (_, _, _, _, _, s) in ctx.saved:
            if s not in streams:
                streams.append(s)
        for s in streams:
            s.wait_stream(cur)
        keep = []
        for i, (q, Ac, yc, Qo, xc, s) in enumerate(ctx.saved):
            with torch.cuda.stream(s):
                Ab = B.colmajor_empty(m, n, Abar.dtype)
                Ab.zero_()
                if Qbar is not None or Rbar is not None:
                    Qb = _cm(Qbar[i], rows=q.geo["m_pad"]) if Qbar is not None else None
                    Rb = _cm(torch.triu(Rbar[i])) if Rbar is not None else None
                    q.adjoint_qr(Qo, Qb, Rb, Ab)
                    keep += [t_ for t_ in (Qb, Rb) if t_ is not None]
                if xbar is not None:
                    yb = B.colmajor_empty(m, k, Abar.dtype)
                    yb.zero_()
                    xb = _cm(xbar[i])
                    q.adjoint_lstsq(Ac, yc, xc, xb, Ab, yb)
                    ybar[i].copy_(yb)
                    keep += [yb, xb]
                Abar[i].copy_(Ab)
                keep.append(Ab)
        for s in streams:
            cur.wait_stream(s)
        for t_ in keep:
            t_.record_stream(cur)
        for (q, *_rest) in ctx.saved:
            q.close()  # synchronises the handle's stream before freeing its memory
        ctx.saved = None
        return Abar, ybar, None


def coded_lstsq(A, y, p_r, p_c, f, b, seed=1, erasures=None, mma=None, tau=0.0):
    """Q (batch, m, n), R (batch, n, n), x (batch, n, k) of the coded least-squares path.

    A: (batch, m, n) or (m, n) CUDA tensor (float32 or float64); y: (batch, m, k), (batch, m),
    (m, k) or (m,).  erasures: {panel t: [(grid row, grid column), ...]} lost at the start of
    panel t (the same for every problem).  Differentiable in A and y.
    """
    squeeze = A.dim() == 2
    if squeeze:
        A = A.unsqueeze(0)
        y = y.unsqueeze(0)
    vec = y.dim() == 2
    if vec:
        y = y.unsqueeze(2)
    opts = dict(p_r=p_r, p_c=p_c, f=f, b=b, seed=seed, erasures=erasures, tau=tau)
    if mma is not None:
        opts["mma"] = mma
    Q, R, x = CodedLstsqFunction.apply(A, y, opts)
    if vec:
        x = x.squeeze(2)
    if squeeze:
        Q, R, x = Q[0], R[0], x[0]
    return Q, R, x
