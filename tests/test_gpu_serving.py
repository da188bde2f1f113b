"""Serving loop (continuous batching) through the C ABI (lspca_srv_*).

* every request's result is bit-identical alone and in a mix that admits
  requests while others are running;
* projections match the FP64 product of the stored values (relative
  Frobenius 1e-5 for BF16 X, 2e-6 for FP32 X);
* fits (Algorithm 4 slices) span the FP64 oracle's subspace and match its
  singular values;
* admission by HBM footprint: with a small arena a second fit waits until the
  first one has released its workspace, and both still complete.
"""
import numpy as np
import pytest
import torch

from oracle import lspca as O
from oracle import metrics as M
from oracle import philox as P
from paper_1709_07175_gb300 import lspca as L
from paper_1709_07175_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


def _orth(n, k, seed):
    g = torch.Generator().manual_seed(seed)
    q, _ = torch.linalg.qr(torch.randn(n, k, generator=g, dtype=torch.float64))
    return q.float().contiguous()


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1709_07175_gb300 import build
    build.build()
    n = 1024
    Vs = {64: _orth(n, 64, 1).cuda(), 128: _orth(n, 128, 2).cuda()}
    proj = []
    for i, (rows, dt) in enumerate([(1, "bf16"), (7, "f32"), (128, "bf16"), (129, "f32"), (1000, "bf16"),
                                    (5000, "f32"), (3, "bf16"), (20000, "bf16")]):
        w = (S.WORKLOADS["bf16_dense"] if dt == "bf16" else S.WORKLOADS["fp32_sparse"]).scaled(m=rows, n=n)
        from dataclasses import replace
        w = replace(w, data_seed=100 + i)
        proj.append((S.generate(w).cuda(), 64 if i % 2 == 0 else 128))
    fw1 = S.WORKLOADS["fp32_sparse"].scaled(m=70000, n=n, k=64)
    fw2 = S.WORKLOADS["bf16_dense"].scaled(m=20000, n=n, k=64)
    fits = [(fw1, S.generate(fw1).cuda()), (fw2, S.generate(fw2).cuda())]
    return Vs, proj, fits


def _om(w):
    return L.omega(w.omega, w.omega_seed, w.p)


def _run(srv, Vs, proj, fits, order, alone):
    vid = {k: srv.register_v(V) for k, V in Vs.items()}
    out = {}
    pending = []
    for kind, i in order:
        if kind == "p":
            X, k = proj[i]
            req, Y = srv.submit_project(vid[k], X)
            out[("p", i)] = (req, Y)
        else:
            w, X = fits[i]
            req, V, sig = srv.submit_fit(X, w.k, _om(w))
            out[("f", i)] = (req, V, sig)
        pending.append(out[(kind, i)][0])
        if alone:
            srv.wait(pending[-1], 60000)
        else:
            srv.step()  # later submissions arrive while earlier work runs
    for req in pending:
        srv.wait(req, 60000)
    torch.cuda.synchronize()
    return out


def test_serving_alone_equals_mix_and_matches_references(setup):
    Vs, proj, fits = setup
    order = [("f", 0)] + [("p", i) for i in range(4)] + [("f", 1)] + [("p", i) for i in range(4, len(proj))]
    srv_a = L.Server(0, 2 << 30, 64)
    alone = _run(srv_a, Vs, proj, fits, order, alone=True)
    srv_a.close()
    srv_m = L.Server(0, 2 << 30, 64)
    mix = _run(srv_m, Vs, proj, fits, order, alone=False)
    srv_m.close()
    for key in alone:
        a, b = alone[key], mix[key]
        for ta, tb in zip(a[1:], b[1:]):
            assert torch.equal(ta, tb), key
    # projections against the FP64 product of the stored values
    for i, (X, k) in enumerate(proj):
        Y = mix[("p", i)][1].double().cpu().numpy()
        ref = X.double().cpu().numpy() @ Vs[k].double().cpu().numpy()
        tol = 1e-5 if X.dtype == torch.bfloat16 else 2e-6
        assert np.linalg.norm(Y - ref) / max(np.linalg.norm(ref), 1e-30) < tol, i
    # fits against the oracle (sliced accumulation: same subspace and sigma)
    for i, (w, X) in enumerate(fits):
        Xd = X.double().cpu().numpy()
        Om = P.omega_sparse(w.omega_seed, w.n, w.k, w.p) if w.omega == "sparse" else \
            P.bf16_rne(P.omega_gaussian(w.omega_seed, w.n, w.k))
        ref = O.lspca_fit(Xd, Om, route="eig")
        _, V, sig = mix[("f", i)]
        V = V.double().cpu().numpy()
        assert M.max_sine(ref["V"], V) < 1e-4
        tol = 1e-5 if X.dtype == torch.float32 else 1e-4
        assert np.max(np.abs(sig.cpu().numpy() - ref["sigma"]) / ref["sigma"]) < tol


def test_serving_admission_by_memory(setup):
    Vs, proj, fits = setup
    w, X = fits[0]
    srv = L.Server(0, 256 << 20, 8)  # room for one fit workspace at a time
    r1, V1, s1 = srv.submit_fit(X, w.k, _om(w))
    r2, V2, s2 = srv.submit_fit(X, w.k, _om(w))
    srv.step()
    # the second fit cannot be admitted while the first holds the arena
    assert not srv.done(r2)
    srv.wait(r1, 60000)
    srv.wait(r2, 60000)
    torch.cuda.synchronize()
    assert torch.equal(V1, V2) and torch.equal(s1, s2)
    srv.close()
