"""Learned warm start on the GPU: the library's BF16 network kernels against
the FP64 numpy network oracle (forward and gradients), the trilinear transfers
against the oracle's, training, and warm-started solves (gain and fallback).

Tolerances: activations are stored in BF16 (8 significant bits, rounding
2^-9 relative) and re-read by every later layer, so the forward output and
the gradient vector are checked to 3e-2 relative (L2) with cosine similarity
>= 0.999 against the FP64 oracle; the FP64 transfers to 1e-12."""
import numpy as np
import pytest

import oracle as O
import oracle.no_oracle as NO
from paper_2502_03611_gb300.inputs import random_field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qn():
    import torch  # noqa: F401
    from paper_2502_03611_gb300 import build as B
    from paper_2502_03611_gb300 import qn as Q
    B.build()
    Q.load_library()
    return Q


def dev32(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32).reshape(-1)).cuda()


@pytest.mark.parametrize("m_from,m_to,B", [(255, 64, 1), (17, 9, 3), (9, 17, 2), (64, 255, 1)])
def test_interp3d_matches_oracle(qn, m_from, m_to, B):
    import torch
    src = random_field((B, m_from, m_from, m_from), 3)
    dst = torch.empty(B * m_to ** 3, dtype=torch.float64, device="cuda")
    qn.qn_interp3d(torch.from_numpy(src.reshape(-1)).cuda(), m_from, dst, m_to, B)
    got = dst.cpu().numpy().reshape(B, m_to, m_to, m_to)
    A = NO.interp_matrix(m_from, m_to)
    for b in range(B):
        want = np.einsum("pz,qy,rx,zyx->pqr", A, A, A, src[b], optimize=True)
        assert np.abs(got[b] - want).max() <= 1e-12 * max(1.0, np.abs(want).max())


@pytest.mark.parametrize("G,M,L,B", [(8, 3, 2, 2), (12, 4, 3, 3), (16, 6, 4, 2)])
def test_forward_and_gradients_match_oracle(qn, G, M, L, B):
    import torch
    C = 32
    net = qn.QnNet(G, M, L, max_batch=4)
    p = (random_field((net.nparams,), 21) * 0.2).astype(np.float64)
    p[:C] = random_field((C,), 22)          # lift weights O(1)
    net.set_params(p.astype(np.float32))
    pf = net.get_params().astype(np.float64)      # the parameters the GPU actually holds
    f = random_field((B, G, G, G), 23)
    t = random_field((B, G, G, G), 24) * 0.3
    out = torch.empty(B * G ** 3, dtype=torch.float32, device="cuda")
    net.forward(dev32(f), out, B)
    want_out, _ = NO.forward(pf, f, C, M, L)
    got_out = out.cpu().numpy().astype(np.float64).reshape(want_out.shape)
    rel = np.linalg.norm(got_out - want_out) / np.linalg.norm(want_out)
    assert rel < 3e-2, rel
    grads = torch.empty(net.nparams, dtype=torch.float32, device="cuda")
    loss = net.gradients(dev32(f), dev32(t), B, grads)
    want_loss, _, want_g = NO.loss_and_grads(pf, f, t, C, M, L)
    assert loss == pytest.approx(want_loss, rel=3e-2)
    g = grads.cpu().numpy().astype(np.float64)
    rel_g = np.linalg.norm(g - want_g) / np.linalg.norm(want_g)
    cos = float(g @ want_g / (np.linalg.norm(g) * np.linalg.norm(want_g)))
    assert rel_g < 3e-2 and cos > 0.999, (rel_g, cos)
    # every parameter group individually (a wrong index in one group would hide in the total)
    K = M ** 3
    sizes = [C, C] + [K * C * C, C * C, C] * L + [C, 1]
    o = 0
    for sz in sizes:
        a, b = g[o:o + sz], want_g[o:o + sz]
        if np.linalg.norm(b) > 1e-6 * np.linalg.norm(want_g):
            assert np.linalg.norm(a - b) / np.linalg.norm(b) < 6e-2
        o += sz


@pytest.mark.parametrize("G,M,L,n", [(16, 4, 2, 31), (12, 6, 3, 47), (64, 6, 4, 255), (10, 2, 1, 21)])
def test_fused_inference_matches_oracle_and_training_forward(qn, G, M, L, n):
    """qn_net_predict runs the fused inference kernels (analysis and mode mixing in one
    kernel, the synthesis with the pointwise path in another, the projection in the last
    block, the prolongation): against the FP64 oracle's restriction, network and
    prolongation at the BF16 tolerance, and against the unfused training forward on the
    same restricted input."""
    import torch
    C = 32
    net = qn.QnNet(G, M, L, max_batch=2)
    p = (random_field((net.nparams,), 51) * 0.2).astype(np.float64)
    p[:C] = random_field((C,), 52)
    net.set_params(p.astype(np.float32))
    pf = net.get_params().astype(np.float64)
    f = random_field((n, n, n), 53)
    fd = torch.from_numpy(f.reshape(-1)).cuda()
    U0 = torch.empty(n ** 3, dtype=torch.float64, device="cuda")
    in_scale, out_scale = 0.7, 1.3
    for _ in range(2):   # twice: the second call reuses the network's buffers
        net.predict(fd, n, U0, in_scale, out_scale)
    got = U0.cpu().numpy().reshape(n, n, n)
    Ar, Ap = NO.interp_matrix(n, G), NO.interp_matrix(G, n)
    fc = np.einsum("pz,qy,rx,zyx->pqr", Ar, Ar, Ar, f, optimize=True) * in_scale
    want_c, _ = NO.forward(pf, fc[None], C, M, L)
    want = np.einsum("pz,qy,rx,zyx->pqr", Ap, Ap, Ap, np.asarray(want_c).reshape(G, G, G), optimize=True) * out_scale
    rel = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert rel < 3e-2, rel
    fcd = torch.empty(G ** 3, dtype=torch.float32, device="cuda")
    qn.qn_interp3d(fd, n, fcd, G, 1, in_scale)
    out = torch.empty(G ** 3, dtype=torch.float32, device="cuda")
    net.forward(fcd, out, 1)
    unf = np.einsum("pz,qy,rx,zyx->pqr", Ap, Ap, Ap, out.cpu().numpy().astype(np.float64).reshape(G, G, G),
                    optimize=True) * out_scale
    assert np.linalg.norm(got - unf) / np.linalg.norm(unf) < 2e-2


def test_training_reduces_loss_and_warm_start_solves(qn):
    import torch
    from paper_2502_03611_gb300 import warmstart as W
    n, G = 47, 16
    ctx = qn.QnContext(3, n, "bf16x3")
    f_c, u_c, its = W.generate(ctx, G, n, range(0, 96), scale=100.0)
    out_scale = float(torch.sqrt(torch.mean(u_c.double() ** 2)))
    in_scale = 1.0 / float(torch.sqrt(torch.mean(f_c.double() ** 2)))
    net = qn.QnNet(G, 4, 2, max_batch=8)
    net.set_params(W.init_params(32, 4, 2))
    losses = W.train(net, f_c, u_c, in_scale, out_scale, epochs=15, batch=8, lr=3e-3)
    assert losses[-1] < 0.2 * losses[0], losses
    rows = W.evaluate(ctx, net, n, range(5000, 5006), 100.0, in_scale, out_scale)
    for r in rows:
        assert r["zero"]["status"] == 0 and r["warm"]["status"] == 0
        assert r["warm"]["rel"] <= 1e-10
        assert r["u0_rel_error"] < 0.2             # the network's U0 is close to the solution
        assert r["warm"]["used_warm"]
    s = W.summarise(rows)
    # on this strongly nonlinear variant (sources x100) the trained network must save iterations
    assert s["warm_iterations_mean"] < s["zero_iterations_mean"], s
    # the warm-started solution is the oracle's solution (same tolerances as every solve)
    from paper_2502_03611_gb300.inputs import grf_source
    f_np = grf_source(n, 5000, scale=100.0)
    U = torch.zeros(n ** 3, dtype=torch.float64, device="cuda")
    r = qn.qn_solve_warm(ctx, net, U, torch.from_numpy(f_np.reshape(-1)).cuda(), in_scale=in_scale,
                         out_scale=out_scale)
    assert r["status"] == 0 and r["used_warm"]
    Uo, ho, ok = O.qn_solve(f_np)
    assert ok
    Ug = U.cpu().numpy().reshape(f_np.shape)
    assert np.abs(Ug - Uo).max() <= 1e-9 * np.abs(Uo).max()
    assert np.linalg.norm(O.residual(Ug, f_np)) <= 1e-10 * np.linalg.norm(f_np)


def test_warm_start_falls_back_to_zero_start(qn):
    import torch
    from paper_2502_03611_gb300.inputs import grf_source_torch
    n, G = 31, 8
    ctx = qn.QnContext(3, n, "bf16x3")
    net = qn.QnNet(G, 2, 1, max_batch=1)
    p = random_field((net.nparams,), 5).astype(np.float32) * 1e3   # a corrupted network
    net.set_params(p)
    f = grf_source_torch(n, 7, scale=10.0).reshape(-1).contiguous()
    U = torch.zeros(n ** 3, dtype=torch.float64, device="cuda")
    res = qn.qn_solve_warm(ctx, net, U, f, out_scale=1.0)
    assert res["used_warm"] is False and res["status"] == 0 and res["rel"] <= 1e-10
    U2 = torch.zeros_like(U)
    res2, _ = qn.qn_solve(ctx, U2, f)
    assert res2["iterations"] == res["iterations"]
    assert torch.equal(U, U2)
