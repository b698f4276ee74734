"""The six-product backward level (QN_PREC_BF16X6) against the FP64 oracle.

A BF16X3 correction's error is spread over all modes by the backward products and
A_h amplifies it by up to its stiffness ratio, so for a nearly linear problem the
precision, not the nonlinearity, sets the residual after each correction. BF16X6
forms the backward products from three-level operands (six BF16 products, FP32
accumulation) and keeps the forward products three-term.

Tolerances:
* one correction from the zero start (U_1 = A_h^{-1} f): U_1 to 5e-5 max|U_1|
  (the forward products' three-term error dominates the max norm, ~1e-5), and the
  error's residual ||A_h (U_1 - U_1,exact)|| at most 1/8 of BF16X3's (20x in emulation);
* solves: the FP64 tolerances of the parity tests (rel <= 1e-10 by the oracle's own
  residual, max|U - U_oracle| <= 1e-9 max|U_oracle|), and never more iterations than
  BF16X3.
Neumann data through this level: tests/test_gpu_neumann.py (Example 1 at n = 65, 128).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2502_03611_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qn():
    import torch  # noqa: F401
    from paper_2502_03611_gb300 import build as B
    from paper_2502_03611_gb300 import qn as Q
    B.build()
    Q.load_library()
    return Q


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.cpu().numpy()


def _first_correction(qn, prec, f, bc="dirichlet"):
    import torch
    n = f.shape[0]
    ctx = qn.QnContext(3, n, prec, bc=bc)
    U = torch.zeros(n ** 3, dtype=torch.float64, device="cuda")
    qn.qn_profile_enable(ctx, True)
    qn.qn_step(ctx, U, dev(f).reshape(-1))
    prof = qn.qn_profile_read(ctx)
    ctx.close()
    return host(U).reshape(f.shape), prof


@pytest.mark.parametrize("n", [65, 127, 128, 200])
@pytest.mark.parametrize("source", ["grf", "manufactured"])
def test_first_correction_matches_oracle(qn, n, source):
    """U_1 = (A_h)^{-1} f (beta = 0 at U_0 = 0) through the reflection-split products:
    odd and even n, P = 128 and 256, ragged tails."""
    f = I.grf_source(n, 100000) if source == "grf" else I.manufactured_problem(n, 3, seed=5)[1]
    S, Si, lam = O.eig_1d(n)
    want = O.fast_diag_solve(f, S, Si, lam, 0.0)
    U6, prof6 = _first_correction(qn, "bf16x6", f)
    U3, prof3 = _first_correction(qn, "bf16x3", f)
    assert prof6["split_products"] == 1 and prof3["split_products"] == 1
    m = np.abs(want).max()
    assert np.abs(U6 - want).max() <= 5e-5 * m
    # the error of the correction in the residual's units: ||A_h (U_1 - U_1,exact)|| / ||f||
    # (what the next iteration has to remove on top of the nonlinear term)
    fn = np.linalg.norm(f)
    e6 = np.linalg.norm(O.apply_laplacian(U6 - want)) / fn
    e3 = np.linalg.norm(O.apply_laplacian(U3 - want)) / fn
    assert e6 <= e3 / 8, (e6, e3)


@pytest.mark.parametrize("n,seed", [(127, 100000), (127, 100003), (200, 100001)])
def test_solve_grf_matches_oracle(qn, n, seed):
    import torch
    f = I.grf_source(n, seed)
    Uo, ho, ok = O.qn_solve(f, tol=1e-10)
    assert ok
    its = {}
    for prec in ("bf16x6", "bf16x3"):
        ctx = qn.QnContext(3, n, prec)
        U = torch.zeros(n ** 3, dtype=torch.float64, device="cuda")
        res, _ = qn.qn_solve(ctx, U, dev(f).reshape(-1), tol=1e-10)
        ctx.close()
        Ug = host(U).reshape(f.shape)
        assert res["status"] == 0 and res["rel"] <= 1e-10
        assert np.linalg.norm(O.residual(Ug, f)) / np.linalg.norm(f) <= 1.05e-10
        assert np.abs(Ug - Uo).max() <= 1e-9 * np.abs(Uo).max()
        its[prec] = res["iterations"]
    assert its["bf16x6"] <= its["bf16x3"]


@pytest.mark.parametrize("graph", [False, True])
def test_solve_manufactured_matches_oracle(qn, graph):
    """The strongly nonlinear manufactured family (rate set by the nonlinearity):
    the same solution, graph replay included."""
    import torch
    n = 127
    _, f = I.manufactured_problem(n, 3, seed=2)
    Uo, ho, ok = O.qn_solve(f, tol=1e-10)
    assert ok
    ctx = qn.QnContext(3, n, "bf16x6")
    U = torch.zeros(n ** 3, dtype=torch.float64, device="cuda")
    res, _ = qn.qn_solve(ctx, U, dev(f).reshape(-1), tol=1e-10, graph=graph, sync_every=2)
    Ug = host(U).reshape(f.shape)
    assert res["status"] == 0 and res["rel"] <= 1e-10
    assert np.linalg.norm(O.residual(Ug, f)) / np.linalg.norm(f) <= 1.05e-10
    assert np.abs(Ug - Uo).max() <= 1e-9 * np.abs(Uo).max()
    assert abs(res["iterations"] - (len(ho) - 1)) <= 1


def test_fewer_iterations_at_255_grf(qn):
    """Unit-variance GRF at 255^3 (the warm-start workload's sources): BF16X3 needs
    4 iterations, its first correction leaving ~2e-2 of ||f||; BF16X6 needs the
    FP64 count. Seed 100000 against the oracle's complete solve."""
    import torch
    n = 255
    fs = {s: I.grf_source(n, s) for s in (100000, 100001, 100002)}
    its = {"bf16x3": [], "bf16x6": []}
    sols = {}
    for prec in its:
        ctx = qn.QnContext(3, n, prec)
        for s, f in fs.items():
            U = torch.zeros(n ** 3, dtype=torch.float64, device="cuda")
            res, hist = qn.qn_solve(ctx, U, dev(f).reshape(-1), tol=1e-10, history_len=16)
            assert res["status"] == 0 and res["rel"] <= 1e-10
            its[prec].append(res["iterations"])
            if s == 100000:
                sols[prec] = host(U).reshape(f.shape)
        ctx.close()
    assert sum(its["bf16x6"]) < sum(its["bf16x3"]), its
    f = fs[100000]
    Uo, ho, ok = O.qn_solve(f, tol=1e-10)
    assert ok
    assert its["bf16x6"][0] <= len(ho) - 1
    Ug = sols["bf16x6"]
    assert np.linalg.norm(O.residual(Ug, f)) / np.linalg.norm(f) <= 1.05e-10
    assert np.abs(Ug - Uo).max() <= 1e-9 * np.abs(Uo).max()


@pytest.mark.parametrize("dim,n", [(2, 127), (3, 130), (3, 63)])
def test_unsupported_shapes_rejected(qn, dim, n):
    """No reflection-split products (2-D, or P not a multiple of 128): QN_EUNSUPPORTED
    at context creation, with a message."""
    with pytest.raises(RuntimeError, match="BF16X6"):
        qn.QnContext(dim, n, "bf16x6")


# --------------------------------------------------------------------------------------------
# precision escalation of BF16X3 solves (qn_set_escalation)
# --------------------------------------------------------------------------------------------
def _solve(qn, ctx, f, graph=False, sync_every=2):
    import torch
    n = f.shape[0]
    U = torch.zeros(n ** 3, dtype=torch.float64, device="cuda")
    res, hist = qn.qn_solve(ctx, U, dev(f).reshape(-1), tol=1e-10, graph=graph, sync_every=sync_every,
                            history_len=32)
    return res, hist, host(U).reshape(f.shape), qn.qn_profile_read(ctx)["x6_from"]


@pytest.mark.parametrize("n,graph", [(127, False), (255, True)])
def test_escalation_on_precision_bound_contraction(qn, n, graph):
    """GRF source (nearly linear): the first correction's contraction (~1e-2) is far above
    the nonlinear bound (~1e-4), so the solve switches at the first check (after
    iterations 0 and 1) and matches the oracle."""
    f = I.grf_source(n, 100002)
    ctx = qn.QnContext(3, n, "bf16x3")
    res3, h3, U3, at3 = _solve(qn, ctx, f, graph)
    assert at3 == -1
    qn.qn_set_escalation(ctx, 1e-3)
    res, hist, Ug, at = _solve(qn, ctx, f, graph)
    assert at == 2, (at, [x["rel"] for x in hist])
    assert res["status"] == 0 and res["rel"] <= 1e-10
    assert res["iterations"] <= res3["iterations"]
    # iterations 0 and 1 are the BF16X3 ones
    for a, b in zip(hist[:2], h3[:2]):
        assert a["rel"] == b["rel"]
    assert np.linalg.norm(O.residual(Ug, f)) / np.linalg.norm(f) <= 1.05e-10
    if n <= 127:
        Uo, ho, ok = O.qn_solve(f, tol=1e-10)
        assert ok
        assert np.abs(Ug - Uo).max() <= 1e-9 * np.abs(Uo).max()
    # off again: the BF16X3 iterates
    qn.qn_set_escalation(ctx, 0.0)
    res0, h0, U0, at0 = _solve(qn, ctx, f, graph)
    assert at0 == -1 and np.array_equal(U0, U3)
    ctx.close()


def test_escalation_stays_off_when_nonlinearity_bound(qn):
    """The manufactured family contracts at ~0.2 with a bound of ~0.26: the rate is the
    nonlinearity's, the solve stays at three products and gives the same iterates."""
    n = 127
    _, f = I.manufactured_problem(n, 3, seed=4)
    ctx = qn.QnContext(3, n, "bf16x3")
    res3, h3, U3, _ = _solve(qn, ctx, f)
    qn.qn_set_escalation(ctx, 1e-3)
    res, hist, Ug, at = _solve(qn, ctx, f)
    assert at == -1
    assert res["iterations"] == res3["iterations"] and np.array_equal(Ug, U3)
    ctx.close()


def test_escalation_arguments(qn):
    ctx6 = qn.QnContext(3, 65, "bf16x6")
    qn.qn_set_escalation(ctx6, 0.5)   # recorded; every iteration is at that level already
    res, hist, Ug, at = _solve(qn, ctx6, I.grf_source(65, 100001))
    assert at == 0 and res["status"] == 0
    ctx6.close()
    ctx = qn.QnContext(3, 65, "bf16x3")
    for bad in (-1.0, math.inf, math.nan):
        with pytest.raises(RuntimeError):
            qn.qn_set_escalation(ctx, bad)
    ctx.close()
    for dim, n, prec in ((2, 127, "bf16x3"), (3, 63, "bf16x3"), (3, 65, "fp64")):
        c = qn.QnContext(dim, n, prec)
        with pytest.raises(RuntimeError, match="reflection-split"):
            qn.qn_set_escalation(c, 0.5)
        qn.qn_set_escalation(c, 0.0)   # off is always accepted
        c.close()


def test_eigenproblem_at_six_products(qn):
    """The nonlinear eigenproblem (Sec. 4.4, Example 2 of Sec. 6.3) runs its shifted inverse
    through the same split products, so a BF16X6 context takes it at the six-product level:
    lambda and U against the oracle as for BF16X3 (tests/test_gpu_eig.py)."""
    import torch
    from oracle import qn_oracle_bc as ob
    n = 65
    v, h, x = I.ex2_problem(n)
    U0 = I.ex2_start(n, seed=1)
    Uo, lam_o, ho, ok = ob.qn_eig_solve(U0, h, "dirichlet", b=I.EX2_ALPHA, V=ob.potential(v, 3, n))
    assert ok
    its = {}
    for prec in ("bf16x6", "bf16x3"):
        ctx = qn.QnContext(3, n, prec, lam=0.0, b=I.EX2_ALPHA, bc="dirichlet", length=I.EX2_LENGTH, potential=v)
        U = dev(U0).reshape(-1).clone()
        res, _ = qn.qn_eig_solve(ctx, U)
        ctx.close()
        assert res["status"] == 0 and res["rel"] <= 1e-10, res
        assert res["lambda"] == pytest.approx(lam_o, rel=1e-9)
        Ug = host(U).reshape(U0.shape)
        assert np.abs(Ug - Uo).max() <= 1e-7 * np.abs(Uo).max()
        its[prec] = res["iterations"]
    assert its["bf16x6"] <= its["bf16x3"] + 2
