"""The whole-solve persistent kernel of small 2-D FP64 problems (qn_small.cu) against the
FP64 oracle and against the per-phase launches of the same solve (QN_SMALL=0).

Tolerances: FP64 throughout, so the iterates agree with the oracle's to the FP64 rounding
of the two summation orders: beta to 1e-12, U to 1e-12 of max|U|, the same iteration count,
and the relative residual of each iterate to 1e-6 (near convergence it is itself a ~1e-9
quantity formed from rounding-level differences) or 1e-13 absolute; the two GPU paths agree
to 1e-13 of max|U|.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import qn_oracle_bc as OB
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


def _solve(qn, n, f, prec="fp64", U0=None, profile=False, **kw):
    import torch
    ctx = qn.QnContext(2, n, prec, **{k: v for k, v in kw.items() if k in ("lam", "b", "bc", "length")})
    U = dev(U0).reshape(-1).clone() if U0 is not None else torch.zeros(n * n, dtype=torch.float64, device="cuda")
    if profile:
        qn.qn_profile_enable(ctx, True)
    opts = {k: v for k, v in kw.items() if k in ("tol", "max_it", "beta", "step", "sync_every", "graph", "check")}
    res, hist = qn.qn_solve(ctx, U, dev(f).reshape(-1), history_len=256, **opts)
    prof = qn.qn_profile_read(ctx)
    ctx.close()
    return res, hist, host(U).reshape(f.shape), prof


@pytest.mark.parametrize("n", [1, 2, 17, 63, 64, 100, 128])
def test_matches_oracle_and_launches_once(qn, n):
    _, f = I.manufactured_problem(n, 2, seed=7)
    res, hist, Ug, prof = _solve(qn, n, f)
    Uo, ho, ok = O.qn_solve(f, tol=1e-10)
    assert ok and res["status"] == 0 and res["rel"] <= 1e-10
    assert res["iterations"] == len(ho) - 1
    for a, b in zip(hist, ho):
        assert a["rel"] == pytest.approx(b["rel"], rel=1e-6, abs=1e-13)
        assert a["beta"] == pytest.approx(b["beta"], rel=1e-12, abs=1e-14)
    assert np.abs(Ug - Uo).max() <= 1e-12 * np.abs(Uo).max()
    # one kernel for the solve (the state-set and state-mirror kernels aside)
    assert prof["launches"] <= 4, prof


@pytest.mark.parametrize("seed", [0, 3])
def test_agrees_with_per_phase_launches(qn, monkeypatch, seed):
    n = 63
    _, f = I.manufactured_problem(n, 2, seed=seed)
    out = []
    for flag in ("1", "0"):
        monkeypatch.setenv("QN_SMALL", flag)
        res, hist, Ug, prof = _solve(qn, n, f)
        out.append((res, Ug, prof))
    assert out[0][0]["iterations"] == out[1][0]["iterations"]
    assert np.abs(out[0][1] - out[1][1]).max() <= 1e-13 * np.abs(out[1][1]).max()
    assert out[0][2]["launches"] < out[1][2]["launches"]


@pytest.mark.parametrize("beta,step", [(4.0, 1.0), (None, 0.8)])
def test_fixed_beta_and_damped_step(qn, beta, step):
    n = 40
    _, f = I.manufactured_problem(n, 2, seed=2)
    res, hist, Ug, _ = _solve(qn, n, f, beta=beta, step=step, max_it=400)
    Uo, ho, ok = O.qn_solve(f, tol=1e-10, beta=beta, step=step, max_it=400)
    assert ok and res["status"] == 0
    assert abs(res["iterations"] - (len(ho) - 1)) <= 1
    assert np.abs(Ug - Uo).max() <= 1e-11 * np.abs(Uo).max()


def test_neumann_with_linear_term(qn):
    """Sec. 6.2 Example 1 in 2-D: -Lap u + u + u^3 = f on (-1,1)^2, zero normal derivative."""
    n = 50
    u, f, h = I.ex2d1_problem(n)
    U0 = u + 0.1 * np.cos(0.5 * np.arange(n))[None, :] * np.ones((n, 1))
    res, hist, Ug, _ = _solve(qn, n, f, U0=U0, lam=1.0, b=1.0, bc="neumann", length=2.0)
    Uo, ho, ok = OB.qn_solve(f, h, "neumann", U0=U0, lam=1.0, b=1.0, tol=1e-10, max_it=200)
    assert ok and res["status"] == 0
    assert abs(res["iterations"] - (len(ho) - 1)) <= 1
    assert np.abs(Ug - Uo).max() <= 1e-11 * np.abs(Uo).max()


def test_status_codes(qn):
    n = 31
    _, f = I.manufactured_problem(n, 2, seed=1)
    res, hist, Ug, _ = _solve(qn, n, f, max_it=2, check=False)
    assert res["status"] == qn.QN_ENOTCONV and res["iterations"] == 2
    # beta = -5 lambda_min(A_h) makes A_h + beta I indefinite: the solve must stop as diverged
    lam_min = 2 * 4 * (n + 1) ** 2 * math.sin(math.pi / (2 * (n + 1))) ** 2
    res, hist, Ug, _ = _solve(qn, n, f, beta=-5 * lam_min, max_it=100, check=False)
    assert res["status"] == qn.QN_EDIVERGED and res["iterations"] < 100
    # a zero source converges at once
    res, hist, Ug, _ = _solve(qn, n, np.zeros((n, n)))
    assert res["status"] == 0 and res["iterations"] == 0 and not np.any(Ug)


def test_deterministic(qn):
    n = 63
    _, f = I.manufactured_problem(n, 2, seed=5)
    a = _solve(qn, n, f)[2]
    b = _solve(qn, n, f)[2]
    assert np.array_equal(a, b)
