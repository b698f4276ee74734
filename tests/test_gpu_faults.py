"""Failure detection without a GPU fault. These are the library's status codes; the paper
has none.

* A tensor-core wait that runs out: the test hook makes one launch's producer withhold a
  stage. The bounded waits give up after 2 s, the solve returns QN_ETIMEOUT, and the same
  context then solves normally.
* A fixed beta below -lambda_min(A_h) makes (A_h + beta I) indefinite, and the iteration
  blows up. The solve reports QN_EDIVERGED instead of running to max_it.
"""
import time

import numpy as np
import pytest

import oracle as O
from paper_2502_03611_gb300.inputs import manufactured_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qn():
    import torch  # noqa: F401
    from paper_2502_03611_gb300 import build as B
    from paper_2502_03611_gb300 import qn as Q
    B.build()
    Q.load_library()
    return Q


def _problem(n, seed):
    import torch
    u, f = manufactured_problem(n, 2, seed=seed)
    fd = torch.from_numpy(np.ascontiguousarray(f.reshape(-1))).cuda()
    U = torch.zeros(n * n, dtype=torch.float64, device="cuda")
    return f, fd, U


def test_withheld_arrival_times_out_and_context_recovers(qn):
    n = 63
    f, fd, U = _problem(n, 5)
    ctx = qn.QnContext(2, n, "bf16x3")
    qn.qn_test_withhold_arrival()
    t0 = time.time()
    with pytest.raises(qn.QnError) as e:
        qn.qn_solve(ctx, U, fd)
    assert e.value.code == qn.QN_ETIMEOUT
    assert time.time() - t0 >= 1.5          # the waits ran to their 2 s limit
    # the hook affected one launch only: the same context now solves as usual
    U.zero_()
    out, _ = qn.qn_solve(ctx, U, fd)
    assert out["status"] == qn.QN_OK and out["rel"] <= 1e-10
    Uo, _, ok = O.qn_solve(f)
    assert ok
    assert np.abs(U.cpu().numpy().reshape(n, n) - Uo).max() <= 1e-9 * np.abs(Uo).max()


@pytest.mark.parametrize("precision", ["bf16x3", "fp64"])
def test_fixed_beta_below_minus_lambda_min_diverges(qn, precision):
    n = 63
    f, fd, U = _problem(n, 6)
    # lambda_min(A_h) = 2 (4/h^2) sin^2(pi h / 2) ~ 2 pi^2 ~ 19.7 on the unit square
    h = 1.0 / (n + 1)
    lam_min = 2 * 4 / h ** 2 * np.sin(np.pi * h / 2) ** 2
    ctx = qn.QnContext(2, n, precision)
    out, _ = qn.qn_solve(ctx, U, fd, beta=-5.0 * lam_min, max_it=100)
    assert out["status"] == qn.QN_EDIVERGED
    assert out["iterations"] < 100
