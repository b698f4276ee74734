"""C-ABI checks that need no GPU: the library builds and loads, exports every
entry point include/qn.h declares, its host-only 1-D diagonalisation matches
the oracle, and argument validation fails before anything is launched."""
import math
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qn.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2502_03611_gb300 import build as B
    from paper_2502_03611_gb300 import qn
    B.build()
    return qn.load_library()


def declared_entry_points():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qn_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_core_calls():
    names = declared_entry_points()
    for want in ("qn_setup_1d_eig", "qn_residual", "qn_step", "qn_solve", "qn_ctx_create",
                 "qn_fast_diag_solve"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2502_03611_gb300 import qn
    out = subprocess.run(["nm", "-D", "--defined-only", qn.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\sT\s(qn_[a-z0-9_]+)", out))
    missing = [s for s in declared_entry_points() if s not in exported]
    assert not missing, f"declared but not exported: {missing}"
    for s in declared_entry_points():
        assert hasattr(lib, s)


def test_version(lib):
    from paper_2502_03611_gb300 import qn
    assert qn.qn_version() >= 10000


@pytest.mark.parametrize("n", [1, 2, 7, 63, 255, 511])
def test_setup_1d_eig_matches_oracle(lib, n):
    import oracle as O
    from paper_2502_03611_gb300 import qn
    S, Si, lam = qn.qn_setup_1d_eig(n)
    So, _, lamo = O.eig_1d(n)
    assert np.abs(lam - lamo).max() <= 1e-12 * lamo.max()
    # eigenvectors are unique up to sign: compare |<s_k, o_k>| = 1 and validity
    dots = np.abs(np.sum(S * So, axis=0))
    assert np.abs(dots - 1.0).max() < 1e-10
    assert np.abs(Si @ S - np.eye(n)).max() < 1e-12
    H = O.fd_matrix_1d(n)
    assert np.abs(H @ S - S * lam[None, :]).max() < 1e-12 * lam.max()


@pytest.mark.parametrize("n", [2, 3, 8, 201])
def test_setup_1d_eig_neumann_matches_oracle(lib, n):
    """Closed-form cosine pairs of the library against the oracle's diagonalisation
    of the ghost-point matrix (Sec. 3.2 Neumann rows)."""
    from oracle import qn_oracle_bc as ob
    from paper_2502_03611_gb300 import qn
    h = 2.0 / (n - 1)
    S, Si, lam = qn.qn_setup_1d_eig(n, h, qn.QN_BC_NEUMANN)
    So, Sio, lamo = ob.eig_1d(n, h, "neumann")
    assert np.abs(lam - lamo).max() <= 1e-12 * lamo.max()
    assert np.abs(Si @ S - np.eye(n)).max() < 1e-12
    H = ob.fd_matrix_1d(n, h, "neumann")
    assert np.abs(H @ S - S * lam[None, :]).max() < 1e-12 * lam.max()
    # both normalise W^{1/2} S to orthonormal columns (W the trapezoid weights), so the
    # columns agree up to sign: |sum_j w_j S_jk So_jk| = 1
    w = ob.trapezoid_weights(n, "neumann")
    assert np.abs(np.abs(np.sum(w[:, None] * S * So, axis=0)) - 1.0).max() < 1e-10


def test_setup_rejects_bad_arguments(lib):
    from paper_2502_03611_gb300 import qn
    assert lib.qn_setup_1d_eig(0, 0.5, 0, None, None, None) == qn.QN_EINVAL
    assert lib.qn_setup_1d_eig(7, 0.0, 0, None, None, None) == qn.QN_EINVAL    # h must be > 0
    assert lib.qn_setup_1d_eig(7, -1.0, 1, None, None, None) == qn.QN_EINVAL
    assert lib.qn_setup_1d_eig(1, 0.5, 1, None, None, None) == qn.QN_EINVAL    # Neumann needs n >= 2
    assert lib.qn_setup_1d_eig(7, 0.125, 5, None, None, None) == qn.QN_EINVAL  # unknown bc
    assert "boundary" in qn.qn_last_error()


def test_ctx_create_validates_before_cuda(lib):
    import ctypes
    from paper_2502_03611_gb300 import qn
    h = ctypes.c_void_p()
    for prob in (qn.QnProblem(4, 10, 0, 0, 0.0, 1.0), qn.QnProblem(3, 0, 0, 0, 0.0, 1.0),
                 qn.QnProblem(3, 2000, 0, 0, 0.0, 1.0), qn.QnProblem(3, 10, 0, 9, 0.0, 1.0),
                 qn.QnProblem(3, 10, 0, 0, math.inf, 1.0), qn.QnProblem(3, 1, 1, 0, 0.0, 1.0),
                 qn.QnProblem(3, 10, 7, 0, 0.0, 1.0), qn.QnProblem(3, 10, 1, 0, 0.0, 1.0, -2.0),
                 qn.QnProblem(3, 10, 1, 0, 0.0, 1.0, math.nan)):
        assert lib.qn_ctx_create(ctypes.byref(prob), ctypes.byref(h)) == qn.QN_EINVAL
    bad = np.zeros(30)
    bad[17] = math.inf
    prob = qn.QnProblem(3, 10, 1, 0, 0.0, 1.0, 2.0, bad.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    assert lib.qn_ctx_create(ctypes.byref(prob), ctypes.byref(h)) == qn.QN_EINVAL
    assert "potential" in qn.qn_last_error()
    assert lib.qn_ctx_create(None, ctypes.byref(h)) == qn.QN_EINVAL
    assert lib.qn_residual(None, None, None, None, None, None) == qn.QN_EINVAL
    assert lib.qn_solve(None, None, None, None, None, None, 0, None) == qn.QN_EINVAL
    assert lib.qn_set_escalation(None, ctypes.c_double(1.0)) == qn.QN_EINVAL
    assert lib.qn_set_fused_residual(None, 1) == qn.QN_EINVAL
    assert lib.qn_set_fused_residual(None, 0) == qn.QN_EINVAL
    assert lib.qn_ctx_destroy(None) == qn.QN_OK


@pytest.mark.parametrize("n,k,bc", [(9, 1, 0), (15, 2, 0), (33, 4, 1), (59, 3, 0), (63, 8, 0), (41, 5, 1)])
def test_setup_1d_sem_matches_oracle(lib, n, k, bc):
    """The library's Q^k matrices (its own Gauss-Lobatto rule, assembly and symmetric
    eigensolver) against the oracle's (numpy Legendre roots, eigh)."""
    from oracle import qn_oracle_sem as so
    from paper_2502_03611_gb300 import qn
    L = 2.5
    H, S, Si, lam, x = qn.qn_setup_1d_sem(n, k, L, bc)
    bcs = "dirichlet" if bc == 0 else "neumann"
    So, Sio, lamo, Ho = so.eig_1d(n, k, L, bcs)
    _, _, xo = so.assemble_1d(n, k, L, bcs)
    assert np.abs(x - xo).max() < 1e-14 * L
    assert np.abs(H - Ho).max() <= 1e-11 * np.abs(Ho).max()
    assert np.abs(lam - lamo).max() <= 1e-11 * np.abs(lamo).max()
    assert np.abs(Si @ S - np.eye(n)).max() < 1e-11
    assert np.abs(H @ S - S * lam[None, :]).max() < 1e-11 * np.abs(lam).max()


def test_setup_1d_sem_large_and_rejects_bad_sizes(lib):
    import time
    from paper_2502_03611_gb300 import qn
    t0 = time.time()
    H, S, Si, lam, x = qn.qn_setup_1d_sem(511, 4, 1.0, 0)
    assert time.time() - t0 < 60
    assert np.all(np.diff(lam) >= 0) and lam[0] > 0
    assert np.abs(H @ S - S * lam[None, :]).max() < 1e-10 * lam.max()
    assert np.abs(Si @ S - np.eye(511)).max() < 1e-10
    assert lib.qn_setup_1d_sem(10, 4, 1.0, 0, None, None, None, None, None) == qn.QN_EINVAL   # 11 % 4 != 0
    assert lib.qn_setup_1d_sem(9, 0, 1.0, 0, None, None, None, None, None) == qn.QN_EINVAL
    assert lib.qn_setup_1d_sem(9, 2, -1.0, 0, None, None, None, None, None) == qn.QN_EINVAL


@pytest.mark.parametrize("n,kappa", [(2, 1.0), (3, 0.0), (9, 2.5), (40, 0.3)])
def test_setup_1d_robin_matches_oracle(lib, n, kappa):
    from oracle import qn_oracle_bc as ob
    from paper_2502_03611_gb300 import qn
    h = ob.mesh_width(n, "robin", 2.0)
    S, Si, lam = qn.qn_setup_1d_robin(n, h, kappa)
    _, _, lamo = ob.eig_1d(n, h, "robin", kappa)
    assert np.abs(lam - lamo).max() <= 1e-11 * np.abs(lamo).max()
    H = ob.fd_matrix_1d(n, h, "robin", kappa)
    assert np.abs(H @ S - S * lam[None, :]).max() < 1e-11 * np.abs(lam).max()
    assert np.abs(Si @ S - np.eye(n)).max() < 1e-12
