"""Pins for the warm-start network oracle (oracle/no_oracle.py) and the GRF
generator: finite differences for every parameter's gradient, a closed-form
special case of the spectral block, orthonormality of the sine basis,
exactness and second-order accuracy of the trilinear transfers, and the GRF's
normalisation and spectrum."""
import math

import numpy as np
import pytest

import oracle.no_oracle as N
from paper_2502_03611_gb300.inputs import (grf_coeffs, grf_source, grid_points, mode_wavenumber_sq,
                                           random_field, sine_series)


def test_sine_basis_orthonormal():
    for G, M in ((8, 3), (64, 6), (5, 5)):
        B = N.sine_analysis_basis(G, M)
        assert np.abs(B.T @ B - np.eye(M)).max() < 1e-13


def test_gelu_derivative_by_finite_differences():
    x = np.linspace(-4, 4, 41)
    h = 1e-6
    fd = (N.gelu(x + h) - N.gelu(x - h)) / (2 * h)
    assert np.abs(fd - N.gelu_grad(x)).max() < 1e-8
    assert N.gelu(0.0) == 0.0
    assert abs(N.gelu(10.0) - 10.0) < 1e-6 and abs(N.gelu(-10.0)) < 1e-6


def _params(C, M, L, seed, scale=0.3):
    return random_field((N.param_count(C, M, L),), seed) * scale


@pytest.mark.parametrize("C,M,L", [(3, 2, 2), (2, 3, 1)])
def test_gradients_by_finite_differences(C, M, L):
    G, B = 5, 2
    p = _params(C, M, L, 7)
    f = random_field((B, G, G, G), 8)
    t = random_field((B, G, G, G), 9) * 0.5
    loss, _, g = N.loss_and_grads(p, f, t, C, M, L)
    h = 1e-5
    fd = np.empty_like(g)
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = h
        lp = N.loss_and_grads(p + e, f, t, C, M, L)[0]
        lm = N.loss_and_grads(p - e, f, t, C, M, L)[0]
        fd[i] = (lp - lm) / (2 * h)
    # central differences are accurate to O(h^2) plus rounding ~1e-16/h
    err = np.abs(fd - g)
    assert err.max() <= 1e-7 * np.abs(g).max(), err.max() / np.abs(g).max()


def test_spectral_block_projects_on_low_modes():
    # C = 1, one block, R = 1 on every mode, W = 0, b = 0, identity lift and
    # projection: out = synthesis(analysis(f)) keeps sine modes <= M, drops the rest
    G, M = 9, 3
    C, L = 1, 1
    p = np.zeros(N.param_count(C, M, L))
    P = N.unpack(p, C, M, L)   # views into p
    P["wl"][:] = 1.0
    P["blocks"][0][0][:] = 1.0
    P["wp"][:] = 1.0
    x = np.arange(1, G + 1) / (G + 1)

    def mode(k):
        s = [np.sin(ki * math.pi * x) for ki in k]
        return np.einsum("z,y,x->zyx", s[2], s[1], s[0])

    for k, keep in (((1, 2, 3), True), ((3, 3, 1), True), ((4, 1, 1), False), ((2, 5, 9), False)):
        f = mode(k)[None]
        out, _ = N.forward(p, f, C, M, L)
        want = f if keep else np.zeros_like(f)
        assert np.abs(out - want).max() < 1e-12


def test_interp_identity_and_linear_exactness():
    assert np.abs(N.interp_matrix(7, 7) - np.eye(7)).max() < 1e-15
    # a function that is linear between the coarse nodes (hat functions) is interpolated exactly
    m_from, m_to = 5, 17
    A = N.interp_matrix(m_from, m_to)
    xf = np.arange(1, m_from + 1) / (m_from + 1)
    xt = np.arange(1, m_to + 1) / (m_to + 1)
    for j in range(m_from):
        a = np.zeros(m_from)
        a[j] = 1.0
        hat = np.maximum(0.0, 1.0 - np.abs(xt - xf[j]) * (m_from + 1))
        assert np.abs(A @ a - hat).max() < 1e-14


def test_transfer_second_order():
    def field(m):
        x = np.arange(1, m + 1) / (m + 1)
        s = np.sin(math.pi * x)
        return np.einsum("z,y,x->zyx", s, s * s, s)

    errs = []
    for G in (8, 16, 32):
        fine = field(63)
        back = N.prolong(N.restrict(fine, G), 63)
        errs.append(np.abs(back - fine).max())
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0, errs


def test_grf_unit_variance_and_spectrum():
    f = grf_source(31, 3)
    assert abs(np.sqrt(np.mean(f * f)) - 1.0) < 1e-12
    # coefficient amplitudes follow (1 + |k|^2)^-1: the sample variance of
    # c_k (1 + |k|^2) over many modes is ~1
    c = grf_coeffs(11, 16)
    z = c * (1.0 + mode_wavenumber_sq(16, 3))
    assert abs(np.var(z) - 1.0) < 0.06 and abs(np.mean(z)) < 0.06
    # the field is the sine series of those coefficients
    g = sine_series(grf_coeffs(3), 31)
    assert np.abs(f - g / np.sqrt(np.mean(g * g))).max() < 1e-12
