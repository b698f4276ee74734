"""FP64 CPU oracle for the learned warm start (test infrastructure only).

Plain numpy forward and backward passes of the small neural operator that
maps the source term f (on a coarse G^3 grid) to an initial iterate U_0, and
the trilinear transfer operators between the fine n^3 grid and the coarse
grid. Only tests (gradient checks, transfer checks) use it; the CUDA
training and inference kernels share no code with it.

The paper has no learned component; this part follows the network the warm
start is built on:

* sine basis (Dirichlet-consistent): Bm[j, k] = sqrt(2/(G+1)) sin(pi (j+1)(k+1)/(G+1)),
  j < G, k < M; its columns are orthonormal, so synthesis is the adjoint of
  analysis;
* layout of an activation: [batch, z, y, x, channel];
* lift:       h0 = f * wl + bl                                  (1 -> C channels)
* block l:    hh = analysis_xyz(h_l)                            (M^3 modes x C)
              g[k, o] = sum_i hh[k, i] R_l[k, i, o]             (per-mode channel mixing)
              z_l = synthesis_xyz(g) + h_l W_l + b_l
              h_{l+1} = gelu(z_l) for l < L-1, z_l for the last block
* projection: out = h_L wp + bp                                 (C -> 1)
* loss:       mean over batch and nodes of (out - target)^2
* gelu:       0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3)))

Flat parameter order: wl (C), bl (C), then per block R (M^3 C C, index
[kz, ky, kx, i, o]), W (C C, index [i, o]), b (C), then wp (C), bp (1).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["sine_analysis_basis", "gelu", "gelu_grad", "param_count", "unpack", "forward",
           "loss_and_grads", "interp_matrix", "restrict", "prolong"]

_GC = math.sqrt(2.0 / math.pi)


def sine_analysis_basis(G: int, M: int) -> np.ndarray:
    j = np.arange(1, G + 1)[:, None]
    k = np.arange(1, M + 1)[None, :]
    return math.sqrt(2.0 / (G + 1)) * np.sin(math.pi * j * k / (G + 1))


def gelu(x):
    return 0.5 * x * (1.0 + np.tanh(_GC * (x + 0.044715 * x ** 3)))


def gelu_grad(x):
    t = np.tanh(_GC * (x + 0.044715 * x ** 3))
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * _GC * (1.0 + 3 * 0.044715 * x * x)


def param_count(C: int, M: int, L: int) -> int:
    return 2 * C + L * (M ** 3 * C * C + C * C + C) + C + 1


def unpack(p: np.ndarray, C: int, M: int, L: int):
    p = np.asarray(p, dtype=np.float64)
    o = 0

    def take(k, shape):
        nonlocal o
        a = p[o:o + k].reshape(shape)
        o += k
        return a

    out = {"wl": take(C, (C,)), "bl": take(C, (C,)), "blocks": []}
    for _ in range(L):
        R = take(M ** 3 * C * C, (M, M, M, C, C))
        W = take(C * C, (C, C))
        b = take(C, (C,))
        out["blocks"].append((R, W, b))
    out["wp"] = take(C, (C,))
    out["bp"] = take(1, (1,))
    assert o == p.size
    return out


def _analysis(h, B):
    # h: [b, z, y, x, c] -> [b, kz, ky, kx, c]
    return np.einsum("zp,yq,xr,bzyxc->bpqrc", B, B, B, h, optimize=True)


def _synthesis(g, B):
    return np.einsum("zp,yq,xr,bpqrc->bzyxc", B, B, B, g, optimize=True)


def forward(p, f, C: int, M: int, L: int):
    """f: [batch, G, G, G]. Returns (out [batch, G, G, G], cache)."""
    P = unpack(p, C, M, L)
    G = f.shape[1]
    B = sine_analysis_basis(G, M)
    h = f[..., None] * P["wl"] + P["bl"]
    cache = {"f": f, "B": B, "h": [h], "z": [], "hh": []}
    for l, (R, W, b) in enumerate(P["blocks"]):
        hh = _analysis(h, B)
        g = np.einsum("bpqri,pqrio->bpqro", hh, R)
        z = _synthesis(g, B) + h @ W + b
        cache["hh"].append(hh)
        cache["z"].append(z)
        h = gelu(z) if l < L - 1 else z
        cache["h"].append(h)
    out = h @ P["wp"] + P["bp"][0]
    return out, cache


def loss_and_grads(p, f, target, C: int, M: int, L: int):
    """Mean-squared loss and its gradient with respect to the flat parameters."""
    P = unpack(p, C, M, L)
    out, cache = forward(p, f, C, M, L)
    N = out.size
    diff = out - target
    loss = float(np.sum(diff * diff) / N)
    dout = 2.0 * diff / N
    B = cache["B"]
    hL = cache["h"][L]
    g_wp = np.einsum("bzyxc,bzyx->c", hL, dout)
    g_bp = np.array([dout.sum()])
    dh = dout[..., None] * P["wp"]
    blocks_g = [None] * L
    for l in reversed(range(L)):
        R, W, b = P["blocks"][l]
        z = cache["z"][l]
        dz = dh * gelu_grad(z) if l < L - 1 else dh
        h_in = cache["h"][l]
        gW = np.einsum("bzyxi,bzyxo->io", h_in, dz)
        gb = dz.sum(axis=(0, 1, 2, 3))
        dg = _analysis(dz, B)                           # adjoint of synthesis
        gR = np.einsum("bpqri,bpqro->pqrio", cache["hh"][l], dg)
        dhh = np.einsum("bpqro,pqrio->bpqri", dg, R)
        dh = _synthesis(dhh, B) + dz @ W.T               # adjoint of analysis + pointwise path
        blocks_g[l] = (gR, gW, gb)
    g_wl = np.einsum("bzyx,bzyxc->c", cache["f"], dh)
    g_bl = dh.sum(axis=(0, 1, 2, 3))
    parts = [g_wl, g_bl]
    for gR, gW, gb in blocks_g:
        parts += [gR.ravel(), gW.ravel(), gb]
    parts += [g_wp, g_bp]
    return loss, out, np.concatenate([q.ravel() for q in parts])


# ---------------------------------------------------------------------------
# trilinear transfer between the fine n^3 and the coarse G^3 interior grids
# ---------------------------------------------------------------------------
def interp_matrix(m_from: int, m_to: int) -> np.ndarray:
    """1-D linear interpolation from nodes j/(m_from+1) (j = 1..m_from, zero at
    0 and 1) to nodes i/(m_to+1) (i = 1..m_to): matrix [m_to, m_from]."""
    A = np.zeros((m_to, m_from))
    for i in range(1, m_to + 1):
        t = i * (m_from + 1) / (m_to + 1)
        j0 = int(math.floor(t))
        w = t - j0
        if 1 <= j0 <= m_from:
            A[i - 1, j0 - 1] += 1.0 - w
        if 1 <= j0 + 1 <= m_from:
            A[i - 1, j0] += w
    return A


def _apply3(a, A):
    return np.einsum("pz,qy,rx,zyx->pqr", A, A, A, a, optimize=True)


def restrict(fine: np.ndarray, G: int) -> np.ndarray:
    """Trilinear interpolation of an n^3 interior field at the coarse nodes J/(G+1)."""
    return _apply3(fine, interp_matrix(fine.shape[0], G))


def prolong(coarse: np.ndarray, n: int) -> np.ndarray:
    """Trilinear interpolation of a G^3 interior field at the fine nodes i/(n+1)."""
    return _apply3(coarse, interp_matrix(coarse.shape[0], n))
