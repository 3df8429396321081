"""Learned right preconditioner M: a linear, gauge-equivariant parallel-transport
convolution (PTC) network, float64 (test infrastructure).

One layer maps C_in to C_out quark-field channels:

    out[c](x) = sum_{h in HOPS} sum_{c'} W[h, c, c'] (T_h in[c'])(x),

with HOPS = (0, +x, -x, +y, -y, +z, -z, +t, -t), T_0 = 1,
T_{+mu} f(x) = U_mu(x) f(x + mu), T_{-mu} f(x) = U_mu(x - mu)^+ f(x - mu) (the fermion
boundary phase multiplies hops that wrap, as in the Wilson matrix), and
W[h, c, c'] a complex 4x4 matrix acting on spin (colour is acted on only by
the transport). M = L2 o L1 with channels 1 -> 12 -> 1; it acts on an even-site
vector embedded in the full lattice (odd sites zero) and its output is
restricted to the even sites. There is no activation: M is a fixed linear
operator, used as a right preconditioner of the even-odd operator A.

Training loss over samples (v, y = A^{-1} v):
    L = sum |M v - y|^2 / |y|^2 + mu sum |A M v - v|^2 / |v|^2.
Weight gradients come from torch autograd on this float64 definition; the
tests pin them by central finite differences.
"""

from __future__ import annotations

import torch

from . import wilson as W

CDT = torch.complex128
HOPS = [(None, 0), (0, 1), (0, -1), (1, 1), (1, -1), (2, 1), (2, -1), (3, 1), (3, -1)]
C_MID = 12


def transport(U, f, hop, bc=(1, 1, 1, -1)):
    """T_h f for f of shape [..., Lt, Lz, Ly, Lx, 4, 3] (leading channel axes allowed)."""
    mu, step = hop
    if mu is None:
        return f
    ax = f.dim() - 6 + (3 - mu)          # lattice axis of direction mu
    L = f.shape[ax]
    g = torch.roll(f, shifts=-step, dims=ax)
    if bc[mu] != 1:
        idx = [slice(None)] * g.dim()
        idx[ax] = L - 1 if step > 0 else 0
        g = g.clone()
        g[tuple(idx)] = g[tuple(idx)] * bc[mu]
    if step > 0:
        return g @ U[mu].transpose(-1, -2)                 # U_mu(x) f(x+mu)
    u_back = torch.roll(U[mu], shifts=1, dims=3 - mu)      # U_mu(x-mu)
    return g @ u_back.conj()                               # U_mu(x-mu)^+ f(x-mu)


def layer(U, w, f, bc=(1, 1, 1, -1)):
    """w: [9, C_out, C_in, 4, 4] complex; f: [C_in, Lt, Lz, Ly, Lx, 4, 3] -> [C_out, ...]."""
    out = None
    for k, hop in enumerate(HOPS):
        t = transport(U, f, hop, bc)                       # [C_in, ..., 4, 3]
        term = torch.einsum("oist,i...tc->o...sc", w[k], t)
        out = term if out is None else out + term
    return out


def apply(U, w1, w2, psi_e, bc=(1, 1, 1, -1)):
    """M psi_e: even input embedded in the full lattice, output restricted to even sites."""
    f = W.restrict(psi_e, 0)[None]
    h = layer(U, w1, f, bc)
    return W.restrict(layer(U, w2, h, bc)[0], 0)


def identity_weights(c_mid: int = C_MID):
    """W1[0, 0, 0] = W2[0, 0, 0] = 1 (spin identity), all else 0: M = 1."""
    w1 = torch.zeros((9, c_mid, 1, 4, 4), dtype=CDT)
    w2 = torch.zeros((9, 1, c_mid, 4, 4), dtype=CDT)
    w1[0, 0, 0] = torch.eye(4, dtype=CDT)
    w2[0, 0, 0] = torch.eye(4, dtype=CDT)
    return w1, w2


def random_weights(seed: int, scale: float = 0.1, c_mid: int = C_MID):
    """Identity weights plus complex Gaussian noise of the given scale (seeded)."""
    g = torch.Generator().manual_seed(seed)
    w1, w2 = identity_weights(c_mid)
    w1 = w1 + scale * torch.randn(w1.shape, dtype=CDT, generator=g)
    w2 = w2 + scale * torch.randn(w2.shape, dtype=CDT, generator=g)
    return w1, w2


def loss(U, w1, w2, vs, ys, kappa, mu, bc=(1, 1, 1, -1)):
    """Training loss over samples (v, y = A^{-1} v), both even-site fields."""
    tot = 0.0
    for v, y in zip(vs, ys):
        m = apply(U, w1, w2, v, bc)
        e1 = m - y
        e2 = W.eo_operator(U, m, kappa, bc) - W.restrict(v, 0)
        tot = tot + (e1.abs() ** 2).sum() / (y.abs() ** 2).sum() + mu * (e2.abs() ** 2).sum() / (v.abs() ** 2).sum()
    return tot


def grads(U, w1, w2, vs, ys, kappa, mu, bc=(1, 1, 1, -1)):
    """(L, dL/dW1, dL/dW2) with dL/dW = dL/dRe W + i dL/dIm W."""
    a = w1.clone().requires_grad_(True)
    b = w2.clone().requires_grad_(True)
    L = loss(U, a, b, vs, ys, kappa, mu, bc)
    L.backward()
    # torch returns the conjugate Wirtinger form dL/d conj(w) * 2 = dL/dRe + i dL/dIm
    return float(L.item()), a.grad.detach(), b.grad.detach()


# --- flat weight layout shared with the C ABI (see include/wd.h) --------------

def to_flat(w1, w2) -> torch.Tensor:
    """float32-ready flat layout: W1 as [9][12][4][4][2], then W2 as [9][12][4][4][2]."""
    a = torch.view_as_real(w1[:, :, 0].contiguous()).reshape(-1)
    b = torch.view_as_real(w2[:, 0, :].contiguous()).reshape(-1)
    return torch.cat([a, b])


def from_flat(flat: torch.Tensor, c_mid: int = C_MID):
    n = 9 * c_mid * 16 * 2
    a = torch.view_as_complex(flat[:n].to(torch.float64).reshape(9, c_mid, 4, 4, 2).contiguous())
    b = torch.view_as_complex(flat[n:2 * n].to(torch.float64).reshape(9, c_mid, 4, 4, 2).contiguous())
    return a[:, :, None], b[:, None, :]
