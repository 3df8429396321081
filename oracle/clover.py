"""Clover (Sheikholeslami-Wohlert) term and the even-odd system with
non-trivial diagonal blocks, float64 -- test infrastructure only.

The paper uses the plain Wilson matrix and names the clover matrix as the
next one to study (Sec. 7); its even-odd equations (Eqs. 4-5) are written for
general diagonal blocks D_ee, D_oo. With the clover term the Wilson-clover
matrix is

    D_sw = C - kappa H,   C(x) = 1 - c_sw kappa sum_{mu<nu} sigma_mu_nu (x) Fh_mu_nu(x),

a site-local 12 x 12 Hermitian block C (spin x colour) with
sigma_mu_nu = (i/2) [gamma_mu, gamma_nu] and the four-leaf clover field
strength Fh_mu_nu = traceless part of (Q_mu_nu - Q_mu_nu^+) / (8 i), Q the sum
of the four plaquettes of the mu-nu plane that touch x, all oriented
mu-then-nu. The links are periodic; the fermion boundary phases enter only
through H. Then D_ee = C_ee, D_oo = C_oo, D_eo = -kappa H_eo, and Eqs. 4-5 read

    A = 1 - kappa^2 C_ee^{-1} H_eo C_oo^{-1} H_oe,
    b^ = C_ee^{-1} (eta_e + kappa H_eo C_oo^{-1} eta_o),
    xi_o = C_oo^{-1} (eta_o + kappa H_oe xi_e).

Matrices are [Lt, Lz, Ly, Lx, 12, 12] complex128 with the spin-colour index
3 s + a; a quark field [..., 4, 3] is flattened to [..., 12] for them.
"""

from __future__ import annotations

import torch

from .gamma import gammas
from .wilson import _neighbour, hop, hop_pq, restrict

CDT = torch.complex128


def _dag(m: torch.Tensor) -> torch.Tensor:
    return m.conj().transpose(-1, -2)


def _sh(f: torch.Tensor, mu: int, step: int) -> torch.Tensor:
    """f(x + step mu-hat) for a periodic link field."""
    return _neighbour(f, mu, step, 1)


def clover_leaves(U: torch.Tensor, mu: int, nu: int) -> torch.Tensor:
    """Q_mu_nu(x): the four plaquettes of the mu-nu plane with a corner at x,
    each traversed mu-then-nu (counterclockwise), as closed loops from x."""
    um, un = U[mu], U[nu]
    l1 = um @ _sh(un, mu, 1) @ _dag(_sh(um, nu, 1)) @ _dag(un)
    l2 = un @ _dag(_sh(_sh(um, mu, -1), nu, 1)) @ _dag(_sh(un, mu, -1)) @ _sh(um, mu, -1)
    l3 = _dag(_sh(um, mu, -1)) @ _dag(_sh(_sh(un, mu, -1), nu, -1)) @ _sh(_sh(um, mu, -1), nu, -1) @ _sh(un, nu, -1)
    l4 = _dag(_sh(un, nu, -1)) @ _sh(um, nu, -1) @ _sh(_sh(un, nu, -1), mu, 1) @ _dag(um)
    return l1 + l2 + l3 + l4


def field_strength(U: torch.Tensor, mu: int, nu: int) -> torch.Tensor:
    """Fh_mu_nu(x): traceless part of (Q - Q^+) / (8 i), a Hermitian 3 x 3 per site."""
    q = clover_leaves(U, mu, nu)
    f = (q - _dag(q)) / 8j
    tr = torch.diagonal(f, dim1=-2, dim2=-1).sum(-1)
    return f - (tr / 3)[..., None, None] * torch.eye(3, dtype=CDT)


def sigma(mu: int, nu: int) -> torch.Tensor:
    g = gammas()
    return 0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])


def clover_matrix(U: torch.Tensor, csw: float, kappa: float) -> torch.Tensor:
    """C(x) = 1 - c_sw kappa sum_{mu<nu} sigma_mu_nu (x) Fh_mu_nu(x), [..., 12, 12]."""
    shape = U.shape[1:5]
    c = torch.zeros(shape + (4, 3, 4, 3), dtype=CDT)
    for mu in range(4):
        for nu in range(mu + 1, 4):
            f = field_strength(U, mu, nu)
            c -= csw * kappa * torch.einsum("st,...ab->...satb", sigma(mu, nu), f)
    c = c.reshape(shape + (12, 12))
    return c + torch.eye(12, dtype=CDT)


def apply_block(C: torch.Tensor, psi: torch.Tensor) -> torch.Tensor:
    """(C psi)(x) site by site."""
    flat = psi.reshape(psi.shape[:4] + (12,))
    return (C @ flat[..., None])[..., 0].reshape(psi.shape)


def dirac_sw(U, C, psi, kappa: float, bc=(1, 1, 1, -1)) -> torch.Tensor:
    """D_sw psi = C psi - kappa H psi."""
    return apply_block(C, psi) - kappa * hop(U, psi, bc)


def eo_operator_sw(U, Cinv, psi_e, kappa: float, bc=(1, 1, 1, -1)) -> torch.Tensor:
    """A psi_e = psi_e - kappa^2 C_ee^{-1} H_eo C_oo^{-1} H_oe psi_e (Eq. 4 with the clover blocks)."""
    t = restrict(apply_block(Cinv, hop_pq(U, psi_e, 1, bc)), 1)
    return restrict(psi_e, 0) - kappa * kappa * restrict(apply_block(Cinv, hop_pq(U, t, 0, bc)), 0)


def eo_source_sw(U, Cinv, eta, kappa: float, bc=(1, 1, 1, -1)) -> torch.Tensor:
    """b^ = C_ee^{-1} (eta_e + kappa H_eo C_oo^{-1} eta_o) (right-hand side of Eq. 4)."""
    t = restrict(apply_block(Cinv, restrict(eta, 1)), 1)
    return restrict(apply_block(Cinv, restrict(eta, 0) + kappa * hop_pq(U, t, 0, bc)), 0)


def eo_reconstruct_sw(U, Cinv, xi_e, eta, kappa: float, bc=(1, 1, 1, -1)) -> torch.Tensor:
    """Eq. 5: xi_o = C_oo^{-1} (eta_o + kappa H_oe xi_e); returns xi_e + xi_o."""
    xi_o = restrict(apply_block(Cinv, restrict(eta, 1) + kappa * hop_pq(U, xi_e, 1, bc)), 1)
    return restrict(xi_e, 0) + xi_o


def plaquette_sum(U: torch.Tensor, mu: int, nu: int) -> torch.Tensor:
    """sum_x Re tr P_mu_nu(x) with P_mu_nu(x) = U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+."""
    p = U[mu] @ _sh(U[nu], mu, 1) @ _dag(_sh(U[mu], nu, 1)) @ _dag(U[nu])
    return torch.diagonal(p, dim1=-2, dim2=-1).sum(-1).real.sum()
