"""Pins of the oracle's clover term (Sheikholeslami-Wohlert) and of the
even-odd system with clover diagonal blocks (Eqs. 4-5 with D_ee = C_ee,
D_oo = C_oo)."""

import numpy as np
import pytest
import torch

from oracle import clover as cl
from oracle import solvers as S
from oracle import wilson as w
from paper_2602_14450_gb300 import synth

BC = (1, 1, 1, -1)
CSW = 1.0


def rand_field(dims, seed):
    g = torch.Generator().manual_seed(seed)
    lx, ly, lz, lt = dims
    return torch.randn((lt, lz, ly, lx, 4, 3), dtype=torch.complex128, generator=g)


def test_free_field_clover_is_identity():
    dims = (4, 4, 4, 4)
    c = cl.clover_matrix(synth.gauge_unit(dims), CSW, 0.13)
    assert torch.allclose(c, torch.eye(12, dtype=torch.complex128).expand_as(c), atol=1e-15, rtol=0)


def test_clover_hermitian_and_leaf_orientation():
    dims = (4, 2, 4, 6)
    u = synth.gauge_random(dims, 0.5, seed=21)
    c = cl.clover_matrix(u, CSW, 0.13)
    assert torch.allclose(c, c.conj().transpose(-1, -2), atol=1e-14, rtol=0)
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            # swapping the plane reverses every loop: Q_nu_mu = Q_mu_nu^+
            q1, q2 = cl.clover_leaves(u, mu, nu), cl.clover_leaves(u, nu, mu)
            assert torch.allclose(q2, q1.conj().transpose(-1, -2), atol=1e-13, rtol=0)
            # every plaquette is a leaf of its four corners
            tot = torch.diagonal(q1, dim1=-2, dim2=-1).sum(-1).real.sum()
            assert abs(tot - 4 * cl.plaquette_sum(u, mu, nu)) <= 1e-10 * abs(tot)


def test_abelian_field_strength_closed_form():
    """Diagonal (commuting) links diag(e^{i a}, e^{i b}, e^{-i(a+b)}): every
    leaf is exp(i phi) with phi the oriented sum of angles around its
    plaquette, so Fh = traceless part of sum over the four corners of
    sin(phi) / 4 -- written here directly from the angles."""
    dims = (4, 6, 4, 2)
    lx, ly, lz, lt = dims
    rng = np.random.default_rng(7)
    ang = rng.uniform(-np.pi, np.pi, size=(4, 2, lt, lz, ly, lx))
    th = np.concatenate([ang, -ang.sum(axis=1, keepdims=True)], axis=1)   # [mu, k, t, z, y, x]
    u = torch.zeros((4, lt, lz, ly, lx, 3, 3), dtype=torch.complex128)
    for k in range(3):
        u[:, :, :, :, :, k, k] = torch.from_numpy(np.exp(1j * th[:, k]))

    def shift(a, mu, step):            # a(x + step mu) on [t, z, y, x]
        return np.roll(a, -step, axis=3 - mu)

    for mu, nu in [(0, 1), (0, 3), (1, 2), (2, 3)]:
        want = np.zeros((3, lt, lz, ly, lx))
        for k in range(3):
            phi = th[mu, k] + shift(th[nu, k], mu, 1) - shift(th[mu, k], nu, 1) - th[nu, k]
            corners = [phi, shift(phi, mu, -1), shift(phi, nu, -1), shift(shift(phi, mu, -1), nu, -1)]
            want[k] = sum(np.sin(c) for c in corners) / 4
        want -= want.mean(axis=0, keepdims=True)
        got = cl.field_strength(u, mu, nu)
        for k in range(3):
            assert np.allclose(got[..., k, k].numpy(), want[k], atol=1e-14)
        off = got - torch.diag_embed(torch.diagonal(got, dim1=-2, dim2=-1))
        assert off.abs().max() == 0


def test_clover_gauge_covariance_and_gamma5_hermiticity():
    dims = (4, 2, 4, 6)
    u = synth.gauge_random(dims, 0.5, seed=5)
    g = synth.gauge_transform_field(dims, seed=6)
    ug = torch.empty_like(u)
    for mu in range(4):
        g_next = torch.roll(g, shifts=-1, dims=3 - mu)
        ug[mu] = g @ u[mu] @ g_next.conj().transpose(-1, -2)
    kappa = 0.124
    c, cg = cl.clover_matrix(u, CSW, kappa), cl.clover_matrix(ug, CSW, kappa)
    psi, chi = rand_field(dims, 7), rand_field(dims, 8)
    lhs = cl.dirac_sw(ug, cg, psi @ g.transpose(-1, -2), kappa, BC)
    rhs = cl.dirac_sw(u, c, psi, kappa, BC) @ g.transpose(-1, -2)
    assert torch.allclose(lhs, rhs, atol=1e-12, rtol=0)
    from oracle.gamma import gamma5
    g5 = gamma5()
    g5d = (g5 @ cl.dirac_sw(u, c, g5 @ psi, kappa, BC))
    assert abs(S.dot(chi, g5d) - S.dot(cl.dirac_sw(u, c, chi, kappa, BC), psi)) <= 1e-11 * S.norm(psi) * S.norm(chi)


@pytest.mark.parametrize("dims", [(2, 2, 2, 4), (4, 2, 2, 2)])
def test_even_odd_clover_solve_equals_lu(dims):
    """Eqs. 4-5 with clover blocks: BiCGStab on A = 1 - kappa^2 C_ee^-1 H_eo C_oo^-1 H_oe
    and the odd reconstruction give the LU solution of the dense D_sw."""
    u = synth.gauge_random(dims, 0.5, seed=31)
    kappa = 0.12
    c = cl.clover_matrix(u, CSW, kappa)
    cinv = torch.linalg.inv(c)
    eta = rand_field(dims, 32)
    n = eta.numel()
    cols = []
    for j in range(n):
        e = torch.zeros(n, dtype=torch.complex128)
        e[j] = 1
        cols.append(cl.dirac_sw(u, c, e.reshape(eta.shape), kappa, BC).reshape(-1))
    dense = torch.stack(cols, dim=1)
    want = torch.linalg.solve(dense, eta.reshape(-1)).reshape(eta.shape)
    b = cl.eo_source_sw(u, cinv, eta, kappa, BC)
    xe, info = S.bicgstab(lambda f: cl.eo_operator_sw(u, cinv, f, kappa, BC), b, 1e-14, bref=S.norm(b))
    assert info.converged
    got = cl.eo_reconstruct_sw(u, cinv, xe, eta, kappa, BC)
    assert S.norm(got - want) / S.norm(want) <= 1e-11
    assert S.norm(eta - cl.dirac_sw(u, c, got, kappa, BC)) / S.norm(eta) <= 1e-11
