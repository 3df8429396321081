"""Pins of the oracle's Wilson matrix (Eq. 1) and even-odd form (Eqs. 4-5).

Each check is fixed by mathematics, not by re-running the oracle's formula:
dense block assembly, gamma5-hermiticity, gauge covariance, free-field plane
waves, and LU solves of the dense matrix.
"""

import math

import pytest
import torch

from oracle import wilson as w
from oracle.gamma import gamma5, gammas
from paper_2602_14450_gb300 import synth

BC = (1, 1, 1, -1)
CDT = torch.complex128


def rand_field(dims, seed):
    return synth.gaussian_source(dims, seed)


def inner(a, b):
    return torch.vdot(a.reshape(-1), b.reshape(-1))


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 2, 4, 2)])
def test_dense_columns_match_block_assembly(dims):
    u = synth.gauge_random(dims, 0.7, seed=3)
    kappa = 0.13
    a = w.dense_by_columns(u, kappa, BC)
    b = w.dense_by_blocks(u, kappa, BC)
    assert torch.allclose(a, b, atol=1e-14, rtol=0)


def test_gamma5_hermiticity():
    dims = (4, 4, 4, 4)
    u = synth.gauge_random(dims, 0.5, seed=11)
    chi, psi = rand_field(dims, 1), rand_field(dims, 2)
    g5 = gamma5()
    lhs = inner(chi, g5 @ w.dirac(u, g5 @ psi, 0.12, BC))
    rhs = inner(w.dirac(u, chi, 0.12, BC), psi)
    assert abs(lhs - rhs) <= 1e-12 * abs(rhs)


def test_gauge_covariance():
    dims = (4, 2, 4, 6)
    u = synth.gauge_random(dims, 0.5, seed=5)
    g = synth.gauge_transform_field(dims, seed=6)
    ug = torch.empty_like(u)
    for mu in range(4):
        g_next = torch.roll(g, shifts=-1, dims=3 - mu)
        ug[mu] = g @ u[mu] @ g_next.conj().transpose(-1, -2)
    psi = rand_field(dims, 7)
    # (g psi)(x) = g(x) psi(x) on colour: psi @ g^T
    gpsi = psi @ g.transpose(-1, -2)
    lhs = w.dirac(ug, gpsi, 0.124, BC)
    rhs = w.dirac(u, psi, 0.124, BC) @ g.transpose(-1, -2)
    assert torch.allclose(lhs, rhs, atol=1e-12, rtol=0)


def test_free_field_plane_waves():
    # U = 1: D e^{ipx} u = e^{ipx} D(p) u with
    # D(p) = 1 - 2 kappa sum cos p_mu + 2 i kappa sum gamma_mu sin p_mu,
    # p_k = 2 pi n_k / L_k (periodic), p_t = (2 n_t + 1) pi / L_t (antiperiodic).
    dims = (4, 6, 4, 8)
    lx, ly, lz, lt = dims
    u = synth.gauge_unit(dims)
    kappa = 0.11
    g = gammas()
    gen = torch.Generator().manual_seed(0)
    for n in [(0, 0, 0, 0), (1, 2, 3, 1), (3, 5, 1, 6)]:
        p = [2 * math.pi * n[0] / lx, 2 * math.pi * n[1] / ly, 2 * math.pi * n[2] / lz,
             (2 * n[3] + 1) * math.pi / lt]
        f64 = torch.float64
        t = torch.arange(lt, dtype=f64).view(lt, 1, 1, 1)
        z = torch.arange(lz, dtype=f64).view(1, lz, 1, 1)
        y = torch.arange(ly, dtype=f64).view(1, 1, ly, 1)
        x = torch.arange(lx, dtype=f64).view(1, 1, 1, lx)
        phase = torch.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
        spinor = torch.randn(4, 3, dtype=CDT, generator=gen)
        psi = phase[..., None, None] * spinor
        dp = torch.eye(4, dtype=CDT) * (1 - 2 * kappa * sum(math.cos(q) for q in p))
        for mu in range(4):
            dp = dp + 2j * kappa * math.sin(p[mu]) * g[mu]
        expect = phase[..., None, None] * (dp @ spinor)
        assert torch.allclose(w.dirac(u, psi, kappa, BC), expect, atol=1e-12, rtol=0)
        # eigenvalues 1 - 2k sum cos +- 2 i k sqrt(sum sin^2), each twice in spin
        ev = torch.linalg.eigvals(dp)
        c = 1 - 2 * kappa * sum(math.cos(q) for q in p)
        s = 2 * kappa * math.sqrt(sum(math.sin(q) ** 2 for q in p))
        want = torch.tensor([c - 1j * s, c - 1j * s, c + 1j * s, c + 1j * s], dtype=CDT)
        got = ev[torch.argsort(ev.imag)]
        assert torch.allclose(got, want, atol=1e-12)


def test_hop_at_sites_matches_full_hop():
    dims = (4, 6, 2, 8)
    u = synth.gauge_random(dims, 0.5, seed=9)
    psi = rand_field(dims, 10)
    full = w.hop(u, psi, BC).reshape(-1, 4, 3)
    sites = torch.tensor([0, 1, 5, 47, 95, 190, 383])
    assert torch.allclose(w.hop_at_sites(u, psi, sites, BC), full[sites], atol=1e-13, rtol=0)


def _eo_index(dims):
    par = w.parity(dims).reshape(-1)
    ev = torch.nonzero(par == 0).reshape(-1)
    od = torch.nonzero(par == 1).reshape(-1)
    expand = lambda s: (12 * s[:, None] + torch.arange(12)[None, :]).reshape(-1)
    return expand(ev), expand(od)


def test_even_odd_blocks_and_schur_complement():
    dims = (2, 2, 2, 2)
    u = synth.gauge_random(dims, 0.6, seed=21)
    kappa = 0.125
    d = w.dense_by_blocks(u, kappa, BC)
    ie, io = _eo_index(dims)
    dee, deo = d[ie][:, ie], d[ie][:, io]
    doe, doo = d[io][:, ie], d[io][:, io]
    n = len(ie)
    assert torch.allclose(dee, torch.eye(n, dtype=CDT), atol=0)
    assert torch.allclose(doo, torch.eye(n, dtype=CDT), atol=0)
    schur = torch.eye(n, dtype=CDT) - deo @ doe
    # columns of the oracle's A on even unit vectors
    cols = []
    for j in range(n):
        e = torch.zeros(12 * 16, dtype=CDT)
        e[ie[j]] = 1
        a = w.eo_operator(u, e.reshape(2, 2, 2, 2, 4, 3), kappa, BC).reshape(-1)
        cols.append(a[ie])
    assert torch.allclose(torch.stack(cols, 1), schur, atol=1e-14)


def test_even_odd_solve_equals_lu():
    dims = (2, 2, 2, 4)
    u = synth.gauge_random(dims, 0.6, seed=22)
    kappa = 0.12
    d = w.dense_by_blocks(u, kappa, BC)
    eta = rand_field(dims, 23)
    exact = torch.linalg.solve(d, eta.reshape(-1)).reshape(eta.shape)
    from oracle.solvers import solve_wilson
    xi, info = solve_wilson(u, eta, kappa, BC, tol=1e-14)
    assert info.converged
    assert torch.allclose(xi, exact, atol=1e-12 * exact.abs().max().item(), rtol=0)
    # Eq. 4 right-hand side and Eq. 5 reconstruction against the dense blocks
    ie, io = _eo_index(dims)
    deo, doe = d[ie][:, io], d[io][:, ie]
    b = w.eo_source(u, eta, kappa, BC).reshape(-1)
    assert torch.allclose(b[ie], eta.reshape(-1)[ie] - deo @ eta.reshape(-1)[io], atol=1e-14)
    assert torch.allclose(b[io], torch.zeros(len(io), dtype=CDT))
    rec = w.eo_reconstruct(u, w.restrict(exact, 0), eta, kappa, BC).reshape(-1)
    assert torch.allclose(rec[io], eta.reshape(-1)[io] - doe @ exact.reshape(-1)[ie], atol=1e-13)


@pytest.mark.parametrize("p", [0, 1])
def test_parity_hop_equals_masked_full_hop(p):
    dims = (4, 6, 2, 8)
    u = synth.gauge_random(dims, 0.5, seed=24)
    psi = rand_field(dims, 25)
    for bc in [(1, 1, 1, -1), (-1, 1, -1, 1)]:
        assert torch.allclose(w.hop_pq(u, psi, p, bc), w.hop_pq_full(u, psi, p, bc), atol=1e-13, rtol=0)
