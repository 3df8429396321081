"""Pins of the oracle's learned preconditioner (parallel-transport convolution)."""

import pytest
import torch

from oracle import ptc
from oracle import wilson as W
from paper_2602_14450_gb300 import synth

BC = (1, 1, 1, -1)
CDT = torch.complex128
DIMS = (4, 4, 2, 4)


@pytest.fixture(scope="module")
def field():
    u = synth.gauge_random(DIMS, 0.6, seed=12)
    psi = W.restrict(synth.gaussian_source(DIMS, seed=13), 0)
    return u, psi


def test_identity_weights_give_identity(field):
    u, psi = field
    w1, w2 = ptc.identity_weights()
    assert torch.allclose(ptc.apply(u, w1, w2, psi, BC), psi, atol=1e-15, rtol=0)


@pytest.mark.parametrize("mu", [0, 3])
def test_hop_then_reverse_hop_is_site_local(field, mu):
    # W1 only on +mu, W2 only on -mu: M psi(x) = W2 W1 U(x-mu)^+ U(x-mu) psi(x) = W2 W1 psi(x)
    # (unitary links; the boundary phase enters twice).
    u, psi = field
    g = torch.Generator().manual_seed(mu)
    a = torch.randn(4, 4, dtype=CDT, generator=g)
    b = torch.randn(4, 4, dtype=CDT, generator=g)
    w1 = torch.zeros((9, 12, 1, 4, 4), dtype=CDT)
    w2 = torch.zeros((9, 1, 12, 4, 4), dtype=CDT)
    kp = ptc.HOPS.index((mu, 1))
    km = ptc.HOPS.index((mu, -1))
    w1[kp, 3, 0] = a
    w2[km, 0, 3] = b
    got = ptc.apply(u, w1, w2, psi, BC)
    want = (b @ a) @ psi
    assert torch.allclose(got, want, atol=1e-13, rtol=0)


def test_gauge_equivariance(field):
    u, psi = field
    g = synth.gauge_transform_field(DIMS, seed=14)
    ug = torch.empty_like(u)
    for mu in range(4):
        ug[mu] = g @ u[mu] @ torch.roll(g, -1, 3 - mu).conj().transpose(-1, -2)
    w1, w2 = ptc.random_weights(seed=3)
    lhs = ptc.apply(ug, w1, w2, psi @ g.transpose(-1, -2), BC)
    rhs = ptc.apply(u, w1, w2, psi, BC) @ g.transpose(-1, -2)
    assert torch.allclose(lhs, rhs, atol=1e-12, rtol=0)


def test_linearity(field):
    u, psi = field
    chi = W.restrict(synth.gaussian_source(DIMS, seed=15), 0)
    w1, w2 = ptc.random_weights(seed=4)
    a, b = 0.3 - 1.2j, 2.5 + 0.1j
    lhs = ptc.apply(u, w1, w2, a * psi + b * chi, BC)
    rhs = a * ptc.apply(u, w1, w2, psi, BC) + b * ptc.apply(u, w1, w2, chi, BC)
    assert torch.allclose(lhs, rhs, atol=1e-12, rtol=0)


def test_gradients_match_finite_differences(field):
    u, _ = field
    kappa, mu = 0.12, 0.3
    vs = [W.restrict(synth.gaussian_source(DIMS, seed=20 + i), 0) for i in range(2)]
    ys = [W.restrict(synth.gaussian_source(DIMS, seed=30 + i), 0) for i in range(2)]
    w1, w2 = ptc.random_weights(seed=5)
    L, g1, g2 = ptc.grads(u, w1, w2, vs, ys, kappa, mu, BC)
    h = 1e-6
    for (w, g, idx) in [(w1, g1, (0, 3, 0, 1, 2)), (w1, g1, (5, 7, 0, 0, 0)), (w2, g2, (2, 0, 4, 3, 1)),
                        (w2, g2, (0, 0, 0, 2, 2))]:
        for comp, unit in (("re", 1.0), ("im", 1j)):
            wp, wm = w.clone(), w.clone()
            wp[idx] += unit * h
            wm[idx] -= unit * h
            a1, a2 = (wp, w2) if w is w1 else (w1, wp)
            b1, b2 = (wm, w2) if w is w1 else (w1, wm)
            fd = (ptc.loss(u, a1, a2, vs, ys, kappa, mu, BC) - ptc.loss(u, b1, b2, vs, ys, kappa, mu, BC)).item() / (2 * h)
            an = g[idx].real.item() if comp == "re" else g[idx].imag.item()
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (idx, comp, fd, an)


def test_flat_layout_roundtrip():
    w1, w2 = ptc.random_weights(seed=6)
    flat = ptc.to_flat(w1, w2)
    assert flat.numel() == 2 * 9 * 12 * 16 * 2
    a, b = ptc.from_flat(flat)
    assert torch.equal(a, w1) and torch.equal(b, w2)
