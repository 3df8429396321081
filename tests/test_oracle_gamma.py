"""Pins of the oracle's Dirac matrices against Eq. 2 and the Clifford algebra."""

import pytest
import torch

from oracle.gamma import gamma5, gammas, projectors
from tests.golden_util import read_complex_matrix, read_numbers

pytestmark = pytest.mark.filterwarnings("ignore")


def test_printed_one_minus_gamma1():
    printed = read_complex_matrix("eq2_one_minus_gamma1.txt")
    pm, _ = projectors()
    assert torch.equal(pm[0], printed)


def test_projected_component_identities():
    # Eq. 2: phi3+ = -i phi2+, phi4+ = -i phi1+ for (1 - gamma_1) phi.
    g = torch.Generator().manual_seed(1)
    phi = torch.randn(4, 3, dtype=torch.complex128, generator=g)
    pm, _ = projectors()
    out = pm[0] @ phi
    assert torch.allclose(out[2], -1j * out[1], atol=0, rtol=0)
    assert torch.allclose(out[3], -1j * out[0], atol=0, rtol=0)


def test_clifford_algebra_and_hermiticity():
    g = gammas()
    eye = torch.eye(4, dtype=torch.complex128)
    for mu in range(4):
        assert torch.equal(g[mu], g[mu].conj().T)
        for nu in range(4):
            anti = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert torch.equal(anti, 2 * eye * (mu == nu))
    g5 = gamma5()
    assert torch.allclose(g5 @ g5, eye)
    assert torch.allclose(g5, g5.conj().T)
    for mu in range(4):
        assert torch.allclose(g5 @ g[mu], -g[mu] @ g5)


def test_projectors_rank_two():
    # Sec. 2: (1 -+ gamma_mu) keeps two of the four spin components
    pm, pp = projectors()
    for mu in range(4):
        for p in (pm[mu], pp[mu]):
            assert torch.linalg.matrix_rank(p).item() == 2
            assert torch.allclose(p @ p, 2 * p)
