"""Pins of the three-step hop of Sec. 2 and of its operation count.

oracle.flops evaluates H_pq with numbers that count their own real
operations. Its result must equal the oracle's Eq. 1 (full 4x4 spin
matrices, no projection), and the operations it performs must give the
paper's 168 per hop (Sec. 2) for every projector of the form printed in
Eq. 2 -- so a dropped, doubled or misplaced term in the projection, the
link product or the rebuild fails one of the two.
"""

import pytest
import torch

from oracle import flops as F
from oracle import wilson as W
from paper_2602_14450_gb300 import synth
from tests.golden_util import read_numbers

BC = (1, 1, 1, -1)


@pytest.fixture(scope="module")
def fields():
    dims = (4, 2, 2, 4)
    return dims, synth.gauge_random(dims, 0.5, seed=5), synth.gaussian_source(dims, seed=6)


@pytest.mark.parametrize("p", [0, 1])
def test_three_step_hop_equals_eq1(fields, p):
    dims, u, psi = fields
    got, _ = F.hop_pq_counted(u, psi, p, BC)
    want = W.hop_pq(u, psi, p, BC)
    assert torch.allclose(got, want, rtol=0, atol=1e-14 * want.abs().max().item())


def test_168_flops_per_hop(fields):
    dims, u, psi = fields
    nums = read_numbers()
    _, counts = F.hop_pq_counted(u, psi, 0, BC)
    # x, y, z: projectors with two nonzeros per row, as the printed (1 - gamma_1)
    for mu in range(3):
        for sign in (+1, -1):
            assert counts[(mu, sign)] == {nums["flops_per_hop_projected"]}, (mu, sign, counts[(mu, sign)])
    # t in the Dirac basis: (1 -+ gamma_4) is diagonal (2 on two rows, 0 on the
    # others), so step 1 scales (12) instead of adding (12) and step 3
    # accumulates six complex numbers (12) instead of twelve (24)
    for sign in (+1, -1):
        assert counts[(3, sign)] == {12 + 132 + 12}
    per_site = sum(next(iter(c)) for c in counts.values())
    assert per_site == 6 * 168 + 2 * 156 == 1320


def test_dense_12x12_block_flops():
    nums = read_numbers()
    g = torch.Generator().manual_seed(3)
    block = torch.randn(12, 12, dtype=torch.complex128, generator=g)
    vec = torch.randn(12, dtype=torch.complex128, generator=g)
    out = torch.randn(12, dtype=torch.complex128, generator=g)
    got, n = F.dense_block_flops(block, vec, out)
    assert n == nums["flops_per_hop_dense12"]
    assert torch.allclose(got, out + block @ vec, rtol=0, atol=1e-13)


def test_count_follows_the_operations():
    """The count is that of the operations performed: the same hop on a link
    stored as a dense 3x3 product M = A B (formed on the counted numbers)
    costs the 27 complex products and 18 sums of forming M on top."""
    g = torch.Generator().manual_seed(4)
    ctr = F.Counter()
    num = lambda z: F.Num(z.real, z.imag, ctr)
    a = torch.randn(3, 3, dtype=torch.complex128, generator=g)
    b = torch.randn(3, 3, dtype=torch.complex128, generator=g)
    src = [[num(z) for z in row] for row in torch.randn(4, 3, dtype=torch.complex128, generator=g).tolist()]
    from oracle.gamma import projectors
    pm, _ = projectors()
    out = [[num(0j) for _ in range(3)] for _ in range(4)]
    n0 = ctr.n
    A = [[num(z) for z in row] for row in a.tolist()]
    B = [[num(z) for z in row] for row in b.tolist()]
    M = [[A[i][0] * B[0][j] + A[i][1] * B[1][j] + A[i][2] * B[2][j] for j in range(3)] for i in range(3)]
    assert F.one_hop(pm[0], M, src, out, ctr) == 168
    assert ctr.n - n0 == 168 + 27 * 6 + 18 * 2
