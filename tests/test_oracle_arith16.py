"""Pins of the oracle's FP16-arithmetic hop (oracle.arith16): exact where FP16
arithmetic is exact, IEEE scaling behaviour, the projector split of the printed
(1 - gamma_1), and an error between that of exact arithmetic on rounded inputs
and the bound the FP16-arithmetic kernel is held to."""

import numpy as np
import pytest
import torch

from oracle import arith16 as A
from oracle import solvers as S
from oracle import wilson as W
from oracle.gamma import projectors
from paper_2602_14450_gb300 import synth
from tests.golden_util import read_complex_matrix

BC = (1, 1, 1, -1)


def rel(a, b):
    return (torch.linalg.vector_norm((a - b).reshape(-1)) / torch.linalg.vector_norm(b.reshape(-1))).item()


def signed_permutation_links(dims, seed):
    """Links whose entries are 0, +-1 or +-i, one per row and column: every
    product with an FP16 value is exact."""
    g = torch.Generator().manual_seed(seed)
    lx, ly, lz, lt = dims
    v = lx * ly * lz * lt
    units = torch.tensor([1, -1, 1j, -1j], dtype=torch.complex128)
    u = torch.zeros((4, v, 3, 3), dtype=torch.complex128)
    for mu in range(4):
        perm = torch.argsort(torch.rand((v, 3), generator=g), dim=1)
        ph = units[torch.randint(4, (v, 3), generator=g)]
        u[mu, torch.arange(v)[:, None], torch.arange(3)[None, :], perm] = ph
    return u.reshape(4, lt, lz, ly, lx, 3, 3)


def test_split_of_the_printed_projector():
    # Eq. 2: (1 - gamma_1) keeps rows 0 and 1; row 2 = -i row 1, row 3 = -i row 0
    p = read_complex_matrix("eq2_one_minus_gamma1.txt").numpy()
    terms, rebuild = A.split_projector(p)
    assert terms == [[(0, 1 + 0j), (3, 1j)], [(1, 1 + 0j), (2, 1j)]]
    assert sorted(rebuild) == [(0, 0, 1 + 0j), (1, 1, 1 + 0j), (2, 1, -1j), (3, 0, -1j)]
    # every projector of Eq. 1 splits into two rows that rebuild it exactly
    pm, pp = projectors()
    for m in list(pm) + list(pp):
        m = m.numpy()
        terms, rebuild = A.split_projector(m)
        lead = [np.array([dict(t).get(s, 0) for s in range(4)]) for t in terms]
        back = np.zeros((4, 4), dtype=complex)
        for r, j, c in rebuild:
            back[r] = c * lead[j]
        assert np.array_equal(back, m)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 6, 4)])
@pytest.mark.parametrize("p", [0, 1])
def test_exact_where_fp16_arithmetic_is_exact(dims, p):
    """Small integer spinors and links with entries 0, +-1, +-i: every
    intermediate is an integer below 2^11, so FP16 arithmetic is exact and the
    result equals Eq. 1 in float64, boundary phases included."""
    u = signed_permutation_links(dims, seed=11 + p)
    g = torch.Generator().manual_seed(5)
    shape = (dims[3], dims[2], dims[1], dims[0], 4, 3)
    psi = (torch.randint(-8, 9, shape, generator=g) + 1j * torch.randint(-8, 9, shape, generator=g)).to(torch.complex128)
    for bc in (BC, (-1, 1, -1, 1)):
        assert torch.equal(A.hop_pq_fp16(u, psi, p, bc), W.hop_pq(u, psi, p, bc))


def test_scaling_by_two_commutes():
    """Every operation is one IEEE rounding, so doubling the input doubles the
    output exactly while no value leaves the normal range."""
    dims = (4, 4, 4, 4)
    st = S.make_store("fp16")
    u = st(synth.gauge_random(dims, 0.5, seed=3))
    psi = st(16 * synth.gaussian_source(dims, seed=4))
    h = A.hop_pq_fp16(u, psi, 0, BC)
    assert torch.equal(A.hop_pq_fp16(u, 2 * psi, 0, BC), 2 * h)


def test_error_between_exact_arithmetic_and_the_kernel_bound():
    """On FP16-rounded SU(3) links and spinor, exact arithmetic gives the
    rounded inputs' hop; FP16 arithmetic adds about 20 roundings per output real,
    so its distance from that is several times the unit roundoff 2^-11 / sqrt(3)
    and stays below the 2e-3 bound the FP16 hopping term is held to."""
    dims = (8, 6, 4, 10)
    st = S.make_store("fp16")
    u64 = synth.gauge_random(dims, 0.5, seed=7)
    p64 = synth.gaussian_source(dims, seed=8)
    u, psi = st(u64), st(p64)
    h16 = A.hop_pq_fp16(u, psi, 0, BC)
    exact = W.hop_pq(u, psi, 0, BC)
    e_arith = rel(h16, exact)
    assert 2.0 ** -11 / np.sqrt(3) < e_arith < 2e-3
    assert rel(h16, W.hop_pq(u64, p64, 0, BC)) < 2e-3
    # the result is made of FP16 values
    assert torch.equal(st(h16), h16)


def test_mixed_solve_with_fp16_arithmetic_reaches_fp64_tolerance():
    """Alg. 3 + Alg. 4 with the inner operator in FP16 arithmetic: the FP64
    refinement still reaches 1e-10 in the full system."""
    dims = (4, 4, 4, 4)
    u = synth.gauge_random(dims, 0.5, seed=21)
    eta = synth.gaussian_source(dims, seed=22)
    kappa = 0.12
    x, tr = S.solve_wilson_mixed(u, eta, kappa, BC, fmt="fp16", outer=S.OuterParams(s=128.0),
                                 inner=S.InnerParams(sigma=64.0), arith16=True)
    res = S.norm(eta - W.dirac(u, x, kappa, BC)) / S.norm(eta)
    assert res <= 1e-10
    with pytest.raises(ValueError):
        S.low_precision_operator(u, kappa, "fp32", BC, arith16=True)


def su3_signed_permutations(dims, seed):
    """SU(3) links with entries 0, +-1, +-i: rows 0 and 1 from a signed
    permutation, row 2 = conj(row 0 x row 1) (exact for such entries)."""
    u = signed_permutation_links(dims, seed)
    r0, r1 = u[..., 0, :], u[..., 1, :]
    u[..., 2, :] = torch.linalg.cross(r0, r1).conj()
    return u


@pytest.mark.parametrize("p", [0, 1])
def test_twelve_real_rebuild_exact_for_exact_links(p):
    """With SU(3) links whose entries are 0, +-1, +-i, the FP16 rebuild of the
    third row is exact, so the 12-real FP16 hop equals Eq. 1 in float64."""
    dims = (4, 2, 6, 4)
    u = su3_signed_permutations(dims, seed=31 + p)
    assert torch.allclose(torch.linalg.det(u), torch.ones((), dtype=torch.complex128), atol=0)
    m = torch.view_as_real(u.contiguous()).numpy()
    mr, mi = m[..., 0].copy(), m[..., 1].copy()
    A.rebuild_third_row(mr, mi)
    assert np.array_equal(mr, m[..., 0]) and np.array_equal(mi, m[..., 1])
    g = torch.Generator().manual_seed(6)
    shape = (dims[3], dims[2], dims[1], dims[0], 4, 3)
    psi = (torch.randint(-8, 9, shape, generator=g) + 1j * torch.randint(-8, 9, shape, generator=g)).to(torch.complex128)
    assert torch.equal(A.hop_pq_fp16(u, psi, p, BC, recon=12), W.hop_pq(u, psi, p, BC))


def test_twelve_real_rebuild_on_generic_links():
    """On FP16-rounded SU(3) links the rebuilt third row is the true one to a
    few FP16 units (rows 0, 1 carry 2^-12 relative rounding, each rebuilt
    element sums two products of them in four roundings), and the 12-real hop
    stays within the FP16-arithmetic bound of float64."""
    dims = (4, 4, 4, 4)
    u64 = synth.gauge_random(dims, 0.5, seed=9)
    m = A.r16(torch.view_as_real(u64.contiguous()).numpy())
    mr, mi = m[..., 0].copy(), m[..., 1].copy()
    A.rebuild_third_row(mr, mi)
    true = torch.view_as_real(u64.contiguous()).numpy()[..., 2, :, :]
    err = np.abs(np.stack([mr[..., 2, :], mi[..., 2, :]], -1) - true).max()
    assert err < 8 * 2.0 ** -11
    psi = synth.gaussian_source(dims, seed=10)
    assert rel(A.hop_pq_fp16(u64, psi, 0, BC, recon=12), W.hop_pq(u64, psi, 0, BC)) < 2e-3
    with pytest.raises(ValueError):
        A.hop_pq_fp16(u64, psi, 0, BC, recon=8)
