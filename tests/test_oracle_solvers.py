"""Pins of the oracle's solvers (Sec. 3, Algorithms 2-5).

Pinned by: a dense LU solve; exact invariances of the rescaled recurrences in
float64 (rescaling by any sigma, solution rescaling, gamma = 1 and omega_0 = 0
reduce to textbook BiCGStab); beta = 1 on the first step; one-step exactness of
the refinement with an exact inner solve; the paper's single-nonzero first
inner input; and final residuals checked with the independently pinned D_W.
"""

import math

import pytest
import torch

from oracle import solvers as S
from oracle import wilson as w
from paper_2602_14450_gb300 import synth
from tests.golden_util import read_numbers

BC = (1, 1, 1, -1)
DIMS = (4, 4, 4, 4)
KAPPA = 0.13


@pytest.fixture(scope="module")
def system():
    u = synth.gauge_smeared(DIMS, seed=20260214)
    eta = synth.gaussian_source(DIMS, seed=450)
    b = w.eo_source(u, eta, KAPPA, BC)
    a = lambda f: w.eo_operator(u, f, KAPPA, BC)
    return u, eta, b, a


def rel(a, b):
    return S.norm(a - b) / S.norm(b)


def test_bicgstab_matches_lu_on_dense_matrix():
    n = 60
    g = torch.Generator().manual_seed(3)
    m = torch.eye(n, dtype=torch.complex128) + 0.4 * torch.randn(n, n, dtype=torch.complex128, generator=g) / math.sqrt(n)
    b = torch.randn(n, dtype=torch.complex128, generator=g)
    x, info = S.bicgstab(lambda v: m @ v, b, 1e-14)
    assert info.converged
    assert rel(x, torch.linalg.solve(m, b)) < 1e-12


def test_gamma_one_omega0_zero_is_textbook(system):
    _, _, b, a = system
    k = 8
    x_ref, _ = S.bicgstab(a, b, 0.0, maxiter=k)
    prm = S.InnerParams(sigma=None, eps=0.0, omega0=0.0, max_matvecs=2 * k)
    x, tr = S.bicgstab_rescaled(a, b, prm)
    assert tr.iterations == k
    assert rel(x, x_ref) < 1e-12


@pytest.mark.parametrize("sigma,recalc", [(64.0, True), (64.0, False), (1e4, True), (1e-3, True)])
def test_residual_rescaling_is_exact_in_fp64(system, sigma, recalc):
    # Alg. 4 with any sigma computes the same iterates as gamma = 1 in exact
    # arithmetic; in float64 they agree to rounding.
    _, _, b, a = system
    base = S.InnerParams(sigma=None, eps=0.0, max_matvecs=24)
    _, t0 = S.bicgstab_rescaled(a, b, base, keep_iterates=True)
    prm = S.InnerParams(sigma=sigma, recalc_gamma=recalc, eps=0.0, max_matvecs=24)
    _, t1 = S.bicgstab_rescaled(a, b, prm, keep_iterates=True)
    assert len(t0.iterates) == len(t1.iterates) == 12
    for x0, x1 in zip(t0.iterates, t1.iterates):
        assert rel(x1, x0) < 1e-11
    for r0, r1 in zip(t0.residuals, t1.residuals):
        assert abs(r1 - r0) <= 1e-11 * r0


def test_solution_rescaling_alg5_equals_alg4_in_fp64(system):
    _, _, b, a = system
    p3 = S.InnerParams(sigma=256.0, eps=0.0, max_matvecs=24)
    p4 = S.InnerParams(sigma=256.0, rescale_x=True, sigma_lambda=256.0, eps=0.0, max_matvecs=24)
    _, t3 = S.bicgstab_rescaled(a, b, p3, keep_iterates=True)
    _, t4 = S.bicgstab_rescaled(a, b, p4, keep_iterates=True)
    for x3, x4 in zip(t3.iterates, t4.iterates):
        assert rel(x4, x3) < 1e-11


@pytest.mark.parametrize("scale", [1e-6, 1.0, 1e6])
def test_first_beta_is_one(system, scale):
    # Sec. 3: rho' = |r|^2 makes beta = 1 in the first iteration for any |b|.
    _, _, b, a = system
    _, tr = S.bicgstab_rescaled(a, scale * b, S.InnerParams(eps=0.0, max_matvecs=2))
    assert abs(tr.first_beta - 1) < 1e-14


def test_refinement_one_step_exact_with_exact_inner(system):
    # Reading of Alg. 3's correction: x += (|r| / s-hat) t makes one exact
    # inner solve give r = 0. The literal x += t / s-hat does not (|r| != 1).
    _, _, b, a = system
    b = 1e3 * b
    exact_inner = lambda y: (S.bicgstab(a, y, 1e-15)[0], S.InnerTrace())
    ident = S.make_store("fp64")
    prm = S.OuterParams(s=128.0, tol=0.0, max_outer=1)
    x, tr = S.refine(a, b, exact_inner, ident, prm)
    assert tr.outer == 1
    assert S.norm(b - a(x)) <= 1e-12 * S.norm(b)
    y = (128.0 / S.norm(b)) * b
    t, _ = exact_inner(y)
    literal = t / S.norm(y)
    assert S.norm(b - a(literal)) > 0.5 * S.norm(b)


def test_first_inner_input_has_one_nonzero():
    # Sec. 6: for b = (1, 0, ..., 0) the first inner input has 1 nonzero
    # among the 25,165,824 reals of an even-odd vector at 32^3 x 64.
    nums = read_numbers()
    assert (32 ** 3 * 64 // 2) * 24 == nums["first_inner_input_elements"]
    u = synth.gauge_smeared(DIMS, seed=1)
    b = synth.point_source(DIMS, 0, 0, site=0)        # even site 0 of the even-odd system
    a = lambda f: w.eo_operator(u, f, KAPPA, BC)
    a_low, store = S.low_precision_operator(u, KAPPA, "fp16", BC)
    inner = lambda y: S.bicgstab_rescaled(a_low, y, S.InnerParams(sigma=64.0), store)
    _, tr = S.refine(a, b, inner, store, S.OuterParams(s=128.0, tol=1e-6, max_outer=2))
    assert tr.nonzeros[0] == nums["first_inner_input_nonzero"]
    assert tr.nonzeros[1] > 1


@pytest.mark.parametrize("fmt,outer,inner", [
    ("fp16", S.OuterParams(s=128.0), S.InnerParams(sigma=64.0)),
    ("fp16", S.OuterParams(s=4096.0), S.InnerParams(sigma=None)),
    ("fp16", S.OuterParams(s=128.0), S.InnerParams(sigma=256.0, rescale_x=True, sigma_lambda=256.0)),
    ("fp32", S.OuterParams(s=1.0, use_shat=False), S.InnerParams(sigma=None)),
])
def test_mixed_solver_reaches_fp64_residual(system, fmt, outer, inner):
    u, eta, _, _ = system
    xi, tr = S.solve_wilson_mixed(u, eta, KAPPA, BC, fmt=fmt, outer=outer, inner=inner)
    assert tr.converged
    assert S.norm(eta - w.dirac(u, xi, KAPPA, BC)) <= 1e-10 * S.norm(eta)
    ref, info = S.solve_wilson(u, eta, KAPPA, BC, tol=1e-12)
    assert rel(xi, ref) < 1e-8
    # Sec. 1 / Table 2: low-precision inner solves cost at most ~20% more
    # matrix-vector products than the float64 solver (soft band).
    nums = read_numbers()
    assert tr.matvecs <= nums["fp16_overhead_bound"] * info.matvecs + 20


def test_storage_rounding_formats():
    # FP16: 11-bit significand, max 65504, min normal 2^-14 ~ 6.10e-5 (Sec. 5, Table 1).
    st = S.make_store("fp16")
    v = torch.tensor([1 + 2 ** -11, 1 + 3 * 2 ** -11, 65504.0, 65520.0, 2 ** -24, 2 ** -25], dtype=torch.float64)
    got = torch.view_as_real(st(torch.complex(v, torch.zeros_like(v))))[:, 0]
    want = torch.tensor([1.0, 1 + 2 ** -9, 65504.0, math.inf, 2 ** -24, 0.0], dtype=torch.float64)
    assert torch.equal(got, want)
    bf = S._round_bf16(torch.tensor([1 + 2 ** -8, 1 + 3 * 2 ** -8, 2 ** -130, 3.0e38]).numpy())
    assert list(bf) == [1.0, 1 + 2 ** -6, 2 ** -130, float(torch.tensor(3.0e38).to(torch.bfloat16).double())]


def test_inner_breakdown_stops_without_raising():
    """Algorithm 4 breaks down when (r*, v) = 0 (here A = 0): the oracle stops
    the inner solve with x = 0 and flags it, as the device recurrence does
    (status breakdown, the refinement continues), instead of dividing by zero."""
    b = torch.randn(40, dtype=torch.complex128, generator=torch.Generator().manual_seed(3))
    x, tr = S.bicgstab_rescaled(lambda f: torch.zeros_like(f), b, S.InnerParams(sigma=64.0))
    assert tr.breakdown and not tr.converged
    assert tr.iterations == 0 and tr.matvecs == 0
    assert torch.count_nonzero(x) == 0


def test_fp16_flush_to_zero_slows_unrescaled_inner_solve():
    """Sec. 6: with the paper's unit source and FP16 subnormals flushed to zero
    (its -Kfz build), the unrescaled inner solve of Alg. 2 loses vector
    elements to underflow and needs far more matvecs, while Alg. 3 + Alg. 4
    (s = 128, sigma = 64) keeps its vectors in range and is unaffected. Without
    the flush the two cost the same. (On 8^3 x 16 the gap is 3804 vs 434.)"""
    from oracle import wilson as W
    from paper_2602_14450_gb300 import synth
    dims = (4, 4, 4, 8)
    u = synth.gauge_smeared(dims, seed=5)
    eta = synth.point_source(dims, 0, 0, 0)
    runs = {}
    for ftz in (False, True):
        for name, outer, inner in [
            ("alg2", S.OuterParams(s=1.0, use_shat=False, tol=1e-13, max_outer=25),
             S.InnerParams(sigma=None, max_matvecs=600)),
            ("alg34", S.OuterParams(s=128.0, use_shat=True, tol=1e-13, max_outer=25),
             S.InnerParams(sigma=64.0, max_matvecs=600)),
        ]:
            x, tr = S.solve_wilson_mixed(u, eta, 0.124, fmt="fp16", outer=outer, inner=inner, ftz=ftz)
            assert tr.converged and S.norm(eta - W.dirac(u, x, 0.124)) / S.norm(eta) <= 1e-13
            runs[name, ftz] = tr
    n = 2 * dims[0] * dims[1] * dims[2] * dims[3] // 2 * 12       # reals of an even-site vector
    assert runs["alg2", False].nonzeros[1] == n and runs["alg2", True].nonzeros[1] < n
    assert runs["alg2", True].matvecs >= 1.4 * runs["alg2", False].matvecs
    assert abs(runs["alg34", True].matvecs - runs["alg34", False].matvecs) <= 0.1 * runs["alg34", False].matvecs
