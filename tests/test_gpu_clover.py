"""The clover term on the GPU (wd_set_clover) against the oracle: the even-odd
operator of Eq. 4 and the full matrix with clover blocks, and the solvers."""

import pytest
import torch

from oracle import clover as cl
from oracle import solvers as S
from paper_2602_14450_gb300 import synth, wd
from tests.gpu_util import TOL, apply_op, from_lex, lattice, lex_dev, rel_l2

pytestmark = pytest.mark.gpu
BC = (1, 1, 1, -1)
CSW = 1.0


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 4, 8)])
@pytest.mark.parametrize("prec,recon", [("fp64", 18), ("fp32", 18), ("fp32", 12), ("fp16", 12), ("bf16", 12)])
def test_clover_operators_match_oracle(dims, prec, recon):
    u = synth.gauge_random(dims, 0.5, seed=41)
    psi = synth.gaussian_source(dims, seed=42)
    kappa = 0.125
    lat = lattice(u, kappa, dims)
    lat.set_clover(CSW)
    c = cl.clover_matrix(u, CSW, kappa)
    cinv = torch.linalg.inv(c)
    from oracle import wilson as w
    want_a = cl.eo_operator_sw(u, cinv, w.restrict(psi, 0), kappa, BC)
    want_d = cl.dirac_sw(u, c, psi, kappa, BC)
    # FP16: the bound the FP16 hopping term is specified to meet; the other
    # precisions allow twice theirs, since the blocks are stored in the
    # operator's precision too
    tol = TOL[prec] if prec == "fp16" else 2 * TOL[prec]
    assert rel_l2(apply_op(lat, prec, recon, wd.WD_OP_EO_A, psi, dims), want_a) <= tol
    assert rel_l2(apply_op(lat, prec, recon, wd.WD_OP_FULL, psi, dims), want_d) <= tol
    # the hopping operators are the plain ones
    assert rel_l2(apply_op(lat, prec, recon, wd.WD_OP_HOP_EO, psi, dims), w.hop_pq(u, psi, 0, BC)) <= TOL[prec]
    lat.set_clover(0.0)
    assert rel_l2(apply_op(lat, prec, recon, wd.WD_OP_FULL, psi, dims), w.dirac(u, psi, kappa, BC)) <= TOL[prec]


@pytest.mark.parametrize("scheme", ["fp64", "mixed_fp32", "mixed_fp16", "mixed_bf16"])
def test_clover_solves_reach_fp64_residual(scheme):
    dims = (8, 8, 8, 8)
    u = synth.gauge_smeared(dims, seed=43)
    eta = synth.gaussian_source(dims, seed=44)
    kappa = 0.124
    lat = lattice(u, kappa, dims)
    lat.set_clover(CSW)
    b = lex_dev(eta)
    x = torch.zeros_like(b)
    st = lat.solve(b, x, 1e-10, scheme)
    assert st.status == wd.WD_OK and st.true_residual <= 1e-10
    c = cl.clover_matrix(u, CSW, kappa)
    res = S.norm(eta - cl.dirac_sw(u, c, from_lex(x, dims), kappa, BC)) / S.norm(eta)
    assert res <= 1e-10 and abs(res - st.true_residual) <= 1e-3 * res + 1e-14


def test_clover_batch_and_guards():
    dims = (4, 4, 4, 8)
    u = synth.gauge_random(dims, 0.5, seed=45)
    kappa = 0.12
    lat = wd.Lattice(dims, kappa)
    with pytest.raises(wd.WDError) as e:
        lat.set_clover(CSW)
    assert e.value.code == wd.WD_ERR_NO_GAUGE
    lat = lattice(u, kappa, dims)
    lat.set_clover(CSW)
    etas = [synth.gaussian_source(dims, seed=46 + i) for i in range(3)]
    b = torch.stack([lex_dev(e) for e in etas])
    x = torch.zeros_like(b)
    stats = lat.solve_rhs(b, x, 1e-10, "mixed_fp16")
    c = cl.clover_matrix(u, CSW, kappa)
    for i, st in enumerate(stats):
        assert st.status == wd.WD_OK
        res = S.norm(etas[i] - cl.dirac_sw(u, c, from_lex(x[i], dims), kappa, BC)) / S.norm(etas[i])
        assert res <= 1e-10
    lat.precond_set(torch.zeros(wd.PRECOND_FLOATS))
    with pytest.raises(wd.WDError) as e:
        lat.solve(b[0], x[0], 1e-10, "mixed_fp16_learned")
    assert e.value.code == wd.WD_ERR_INVALID_ARG


@pytest.mark.parametrize("recon", [12, 18])
def test_clover_operators_fp16_arithmetic(recon):
    """The clover blocks in the epilogue of the FP16-arithmetic hop
    (wd_set_arith(16)): the even-odd operator and the full matrix."""
    dims = (6, 4, 4, 8)
    u = synth.gauge_random(dims, 0.5, seed=47)
    psi = synth.gaussian_source(dims, seed=48)
    kappa = 0.125
    lat = lattice(u, kappa, dims)
    lat.set_clover(CSW)
    lat.set_arith(16)
    c = cl.clover_matrix(u, CSW, kappa)
    from oracle import wilson as w
    want_a = cl.eo_operator_sw(u, torch.linalg.inv(c), w.restrict(psi, 0), kappa, BC)
    want_d = cl.dirac_sw(u, c, psi, kappa, BC)
    assert rel_l2(apply_op(lat, "fp16", recon, wd.WD_OP_EO_A, psi, dims), want_a) <= TOL["fp16a"]
    assert rel_l2(apply_op(lat, "fp16", recon, wd.WD_OP_FULL, psi, dims), want_d) <= TOL["fp16a"]
