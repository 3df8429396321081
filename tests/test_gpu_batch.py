"""Batched solves (several right-hand sides and lattices per call) against the oracle."""

import pytest
import torch

from oracle import solvers as S
from oracle import wilson as W
from paper_2602_14450_gb300 import synth, wd
from tests.gpu_util import from_lex, lattice, lex_dev

pytestmark = pytest.mark.gpu
BC = (1, 1, 1, -1)
TOL = 1e-10


def residual(u, eta, kappa, x):
    return S.norm(eta - W.dirac(u, x, kappa, BC)) / S.norm(eta)


@pytest.mark.parametrize("arith", [32, 16])
@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (6, 4, 4, 8)])
def test_twelve_spin_colour_point_sources(dims, arith):
    u = synth.gauge_smeared(dims, seed=31)
    kappa = 0.125
    lat = lattice(u, kappa, dims)
    lat.set_arith(arith)
    etas = [synth.point_source(dims, s, c, site=0) for s in range(4) for c in range(3)]
    b = torch.stack([lex_dev(e) for e in etas])
    x = torch.zeros_like(b)
    stats = lat.solve_rhs(b, x, TOL, "mixed_fp16")
    assert len(stats) == 12
    for k, (eta, st) in enumerate(zip(etas, stats)):
        assert st.status == wd.WD_OK and st.true_residual <= TOL
        xi = from_lex(x[k], dims)
        assert residual(u, eta, kappa, xi) <= TOL
    # the batched solution of one source equals its single-source solve
    x1 = torch.zeros_like(b[5])
    lat.solve(b[5].contiguous(), x1, TOL, "mixed_fp16")
    ref = from_lex(x1, dims)
    assert S.norm(from_lex(x[5], dims) - ref) / S.norm(ref) < 1e-8


@pytest.mark.parametrize("arith", [32, 16])
def test_uneven_batch_of_lattices(arith):
    specs = [((4, 4, 4, 4), 0.12, 41), ((6, 4, 4, 8), 0.12, 42), ((8, 8, 8, 8), 0.12, 43)]
    lats, bs, xs, etas, us = [], [], [], [], []
    for dims, kappa, seed in specs:
        u = synth.gauge_random(dims, 0.5, seed=seed)
        us.append(u)
        lats.append(lattice(u, kappa, dims))
        lats[-1].set_arith(arith)
        e = [synth.gaussian_source(dims, seed=100 * seed + j) for j in range(4)]
        etas.append(e)
        bs.append(torch.stack([lex_dev(v) for v in e]))
        xs.append(torch.zeros_like(bs[-1]))
    for scheme in ("mixed_fp16", "fp64"):
        for x in xs:
            x.zero_()
        stats = wd.solve_batch(lats, bs, xs, TOL, scheme)
        assert len(stats) == 12
        k = 0
        for (dims, kappa, _), u, e, x in zip(specs, us, etas, xs):
            for j in range(4):
                assert stats[k].status == wd.WD_OK
                assert residual(u, e[j], kappa, from_lex(x[j], dims)) <= TOL
                k += 1


def test_converged_rhs_are_left_alone():
    # a zero source converges at once; its neighbours in the batch still solve
    dims = (4, 4, 4, 8)
    u = synth.gauge_random(dims, 0.5, seed=5)
    lat = lattice(u, 0.12, dims)
    e = [synth.gaussian_source(dims, seed=1), torch.zeros_like(synth.gaussian_source(dims, seed=1)),
         synth.gaussian_source(dims, seed=2)]
    b = torch.stack([lex_dev(v) for v in e])
    x = torch.full_like(b, 7.0)
    stats = lat.solve_rhs(b, x, TOL, "mixed_fp16")
    assert stats[1].outer_iterations == 0 and torch.count_nonzero(x[1]) == 0
    for j in (0, 2):
        assert stats[j].status == wd.WD_OK
        assert residual(u, e[j], 0.12, from_lex(x[j], dims)) <= TOL
