"""Batched operators (wd_apply_batch) and the FP16-arithmetic hop over K
right-hand sides per thread: identical bits to one right-hand side at a time
for every K and link placement, the oracle's Eq. 1 at the 24^3 x 48 size of
the batched workload, and the 12-point-source batch solve checked with Eq. 1
at sampled sites."""

import pytest
import torch

from oracle import wilson as W
from paper_2602_14450_gb300 import synth, wd
from tests.gpu_util import TOL, lattice, lex_dev

pytestmark = pytest.mark.gpu
BC = (1, 1, 1, -1)
NRHS = 12


def packed_batch(lat, prec, fields, parity=None):
    nb = lat.vector_bytes(prec)
    full = parity is None
    per = 2 * nb if full else nb
    buf = torch.empty(len(fields) * per, dtype=torch.uint8, device="cuda")
    for r, f in enumerate(fields):
        lex = lex_dev(f)
        if full:
            lat.pack(prec, 0, lex, buf[r * per: r * per + nb])
            lat.pack(prec, 1, lex, buf[r * per + nb: (r + 1) * per])
        else:
            lat.pack(prec, parity, lex, buf[r * per: (r + 1) * per])
    return buf


OPS = [(wd.WD_OP_HOP_EO, 1), (wd.WD_OP_HOP_OE, 0), (wd.WD_OP_EO_A, 0), (wd.WD_OP_FULL, None)]


@pytest.mark.parametrize("dims", [(6, 4, 4, 8), (8, 6, 4, 10)])
@pytest.mark.parametrize("prec,recon,arith", [("fp16", 12, 16), ("fp16", 18, 16), ("fp16", 12, 32), ("bf16", 12, 32),
                                              ("fp32", 18, 32), ("fp64", 18, 32)])
def test_batch_apply_equals_one_at_a_time(dims, prec, recon, arith):
    u = synth.gauge_random(dims, 0.5, seed=51)
    lat = lattice(u, 0.125, dims)
    lat.set_arith(arith)
    fields = [synth.gaussian_source(dims, seed=520 + r) for r in range(NRHS)]
    shapes = [(1, 0)] + ([(k, s) for k in (2, 3, 4, 6, 12) for s in (0, 1)] if arith == 16 and prec == "fp16" else [])
    for op, pin in OPS:
        src = packed_batch(lat, prec, fields, pin)
        per = src.numel() // NRHS
        want = torch.empty_like(src)
        for r in range(NRHS):
            lat.apply(prec, recon, op, src[r * per:(r + 1) * per], want[r * per:(r + 1) * per])
        for k, smem in shapes:
            lat.set_rhs_per_thread(recon, k, k, smem)
            got = torch.full_like(src, 0x7F)
            lat.apply_batch(prec, recon, op, NRHS, src, got)
            torch.cuda.synchronize()
            assert torch.equal(got, want), (op, k, smem)


def test_batch_hop_at_the_batched_size_matches_eq1():
    """H_oe of 12 Gaussian sources on 24^3 x 48 in one launch (FP16 arithmetic,
    12 right-hand sides per thread): the oracle's Eq. 1 at sampled sites, and
    every right-hand side against its own single-source result."""
    dims = (24, 24, 24, 48)
    u = synth.gauge_smeared(dims, seed=20260215, device="cuda").cpu()
    lat = lattice(u, 0.1265, dims)
    lat.set_arith(16)
    lat.set_rhs_per_thread(12, 12, 12, 1)
    fields = [synth.gaussian_source(dims, seed=530 + r) for r in range(NRHS)]
    src = packed_batch(lat, "fp16", fields, 0)
    out = torch.empty_like(src)
    lat.apply_batch("fp16", 12, wd.WD_OP_HOP_OE, NRHS, src, out)
    per = src.numel() // NRHS
    par = W.parity(dims).reshape(-1)
    odd = torch.nonzero(par == 1).reshape(-1)
    g = torch.Generator().manual_seed(5)
    sites = odd[torch.randint(len(odd), (1500,), generator=g)]
    corner = torch.tensor([1, 24 ** 3 * 48 - 2])
    sites = torch.cat([sites, corner[par[corner] == 1]])
    for r in (0, 5, 11):
        lex = torch.zeros(24 ** 3 * 48 * 24, dtype=torch.float64, device="cuda")
        lat.unpack("fp16", 1, out[r * per:(r + 1) * per], lex)
        got = synth.from_host_layout(lex.cpu(), dims).reshape(-1, 4, 3)[sites]
        want = W.hop_at_sites(u, fields[r], sites, BC)
        err = (torch.linalg.vector_norm(got - want) / torch.linalg.vector_norm(want)).item()
        assert err <= TOL["fp16a"], (r, err)
        one = torch.empty(per, dtype=torch.uint8, device="cuda")
        lat.apply("fp16", 12, wd.WD_OP_HOP_OE, src[r * per:(r + 1) * per], one)
        assert torch.equal(one, out[r * per:(r + 1) * per])


def test_twelve_point_source_batch_solve_at_24x24x24x48_satisfies_eq1():
    """The batched form's workload: the 12 spin-colour point sources at site 0
    of 24^3 x 48, one wd_solve_batch with the tuned batched kernels; every
    solution's residual eta - D_W x, evaluated by the oracle's Eq. 1 at sampled
    sites (site 0 and its neighbours among them), is within the 1e-10 bound."""
    dims = (24, 24, 24, 48)
    kappa = 0.1265
    u = synth.gauge_smeared(dims, seed=20260215, device="cuda").cpu()
    lat = lattice(u, kappa, dims)
    lat.set_arith(16)
    r = lat.tune("fp16", 12, NRHS)
    assert r["candidates16"] >= 6
    etas = [synth.point_source(dims, s, c) for s in range(4) for c in range(3)]
    b = torch.stack([lex_dev(e) for e in etas])
    x = torch.zeros_like(b)
    stats = lat.solve_rhs(b, x, 1e-10, "mixed_fp16")
    assert all(st.status == wd.WD_OK and st.true_residual <= 1e-10 for st in stats)
    g = torch.Generator().manual_seed(6)
    v = 24 ** 3 * 48
    near = torch.tensor([0, 1, 24, 24 * 24, 24 ** 3, 23, 24 * 23, v - 24 ** 3])
    sites = torch.cat([near, torch.randint(v, (2000,), generator=g)])
    for k in (0, 7, 11):
        xi = synth.from_host_layout(x[k].cpu(), dims)
        res = etas[k].reshape(-1, 4, 3)[sites] - xi.reshape(-1, 4, 3)[sites] + kappa * W.hop_at_sites(u, xi, sites, BC)
        assert torch.linalg.vector_norm(res).item() <= 1e-10 * torch.linalg.vector_norm(etas[k]).item(), k
