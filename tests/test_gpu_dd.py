"""The split hopping term on the GPU (wd_dd_* through paper_2602_14450_gb300.dd):
several sub-lattice handles in one process, faces moved by copies between
launches (no kernel waits on another), against the undivided oracle (Eq. 1,
Eq. 4), the undivided library operator, and an FP64 BiCGStab solve across
the sub-lattices."""

import ctypes as C

import pytest
import torch

from oracle import solvers as S
from oracle import wilson as W
from paper_2602_14450_gb300 import dd, synth, wd
from tests.gpu_util import TOL, apply_op, gauge_host, lattice, rel_l2

pytestmark = pytest.mark.gpu
BC = (1, 1, 1, -1)
KAPPA = 0.12
DIMS = (4, 4, 8, 8)


def gpu_set(u, grid, prec, recon, arith=32, dims=DIMS):
    parts = [dd.Partition(dims, grid, r) for r in range(dd.Partition(dims, grid, 0).size)]
    doms = [dd.GpuDomain(p, KAPPA, gauge_host(p.scatter_gauge(u)), prec, recon, BC, arith) for p in parts]
    return parts, dd.DomainSet(doms, dd.LocalComm(parts))


def to_packed(parts, ds, field, parity):
    vs = []
    for q, d in zip(parts, ds.domains):
        v = d.new_vector()
        d.pack_field(parity, synth.to_host_layout(q.scatter_field(field)).cuda(), v)
        vs.append(v)
    return vs


def from_packed(parts, ds, vs, parity):
    out = []
    for q, d, v in zip(parts, ds.domains, vs):
        lex = torch.zeros(q.local_dims[0] * q.local_dims[1] * q.local_dims[2] * q.local_dims[3] * 24,
                          dtype=torch.float64, device="cuda")
        d.unpack_field(parity, v, lex)
        out.append(synth.from_host_layout(lex.cpu(), q.local_dims))
    torch.cuda.synchronize()
    return dd.Partition.gather_field(out, [q.block() for q in parts])


CASES = [("fp64", 18, 32, "fp64"), ("fp32", 18, 32, "fp32"), ("fp32", 12, 32, "fp32"), ("fp16", 12, 32, "fp16"),
         ("fp16", 12, 16, "fp16a"), ("bf16", 12, 32, "bf16")]


@pytest.mark.parametrize("grid", [(1, 1, 1, 2), (1, 1, 2, 2), (2, 2, 2, 2), (1, 2, 1, 4)])
@pytest.mark.parametrize("prec,recon,arith,tol", CASES)
def test_split_hop_matches_oracle(grid, prec, recon, arith, tol):
    u = synth.gauge_random(DIMS, 0.5, seed=21)
    psi = synth.gaussian_source(DIMS, seed=22)
    parts, ds = gpu_set(u, grid, prec, recon, arith)
    for p in (0, 1):
        xs = to_packed(parts, ds, psi, 1 - p)
        outs = ds.new_vectors()
        dd.hop(ds, p, xs, outs)
        got = from_packed(parts, ds, outs, p)
        want = W.hop_pq(u, psi, p, BC)
        assert rel_l2(got, want) <= TOL[tol], (p, rel_l2(got, want))
        if prec == "fp64":
            assert torch.allclose(got, want, rtol=0, atol=1e-13 * want.abs().max().item())


@pytest.mark.parametrize("prec,recon,arith,tol", CASES)
def test_split_eo_operator_matches_undivided_library(prec, recon, arith, tol):
    """The split A = 1 - kappa^2 H_eo H_oe (Eq. 4) against wd_apply(WD_OP_EO_A)
    on the undivided lattice and against the oracle."""
    u = synth.gauge_random(DIMS, 0.5, seed=23)
    psi = W.restrict(synth.gaussian_source(DIMS, seed=24), 0)
    parts, ds = gpu_set(u, (1, 1, 2, 2), prec, recon, arith)
    xs = to_packed(parts, ds, psi, 0)
    outs, tmps = ds.new_vectors(), ds.new_vectors()
    dd.eo_operator(ds, xs, outs, tmps)
    got = from_packed(parts, ds, outs, 0)
    lat = lattice(u, KAPPA, DIMS)
    lat.set_arith(arith)
    whole = apply_op(lat, prec, recon, wd.WD_OP_EO_A, psi, DIMS)
    want = W.eo_operator(u, psi, KAPPA, BC)
    assert rel_l2(got, want) <= TOL[tol]
    assert rel_l2(got, whole) <= (1e-14 if prec == "fp64" else TOL[tol])


def test_split_fp64_bicgstab_matches_oracle_and_undivided_solve():
    """FP64 BiCGStab across four sub-lattices (global FP64 dot products) solves
    the even-odd system like the undivided oracle and the library's wd_solve."""
    u = synth.gauge_random(DIMS, 0.5, seed=25)
    eta = synth.gaussian_source(DIMS, seed=26)
    b = W.eo_source(u, eta, KAPPA, BC)
    parts, ds = gpu_set(u, (1, 1, 2, 2), "fp64", 18)
    xs = ds.new_vectors()
    it, res = dd.bicgstab(ds, to_packed(parts, ds, b, 0), xs, 1e-12)
    x = from_packed(parts, ds, xs, 0)
    x0, info = S.bicgstab(lambda v: W.eo_operator(u, v, KAPPA, BC), b, 1e-12)
    assert res <= 1e-12
    assert abs(it - info.iterations) <= 2
    assert S.norm(x - x0) <= 1e-11 * S.norm(x0)
    xi = W.eo_reconstruct(u, x, eta, KAPPA, BC)
    assert S.norm(eta - W.dirac(u, xi, KAPPA, BC)) <= 1e-11 * S.norm(eta)
    lat = lattice(u, KAPPA, DIMS)
    bl = synth.to_host_layout(eta).cuda()
    xl = torch.zeros_like(bl)
    st = lat.solve(bl, xl, 1e-12, "fp64")
    assert st.status == wd.WD_OK
    x_lib = W.restrict(synth.from_host_layout(xl.cpu(), DIMS), 0)
    assert S.norm(x - x_lib) <= 1e-10 * S.norm(x_lib)


def test_split_handle_refuses_whole_lattice_calls():
    u = synth.gauge_random(DIMS, 0.5, seed=27)
    parts, ds = gpu_set(u, (1, 1, 1, 2), "fp16", 12)
    d = ds.domains[0]
    x, y = d.new_vector(), d.new_vector()
    with pytest.raises(wd.WDError) as e:
        d.lat.apply("fp16", 12, wd.WD_OP_EO_A, x, y)
    assert e.value.code == wd.WD_ERR_INVALID_ARG
    # face buffers: 12 FP16 reals per face site, V_local / 2 / L_t face sites
    assert d.lat.dd_face_bytes("fp16", 3) == (4 * 4 * 8 * 4 // 2 // 4) * 12 * 2
    with pytest.raises(wd.WDError):
        d.lat.dd_set_partition((1, 1, 1, 2), (0, 0, 0, 2))
    # undoing the split gives the whole-lattice operator back
    d.lat.dd_set_partition((1, 1, 1, 1), (0, 0, 0, 0))
    d.lat.apply("fp16", 12, wd.WD_OP_HOP_EO, x, y)
    rc = wd.lib().wd_dd_pack(d.lat.h, wd.WD_FP16, 0, C.c_void_p(x.data_ptr()), None, None)
    assert rc == wd.WD_ERR_INVALID_ARG
