"""wd_apply_eo_noalloc: the even-odd operator for callers that cannot allocate.

Some callers must not have the library call cudaMalloc: code running under a
caching allocator that owns all device memory, or code that must avoid the
implicit device synchronization of cudaMalloc/cudaFree. This entry point keeps
its odd-site intermediate in a fixed array of the library's device memory. It
must give the same result as wd_apply(WD_OP_EO_A), call after call.
"""

import ctypes as C

import pytest
import torch

from paper_2602_14450_gb300 import synth, wd
from tests.gpu_util import TOL, gauge_host, lex_dev, rel_l2

pytestmark = pytest.mark.gpu


def packed_even(lat, prec, field):
    buf = torch.empty(lat.vector_bytes(prec), dtype=torch.uint8, device="cuda")
    lat.pack(prec, 0, lex_dev(field), buf)
    return buf


def as_even(lat, prec, buf, dims):
    out = torch.zeros(lex_dev(synth.gaussian_source(dims, 0)).shape, dtype=torch.float64, device="cuda")
    lat.unpack(prec, 0, buf, out)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("prec,recon,arith", [("fp16", 12, 32), ("fp16", 12, 16), ("fp32", 18, 32), ("fp64", 18, 32)])
def test_noalloc_matches_wd_apply_twice(prec, recon, arith):
    dims = (8, 6, 4, 10)
    lat = wd.Lattice(dims, 0.125)
    lat.set_gauge(gauge_host(synth.gauge_random(dims, 0.5, seed=71)))
    lat.set_arith(arith)
    src = packed_even(lat, prec, synth.gaussian_source(dims, seed=72))
    ref = torch.empty_like(src)
    lat.apply(prec, recon, wd.WD_OP_EO_A, src, ref)        # existing entry point (also builds the links)
    want = as_even(lat, prec, ref, dims)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        out = torch.full_like(src, 0xFF)
        rc = wd.lib().wd_apply_eo_noalloc(lat.h, wd.PREC[prec], recon, C.c_void_p(src.data_ptr()),
                                          C.c_void_p(out.data_ptr()), stream)
        assert rc == wd.WD_OK, wd.lib().wd_last_error(lat.h)
        got = as_even(lat, prec, out, dims)
        assert rel_l2(got, want) <= TOL["fp16a" if arith == 16 else prec]
        assert torch.equal(got, want)


def _noalloc(lat, prec, recon, src):
    out = torch.full_like(src, 0xFF)
    rc = wd.lib().wd_apply_eo_noalloc(lat.h, wd.PREC[prec], recon, C.c_void_p(src.data_ptr()),
                                      C.c_void_p(out.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, out


@pytest.mark.parametrize("prec,recon,arith", [("fp16", 12, 16), ("fp32", 18, 32), ("fp64", 18, 32)])
def test_noalloc_with_clover_matches_wd_apply(prec, recon, arith):
    """With a clover term both entry points give in - kappa^2 C_ee^-1 H_eo C_oo^-1 H_oe in (Eq. 4)."""
    dims = (8, 6, 4, 10)
    lat = wd.Lattice(dims, 0.125)
    lat.set_gauge(gauge_host(synth.gauge_random(dims, 0.5, seed=73)))
    lat.set_arith(arith)
    src = packed_even(lat, prec, synth.gaussian_source(dims, seed=74))
    plain = torch.empty_like(src)
    lat.apply(prec, recon, wd.WD_OP_EO_A, src, plain)        # Wilson A; builds the links
    lat.set_clover(1.0)
    rc, _ = _noalloc(lat, prec, recon, src)                 # clover blocks of prec not built yet
    assert rc == wd.WD_ERR_INVALID_ARG
    assert b"clover" in wd.lib().wd_last_error(lat.h)
    ref = torch.empty_like(src)
    lat.apply(prec, recon, wd.WD_OP_EO_A, src, ref)          # builds the blocks
    assert not torch.equal(ref, plain)
    for _ in range(2):
        rc, out = _noalloc(lat, prec, recon, src)
        assert rc == wd.WD_OK, wd.lib().wd_last_error(lat.h)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)


@pytest.mark.parametrize("prec,recon", [("fp16", 12), ("bf16", 12), ("fp32", 12)])
def test_noalloc_after_tune_matches_wd_apply(prec, recon):
    """After wd_tune both entry points run the tuned kernels and give the same bits."""
    dims = (8, 8, 8, 16)
    lat = wd.Lattice(dims, 0.125)
    lat.set_gauge(gauge_host(synth.gauge_random(dims, 0.5, seed=75)))
    src = packed_even(lat, prec, synth.gaussian_source(dims, seed=76))
    ref = torch.empty_like(src)
    lat.apply(prec, recon, wd.WD_OP_EO_A, src, ref)
    lat.tune(prec, recon)
    lat.apply(prec, recon, wd.WD_OP_EO_A, src, ref)
    for _ in range(2):
        rc, out = _noalloc(lat, prec, recon, src)
        assert rc == wd.WD_OK, wd.lib().wd_last_error(lat.h)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)


def test_noalloc_refuses_oversized_and_unbuilt():
    dims = (24, 24, 24, 48)                                  # FP64 odd-site vector: 63.7 MB > 16 MiB
    lat = wd.Lattice(dims, 0.12)
    lat.set_gauge(gauge_host(synth.gauge_unit(dims)))
    buf = torch.zeros(lat.vector_bytes("fp64"), dtype=torch.uint8, device="cuda")
    out = torch.zeros_like(buf)
    rc = wd.lib().wd_apply_eo_noalloc(lat.h, wd.WD_FP64, 18, C.c_void_p(buf.data_ptr()), C.c_void_p(out.data_ptr()),
                                      None)
    assert rc == wd.WD_ERR_INVALID_ARG
    assert b"16" in wd.lib().wd_last_error(lat.h)
    # FP16 fits, but its links have not been built by an allocating call yet
    b16 = torch.zeros(lat.vector_bytes("fp16"), dtype=torch.uint8, device="cuda")
    o16 = torch.zeros_like(b16)
    rc = wd.lib().wd_apply_eo_noalloc(lat.h, wd.WD_FP16, 12, C.c_void_p(b16.data_ptr()), C.c_void_p(o16.data_ptr()),
                                      None)
    assert rc == wd.WD_ERR_INVALID_ARG
