"""Bounded device waits that run out (wd_set_wait_limit(h, 0)): the kernel
raises its flag, lets its own copies and tensor-core operations in flight
finish, frees its tensor memory and returns; the call reports
WD_ERR_TIMEOUT and the handle stays usable. No trap, no fault: the waits are
made to give up, the work they wait for still completes."""

import os
import subprocess
import sys

import pytest
import torch

from oracle import ptc
from oracle import wilson as W
from paper_2602_14450_gb300 import synth, wd
from tests.gpu_util import lattice, lex_dev

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _packed_even(lat, prec, field):
    buf = torch.empty(lat.vector_bytes(prec), dtype=torch.uint8, device="cuda")
    lat.pack(prec, 0, lex_dev(field), buf)
    return buf


def test_tensor_core_wait_runs_out_and_the_handle_recovers():
    dims = (8, 8, 8, 8)
    lat = lattice(synth.gauge_random(dims, 0.5, seed=31), 0.12, dims)
    w1, w2 = ptc.random_weights(32, 0.1)
    lat.precond_set(ptc.to_flat(w1, w2).to(torch.float32))
    src = _packed_even(lat, "fp16", W.restrict(synth.gaussian_source(dims, seed=33), 0))
    ref = torch.empty_like(src)
    lat.precond_apply("fp16", src, ref)                       # tensor-core first pass
    torch.cuda.synchronize()
    lat.set_wait_limit(0)
    for _ in range(2):
        out = torch.empty_like(src)
        with pytest.raises(wd.WDError) as e:
            lat.precond_apply("fp16", src, out)
        assert e.value.code == wd.WD_ERR_TIMEOUT
    # a learned solve reports the timeout for its right-hand side (identity weights: M = 1, a preconditioner
    # that cannot spoil the recovery solve below)
    w1, w2 = ptc.identity_weights()
    lat.precond_set(ptc.to_flat(w1, w2).to(torch.float32))
    b = lex_dev(synth.gaussian_source(dims, seed=34))
    x = torch.zeros_like(b)
    prm = wd.default_params("mixed_fp16_learned")
    prm.max_outer, prm.max_inner = 2, 20
    st = lat.solve(b, x, 1e-10, "mixed_fp16_learned", prm, check=False)
    assert st.status == wd.WD_ERR_TIMEOUT
    # back to the default limit: the tensor memory was freed and the same call succeeds, bit for bit
    lat.set_wait_limit(-1)
    st = lat.solve(b, torch.zeros_like(b), 1e-10, "mixed_fp16_learned")
    assert st.status == wd.WD_OK
    lat.precond_set(ptc.to_flat(*ptc.random_weights(32, 0.1)).to(torch.float32))
    again = torch.empty_like(src)
    lat.precond_apply("fp16", src, again)
    torch.cuda.synchronize()
    assert torch.equal(again, ref)


def test_wait_limit_rejects_out_of_range():
    lat = wd.Lattice((4, 4, 4, 4), 0.12)
    with pytest.raises(wd.WDError) as e:
        lat.set_wait_limit(1 << 40)
    assert e.value.code == wd.WD_ERR_INVALID_ARG


_STAGED_HOP = r"""
import sys, torch
sys.path.insert(0, {root!r})
from paper_2602_14450_gb300 import synth, wd
dims = (8, 8, 8, 16)
lat = wd.Lattice(dims, 0.12)
lat.set_gauge(torch.view_as_real(synth.gauge_random(dims, 0.5, seed=35)).contiguous())
b = synth.to_host_layout(synth.gaussian_source(dims, seed=36)).cuda()
prm = wd.default_params("mixed_fp16")
prm.max_outer, prm.max_inner = 2, 20
lat.set_wait_limit(0)
st = lat.solve(b, torch.zeros_like(b), 1e-10, "mixed_fp16", prm, check=False)
assert st.status == wd.WD_ERR_TIMEOUT, st.as_dict()
lat.set_wait_limit(-1)
st = lat.solve(b, torch.zeros_like(b), 1e-10, "mixed_fp16")
assert st.status == wd.WD_OK and st.true_residual <= 1e-10, st.as_dict()
print("staged-hop timeout ok")
"""


def test_bulk_copy_wait_of_the_staged_hop_runs_out():
    """The shared-memory staged hop (kernel variant 3, chosen for the whole
    process by WD_HOP_KERNEL, hence a child process) gives up its wait for the
    bulk copies of a tile at once, lets them land and returns; the solve
    reports WD_ERR_TIMEOUT, and with the default limit the same handle solves."""
    env = dict(os.environ, WD_HOP_KERNEL="3")
    r = subprocess.run([sys.executable, "-c", _STAGED_HOP.format(root=ROOT)], env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "staged-hop timeout ok" in r.stdout
