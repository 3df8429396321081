"""Learned right preconditioner on the GPU against the oracle (forward, gradients),
training, and the preconditioned solve."""

import pytest
import torch

from oracle import ptc
from oracle import solvers as S
from oracle import wilson as W
from paper_2602_14450_gb300 import learned, synth, wd
from tests.gpu_util import from_lex, lattice, lex_dev, rel_l2

pytestmark = pytest.mark.gpu
BC = (1, 1, 1, -1)
DIMS = (4, 4, 4, 8)
KAPPA = 0.12


def bf16_weights(seed, scale=0.1):
    w1, w2 = ptc.random_weights(seed, scale)
    flat = ptc.to_flat(w1, w2).to(torch.float32)
    flat = flat.to(torch.bfloat16).to(torch.float32)        # the kernels use BF16-rounded weights
    return flat, ptc.from_flat(flat)


def packed_even(lat, prec, field):
    buf = torch.empty(lat.vector_bytes(prec), dtype=torch.uint8, device="cuda")
    lat.pack(prec, 0, lex_dev(field), buf)
    return buf


def unpacked_even(lat, prec, buf, dims):
    out = torch.zeros(lex_dev(synth.gaussian_source(dims, 0)).shape, dtype=torch.float64, device="cuda")
    lat.unpack(prec, 0, buf, out)
    return from_lex(out, dims)


@pytest.fixture(scope="module")
def setup():
    u = synth.gauge_random(DIMS, 0.5, seed=61)
    lat = lattice(u, KAPPA, DIMS)
    return u, lat


# FP16 path: BF16 hidden fields (unit roundoff 2^-8) bounded at 1e-2 relative
@pytest.mark.parametrize("prec,tol", [("fp32", 2e-6), ("fp16", 1e-2)])
def test_forward_matches_oracle(setup, prec, tol):
    u, lat = setup
    flat, (w1, w2) = bf16_weights(seed=7)
    lat.precond_set(flat)
    psi = W.restrict(synth.gaussian_source(DIMS, seed=62), 0)
    out = torch.empty(lat.vector_bytes(prec), dtype=torch.uint8, device="cuda")
    lat.precond_apply(prec, packed_even(lat, prec, psi), out)
    got = unpacked_even(lat, prec, out, DIMS)
    want = ptc.apply(u, w1, w2, psi, BC)
    assert rel_l2(got, want) <= tol


def test_identity_weights(setup):
    u, lat = setup
    w1, w2 = ptc.identity_weights()
    lat.precond_set(ptc.to_flat(w1, w2).to(torch.float32))
    psi = W.restrict(synth.gaussian_source(DIMS, seed=63), 0)
    out = torch.empty(lat.vector_bytes("fp32"), dtype=torch.uint8, device="cuda")
    lat.precond_apply("fp32", packed_even(lat, "fp32", psi), out)
    assert rel_l2(unpacked_even(lat, "fp32", out, DIMS), psi) <= 1e-7


def test_gradients_match_oracle(setup):
    """Loss and weight gradients of wd_precond_grad against the oracle's
    autograd (itself pinned by finite differences). The fan-out layers (the
    forward layer 1 and the adjoint of layer 2) mix channels on the tensor cores
    with BF16 operands: loss within 1e-4, gradients within 1e-3 (measured
    2e-5 and 4e-4). With WD_PTC_TC=0 (FP32 cores, a child process) within 1e-5
    and 1e-4."""
    import os
    check_gradients(setup, 1e-4, 1e-3)
    if os.environ.get("WD_PTC_TC") != "0":
        import subprocess
        import sys
        root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
        code = ("import sys; sys.path.insert(0, %r); from tests import test_gpu_precond as t; "
                "from oracle import ptc; from paper_2602_14450_gb300 import synth; "
                "u = synth.gauge_random(t.DIMS, 0.5, seed=61); "
                "t.check_gradients((u, t.lattice(u, t.KAPPA, t.DIMS)), 1e-5, 1e-4); print('fp32 cores ok')" % root)
        r = subprocess.run([sys.executable, "-c", code], env=dict(os.environ, WD_PTC_TC="0"), capture_output=True,
                           text=True, timeout=300, cwd=root)
        assert r.returncode == 0 and "fp32 cores ok" in r.stdout, r.stdout + r.stderr


def check_gradients(setup, loss_tol, grad_tol):
    u, lat = setup
    flat, (w1, w2) = bf16_weights(seed=8)
    lat.precond_set(flat)
    mu = 0.5
    vs = [W.restrict(synth.gaussian_source(DIMS, seed=70 + i), 0) for i in range(2)]
    ys = [W.restrict(synth.gaussian_source(DIMS, seed=80 + i), 0) for i in range(2)]
    v = torch.stack([packed_even(lat, "fp32", f).view(torch.float32) for f in vs])
    y = torch.stack([packed_even(lat, "fp32", f).view(torch.float32) for f in ys])
    loss, g = lat.precond_grad(v, y, mu)
    # the oracle on the same (FP32-rounded) samples
    vs32 = [unpacked_even(lat, "fp32", packed_even(lat, "fp32", f), DIMS) for f in vs]
    ys32 = [unpacked_even(lat, "fp32", packed_even(lat, "fp32", f), DIMS) for f in ys]
    L, g1, g2 = ptc.grads(u, w1, w2, vs32, ys32, KAPPA, mu, BC)
    assert abs(loss - L) <= loss_tol * L
    want = ptc.to_flat(g1, g2)
    got = g.cpu().double()
    assert (torch.linalg.vector_norm(got - want) / torch.linalg.vector_norm(want)).item() <= grad_tol


def test_training_lowers_the_loss_and_preconditioned_solve_converges(setup):
    u, lat = setup
    w1, w2 = ptc.random_weights(seed=9, scale=0.02)
    lat.precond_set(ptc.to_flat(w1, w2).to(torch.float32))
    v, y = learned.make_samples(lat, 8, seed=500)
    losses = learned.train(lat, v, y, steps=40, lr=3e-3, mu=1.0, batch=4)
    assert losses[-1] < 0.8 * losses[0]
    eta = synth.gaussian_source(DIMS, seed=64)
    b = lex_dev(eta)
    x = torch.zeros_like(b)
    st = lat.solve(b, x, 1e-10, "mixed_fp16_learned")
    assert st.status == wd.WD_OK
    assert S.norm(eta - W.dirac(u, from_lex(x, DIMS), KAPPA, BC)) / S.norm(eta) <= 1e-10


def test_learned_scheme_needs_weights():
    dims = (4, 4, 4, 4)
    lat = lattice(synth.gauge_random(dims, 0.5, seed=1), 0.12, dims)
    b = lex_dev(synth.gaussian_source(dims, seed=2))
    x = torch.zeros_like(b)
    with pytest.raises(wd.WDError) as e:
        lat.solve(b, x, 1e-10, "mixed_fp16_learned")
    assert e.value.code == wd.WD_ERR_INVALID_ARG


@pytest.mark.parametrize("dims", [(6, 4, 4, 6), (8, 8, 8, 8)])
def test_collapsed_fp16_path_ragged_tiles(dims):
    """The FP16 path (tensor-core first pass, 128-site tiles) on lattices whose
    odd-site count is not a multiple of 128 (288 sites: two full tiles and a
    ragged one) and on several full tiles, against the oracle's layered network
    and against the FP32 path."""
    u = synth.gauge_random(dims, 0.5, seed=91)
    lat = lattice(u, KAPPA, dims)
    flat, (w1, w2) = bf16_weights(seed=17, scale=0.3)
    lat.precond_set(flat)
    psi = W.restrict(synth.gaussian_source(dims, seed=92), 0)
    want = ptc.apply(u, w1, w2, psi, BC)
    outs = {}
    for prec in ("fp16", "fp32"):
        out = torch.empty(lat.vector_bytes(prec), dtype=torch.uint8, device="cuda")
        lat.precond_apply(prec, packed_even(lat, prec, psi), out)
        outs[prec] = unpacked_even(lat, prec, out, dims)
    assert rel_l2(outs["fp32"], want) <= 2e-6
    assert rel_l2(outs["fp16"], want) <= 1e-2
    assert rel_l2(outs["fp16"], outs["fp32"]) <= 1e-2


def test_trained_network_reduces_matvecs():
    """What the trained network gains over the method without it: M trained on
    (v, A^{-1} v) pairs of one smeared 8^3 x 16 configuration, then the FP16
    solve preconditioned by M needs fewer FP16 matvecs than the plain FP16
    solve on a fresh source (0.55-0.6x on the 32^3 x 64 benchmark workload)."""
    dims = (8, 8, 8, 16)
    kappa = 0.1265
    u = synth.gauge_smeared(dims, seed=20260214)
    lat = lattice(u, kappa, dims)
    lat.precond_set(learned.initial_weights(11))
    v, y = learned.make_samples(lat, 8, seed=3000)
    losses = learned.train(lat, v, y, steps=120, lr=3e-3, mu=1.0, batch=4)
    assert losses[-1] < 0.5 * losses[0]
    eta = synth.gaussian_source(dims, seed=3100)
    b = lex_dev(eta)
    counts = {}
    for scheme in ("mixed_fp16", "mixed_fp16_learned"):
        x = torch.zeros_like(b)
        st = lat.solve(b, x, 1e-10, scheme)
        assert st.status == wd.WD_OK
        assert S.norm(eta - W.dirac(u, from_lex(x, dims), kappa, BC)) / S.norm(eta) <= 1e-10
        counts[scheme] = st.inner_matvecs
    print(f"\nFP16 matvecs to 1e-10, 8^3 x 16: plain {counts['mixed_fp16']}, learned M {counts['mixed_fp16_learned']}")
    assert counts["mixed_fp16_learned"] < 0.9 * counts["mixed_fp16"], counts


def test_training_is_reproducible():
    """Every sum of the training step (the loss's dot products, the weight
    gradients over sites and blocks) is taken in a fixed order, so two runs
    from the same weights on the same samples give the same losses and the
    same weights, bit for bit."""
    dims = (8, 8, 8, 8)
    lat = lattice(synth.gauge_smeared(dims, seed=71), 0.12, dims)
    v, y = learned.make_samples(lat, 4, seed=700)
    runs = []
    for _ in range(2):
        lat.precond_set(learned.initial_weights(5))
        losses = learned.train(lat, v, y, steps=6, lr=3e-3, mu=1.0, batch=2)
        runs.append((losses, lat.precond_get()))
    assert runs[0][0] == runs[1][0]
    assert torch.equal(runs[0][1], runs[1][1])


def test_specified_entry_points_load_and_train():
    """wd_precond_load takes the weights as BF16 values and loads them widened
    exactly to FP32 (the masters then equal the BF16 values); wd_precond_train
    is that many wd_precond_train_step calls on the same samples, bit for bit."""
    dims = (8, 8, 8, 8)
    lat = lattice(synth.gauge_smeared(dims, seed=71), 0.12, dims)
    v, y = learned.make_samples(lat, 2, seed=701)
    wb = learned.initial_weights(5).to(torch.bfloat16)
    lat.precond_load(wb)
    assert torch.equal(lat.precond_get(), wb.to(torch.float32))
    last = lat.precond_train(3, v, y, 1.0, 3e-3)
    trained = lat.precond_get()
    lat.precond_load(wb)
    losses = [lat.precond_train_step(v, y, 1.0, 3e-3) for _ in range(3)]
    assert last == losses[-1]
    assert torch.equal(trained, lat.precond_get())
