"""Training of the learned right preconditioner M through the C ABI.

Samples are (v, y = A^{-1} v) with v a Gaussian even-site vector: the plain
FP64 solver solves D xi = eta for eta = v on the even sites and 0 on the odd
sites, whose even part is exactly A^{-1} v (Eqs. 4-5). All arithmetic runs in
the library's kernels (packing, solves, forward/backward network, Adam);
this module only sequences the calls.
"""

from __future__ import annotations

import torch

from . import synth, wd


def even_only(lat: "wd.Lattice", eta_lex: torch.Tensor) -> torch.Tensor:
    """Zero the odd sites of a device FP64 lexicographic field (pack, then unpack into zeros)."""
    buf = torch.empty(lat.vector_bytes("fp64"), dtype=torch.uint8, device="cuda")
    lat.pack("fp64", 0, eta_lex, buf)
    out = torch.zeros_like(eta_lex)
    lat.unpack("fp64", 0, buf, out)
    return out


def make_samples(lat: "wd.Lattice", n: int, seed: int, tol: float = 1e-10):
    """n training pairs as packed FP32 even-site vectors, shape [n, bytes/4] float32 (device)."""
    nb = lat.vector_bytes("fp32")
    v = torch.empty((n, nb // 4), dtype=torch.float32, device="cuda")
    y = torch.empty_like(v)
    for i in range(n):
        eta = even_only(lat, synth.to_host_layout(synth.gaussian_source(lat.dims, seed=seed + i)).cuda())
        xi = torch.zeros_like(eta)
        lat.solve(eta, xi, tol, "fp64")
        lat.pack("fp32", 0, eta, v[i])
        lat.pack("fp32", 0, xi, y[i])
    return v, y


def train(lat: "wd.Lattice", v, y, steps: int, lr: float = 2e-3, mu: float = 1.0, batch: int = 4, log=None):
    """Adam steps over mini-batches of the samples; returns the loss of every step."""
    losses = []
    n = v.shape[0]
    for k in range(steps):
        i0 = (k * batch) % n
        idx = [(i0 + j) % n for j in range(batch)]
        vb, yb = v[idx].contiguous(), y[idx].contiguous()
        losses.append(lat.precond_train_step(vb, yb, mu, lr) / batch)
        if log and (k % 10 == 0 or k == steps - 1):
            log(f"step {k}: loss {losses[-1]:.4e}")
    return losses


def initial_weights(seed: int, scale: float = 0.02, c_mid: int = 12) -> torch.Tensor:
    """Flat FP32 weights of M = 1 (layer 1 hop 0 -> hidden channel 0 and layer 2
    hidden channel 0 -> output are the spin identity, all else 0) plus real and
    imaginary Gaussian noise of the given scale (seeded, numpy PCG64)."""
    import numpy as np
    per_layer = 9 * c_mid * 16 * 2
    w = np.random.default_rng(seed).normal(0.0, scale, 2 * per_layer)
    w1 = w[:per_layer].reshape(9, c_mid, 4, 4, 2)
    w2 = w[per_layer:].reshape(9, c_mid, 4, 4, 2)
    for s in range(4):
        w1[0, 0, s, s, 0] += 1.0
        w2[0, 0, s, s, 0] += 1.0
    return torch.from_numpy(w).to(torch.float32)
