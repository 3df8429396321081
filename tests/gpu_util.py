"""Helpers of the GPU tests: move oracle fields through the C ABI and back."""

import torch

from paper_2602_14450_gb300 import synth, wd

# Relative L2 bounds of one operator application against the float64 oracle.
# FP16: inputs and links rounded to 11 significant bits (unit roundoff 2^-11)
# and FP32 arithmetic; FP32: 2^-24 rounding; BF16: 8 significant bits
# (2^-8 unit roundoff); FP64: rounding of ~1e3 operations. "fp16a": FP16
# storage and FP16 arithmetic (wd_set_arith(16)), the benchmark's arithmetic:
# held to the same 2e-3 as FP16 storage with FP32 arithmetic, the bound the
# FP16 hopping term is specified to meet against float64. Its roundings
# (projection, rebuilt third link row, packed FMAs, eight accumulations) stay
# well inside it (about 7e-4 measured on smeared and on rough links).
TOL = {"fp64": 1e-13, "fp32": 1e-6, "fp16": 2e-3, "bf16": 1.6e-2, "fp16a": 2e-3}


def gauge_host(u: torch.Tensor) -> torch.Tensor:
    return torch.view_as_real(u.contiguous()).contiguous()


def lattice(u, kappa, dims, bc=(1, 1, 1, -1)):
    lat = wd.Lattice(dims, kappa, bc)
    lat.set_gauge(gauge_host(u))
    return lat


def lex_dev(f: torch.Tensor) -> torch.Tensor:
    return synth.to_host_layout(f).cuda()


def from_lex(t: torch.Tensor, dims) -> torch.Tensor:
    return synth.from_host_layout(t.cpu(), dims)


def packed(lat, prec, n=1):
    return torch.empty(n * lat.vector_bytes(prec), dtype=torch.uint8, device="cuda")


def apply_op(lat, prec, recon, op, psi, dims):
    """Apply a wd_apply operator to a full-lattice complex field; returns the full-lattice result."""
    lex = lex_dev(psi)
    nb = lat.vector_bytes(prec)
    out_lex = torch.zeros_like(lex)
    if op == wd.WD_OP_FULL:
        src, dst = packed(lat, prec, 2), packed(lat, prec, 2)
        lat.pack(prec, 0, lex, src[:nb])
        lat.pack(prec, 1, lex, src[nb:])
        lat.apply(prec, recon, op, src, dst)
        lat.unpack(prec, 0, dst[:nb], out_lex)
        lat.unpack(prec, 1, dst[nb:], out_lex)
    else:
        pin = {wd.WD_OP_HOP_EO: 1, wd.WD_OP_HOP_OE: 0, wd.WD_OP_EO_A: 0}[op]
        pout = {wd.WD_OP_HOP_EO: 0, wd.WD_OP_HOP_OE: 1, wd.WD_OP_EO_A: 0}[op]
        src, dst = packed(lat, prec), packed(lat, prec)
        lat.pack(prec, pin, lex, src)
        lat.apply(prec, recon, op, src, dst)
        lat.unpack(prec, pout, dst, out_lex)
    torch.cuda.synchronize()
    return from_lex(out_lex, dims)


def rel_l2(a, b):
    return (torch.linalg.vector_norm((a - b).reshape(-1)) / torch.linalg.vector_norm(b.reshape(-1))).item()
