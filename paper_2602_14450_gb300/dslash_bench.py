"""Dslash micro-benchmark: the hopping kernel H_eo through wd_apply, and the
learned preconditioner M through wd_precond_apply.

    python -m paper_2602_14450_gb300.dslash_bench --dims 32,32,32,64 --cases fp16_12,fp32_18 --launches 50
    python -m paper_2602_14450_gb300.dslash_bench --dims 32,32,32,64 --cases m_fp16 --launches 20

Case "fp16a_R" is FP16 storage with FP16 arithmetic (wd_set_arith(16)).

Links are exp(i 0.5 H) random SU(3) matrices generated on the GPU; inputs
cycle through four different source vectors so that consecutive launches do
not find their input in L2 (at 32^3 x 64 every launch streams more than L2
holds anyway). Prints one JSON line per case: average launch time from CUDA
events on the launching stream, algorithmic bytes per output site and GB/s.
"""

from __future__ import annotations

import argparse
import json

import torch

BYTES = {"fp64": 8, "fp32": 4, "fp16": 2, "bf16": 2}


def bytes_per_site(prec: str, recon: int) -> int:
    """Input spinor + output spinor (24 reals each) + 8 links of `recon` reals."""
    b = BYTES[prec]
    return 2 * 24 * b + 8 * recon * b


def hop_timing(lat, prec: str, recon: int, launches: int, stream=None) -> dict:
    """Case "fp16" is FP16 storage with FP32 arithmetic, "fp16a" with FP16
    arithmetic, whatever the lattice's setting; the setting is restored."""
    if prec in ("fp16", "fp16a"):
        old = lat.arith
        lat.set_arith(16 if prec == "fp16a" else 32)
        try:
            r = _hop_timing(lat, "fp16", recon, launches, stream)
        finally:
            lat.set_arith(old)
        r["case"] = f"{prec}_{recon}"
        return r
    return _hop_timing(lat, prec, recon, launches, stream)


def _hop_timing(lat, prec: str, recon: int, launches: int, stream=None) -> dict:
    from . import wd
    vh = lat.vector_bytes(prec) // (24 * BYTES[prec])
    nb = lat.vector_bytes(prec)
    ins = []
    for k in range(4):
        f = torch.randn(vh * 24, dtype=torch.float64, device="cuda")
        ins.append(f.to({"fp64": torch.float64, "fp32": torch.float32, "fp16": torch.float16,
                         "bf16": torch.bfloat16}[prec]).view(torch.uint8))
    out = torch.empty(nb, dtype=torch.uint8, device="cuda")
    stream = stream or torch.cuda.current_stream()
    for i in range(5):
        lat.apply(prec, recon, wd.WD_OP_HOP_EO, ins[i % 4], out, stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(launches):
        lat.apply(prec, recon, wd.WD_OP_HOP_EO, ins[i % 4], out, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) * 1e3 / launches
    bps = bytes_per_site(prec, recon)
    return {"case": f"{prec}_{recon}", "us": us, "bytes_per_site": bps, "sites": vh, "gbs": bps * vh / (us * 1e-6) / 1e9}


def precond_timing(lat, prec: str, launches: int, stream=None) -> dict:
    """Average time of one application of M (two kernels) on packed even-site vectors."""
    from . import learned
    lat.precond_set(learned.initial_weights(3, scale=0.1))
    vh = lat.vector_bytes(prec) // (24 * BYTES[prec])
    ins = [torch.randn(vh * 24, dtype=torch.float64, device="cuda").to(
        {"fp32": torch.float32, "fp16": torch.float16}[prec]).view(torch.uint8) for _ in range(4)]
    out = torch.empty(lat.vector_bytes(prec), dtype=torch.uint8, device="cuda")
    stream = stream or torch.cuda.current_stream()
    for i in range(3):
        lat.precond_apply(prec, ins[i % 4], out, stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(launches):
        lat.precond_apply(prec, ins[i % 4], out, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    return {"case": f"m_{prec}", "us": e0.elapsed_time(e1) * 1e3 / launches, "sites": vh}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", default="32,32,32,64")
    ap.add_argument("--cases", default="fp16_12,fp16_18,fp16a_12,fp16a_18,fp32_12,fp32_18,fp64_18,bf16_12")
    ap.add_argument("--launches", type=int, default=50)
    a = ap.parse_args()
    from . import build, synth, wd
    build.build()
    dims = tuple(int(d) for d in a.dims.split(","))
    u = synth.gauge_random(dims, 0.5, seed=1, device="cuda")
    lat = wd.Lattice(dims, 0.12)
    lat.set_gauge(torch.view_as_real(u).contiguous())
    del u
    torch.cuda.empty_cache()
    for c in a.cases.split(","):
        prec, recon = c.split("_")
        if prec == "m":
            print(json.dumps(precond_timing(lat, recon, a.launches)), flush=True)
        else:
            print(json.dumps(hop_timing(lat, prec, int(recon), a.launches)), flush=True)


if __name__ == "__main__":
    main()
