"""In-graph kernel timeline of the benchmark solve (the library's timeline build).

    python -m paper_2602_14450_gb300.timeline [--workload 32x32x32x64] [--arith 16]

Builds libwd_timeline.so (-DWD_TIMELINE, see wd_timeline_set), sets up the
solve as bench.py does (autotuned kernels, warm-up solves), then runs one solve
with recording on and prints, per kernel site:
  - launches and mean duration inside the captured graphs (first block start
    to last block end; the start is after the wait for the preceding kernel),
  - the median gap to the next kernel and the number of gaps above 5 us (graph
    and refinement-trip boundaries),
  - how long the last block outlasts the one before it (the grid reduction's
    last block, which sums the partial sums and runs the scalar stage),
and for the grid reductions the mean time of each phase of their last block.
ncu serialises launches, so this is the view of the kernels as the solver
runs them back to back; the recording adds about 1% to the solve.
"""

from __future__ import annotations

import argparse
import glob
import os
import re

import numpy as np
import torch

from . import build as B

STAGES = {1: "init", 2: "alpha", 3: "omega", 4: "rnorm", 5: "end", 6: "outer", 7: "acc", 8: "acc_set",
          9: "end (fused rescaling)"}
TAGS = {1: "(r*,v)", 2: "(t,s)", 3: "norm"}   # the reduction a hop's records are tagged with
PHASES = ["block sum", "partials out", "ticket", "barrier", "partials summed", "block sum 2", "scalar stage",
          "ticket re-armed"]


def name_hash(s: str) -> int:
    h = 7
    for c in s.encode():
        h = (h * 31 + c) & 0xFFFFFFFF
    return h & 0xFFFF


def kernel_sites() -> dict:
    """(file-name hash, line) of each pdl_begin() -> 'file:line kernel'."""
    sites = {}
    for path in glob.glob(os.path.join(B.CSRC, "*.cu*")):
        lines = open(path).read().splitlines()
        base = os.path.basename(path)
        last_global = 0
        for i, line in enumerate(lines, 1):
            if "__global__" in line:
                last_global = i
            if line.strip().startswith("pdl_begin();") and last_global:
                text = " ".join(lines[last_global - 1: i])
                names = re.findall(r"\b(k_\w+|\w+_kernel)\s*\(", text)
                sites[(name_hash(base), i)] = f"{base}:{i} {names[-1] if names else '?'}"
    return sites


def launches_of(rec: np.ndarray):
    """Group block records into launches: a new launch where the kernel site
    or grid changes, or where a block starts after every earlier block ended."""
    key = rec[:, 0] >> 8
    o = np.argsort(rec[:, 2], kind="stable")
    rec, key = rec[o], key[o]
    end_so_far = np.maximum.accumulate(rec[:, 3])
    new = np.ones(len(rec), dtype=bool)
    new[1:] = (key[1:] != key[:-1]) | (rec[1:, 2] > end_so_far[:-1])
    starts = np.nonzero(new)[0]
    ends = np.append(starts[1:], len(rec))
    out = []
    for s0, s1 in zip(starts, ends):
        r = rec[s0:s1]
        te = np.sort(r[:, 3])
        out.append({"site": int((r[0, 0] >> 32) & 0xFFFFFFFF), "grid": int((r[0, 0] >> 8) & 0xFFFFFF), "blocks": s1 - s0,
                    "start": int(r[:, 2].min()), "end": int(te[-1]),
                    "last_block": float(te[-1] - te[-2]) if s1 - s0 > 1 else 0.0})
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="32x32x32x64")
    ap.add_argument("--arith", type=int, default=16, choices=(16, 32))
    args = ap.parse_args()
    lib_path = B.build(timeline=True)
    from . import synth, wd, workloads
    wd.use_library(lib_path)

    wl = workloads.get(args.workload)
    lat = wd.Lattice(wl.dims, wl.kappa)
    lat.set_gauge(torch.view_as_real(wl.gauge(device="cpu")).contiguous())
    b = synth.to_host_layout(wl.source()).cuda()
    x = torch.zeros_like(b)
    prm = wd.default_params("mixed_fp16")
    stream = torch.cuda.current_stream()
    lat.set_arith(args.arith)
    for p, r in (("fp16", 12), ("fp64", 18), ("fp32", 12)):
        lat.tune(p, r, 1, stream)
    for _ in range(2):
        lat.solve(b, x, 1e-10, "mixed_fp16", prm, stream)
    torch.cuda.synchronize()

    blocks = torch.zeros(1 + 4 * (1 << 24), dtype=torch.int64, device="cuda")
    phases = torch.zeros(1 + 10 * (1 << 20), dtype=torch.int64, device="cuda")
    L = wd.lib()
    if L.wd_timeline_set(blocks.data_ptr(), phases.data_ptr()) != 0:
        raise RuntimeError("wd_timeline_set failed")
    torch.cuda.synchronize()
    st = lat.solve(b, x, 1e-10, "mixed_fp16", prm, stream)
    torch.cuda.synchronize()
    L.wd_timeline_set(None, None)
    nb, nph = int(blocks[0].item()), int(phases[0].item())
    rec = blocks[1: 1 + 4 * min(nb, 1 << 24)].view(-1, 4).cpu().numpy().astype(np.int64)
    ph = phases[1: 1 + 10 * min(nph, 1 << 20)].view(-1, 10).cpu().numpy().astype(np.int64)

    if nb == 0:
        raise RuntimeError("no kernel blocks were recorded (is libwd_timeline.so the library in use?)")
    sites = kernel_sites()
    ls = launches_of(rec)
    span = (ls[-1]["end"] - ls[0]["start"]) / 1e3
    busy = sum(l["end"] - l["start"] for l in ls) / 1e3
    print(f"solve: {st.elapsed_ms:.1f} ms with recording, {st.inner_matvecs} FP16 matvecs, "
          f"{st.outer_iterations} refinement trips; {len(ls)} recorded launches over {span / 1e3:.1f} ms, "
          f"{busy / 1e3:.1f} ms inside them")
    stats = {}
    for j, l in enumerate(ls):
        gap = (ls[j + 1]["start"] - l["end"]) / 1e3 if j + 1 < len(ls) else 0.0
        site, tag = l["site"], (l["site"] >> 12) & 0xF
        name = sites.get((site >> 16, site & 0xFFF), f"site {site:#x}") + (f" {TAGS.get(tag, tag)}" if tag else "")
        k = (name, l["grid"])
        d = stats.setdefault(k, [0, 0.0, 0.0, 0.0, []])
        d[0] += 1
        d[1] += (l["end"] - l["start"]) / 1e3
        d[2] += l["last_block"] / 1e3
        d[4].append(gap)
    print(f"\n{'kernel (file:line of pdl_begin)':<44} {'grid':>6} {'launches':>8} {'mean us':>8} "
          f"{'med gap us':>10} {'gaps>5us':>8} {'last blk us':>11} {'total ms':>9}")
    for (name, grid), d in sorted(stats.items(), key=lambda kv: -kv[1][1]):
        g = np.array(d[4])
        print(f"{name:<44} {grid:>6} {d[0]:>8} {d[1] / d[0]:>8.2f} {np.median(g):>10.2f} {int((g > 5).sum()):>8} "
              f"{d[2] / d[0]:>11.2f} {d[1] / 1e3:>9.2f}")
    if len(ph):
        print(f"\nlast block of the grid reductions, mean us per phase ({' | '.join(PHASES)}):")
        for sg in sorted(set((ph[:, 0] >> 32).tolist())):
            m = (ph[:, 0] >> 32) == sg
            t = np.diff(ph[m][:, 1:], axis=1).mean(axis=0) / 1e3
            print(f"  {STAGES.get(sg, sg):<22} sums {int(ph[m][0, 0] & 0xFFFFFFFF)} x{int(m.sum()):>4}: "
                  + " | ".join(f"{v:.2f}" for v in t))


if __name__ == "__main__":
    main()
