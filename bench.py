#!/usr/bin/env python3
"""Benchmark: time to |b - D x| / |b| <= 1e-10 for the Wilson-Dirac system on
32^3 x 64 with the mixed FP16/FP64 solver (Alg. 3 + Alg. 4), beside the pure
FP64 and FP32-mixed forms, and the FP16 Dslash against the HBM roofline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--arith 16|32]

--arith picks the arithmetic of the FP16 stencil (wd_set_arith): 16, the
default, is the paper's FP16 arithmetic (Sec. 5); 32 widens to FP32. The other
one is reported among the forms.

One step = one full solve (even-odd source, refinement with FP16 inner
BiCGStab, odd reconstruction, FP64 true residual) of a synthetic workload
whose inputs (402 MB FP64 source, 402 MB FP16 links, 1.2 GB FP64 links) are
all larger than the 129 MB L2. Rank 0 prints one JSON line.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# DRAM bytes (read + write) of one launch of the FP16 12-real hop at 32^3 x 64,
# from the ncu captures summarised in profiles/ (hop_fp16_12_32x32x32x64.md for
# FP32 arithmetic, hop16_fp16_12_32x32x32x64.md for FP16 arithmetic); set to
# None whenever that kernel changes until it is captured again.
HOP_FP16_12_TRAFFIC = {32: 269_941_248, 16: 270_509_056}

METRIC = "time to ‖r‖/‖b‖≤1e-10 at 32^3×64, FP16-mixed vs FP64; Dslash GB/s vs HBM peak"
TOL = 1e-10


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="32x32x32x64")
    ap.add_argument("--dslash-launches", type=int, default=60)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the FP64 and FP32-mixed solves")
    ap.add_argument("--no-studies", action="store_true", help="skip the batched and learned-preconditioner sections")
    ap.add_argument("--no-tune", action="store_true", help="keep the default hop kernel configuration")
    ap.add_argument("--arith", type=int, default=16, choices=[16, 32],
                    help="arithmetic of the FP16 stencil of the headline solve (wd_set_arith)")
    return ap.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", self.uuid], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_setup():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return rank, ws, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, ws):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def oracle_iteration_seconds(u_cpu, eta, kappa, iters):
    """Seconds per iteration of the oracle's float64 even-odd solve: the
    Algorithm 4 recurrence with gamma = 1 and the omega_0 prescription, as the
    oracle's kappa calibration counts it (two matrix-vector products each)."""
    import torch

    from oracle import solvers as S
    from oracle import wilson as W
    b = W.eo_source(u_cpu, eta, kappa)
    prm = S.InnerParams(sigma=None, eps=0.0, omega0=0.7, max_matvecs=2 * iters)
    t0 = time.perf_counter()
    S.bicgstab_rescaled(lambda f: W.eo_operator(u_cpu, f, kappa), b, prm)
    return (time.perf_counter() - t0) / iters, torch.get_num_threads()


def cpu_model():
    """The host CPU's model name (lscpu), else what the platform module reports."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def stored_oracle_iterations(dims):
    """Float64 iterations the oracle needs on this workload (written by its kappa calibration)."""
    name = "x".join(str(d) for d in dims)
    path = os.path.join(ROOT, "tests", "golden", f"kappa_calibration_{name}.txt")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        for line in f:
            if line.startswith("iterations"):
                return int(line.split()[1])
    return None


def reference_arm(args, rank, ws):
    """The oracle on the host cores (the reference of this workload); rank 0 only."""
    if rank != 0:
        return
    import torch

    from paper_2602_14450_gb300 import workloads
    wl = workloads.get(args.workload)
    n_iter = stored_oracle_iterations(wl.dims)
    if n_iter is None:
        print(json.dumps({"impl": "reference", "unavailable": "the oracle's float64 iteration count for this "
                          "workload has not been recorded (tests/golden)"}))
        return
    u = wl.gauge(device="cpu")
    eta = wl.source()
    for _ in range(args.warmup):
        oracle_iteration_seconds(u, eta, wl.kappa, 1)
    per = []
    for _ in range(args.steps):
        s, cores = oracle_iteration_seconds(u, eta, wl.kappa, 1)
        per.append(s)
    value = statistics.median(per) * n_iter
    sample = (f"{args.steps} single float64 BiCGStab iterations of the oracle (even-odd, gamma = 1, omega_0 = 0.7) on "
              f"the {args.workload} workload, median scaled by the {n_iter} iterations the oracle needs to 1e-10")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.median(per) * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"wilson_eo_{args.workload}", "kappa": wl.kappa, "tol": TOL},
        "cpu_baseline": {"value": value, "unit": "s", "cores": torch.get_num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    args = parse()
    rank, ws, local = dist_setup()
    if args.impl == "reference":
        return reference_arm(args, rank, ws)
    import torch

    import __graft_entry__
    torch.cuda.set_device(local)
    __graft_entry__.build()
    from paper_2602_14450_gb300 import dslash_bench, synth, wd, workloads

    wl = workloads.get(args.workload)
    vh = wl.volume // 2
    u = wl.gauge(device="cpu")          # the oracle generates the same field on the CPU
    eta = wl.source()
    lat = wd.Lattice(wl.dims, wl.kappa)
    lat.set_gauge(torch.view_as_real(u).contiguous())
    b = synth.to_host_layout(eta).cuda()
    x = torch.zeros_like(b)
    prm = wd.default_params("mixed_fp16")
    stream = torch.cuda.current_stream()
    # the library's autotuner picks the hop kernel variant and block size for the inner and outer precisions
    # (with the headline's stencil arithmetic set, so that the FP16-arithmetic hop's shape is tuned too)
    lat.set_arith(args.arith)
    tuning = {} if args.no_tune else {f"{p}_{r}": lat.tune(p, r, 1, stream)
                                      for p, r in (("fp16", 12), ("fp64", 18), ("fp32", 12))}
    other = 48 - args.arith

    for _ in range(args.warmup):
        st = lat.solve(b, x, TOL, "mixed_fp16", prm, stream)
    props = torch.cuda.get_device_properties(local)
    clocks = Clocks(f"GPU-{props.uuid}" if not str(props.uuid).startswith("GPU-") else str(props.uuid))

    # timed region: K full solves on device-resident inputs
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    e0.record(stream)
    stats = []
    for _ in range(args.steps):
        stats.append(lat.solve(b, x, TOL, "mixed_fp16", prm, stream))
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(ws)
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, ws)
    st = stats[-1]
    launches = sum(s.kernel_launches for s in stats)

    # end to end through the C ABI with pinned host buffers (copies inside)
    bh = b.cpu().pin_memory()
    xh = torch.zeros_like(bh).pin_memory()
    lat.solve(bh, xh, TOL, "mixed_fp16", prm, stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        lat.solve(bh, xh, TOL, "mixed_fp16", prm, stream)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, ws)

    forms = {"mixed_fp16": {"time_s": ms / 1e3, "inner_matvecs": st.inner_matvecs,
                            "outer_iterations": st.outer_iterations, "true_residual": st.true_residual}}
    if not args.no_forms:
        for name in ("mixed_fp32", "fp64", "mixed_bf16", "mixed_fp16_plain", f"mixed_fp16_arith{other}"):
            scheme = name
            if name.startswith("mixed_fp16_arith"):        # the headline solve with the other stencil arithmetic
                scheme = "mixed_fp16"
                lat.set_arith(other)
            p = wd.default_params(scheme)
            if scheme == "mixed_fp16_plain":   # unrescaled FP16 (Alg. 2) crawls: bound its work
                p.max_inner, p.max_outer = 2000, 10
            xs = torch.zeros_like(b)
            q = wd.default_params(scheme)
            q.max_inner, q.max_outer = 4, 1
            lat.solve(b, xs, TOL, scheme, q, stream, check=False)   # links, workspaces and graph
            torch.cuda.synchronize()
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            s2 = lat.solve(b, xs, TOL, scheme, p, stream, check=False)
            f1.record(stream)
            torch.cuda.synchronize()
            forms[name] = {
                "time_s": f0.elapsed_time(f1) / 1e3, "inner_matvecs": s2.inner_matvecs,
                "outer_iterations": s2.outer_iterations, "true_residual": s2.true_residual, "status": s2.status}
            lat.set_arith(args.arith)

    # Dslash: the dominant kernel of the inner solve, timed alone on the launching stream
    sweep = {}
    for prec, recon in (("fp16", 12), ("fp16", 18), ("fp16a", 12), ("fp16a", 18), ("fp32", 12), ("fp32", 18),
                        ("fp64", 18)):
        sweep[f"{prec}_{recon}"] = dslash_bench.hop_timing(lat, prec, recon, args.dslash_launches, stream)
    # arithmetic roofs: GB300's FP64 pipe bounds the FP64 hop (1320 flops per site: 6 x 168 + 2 x 156, the
    # count of the oracle's instrumented three-step hop in this Dirac basis)
    fma_peaks = {f"fp{b}": wd.fma_peak(b, stream=stream) for b in (64, 32, 16)}
    f64 = sweep["fp64_18"]
    f64["tflops"] = 1320 * f64["sites"] / (f64["us"] * 1e-6) / 1e12
    f64["frac_of_measured_fp64_fma_peak"] = f64["tflops"] / fma_peaks["fp64"]
    peak, peak_kind = measured_peaks()
    top = sweep["fp16a_12" if args.arith == 16 else "fp16_12"]
    roof = {"bound": "hbm", "achieved": top["gbs"], "peak": peak, "unit": "GB/s", "frac": top["gbs"] / peak,
            "traffic": HOP_FP16_12_TRAFFIC[args.arith] if wl.dims == (32, 32, 32, 64) else None,
            "kernel": ("hop16_kernel<12,EPI_H,RED_NONE> (H_eo, FP16 storage and arithmetic, 12-real links)"
                       if args.arith == 16 else
                       "hop_kernel<__half,12,EPI_H,RED_NONE> (H_eo, FP16 storage, FP32 arithmetic, 12-real links)"),
            "peak_kind": peak_kind, "bytes_per_site": top["bytes_per_site"], "sites_per_launch": vh,
            "avg_launch_us": top["us"]}

    studies_out = {}
    if not args.no_studies:
        from paper_2602_14450_gb300 import studies
        studies_out["batched"] = studies.batched(workloads.KAPPA["16x16x16x32"], TOL, stream, args.arith)
        studies_out["learned"] = studies.learned_preconditioner(wl.kappa, lat, b, TOL, stream)
        studies_out["tableau"] = studies.tableau(workloads.KAPPA["16x16x16x32"], TOL, stream, arith=args.arith)
        studies_out["tableau_ftz"] = studies.tableau(workloads.KAPPA["16x16x16x32"], TOL, stream, arith=args.arith,
                                                     ftz=1, extras=False)
        if args.workload in workloads.KAPPA_HARD:
            studies_out["harder_system"] = studies.harder_system(wl, workloads.KAPPA_HARD[args.workload], TOL, stream,
                                                                 args.arith, u=u)
        studies_out["table2"] = studies.table2(lat, 1e-13, stream)
        studies_out["clover"] = studies.clover(wl, 1.0, TOL, stream, args.arith)

    line = {
        "metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": (f"f16 storage / f{args.arith} stencil arithmetic, f32 vector arithmetic / f64 refinement"),
        "data": "synthetic",
        "config": {"workload": f"wilson_eo_{args.workload}", "lattice": list(wl.dims), "kappa": wl.kappa,
                   "links": "exp(i 0.5 H) + 3 APE steps (alpha 0.5), SU(3)-reprojected; FP16 12-real in the inner solve",
                   "source": f"Gaussian, seed {wl.source_seed}", "tol": TOL,
                   "scheme": "Alg. 3 + Alg. 4 (s=128, sigma=64, recalculated gamma, eps^2=1e-4)",
                   "stencil_arith_bits": args.arith,
                   "l2": "inputs larger than L2 (no flush)", "parallelism": "replicas" if ws > 1 else "single GPU"},
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": bh.numel() * 8, "d2h_bytes_per_step": xh.numel() * 8},
        "gpu_launches": launches,
        "clocks": clk,
        "roofline": roof,
        "forms": forms,
        "speedup_vs_fp64": (forms["fp64"]["time_s"] / forms["mixed_fp16"]["time_s"]) if "fp64" in forms else None,
        "dslash_sweep": sweep,
        "fma_peaks_tflops": fma_peaks,
        "tuning": tuning,
        "solve": st.as_dict(),
        **studies_out,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        n_iter = stored_oracle_iterations(wl.dims)
        if n_iter:
            import torch as _t
            s_it, cores = oracle_iteration_seconds(u.cpu(), eta, wl.kappa, 2)
            nt = _t.get_num_threads()
            _t.set_num_threads(1)
            try:
                s_one, _ = oracle_iteration_seconds(u.cpu(), eta, wl.kappa, 1)
            finally:
                _t.set_num_threads(nt)
            line["cpu_baseline"] = {
                "value": s_it * n_iter, "unit": "s", "cores": cores, "kind": "oracle", "cpu": cpu_model(),
                "sample": f"2 float64 BiCGStab iterations of the oracle on the full {args.workload} workload "
                          f"({s_it:.2f} s each), scaled by the {n_iter} iterations it needs to 1e-10",
                "one_thread": {"value": s_one * n_iter, "unit": "s", "cores": 1,
                               "sample": f"1 iteration on one thread ({s_one:.2f} s), scaled likewise"}}
        else:
            line["cpu_baseline"] = None
    if rank == 0:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
