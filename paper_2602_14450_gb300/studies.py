"""Measurements beside the headline solve: batched right-hand sides and the
learned preconditioner, run through the C ABI on synthetic workloads.

* ``batched``: the 12 spin-colour point sources at site 0 of a 24^3 x 48
  lattice solved in one wd_solve_batch call against 12 single solves, and an
  uneven batch (8^4, 16^3 x 32 and 24^3 x 48, four Gaussian sources each)
  against the same solves one at a time.
* ``learned``: M trained on 16^3 x 32 smeared-link configurations (four
  gauge seeds, pairs (v, A^{-1} v) from the library's float64 solver) and
  applied as right preconditioner of the FP16 inner solve on a larger lattice,
  against the unpreconditioned FP16-mixed solve of the same system.

Every step runs in the library's kernels; this module only sequences calls
and times them with CUDA events on the launching stream.
"""

from __future__ import annotations

import time

import torch

from . import learned, synth, wd, workloads

SMEARED_SEED = workloads.GAUGE_SEED


def _lattice(dims, kappa, seed, arith=32):
    u = synth.gauge_smeared(dims, seed=seed)
    lat = wd.Lattice(dims, kappa)
    lat.set_gauge(torch.view_as_real(u).contiguous())
    lat.set_arith(arith)
    return lat


def _timed(fn, stream):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return out, e0.elapsed_time(e1) / 1e3


def _summary(stats):
    return {"inner_matvecs": sum(s.inner_matvecs for s in stats),
            "max_true_residual": max(s.true_residual for s in stats),
            "ok": all(s.status == wd.WD_OK for s in stats)}


def batched(kappa: float, tol: float = 1e-10, stream=None, arith: int = 32) -> dict:
    stream = stream or torch.cuda.current_stream()
    res = {}
    d24 = (24, 24, 24, 48)
    lat24 = _lattice(d24, kappa, SMEARED_SEED + 1, arith)
    lat24.tune("fp16", 12, 12, stream)
    b = torch.stack([synth.to_host_layout(synth.point_source(d24, s, c)) for s in range(4) for c in range(3)]).cuda()
    x = torch.zeros_like(b)
    wd.solve_batch([lat24], [b], [x], tol, "mixed_fp16", stream=stream)        # workspaces and graphs
    st_b, t_b = _timed(lambda: wd.solve_batch([lat24], [b], [x.zero_()], tol, "mixed_fp16", stream=stream), stream)
    lat24.solve(b[0], x[0], tol, "mixed_fp16", stream=stream)
    st_s, t_s = _timed(lambda: [lat24.solve(b[i], x[i].zero_(), tol, "mixed_fp16", stream=stream)
                                for i in range(b.shape[0])], stream)
    res["point_sources_24x24x24x48"] = {
        "nrhs": int(b.shape[0]), "batched_s": t_b, "sequential_s": t_s, "speedup": t_s / t_b,
        "batched": _summary(st_b), "sequential": _summary(st_s)}
    del b, x
    torch.cuda.empty_cache()

    lats = [_lattice((8, 8, 8, 8), kappa, SMEARED_SEED + 3, arith), _lattice((16, 16, 16, 32), kappa, SMEARED_SEED, arith),
            lat24]
    bs = [torch.stack([synth.to_host_layout(synth.gaussian_source(l.dims, seed=900 + 10 * i + j)) for j in range(4)]).cuda()
          for i, l in enumerate(lats)]
    xs = [torch.zeros_like(v) for v in bs]
    wd.solve_batch(lats, bs, xs, tol, "mixed_fp16", stream=stream)
    st_b, t_b = _timed(lambda: wd.solve_batch(lats, bs, [v.zero_() for v in xs], tol, "mixed_fp16", stream=stream),
                       stream)

    def one_by_one():
        out = []
        for l, bb, xx in zip(lats, bs, xs):
            for j in range(bb.shape[0]):
                out.append(l.solve(bb[j], xx[j].zero_(), tol, "mixed_fp16", stream=stream))
        return out
    one_by_one()
    st_s, t_s = _timed(one_by_one, stream)
    res["uneven_8x8x8x8_16x16x16x32_24x24x24x48"] = {
        "nrhs": 12, "batched_s": t_b, "sequential_s": t_s, "speedup": t_s / t_b,
        "batched": _summary(st_b), "sequential": _summary(st_s)}
    for l in lats:
        l.close()
    torch.cuda.empty_cache()
    return res


def learned_preconditioner(kappa: float, test_lat: "wd.Lattice", b: torch.Tensor, tol: float = 1e-10, stream=None,
                           configs: int = 4, samples: int = 8, steps: int = 60, lr: float = 3e-3, mu: float = 1.0,
                           seed: int = 11) -> dict:
    stream = stream or torch.cuda.current_stream()
    w = learned.initial_weights(seed)
    t0 = time.perf_counter()
    losses = []
    for c in range(configs):
        lat = _lattice((16, 16, 16, 32), kappa, SMEARED_SEED + 100 + c)
        v, y = learned.make_samples(lat, samples, seed=2000 + 100 * c)
        lat.precond_set(w)
        losses += learned.train(lat, v, y, steps=steps, lr=lr, mu=mu, batch=4)
        w = lat.precond_get()
        lat.close()
        del v, y
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    test_lat.precond_set(w)
    x = torch.zeros_like(b)
    test_lat.solve(b, x, tol, "mixed_fp16_learned", stream=stream)
    st_l, t_l = _timed(lambda: test_lat.solve(b, x.zero_(), tol, "mixed_fp16_learned", stream=stream), stream)
    st_p, t_p = _timed(lambda: test_lat.solve(b, x.zero_(), tol, "mixed_fp16", stream=stream), stream)
    return {
        "train": {"lattice": [16, 16, 16, 32], "configs": configs, "samples_per_config": samples,
                  "adam_steps": steps * configs, "lr": lr, "mu": mu, "first_loss": losses[0],
                  "last_loss": losses[-1], "seconds": train_s},
        "learned": {"time_s": t_l, "inner_matvecs": st_l.inner_matvecs, "outer_iterations": st_l.outer_iterations,
                    "true_residual": st_l.true_residual, "status": st_l.status},
        "plain": {"time_s": t_p, "inner_matvecs": st_p.inner_matvecs, "outer_iterations": st_p.outer_iterations,
                  "true_residual": st_p.true_residual, "status": st_p.status},
        "matvec_ratio": st_l.inner_matvecs / max(1, st_p.inner_matvecs), "time_ratio": t_l / t_p,
    }


def harder_system(wl, kappa: float, tol: float = 1e-10, stream=None, arith: int = 16, u=None) -> dict:
    """The FP16-mixed solve (Alg. 3 + Alg. 4) against FP64 BiCGStab on the
    workload's lattice, links and source at a larger kappa (a system closer to
    critical, as hard as the paper's in FP64 matvecs): times and counts."""
    stream = stream or torch.cuda.current_stream()
    lat = wd.Lattice(wl.dims, kappa)
    lat.set_gauge(torch.view_as_real(wl.gauge() if u is None else u).contiguous())
    lat.set_arith(arith)
    b = synth.to_host_layout(wl.source()).cuda()
    x = torch.zeros_like(b)
    out = {"kappa": kappa, "lattice": list(wl.dims), "arith": arith}
    for scheme in ("mixed_fp16", "fp64"):
        q = wd.default_params(scheme)
        q.max_inner, q.max_outer = 4, 1
        lat.solve(b, x.zero_(), tol, scheme, q, stream=stream, check=False)   # links, workspaces, graphs
        st, t = _timed(lambda: lat.solve(b, x.zero_(), tol, scheme, stream=stream, check=False), stream)
        out[scheme] = {"time_s": t, "inner_matvecs": st.inner_matvecs, "outer_iterations": st.outer_iterations,
                       "true_residual": st.true_residual, "status": st.status}
    out["speedup_vs_fp64"] = out["fp64"]["time_s"] / out["mixed_fp16"]["time_s"]
    lat.close()
    return out


def table2(lat: "wd.Lattice", tol: float = 1e-13, stream=None, max_outer: int = 40) -> dict:
    """The rows of Table 2 on a lattice with the paper's source b = (1, 0, ..., 0)
    (unit real entry at even site 0, spin 0, colour 0) and its stopping rule
    |r|^2 < 1e-26 (|b| = 1, so tol = 1e-13): FP64; FP32 inner (s = 1) with
    eps^2 = 1e-12 and 1e-4; FP16 inner with s = 128, sigma = 64; s = 4096 alone;
    s = 128, sigma = sigma_lambda = 256 with solution rescaling (Alg. 5); and
    unrescaled FP16 (Alg. 2), the paper's unimproved case -- the last and the
    first FP16 row also with subnormals flushed to zero on every store, the
    regime of the paper's build."""
    stream = stream or torch.cuda.current_stream()
    b = synth.to_host_layout(synth.point_source(lat.dims, 0, 0, 0)).cuda()
    x = torch.zeros_like(b)
    rows = {
        "double": ("fp64", {}),
        "fp32_s1_eps2_1e-12": ("mixed_fp32", {"inner_eps": 1e-6}),
        "fp32_s1_eps2_1e-4": ("mixed_fp32", {}),
        "fp16_s128_sigma64": ("mixed_fp16", {}),
        "fp16_s4096": ("mixed_fp16", {"s": 4096.0, "sigma": 0.0}),
        "fp16_s128_sigma256_lambda256": ("mixed_fp16", {"sigma": 256.0, "sigma_lambda": 256.0, "rescale_x": 1}),
        "fp16_unrescaled_alg2": ("mixed_fp16_plain", {}),
        # the paper's build flushes subnormals (-Kfz): the same two FP16 forms with every store flushed
        "fp16_s128_sigma64_ftz": ("mixed_fp16", {"ftz": 1}),
        "fp16_unrescaled_alg2_ftz": ("mixed_fp16_plain", {"ftz": 1}),
    }
    out = {"source": "b = (1, 0, ..., 0): even site 0, spin 0, colour 0", "tol": tol}
    for name, (scheme, kw) in rows.items():
        p = wd.default_params(scheme)
        p.max_outer = max_outer
        for k, v in kw.items():
            setattr(p, k, v)
        lat.solve(b, x.zero_(), tol, scheme, p, stream=stream, check=False)      # graphs and workspaces
        st, t = _timed(lambda: lat.solve(b, x.zero_(), tol, scheme, p, stream=stream, check=False), stream)
        out[name] = {"matvecs": st.inner_matvecs, "outer": st.outer_iterations, "time_s": t, "status": st.status,
                     "true_residual": st.true_residual, "first_inner_nonzeros": st.first_inner_nonzeros}
    return out


def tableau(kappa: float, tol: float = 1e-10, stream=None, s_values=(1.0, 16.0, 128.0, 1024.0, 4096.0),
            sigma_values=(0.0, 1.0, 16.0, 64.0, 256.0, 1024.0), max_outer: int = 30, source: str = "point",
            arith: int = 32, ftz: int = 0, extras: bool = True) -> dict:
    """FP16 low-precision matvecs to 1e-10 over the Alg. 3 scale s and the Alg. 4
    residual norm sigma (sigma = 0: no inner rescaling), recalculated gamma, on
    the 16^3 x 32 workload with the paper's unit source (or the Gaussian one)
    -- the counts Sec. 6 plots in its parameter study --
    plus the four corners of recalculated gamma on/off and solution rescaling
    (Alg. 5, sigma_lambda = sigma) on/off at s = 128, sigma = 64, and Alg. 2
    with unrescaled FP16 (the paper's unimproved case). Inner solves stop at 2000
    matvecs and the refinement at max_outer trips; runs that stop at the caps
    report their status and the matvecs spent. With ftz every low-precision
    store flushes subnormal values to zero, the regime of the paper's build
    (-Ofast implies -Kfz, Sec. 6); extras = False skips the corners and the
    comparison forms."""
    stream = stream or torch.cuda.current_stream()
    dims = (16, 16, 16, 32)
    lat = _lattice(dims, kappa, SMEARED_SEED, arith)
    if source == "point":
        b = synth.to_host_layout(synth.point_source(dims, 0, 0, 0)).cuda()
    else:
        b = synth.to_host_layout(synth.gaussian_source(dims, seed=workloads.SOURCE_SEED)).cuda()
    x = torch.zeros_like(b)

    def run(scheme, **kw):
        p = wd.default_params(scheme)
        p.max_outer = max_outer
        if scheme != "fp64":
            p.max_inner = 2000          # bounds the work of settings that crawl
        p.ftz = ftz
        for k, v in kw.items():
            setattr(p, k, v)
        st = lat.solve(b, x.zero_(), tol, scheme, p, stream=stream, check=False)
        return {"matvecs": st.inner_matvecs, "outer": st.outer_iterations, "status": st.status,
                "true_residual": st.true_residual}

    grid = {}
    for s in s_values:
        for sg in sigma_values:
            grid[f"s={s:g},sigma={sg:g}"] = run("mixed_fp16", s=s, sigma=sg, sigma_lambda=sg if sg > 0 else 64.0)
    out = {"lattice": list(dims), "kappa": kappa, "source": source, "ftz": ftz, "grid": grid}
    if extras:
        corners = {}
        for recalc in (0, 1):
            for lam in (0, 1):
                corners[f"recalc_gamma={recalc},rescale_x={lam}"] = run("mixed_fp16", recalc_gamma=recalc,
                                                                        rescale_x=lam)
        out.update({"corners": corners, "fp16_unrescaled_alg2": run("mixed_fp16_plain"),
                    "fp32_alg2_eps2_1e-4": run("mixed_fp32"), "fp64": run("fp64")})
    lat.close()
    return out



def clover(wl, csw: float = 1.0, tol: float = 1e-10, stream=None, arith: int = 32) -> dict:
    """The clover matrix (wd_set_clover) on a workload: FP16-mixed (Alg. 3 + 4)
    against FP64 time to tol, with the Wilson-only solves of the same system
    beside them, and the clover FP16 hop with its C^-1 block (EO operator)."""
    stream = stream or torch.cuda.current_stream()
    lat = wd.Lattice(wl.dims, wl.kappa)
    lat.set_gauge(torch.view_as_real(wl.gauge()).contiguous())
    lat.set_arith(arith)
    b = synth.to_host_layout(wl.source()).cuda()
    x = torch.zeros_like(b)
    out = {"csw": csw, "kappa": wl.kappa, "arith": arith}
    for name, c in (("wilson", 0.0), ("clover", csw)):
        lat.set_clover(c)
        row = {}
        for scheme in ("mixed_fp16", "fp64"):
            lat.solve(b, x.zero_(), tol, scheme, stream=stream, check=False)
            st, t = _timed(lambda: lat.solve(b, x.zero_(), tol, scheme, stream=stream, check=False), stream)
            row[scheme] = {"time_s": t, "matvecs": st.inner_matvecs, "outer": st.outer_iterations,
                           "status": st.status, "true_residual": st.true_residual}
        row["speedup_fp16_vs_fp64"] = row["fp64"]["time_s"] / row["mixed_fp16"]["time_s"]
        nb = lat.vector_bytes("fp16")
        src = torch.empty(nb, dtype=torch.uint8, device="cuda")
        dst = torch.empty(nb, dtype=torch.uint8, device="cuda")
        src.view(torch.float16).normal_()
        for _ in range(3):
            lat.apply("fp16", 12, wd.WD_OP_EO_A, src, dst, stream)
        _, t = _timed(lambda: [lat.apply("fp16", 12, wd.WD_OP_EO_A, src, dst, stream) for _ in range(20)], stream)
        row["eo_operator_fp16_us"] = t / 20 * 1e6
        out[name] = row
    lat.close()
    return out
