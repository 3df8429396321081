"""Choose the hopping parameter kappa of a smeared-link workload.

Rule (applied to each lattice): with APE-smeared links and a Gaussian source
(seed 450), take the smallest kappa of a grid for which the oracle's float64
even-odd BiCGStab needs between ``LO`` and ``HI`` iterations to reach
|eta - D x| <= 1e-10 |eta|. The smallest, because the iteration count grows
steeply towards the critical kappa, which itself moves down as the volume
grows. Uses only the oracle and the seeded input generator; the grid points
run in parallel worker processes (spawned).

The written file also records each grid point's iteration count; the one of
the chosen kappa is the oracle's float64 iteration count for the workload.

    python -m oracle.calibrate_kappa                      # 16^3 x 32, gauge seed 20260214
    python -m oracle.calibrate_kappa --dims 32,32,32,64 --seed 20260216 \
        --grid 0.1263,0.1264,0.1265 --threads 2
"""

import argparse
import multiprocessing as mp
import os
import time

SOURCE_SEED = 450
LO, HI = 500, 1500
MAXITER = 1600


def _iterations(job):
    dims, seed, kappa, threads = job
    import torch
    torch.set_num_threads(threads)
    from paper_2602_14450_gb300 import synth

    from . import solvers
    u = synth.gauge_smeared(dims, seed=seed)
    eta = synth.gaussian_source(dims, seed=SOURCE_SEED)
    t0 = time.time()
    _, info = solvers.solve_wilson(u, eta, kappa, tol=1e-10, maxiter=MAXITER)
    return kappa, (info.iterations if info.converged else None), time.time() - t0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", default="16,16,16,32")
    ap.add_argument("--seed", type=int, default=20260214)
    ap.add_argument("--grid", default="0.1270,0.1271,0.1272,0.1273,0.1274")
    ap.add_argument("--threads", type=int, default=1)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    dims = tuple(int(d) for d in a.dims.split(","))
    grid = [float(k) for k in a.grid.split(",")]
    name = "x".join(str(d) for d in dims)
    here = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out_path = a.out or os.path.join(here, "tests", "golden", f"kappa_calibration_{name}.txt")
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(grid)) as pool:
        results = sorted(pool.map(_iterations, [(dims, a.seed, k, a.threads) for k in grid]))
    for k, n, t in results:
        print(f"kappa={k:.4f} iterations={n} ({t:.0f}s)", flush=True)
    ok = [(k, n) for k, n, _ in results if n is not None and LO <= n <= HI]
    if not ok:
        raise SystemExit("no kappa on the grid gives an iteration count in the window")
    kappa, n = min(ok)
    with open(out_path, "w") as f:
        f.write("# Written by oracle/calibrate_kappa.py (oracle float64 even-odd BiCGStab, tol 1e-10).\n")
        f.write(f"# lattice {dims}, APE-smeared links seed {a.seed}, Gaussian source seed {SOURCE_SEED},\n")
        f.write(f"# window {LO}..{HI} BiCGStab iterations, smallest kappa in the window; scan: kappa iterations seconds\n")
        for k, m, t in results:
            f.write(f"#   {k:.4f} {m} {t:.0f}\n")
        f.write(f"kappa {kappa:.4f}\n")
        f.write(f"iterations {n}\n")
    print("kappa", f"{kappa:.4f}", "iterations", n)


if __name__ == "__main__":
    main()
