"""Choose the hopping parameter kappa of the smeared-link workloads.

Rule: on the 16^3 x 32 lattice with APE-smeared links (gauge seed 20260214)
and a Gaussian source (seed 450), take the largest kappa of a 5e-4 grid for
which the oracle's float64 even-odd BiCGStab needs between ``LO`` and ``HI``
iterations to reach |eta - D x| <= 1e-10 |eta|. The same kappa is then used
for the 32^3 x 64 lattice. Uses only the oracle and the seeded input
generator; the grid points run in parallel worker processes (spawned, one
thread each).

Writes ``tests/golden/kappa_calibration.txt``. Run:
    python -m oracle.calibrate_kappa
"""

import multiprocessing as mp
import os
import sys
import time

DIMS = (16, 16, 16, 32)
GAUGE_SEED = 20260214
SOURCE_SEED = 450
LO, HI = 500, 1500
MAXITER = 1600
GRID = [0.1270, 0.1275, 0.1280, 0.1285, 0.1290, 0.1295]


def _iterations(kappa):
    import torch
    torch.set_num_threads(1)
    from paper_2602_14450_gb300 import synth

    from . import solvers
    u = synth.gauge_smeared(DIMS, seed=GAUGE_SEED)
    eta = synth.gaussian_source(DIMS, seed=SOURCE_SEED)
    t0 = time.time()
    _, info = solvers.solve_wilson(u, eta, kappa, tol=1e-10, maxiter=MAXITER)
    return kappa, (info.iterations if info.converged else None), time.time() - t0


def main(out_path=None):
    here = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out_path = out_path or os.path.join(here, "tests", "golden", "kappa_calibration.txt")
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(GRID)) as pool:
        results = sorted(pool.map(_iterations, GRID))
    for k, n, t in results:
        print(f"kappa={k:.4f} iterations={n} ({t:.0f}s)", flush=True)
    ok = [(k, n) for k, n, _ in results if n is not None and LO <= n <= HI]
    if not ok:
        raise SystemExit("no kappa on the grid gives an iteration count in the window")
    kappa, n = max(ok)
    with open(out_path, "w") as f:
        f.write("# Written by oracle/calibrate_kappa.py (oracle float64 even-odd BiCGStab, tol 1e-10).\n")
        f.write(f"# lattice {DIMS}, APE-smeared links seed {GAUGE_SEED}, Gaussian source seed {SOURCE_SEED},\n")
        f.write(f"# window {LO}..{HI} BiCGStab iterations; scan: kappa iterations seconds\n")
        for k, m, t in results:
            f.write(f"#   {k:.4f} {m} {t:.0f}\n")
        f.write(f"kappa {kappa:.4f}\n")
        f.write(f"iterations {n}\n")
    print("kappa", f"{kappa:.4f}", "iterations", n)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else None)
