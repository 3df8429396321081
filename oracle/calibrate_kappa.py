"""Choose the hopping parameter kappa of the smeared-link workloads.

Rule: on the 16^3 x 32 lattice with APE-smeared links (gauge seed 20260214)
and a Gaussian source (seed 450), bisect kappa on a 1e-4 grid until the
oracle's float64 even-odd BiCGStab needs between ``LO`` and ``HI`` iterations
to reach |eta - D x| <= 1e-10 |eta|. The same kappa is then used for the
32^3 x 64 lattice. Uses only the oracle and the seeded input generator.

Writes ``tests/golden/kappa_calibration.txt``. Run:
    python -m oracle.calibrate_kappa
"""

import os
import sys
import time

from paper_2602_14450_gb300 import synth

from . import solvers

DIMS = (16, 16, 16, 32)
GAUGE_SEED = 20260214
SOURCE_SEED = 450
LO, HI = 500, 800
MAXITER = 1500


def iterations(u, eta, kappa):
    _, info = solvers.solve_wilson(u, eta, kappa, tol=1e-10, maxiter=MAXITER)
    return info.iterations if info.converged else None


def main(out_path=None):
    here = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out_path = out_path or os.path.join(here, "tests", "golden", "kappa_calibration.txt")
    u = synth.gauge_smeared(DIMS, seed=GAUGE_SEED)
    eta = synth.gaussian_source(DIMS, seed=SOURCE_SEED)
    lo, hi = 1250, 1350                      # kappa * 1e4; lo converges fast, hi does not converge
    log = []
    found = None
    while hi - lo > 1:
        mid = (lo + hi) // 2
        t0 = time.time()
        n = iterations(u, eta, mid * 1e-4)
        log.append((mid * 1e-4, n, time.time() - t0))
        print(f"kappa={mid * 1e-4:.4f} iterations={n} ({time.time() - t0:.0f}s)", flush=True)
        if n is not None and LO <= n <= HI:
            found = (mid * 1e-4, n)
            break
        if n is None or n > HI:
            hi = mid
        else:
            lo = mid
    if found is None:
        raise SystemExit("no kappa on the grid gives an iteration count in the window")
    with open(out_path, "w") as f:
        f.write("# Written by oracle/calibrate_kappa.py (oracle float64 even-odd BiCGStab, tol 1e-10).\n")
        f.write(f"# lattice {DIMS}, APE-smeared links seed {GAUGE_SEED}, Gaussian source seed {SOURCE_SEED},\n")
        f.write(f"# window {LO}..{HI} BiCGStab iterations; bisection log: kappa iterations seconds\n")
        for k, n, t in log:
            f.write(f"#   {k:.4f} {n} {t:.0f}\n")
        f.write(f"kappa {found[0]:.4f}\n")
        f.write(f"iterations {found[1]}\n")
    print("kappa", f"{found[0]:.4f}", "iterations", found[1])


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else None)
