"""Write tests/golden/tableau_ftz_8x8x8x16.txt: the oracle's low-precision
matvec counts of Alg. 3 + Alg. 4 at corner cells of the (s, sigma) parameter
study (Sec. 6, Fig. 6 discussion), with FP16 storage, FP16 arithmetic in the
inner operator's hops and subnormal values kept or flushed to zero on every
store (the paper's -Kfz build), on a small smeared lattice with the unit
source b = (1, 0, ..., 0). Test infrastructure: only the tests read the file.

    python -m oracle.tableau_ftz
"""

from __future__ import annotations

import os

from paper_2602_14450_gb300 import synth

from . import solvers as S

DIMS = (8, 8, 8, 16)
KAPPA = 0.1265
GAUGE_SEED = 5
CELLS = ((128.0, 64.0), (1.0, 64.0), (128.0, 1.0), (1.0, 1.0))
TOL = 1e-12
MAX_OUTER = 40


def counts():
    u = synth.gauge_smeared(DIMS, seed=GAUGE_SEED)
    eta = synth.point_source(DIMS, 0, 0, 0)
    out = []
    for s, sigma in CELLS:
        for ftz in (0, 1):
            _, tr = S.solve_wilson_mixed(u, eta, KAPPA, (1, 1, 1, -1), fmt="fp16",
                                         outer=S.OuterParams(s=s, tol=TOL, max_outer=MAX_OUTER),
                                         inner=S.InnerParams(sigma=sigma), ftz=bool(ftz), arith16=True)
            out.append((s, sigma, ftz, tr.matvecs, tr.outer, int(tr.converged)))
    return out


def main():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    path = os.path.join(root, "tests", "golden", "tableau_ftz_8x8x8x16.txt")
    rows = counts()
    with open(path, "w") as f:
        f.write("# Written by oracle/tableau_ftz.py: oracle Alg. 3 + Alg. 4, FP16 storage and FP16 arithmetic,\n")
        f.write(f"# lattice {DIMS}, APE-smeared links seed {GAUGE_SEED}, kappa {KAPPA}, unit source b = (1,0,...,0),\n")
        f.write(f"# |b^ - A x| <= {TOL:g} |eta|, at most {MAX_OUTER} refinement trips.\n")
        f.write("# s sigma ftz matvecs refinement_trips converged\n")
        for r in rows:
            f.write(f"{r[0]:g} {r[1]:g} {r[2]} {r[3]} {r[4]} {r[5]}\n")
    print(path)


if __name__ == "__main__":
    main()
