"""Synthetic workloads standing in for the paper's lattice (Sec. 6).

The paper solves on 32^3 x 64 with kappa = 0.13, a stout-smeared test
configuration tiled from 4^3 x 8 and the even-odd unit source; that
configuration is not available, so the workloads draw links from the seeded
generator of ``synth``:

* ``8x8x8x8``     links exp(i eps H), eps = 0.5, kappa = 0.12, Gaussian source.
* ``16x16x16x32`` the same links after 3 APE steps (alpha = 0.5) with SU(3)
                  reprojection; kappa chosen by the oracle's calibration so
                  that float64 BiCGStab needs 500-1500 iterations.
* ``32x32x32x64`` 2,097,152 sites, same generator (own seed) and the same
                  kappa rule applied on this lattice (the critical kappa of a
                  field of equal smoothness is lower on the larger lattice).
"""

from __future__ import annotations

from dataclasses import dataclass

from . import synth

GAUGE_SEED = 20260214
SOURCE_SEED = 450
# Smallest kappa of each calibration grid in the 500-1500 iteration window
# (tests/golden/kappa_calibration_<lattice>.txt, written by oracle/calibrate_kappa.py).
KAPPA = {"16x16x16x32": 0.1265, "32x32x32x64": 0.1255}
# A harder system on the same lattice and links: the first kappa of the calibration grid (0.1250, 0.1255, ...)
# at which the FP64 solve needs at least the 775 matrix-vector multiplications of the paper's own FP64 solve
# (Table 2). Measured with the library's FP64 solver on GB300: 714 at 0.1260, 1260 at 0.1265.
KAPPA_HARD = {"32x32x32x64": 0.1265}


@dataclass(frozen=True)
class Workload:
    name: str
    dims: tuple
    smeared: bool
    kappa: float
    gauge_seed: int
    source_seed: int = SOURCE_SEED

    @property
    def volume(self):
        return synth.volume(self.dims)

    def gauge(self, device="cpu"):
        if self.smeared:
            return synth.gauge_smeared(self.dims, seed=self.gauge_seed, device=device)
        return synth.gauge_random(self.dims, 0.5, seed=self.gauge_seed, device=device)

    def source(self):
        return synth.gaussian_source(self.dims, seed=self.source_seed)


def get(name: str) -> Workload:
    if name == "8x8x8x8":
        return Workload(name, (8, 8, 8, 8), False, 0.12, GAUGE_SEED)
    if name not in KAPPA:
        raise KeyError(name)
    if KAPPA[name] is None:
        raise RuntimeError(f"kappa of the {name} workload has not been calibrated")
    if name == "16x16x16x32":
        return Workload(name, (16, 16, 16, 32), True, KAPPA[name], GAUGE_SEED)
    return Workload(name, (32, 32, 32, 64), True, KAPPA[name], GAUGE_SEED + 2)
