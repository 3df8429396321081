"""Synthetic workloads standing in for the paper's lattice (Sec. 5).

The paper solves on 32^3 x 64 with kappa = 0.13, a stout-smeared test
configuration tiled from 4^3 x 8 and the even-odd unit source; that
configuration is not available, so the workloads draw links from the seeded
generator of ``synth``:

* ``8x8x8x8``     links exp(i eps H), eps = 0.5, kappa = 0.12, Gaussian source.
* ``16x16x16x32`` the same links after 3 APE steps (alpha = 0.5) with SU(3)
                  reprojection; kappa chosen by ``oracle/calibrate_kappa.py``
                  so that float64 BiCGStab needs 500-1500 iterations.
* ``32x32x32x64`` 2,097,152 sites, same generator (own seed) and kappa.
"""

from __future__ import annotations

from dataclasses import dataclass

from . import synth

GAUGE_SEED = 20260214
SOURCE_SEED = 450
# Largest kappa of the calibration grid in the 500-1500 iteration window
# (tests/golden/kappa_calibration.txt, written by oracle/calibrate_kappa.py).
KAPPA_SMEARED = None


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
    if KAPPA_SMEARED is None:
        raise RuntimeError("kappa of the smeared workloads has not been calibrated")
    if name == "16x16x16x32":
        return Workload(name, (16, 16, 16, 32), True, KAPPA_SMEARED, GAUGE_SEED)
    if name == "32x32x32x64":
        return Workload(name, (32, 32, 32, 64), True, KAPPA_SMEARED, GAUGE_SEED + 2)
    raise KeyError(name)
