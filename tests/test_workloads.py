"""The smeared-link workloads take their kappa from the oracle's calibration.

Each value of ``workloads.KAPPA`` must be the one the calibration file under
tests/golden records (written by oracle/calibrate_kappa.py from the oracle's
float64 solve alone), and that file must show the rule it applied: the
chosen kappa's count lies in the window and every smaller kappa scanned lies
below it.
"""

import os
import re

import pytest

from paper_2602_14450_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_calibration(name):
    path = os.path.join(GOLDEN, f"kappa_calibration_{name}.txt")
    with open(path) as f:
        text = f.read()
    kappa = float(re.search(r"^kappa (\S+)$", text, re.M).group(1))
    matvecs = int(re.search(r"^matvecs (\d+)$", text, re.M).group(1))
    iterations = int(re.search(r"^iterations (\d+)$", text, re.M).group(1))
    window = tuple(int(v) for v in re.search(r"window (\d+)\.\.(\d+)", text).groups())
    scan = [(float(k), None if n == "None" else int(n))
            for k, n in re.findall(r"^#\s+(0\.\d+) (\d+|None) \d+$", text, re.M)]
    return kappa, matvecs, iterations, window, scan


@pytest.mark.parametrize("name", sorted(workloads.KAPPA))
def test_kappa_matches_calibration(name):
    if workloads.KAPPA[name] is None:
        pytest.skip(f"{name} not calibrated")
    kappa, matvecs, iterations, (lo, hi), scan = read_calibration(name)
    assert workloads.KAPPA[name] == kappa
    assert workloads.get(name).kappa == kappa
    assert lo <= matvecs <= hi
    assert iterations == matvecs // 2
    assert scan[-1] == (kappa, matvecs)
    for k, n in scan[:-1]:
        assert k < kappa and n is not None and n < lo


def test_rough_workload_is_fixed():
    w = workloads.get("8x8x8x8")
    assert w.kappa == 0.12 and not w.smeared and w.dims == (8, 8, 8, 8)
