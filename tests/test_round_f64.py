"""round_f64 (csrc/blas_impl.cuh), the library's FP64 -> FP16 / BF16 / FP32
round-to-nearest-even on the integer pipe, compiled for the host and compared
bit for bit with numpy's direct float64 -> float16 / float32 conversions and,
for BF16, with the IEEE rounding of tests/test_gpu_storage.py (itself pinned to
numpy). The inputs cover every class: zeros, subnormals and normals of each
format, exact ties at both ends of the range, values that round up into the
next binade or to infinity, infinities, NaN and wide random values."""

import os
import subprocess
import tempfile

import numpy as np
import pytest

from paper_2602_14450_gb300 import build as B
from tests.test_gpu_storage import FORMATS, round_ieee, special_values

SRC = r'''
#include "blas_impl.cuh"
#include <cstdio>
void wd::tl::register_unit(int (*)(void*, void*)) {}
int main() {
    unsigned long long bits;
    while (std::scanf("%llx", &bits) == 1) {
        double x;
        memcpy(&x, &bits, sizeof x);
        std::printf("%x %x %x\n", wd::round_f64<10, 5>(x), wd::round_f64<7, 8>(x), wd::round_f64<23, 8>(x));
    }
    return 0;
}
'''


@pytest.fixture(scope="module")
def round_exe():
    d = tempfile.mkdtemp()
    cu, exe = os.path.join(d, "r.cu"), os.path.join(d, "r")
    with open(cu, "w") as f:
        f.write(SRC)
    r = subprocess.run([B.nvcc(), *B.ARCH, *B.FLAGS, "-DWD_TIMELINE", "-I", B.CSRC, cu, "-o", exe],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail(r.stderr)
    return exe


def inputs():
    rng = np.random.default_rng(21)
    spec = special_values()
    ties = []
    for man, emin, emax in FORMATS.values():
        q = 2.0 ** (emin - man)
        for k in range(1, 40):                                  # subnormal ties and near-ties
            ties += [(k + 0.5) * q, (k + 0.5) * q * (1 + 2.0 ** -40), (k + 0.5) * q * (1 - 2.0 ** -40)]
        for e in (emin, -3, 0, 7, emax):
            for k in (0, 1, 2, 2 ** man - 1):
                base = (1 + k * 2.0 ** -man) * 2.0 ** e
                ties += [base + 2.0 ** (e - man - 1), base + 2.0 ** (e - man - 1) * (1 + 2.0 ** -30)]
    wide = rng.standard_normal(60000) * np.exp2(rng.integers(-160, 135, 60000))
    x = np.concatenate([spec, np.array(ties), -np.array(ties), wide, [np.nan, -np.nan, 5e-324, -5e-324]])
    return x.astype(np.float64)


def test_round_f64_is_ieee_round_to_nearest_even(round_exe):
    x = inputs()
    inp = "\n".join(f"{b:016x}" for b in x.view(np.uint64)) + "\n"
    out = subprocess.run([round_exe], input=inp, capture_output=True, text=True, check=True).stdout.split()
    got = np.array([int(w, 16) for w in out], dtype=np.uint64).reshape(-1, 3)
    with np.errstate(over="ignore", invalid="ignore"):
        want16 = x.astype(np.float16).view(np.uint16).astype(np.uint64)
        want32 = x.astype(np.float32).view(np.uint32).astype(np.uint64)
    bf = round_ieee(x, *FORMATS["bf16"]).astype(np.float32).view(np.uint32) >> 16   # exact: bf16 values are floats
    nan = np.isnan(x)
    g16 = got[:, 0].astype(np.uint16).view(np.float16)
    gbf = (got[:, 1].astype(np.uint32) << 16).view(np.float32)
    g32 = got[:, 2].astype(np.uint32).view(np.float32)
    assert np.all(np.isnan(g16[nan])) and np.all(np.isnan(gbf[nan])) and np.all(np.isnan(g32[nan]))
    assert np.array_equal(got[~nan, 0], want16[~nan])
    assert np.array_equal(got[~nan, 1], bf[~nan].astype(np.uint64))
    assert np.array_equal(got[~nan, 2], want32[~nan])


SRC_WIDEN = r'''
#include "blas_impl.cuh"
#include <cstdio>
void wd::tl::register_unit(int (*)(void*, void*)) {}
int main() {
    unsigned bits;
    while (std::scanf("%x", &bits) == 1) {
        float f;
        memcpy(&f, &bits, sizeof f);
        const double d = wd::f32_to_f64(f);
        unsigned long long o;
        memcpy(&o, &d, sizeof o);
        std::printf("%llx\n", o);
    }
    return 0;
}
'''


def test_f32_to_f64_is_the_exact_widening():
    """f32_to_f64 (the integer-pipe widening of k_correct and k_unpack) against
    numpy's float32 -> float64, which is exact: zeros, every float subnormal
    exponent, normals, the largest value, infinities and NaN."""
    d = tempfile.mkdtemp()
    cu, exe = os.path.join(d, "w.cu"), os.path.join(d, "w")
    with open(cu, "w") as f:
        f.write(SRC_WIDEN)
    r = subprocess.run([B.nvcc(), *B.ARCH, *B.FLAGS, "-DWD_TIMELINE", "-I", B.CSRC, cu, "-o", exe],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail(r.stderr)
    rng = np.random.default_rng(41)
    bits = np.concatenate([
        np.array([0, 0x80000000, 1, 0x80000001, 0x7FFFFF, 0x807FFFFF, 0x800000, 0x7F7FFFFF, 0xFF7FFFFF,
                  0x7F800000, 0xFF800000, 0x7FC00000, 0x7FA00001], dtype=np.uint32),
        (np.uint32(1) << np.arange(23, dtype=np.uint32)),                      # one subnormal per exponent
        rng.integers(0, 1 << 23, 2000, dtype=np.uint32),                      # random subnormals
        rng.integers(0, 1 << 32, 20000, dtype=np.uint64).astype(np.uint32),   # anything
    ])
    inp = "\n".join(f"{b:x}" for b in bits) + "\n"
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split()
    got = np.array([int(w, 16) for w in out], dtype=np.uint64).view(np.float64)
    with np.errstate(invalid="ignore"):   # signalling NaNs among the random patterns
        want = bits.view(np.float32).astype(np.float64)
    nan = np.isnan(want)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan].view(np.uint64), want[~nan].view(np.uint64))
