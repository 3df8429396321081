"""The FP32-pair (double-float) additions of the grid reductions
(csrc/common.cuh: two_sum, fast_two_sum, f2_add), compiled for the host and
checked against exact rational arithmetic: TwoSum is error-free, a chain of
pair additions of FP32 values is exact while the running sum fits the pair's
~48 significant bits, and with cancellation and wide exponent ranges the pair
sum stays within a few units of 2^-46 of the exact sum (FP32 accumulation is
not: its error is printed beside it for the same data)."""

import os
import subprocess
import tempfile
from fractions import Fraction

import numpy as np
import pytest

from paper_2602_14450_gb300 import build as B

SRC = r'''
#include "common.cuh"
#include <cstdio>
#include <cstdlib>
void wd::tl::register_unit(int (*)(void*, void*)) {}
int main(int argc, char** argv) {
    // stdin: n, then n floats (as hex bit patterns); stdout: two_sum of the first two, then the pair sum
    // of all n and the plain FP32 sum, each float as a hex bit pattern
    int n = 0;
    if (std::scanf("%d", &n) != 1) return 1;
    float* v = (float*)std::malloc(sizeof(float) * (n > 2 ? n : 2));
    for (int i = 0; i < n; ++i) {
        unsigned u;
        if (std::scanf("%x", &u) != 1) return 1;
        v[i] = *reinterpret_cast<float*>(&u);
    }
    const wd::F2 t = wd::two_sum(v[0], v[1]);
    wd::F2 acc = {0.f, 0.f};
    volatile float plain = 0.f;
    for (int i = 0; i < n; ++i) {
        acc = wd::f2_add(acc, wd::F2{v[i], 0.f});
        plain = plain + v[i];
    }
    const float out[5] = {t.hi, t.lo, acc.hi, acc.lo, plain};
    for (float f : out) std::printf("%08x\n", *reinterpret_cast<const unsigned*>(&f));
    return 0;
}
'''


@pytest.fixture(scope="module")
def pair_sum_exe():
    d = tempfile.mkdtemp()
    cu, exe = os.path.join(d, "pairs.cu"), os.path.join(d, "pairs")
    with open(cu, "w") as f:
        f.write(SRC)
    r = subprocess.run([B.nvcc(), *B.ARCH, *B.FLAGS, "-DWD_TIMELINE", "-I", B.CSRC, cu, "-o", exe],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail(r.stderr)
    return exe


def run(exe, vals):
    v = np.asarray(vals, dtype=np.float32)
    inp = f"{len(v)}\n" + "\n".join(f"{x:08x}" for x in v.view(np.uint32)) + "\n"
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split()
    f = np.array([int(w, 16) for w in out], dtype=np.uint32).view(np.float32)
    return v, f


def exact(vals):
    return sum((Fraction(float(x)) for x in vals), Fraction(0))


def test_two_sum_is_error_free(pair_sum_exe):
    rng = np.random.default_rng(11)
    for _ in range(40):
        a, b = (rng.standard_normal(2) * np.exp2(rng.integers(-60, 60, 2))).astype(np.float32)
        v, f = run(pair_sum_exe, [a, b])
        assert Fraction(float(f[0])) + Fraction(float(f[1])) == Fraction(float(v[0])) + Fraction(float(v[1]))
        assert f[0] == np.float32(v[0] + v[1])   # the high word is the rounded sum


def test_pair_sum_is_exact_within_48_bits(pair_sum_exe):
    rng = np.random.default_rng(12)
    # integers below 2^20 in FP32, 4000 of them: every partial sum fits well inside 48 bits
    vals = rng.integers(-(1 << 20), 1 << 20, 4000).astype(np.float32)
    v, f = run(pair_sum_exe, vals)
    assert Fraction(float(f[2])) + Fraction(float(f[3])) == exact(v)


def test_pair_sum_tracks_the_exact_sum_with_cancellation(pair_sum_exe):
    rng = np.random.default_rng(13)
    for trial in range(6):
        n = 6000
        vals = (rng.standard_normal(n) * np.exp2(rng.integers(-20, 20, n))).astype(np.float32)
        vals[: n // 2] = -vals[n // 2:] * np.float32(1 + 2.0 ** -12)   # heavy cancellation
        v, f = run(pair_sum_exe, vals)
        ex = exact(v)
        scale = sum((abs(Fraction(float(x))) for x in v), Fraction(0))
        err_pair = abs(Fraction(float(f[2])) + Fraction(float(f[3])) - ex)
        err_plain = abs(Fraction(float(f[4])) - ex)
        assert err_pair <= scale * Fraction(8, 2 ** 46), (trial, float(err_pair / scale))
        assert err_plain > 100 * err_pair, (trial, float(err_plain / scale), float(err_pair / scale))
