"""Storage conversions of wd_pack / wd_unpack: FP64 values rounded once to
FP16, BF16 or FP32 storage and widened back to FP64 must equal the IEEE-754
round-to-nearest-even conversion bit for bit. The values span every class of
the narrow formats: signed zeros, subnormals of each format, the largest
finite values, values that overflow to infinity, infinities, NaN and
Gaussian values over 2^-160 .. 2^130."""

import numpy as np
import pytest
import torch

from oracle import wilson as W
from paper_2602_14450_gb300 import wd

DIMS = (4, 4, 4, 8)
# (significand bits after the leading one, smallest normal exponent, largest finite exponent)
FORMATS = {"fp16": (10, -14, 15), "bf16": (7, -126, 127), "fp32": (23, -126, 127)}


def round_ieee(x: np.ndarray, man: int, emin: int, emax: int) -> np.ndarray:
    """x (float64) rounded to nearest-even in a binary format with `man`
    fraction bits and normal exponents emin..emax (gradual underflow below
    2^emin, infinity at or above the overflow threshold). The quantum 2^(e - man)
    of x's binade (2^(emin - man) in the subnormal range) is a power of two, so
    x / quantum is exact and np.rint rounds it half to even."""
    out = x.copy()
    fin = np.isfinite(x) & (x != 0)
    _, e = np.frexp(x[fin])                      # |x| = m 2^e, 0.5 <= m < 1
    q = np.exp2(np.maximum(e - 1, emin) - man)
    r = np.rint(x[fin] / q) * q
    big = np.abs(r) >= np.exp2(emax + 1)        # rounded past the largest finite value
    r[big] = np.copysign(np.inf, r[big])
    out[fin] = r
    return out


def special_values():
    v = [0.0, -0.0, 1.0, -1.0, 0.1, -1.0 / 3.0, np.inf, -np.inf]
    for man, emin, emax in FORMATS.values():
        mx = (2.0 - 2.0 ** -man) * 2.0 ** emax
        tiny, sub = 2.0 ** emin, 2.0 ** (emin - man)
        v += [mx, -mx, tiny, -tiny, sub, -sub, 3 * sub, 0.5 * sub, 0.75 * sub, 1.5 * sub, tiny - sub,
              mx * (1 + 2.0 ** -(man + 2)), mx * (1 + 2.0 ** -(man + 1)), mx * 2, 1 + 2.0 ** -(man + 1),
              1 + 3 * 2.0 ** -(man + 1)]
    return np.array(v, dtype=np.float64)


def test_reference_rounding_is_numpys_ieee_conversion():
    """The rounding above against numpy's direct float64 -> float16 / float32
    conversions (no double rounding), on the same values the GPU test uses."""
    x = np.concatenate([special_values(), np.random.default_rng(3).standard_normal(20000)
                        * np.exp2(np.random.default_rng(4).integers(-160, 130, 20000))])
    for name, dt in (("fp16", np.float16), ("fp32", np.float32)):
        with np.errstate(over="ignore"):
            want = x.astype(dt).astype(np.float64)
        got = round_ieee(x, *FORMATS[name])
        assert np.array_equal(got.view(np.int64), want.view(np.int64)), name


@pytest.mark.gpu
def test_pack_unpack_round_trip_is_the_ieee_conversion():
    lat = wd.Lattice(DIMS, 0.1)
    nsite = DIMS[0] * DIMS[1] * DIMS[2] * DIMS[3]
    rng = np.random.default_rng(77)
    vals = rng.standard_normal(nsite * 24) * np.exp2(rng.integers(-160, 130, nsite * 24))
    spec = special_values()
    vals[: spec.size] = spec
    vals[nsite * 12: nsite * 12 + spec.size] = spec   # again, on sites of the other parity
    vals[5] = np.nan
    lex = torch.from_numpy(vals).cuda()
    par = W.parity(DIMS).reshape(-1).repeat_interleave(24).numpy()
    for prec, fmt in FORMATS.items():
        want = round_ieee(vals, *fmt)
        for parity in (0, 1):
            buf = torch.empty(lat.vector_bytes(prec), dtype=torch.uint8, device="cuda")
            lat.pack(prec, parity, lex, buf)
            out = torch.full_like(lex, 7.0)
            lat.unpack(prec, parity, buf, out)
            torch.cuda.synchronize()
            o = out.cpu().numpy()
            mask = par == parity
            got, exp = o[mask], want[mask]
            nan = np.isnan(exp)
            assert np.array_equal(np.isnan(got), nan), prec
            assert np.array_equal(got[~nan].view(np.int64), exp[~nan].view(np.int64)), (prec, parity)
            assert np.all(o[~mask] == 7.0)
