"""Solvers of Sec. 3, float64 arithmetic with emulated low-precision storage.

* ``bicgstab``          -- textbook BiCGStab (van der Vorst 1992), the plain
                           definition of the solve.
* ``bicgstab_rescaled`` -- Algorithm 4 (residual rescaling, gamma
                           recalculation, omega_0 prescription) and, with
                           ``rescale_x``, Algorithm 5 (solution rescaling).
* ``refine``            -- Algorithm 2 (``s = 1``, no s-hat) and Algorithm 3
                           (rescale the residual to norm s, correct with the
                           norm s-hat of the rounded vector).
* ``solve_wilson``      -- even-odd solve of Eq. 3 via Eqs. 4-5.

Storage emulation: every vector the algorithm assigns is passed through
``store`` (round each real and imaginary part to the storage format with
round-to-nearest-even, subnormals kept unless ``ftz``); arithmetic and all
scalars are float64. Dots are (a, b) = sum conj(a_i) b_i.

Readings of the paper where it is silent or garbled:

* Refinement update (Alg. 2 and 3 print x += t/s and x += t/s-hat): the
  inner solution approximates A^{-1} y with y = (s/|r|) r, so the update
  that makes one exact inner solve give r = 0 is x += (|r|/s-hat) t; for
  Alg. 2, s = 1 and s-hat is replaced by 1.
* Inner stopping rule ("|r|/gamma' not small enough"): |r|/gamma' <= eps * |b|
  with b the inner right-hand side.
* Algorithm 5 returns x / lambda' (the stored x is the rescaled solution).
* Recalculated gamma (Alg. 4/5, "gamma := g/|r|"): the text defines it as the
  ratio of the residual norms after and before rescaling, i.e. the factor
  that was actually applied, |r_stored| / g; the printed g/|r| is its
  reciprocal and would un-scale p and v. Without rounding it equals sigma/g.
* sigma = None means gamma = 1 throughout (Alg. 4 without rescaling).
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

CDT = torch.complex128


def _round_real(a: np.ndarray, fmt: str, ftz: bool) -> np.ndarray:
    if fmt == "fp64":
        return a
    if fmt == "fp32":
        r = a.astype(np.float32).astype(np.float64)
        tiny = np.finfo(np.float32).tiny
    elif fmt == "fp16":
        r = a.astype(np.float16).astype(np.float64)
        tiny = np.finfo(np.float16).tiny
    elif fmt == "bf16":
        r = _round_bf16(a)
        tiny = 2.0 ** -126
    else:
        raise ValueError(fmt)
    if ftz:
        r = np.where(np.abs(r) < tiny, 0.0, r)
    return r


def _round_bf16(a: np.ndarray) -> np.ndarray:
    """Round float64 to bfloat16 (8-bit exponent, 8-bit significand), nearest-even.

    Done on the exact value: x = m * 2^e with 8 significant bits kept;
    np.round rounds halves to even. Overflow to inf past the largest finite
    bfloat16; subnormals below 2^-126 keep a fixed quantum of 2^-133.
    """
    out = a.copy()
    nz = np.isfinite(a) & (a != 0)
    _, e = np.frexp(a[nz])                      # a = m * 2^e, 0.5 <= |m| < 1
    e = np.maximum(e, -125)                     # below 2^-126 the quantum stays 2^-133
    vals = np.ldexp(np.round(np.ldexp(a[nz], 8 - e)), e - 8)
    vals = np.where(np.abs(vals) > 3.3895313892515355e38, np.sign(vals) * np.inf, vals)
    out[nz] = vals
    return out


def make_store(fmt: str = "fp64", ftz: bool = False):
    """Storage rounding for complex fields (identity for ``fp64``)."""
    if fmt == "fp64":
        return lambda f: f

    def store(f: torch.Tensor) -> torch.Tensor:
        a = torch.view_as_real(f.contiguous()).numpy()
        return torch.view_as_complex(torch.from_numpy(_round_real(a, fmt, ftz)).contiguous())

    return store


def dot(a: torch.Tensor, b: torch.Tensor) -> complex:
    return complex(torch.vdot(a.reshape(-1), b.reshape(-1)).item())


def norm(a: torch.Tensor) -> float:
    return float(torch.linalg.vector_norm(a.reshape(-1)).item())


# --- textbook BiCGStab ---------------------------------------------------------

@dataclass
class SolveInfo:
    iterations: int = 0
    matvecs: int = 0
    converged: bool = False
    residuals: list = field(default_factory=list)


def bicgstab(apply_a, b: torch.Tensor, tol: float, maxiter: int = 100000, x0=None, bref=None):
    """Unpreconditioned BiCGStab; stops when |b - A x| (recursive) <= tol * bref."""
    bref = norm(b) if bref is None else bref
    x = torch.zeros_like(b) if x0 is None else x0.clone()
    r = b - apply_a(x) if x0 is not None else b.clone()
    rhat = r.clone()
    rho_old = alpha = omega = 1.0 + 0j
    v = torch.zeros_like(b)
    p = torch.zeros_like(b)
    info = SolveInfo()
    while info.iterations < maxiter:
        rn = norm(r)
        info.residuals.append(rn)
        if rn <= tol * bref:
            info.converged = True
            break
        if not math.isfinite(rn):
            break
        rho = dot(rhat, r)
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = apply_a(p)
        alpha = rho / dot(rhat, v)
        s = r - alpha * v
        t = apply_a(s)
        omega = dot(t, s) / dot(t, t)
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho_old = rho
        info.iterations += 1
        info.matvecs += 2
    return x, info


# --- Algorithms 4 and 5 -----------------------------------------------------------

@dataclass
class InnerParams:
    sigma: float | None = 64.0      # residual norm after rescaling; None -> gamma = 1
    eps: float = 1e-2               # inner tolerance (eps^2 = 1e-4, Table 2)
    omega0: float = 0.7             # Sec. 3
    recalc_gamma: bool = True       # gamma := g / |r_stored|
    rescale_x: bool = False         # Algorithm 5
    sigma_lambda: float | None = None
    max_matvecs: int = 5000


@dataclass
class InnerTrace:
    matvecs: int = 0
    iterations: int = 0
    converged: bool = False
    breakdown: bool = False                         # (r*, v) = 0, (t, t) = 0 or rho' omega' = 0
    first_beta: complex | None = None
    residuals: list = field(default_factory=list)   # |r|/gamma' at each loop test
    iterates: list = field(default_factory=list)    # true solution estimate after each iteration


def bicgstab_rescaled(apply_a_low, b: torch.Tensor, prm: InnerParams, store=None, keep_iterates=False):
    """Algorithm 4 (Alg. 5 with ``prm.rescale_x``) for A x = b, x_0 = 0.

    ``apply_a_low`` is the low-precision operator (it rounds its own output);
    ``b`` is already in storage precision. Returns (t, trace), t = x / lambda'
    in float64.
    """
    store = store or (lambda f: f)
    x = torch.zeros_like(b)
    r = b.clone()                       # r = b - A x_0 with x_0 = 0
    rstar = r.clone()
    p = torch.zeros_like(b)
    v = torch.zeros_like(b)
    rho_p = complex(norm(r) ** 2)       # rho' = |r|^2 gives beta = 1 at the first step
    omega_p = alpha_p = 1.0 + 0j
    gamma_p = 1.0
    lam_p = 1.0
    bnorm = norm(b)
    sig_l = prm.sigma_lambda if prm.sigma_lambda is not None else prm.sigma
    tr = InnerTrace()
    while True:
        res = norm(r) / gamma_p
        tr.residuals.append(res)
        if res <= prm.eps * bnorm:
            tr.converged = True
            break
        if tr.matvecs >= prm.max_matvecs or not math.isfinite(res):
            break
        rho = dot(rstar, r)
        beta = rho * alpha_p / (rho_p * omega_p)
        if tr.first_beta is None:
            tr.first_beta = beta
        p = store(beta * (p - omega_p * v) + r)
        v = apply_a_low(p)
        rv = dot(rstar, v)
        if rv == 0:                         # breakdown: alpha undefined; stop with the current x
            tr.breakdown = True
            break
        alpha = rho / rv
        r = store(r - alpha * v)
        t = apply_a_low(r)
        ts, tt, rr = dot(t, r), dot(t, t).real, dot(r, r).real
        if tt == 0:                         # breakdown: omega undefined
            tr.breakdown = True
            break
        omega = ts / tt
        omega_hat = abs(ts) / math.sqrt(tt * rr) if rr > 0 else math.inf
        if 0 < omega_hat < prm.omega0:      # omega_0 prescription (Sec. 3); omega = 0 stays 0
            omega = omega * prm.omega0 / omega_hat
        x = store(x + (lam_p / gamma_p) * (omega * r + alpha * p))
        r = store(r - omega * t)
        if prm.sigma is not None:
            g = norm(r)
            gamma = prm.sigma / g if g > 0 else math.inf    # r = 0: non-finite, as on the device
            r = store(gamma * r)
            if prm.recalc_gamma:
                gamma = norm(r) / g          # applied factor: stored norm over g
        else:
            gamma = 1.0
        p = store(gamma * p)
        v = store(gamma * v)
        omega_p, alpha_p, rho_p = omega, alpha, gamma * rho
        gamma_p *= gamma
        if prm.rescale_x:
            xn = norm(x)
            lam = sig_l / xn if xn > 0 else math.inf
            x = store(lam * x)
            lam_p *= lam
        tr.iterations += 1
        tr.matvecs += 2                     # matvecs of completed iterations (two each)
        if rho_p * omega_p == 0:            # breakdown: the next beta is undefined
            tr.breakdown = True
            if keep_iterates:
                tr.iterates.append(x / lam_p)
            break
        if keep_iterates:
            tr.iterates.append(x / lam_p)
    return x / lam_p, tr


# --- Algorithms 2 and 3 ------------------------------------------------------------

@dataclass
class OuterParams:
    s: float = 128.0                # target norm of the rescaled residual (Alg. 3)
    use_shat: bool = True           # Alg. 3: correct with |single(low_prec(y))|
    tol: float = 1e-10
    max_outer: int = 100


@dataclass
class RefineTrace:
    outer: int = 0
    matvecs: int = 0
    converged: bool = False
    residuals: list = field(default_factory=list)   # |r| of the FP64 outer residual
    inner: list = field(default_factory=list)
    nonzeros: list = field(default_factory=list)     # nonzero reals in each stored inner input


def refine(apply_a, b: torch.Tensor, inner_solve, store, prm: OuterParams, bref: float | None = None):
    """Algorithm 3 (Alg. 2 with ``s = 1, use_shat = False``); returns (x, trace).

    Stops when |b - A x| <= tol * bref (bref defaults to |b|). ``inner_solve``
    maps a stored right-hand side to (t, InnerTrace) with t ~ A_low^{-1} y.
    """
    bref = norm(b) if bref is None else bref
    x = torch.zeros_like(b)
    r = b.clone()
    tr = RefineTrace()
    while True:
        rn = norm(r)
        tr.residuals.append(rn)
        if rn <= prm.tol * bref:
            tr.converged = True
            break
        if tr.outer >= prm.max_outer or not math.isfinite(rn):
            break
        y = store((prm.s / rn) * r)                 # |y| = s before rounding
        a = torch.view_as_real(y).reshape(-1)
        tr.nonzeros.append(int((a != 0).sum().item()))
        shat = norm(y) if prm.use_shat else prm.s
        t, itr = inner_solve(y)
        tr.inner.append(itr)
        tr.matvecs += itr.matvecs
        x = x + (rn / shat) * t
        r = b - apply_a(x)
        tr.outer += 1
    return x, tr


# --- even-odd Wilson solve -------------------------------------------------------

def solve_wilson(U, eta, kappa: float, bc=(1, 1, 1, -1), tol: float = 1e-12, maxiter: int = 100000):
    """xi = D_W^{-1} eta via Eq. 4 (textbook BiCGStab on the even sites) and Eq. 5.

    The even system is solved to |b_e - A xi_e| <= tol * |eta|; by Eq. 5 this
    is the full-system residual |eta - D_W xi|.
    """
    from . import wilson as w
    b = w.eo_source(U, eta, kappa, bc)
    xi_e, info = bicgstab(lambda f: w.eo_operator(U, f, kappa, bc), b, tol, maxiter, bref=norm(eta))
    return w.eo_reconstruct(U, xi_e, eta, kappa, bc), info


def low_precision_operator(U, kappa: float, fmt: str, bc=(1, 1, 1, -1), ftz: bool = False, arith16: bool = False):
    """The even-odd operator with links and every stored vector in ``fmt``.

    A_low(p) = store(p - kappa^2 H_eo store(H_oe p)) with rounded links: the
    odd intermediate is a stored vector like any other. With ``arith16`` (FP16
    storage only) both hops are evaluated in FP16 arithmetic
    (oracle.arith16), the paper's _Float16 build; otherwise exactly.
    """
    from . import wilson as w
    store = make_store(fmt, ftz)
    ul = store(U)
    if arith16:
        if fmt != "fp16":
            raise ValueError("FP16 arithmetic needs FP16 storage")
        from .arith16 import eo_operator_fp16
        return (lambda p: eo_operator_fp16(ul, p, kappa, store, bc)), store

    def apply(p):
        tmp = store(w.hop_pq(ul, p, 1, bc))
        return store(w.restrict(p, 0) - kappa * kappa * w.hop_pq(ul, tmp, 0, bc))

    return apply, store


def solve_wilson_mixed(U, eta, kappa: float, bc=(1, 1, 1, -1), fmt: str = "fp16",
                       outer: OuterParams | None = None, inner: InnerParams | None = None, ftz: bool = False,
                       arith16: bool = False):
    """Alg. 3 + Alg. 4/5 on the even-odd system, FP64 outer, ``fmt`` inner storage
    (and, with ``arith16``, FP16 arithmetic in the inner operator's hops)."""
    from . import wilson as w
    outer = outer or OuterParams()
    inner = inner or InnerParams()
    b = w.eo_source(U, eta, kappa, bc)
    a_low, store = low_precision_operator(U, kappa, fmt, bc, ftz, arith16)
    xi_e, tr = refine(lambda f: w.eo_operator(U, f, kappa, bc), b,
                      lambda y: bicgstab_rescaled(a_low, y, inner, store), store, outer, bref=norm(eta))
    return w.eo_reconstruct(U, xi_e, eta, kappa, bc), tr
