"""Seeded synthetic inputs: gauge fields and quark sources.

This module is the only code shared by the CPU oracle and the CUDA path's tests
and benchmark. It draws inputs; it holds none of the solver's arithmetic (no
Wilson operator, no BiCGStab, no rescaling).

Conventions (shared by every consumer):

* ``dims = (Lx, Ly, Lz, Lt)``; all extents even and >= 2.
* Lexicographic site index ``x + Lx*(y + Ly*(z + Lz*t))``, i.e. the C-order
  flattening of a ``[Lt, Lz, Ly, Lx]`` block. Direction ``mu = 0,1,2,3`` is
  x, y, z, t and lives on block axis ``3 - mu``.
* Gauge field: complex128 tensor ``U[mu, t, z, y, x, a, b] = (U_mu(x))_ab``,
  the SU(3) link from x to x + mu-hat (Sec. 2 of the paper). Viewed as float64
  with a trailing (re, im) axis this is the host layout of ``wd_set_gauge``.
* Quark field: complex128 tensor ``psi[t, z, y, x, spin, colour]`` (4 x 3 complex
  per site, Sec. 2). As float64 (re, im) this is the host vector layout.

Random numbers come from numpy's PCG64 so that a seed gives the same draws on
x86-64 and aarch64. Floating-point post-processing (exp, smearing) runs in
float64 torch ops on the CPU, or on a CUDA device when ``device`` says so (a
large lattice is generated in seconds there); results may differ between
machines and devices in the last bits, so consumers generate once and hand
the same tensor to both sides.
"""

from __future__ import annotations

import numpy as np
import torch

CDT = torch.complex128


def _check_dims(dims):
    dims = tuple(int(d) for d in dims)
    if len(dims) != 4 or any(d < 2 or d % 2 for d in dims):
        raise ValueError(f"lattice extents must be 4 even numbers >= 2, got {dims}")
    return dims


def volume(dims) -> int:
    lx, ly, lz, lt = _check_dims(dims)
    return lx * ly * lz * lt


def gell_mann() -> torch.Tensor:
    """The eight Gell-Mann matrices lambda_a, shape [8, 3, 3] complex128."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7][0, 0] = lam[7][1, 1] = 1 / np.sqrt(3)
    lam[7][2, 2] = -2 / np.sqrt(3)
    return torch.from_numpy(lam)


def _dagger(m: torch.Tensor) -> torch.Tensor:
    return m.conj().transpose(-1, -2)


def _expi_hermitian(h: torch.Tensor, eps: float) -> torch.Tensor:
    """exp(i*eps*h) for a batch of Hermitian matrices (Pade scaling and squaring)."""
    return torch.linalg.matrix_exp((1j * eps) * h)


def _inverse_and_det(w: torch.Tensor):
    """Inverse and determinant of a batch of 3x3 matrices via the adjugate."""
    n = w.shape[0]
    a = w.reshape(n, 9).T.contiguous()          # a[3 i + j] = w[:, i, j]
    cof = [None] * 9
    for i in range(3):
        r0, r1 = [k for k in range(3) if k != i]
        for j in range(3):
            c0, c1 = [k for k in range(3) if k != j]
            minor = a[3 * r0 + c0] * a[3 * r1 + c1] - a[3 * r0 + c1] * a[3 * r1 + c0]
            cof[3 * i + j] = minor if (i + j) % 2 == 0 else -minor
    det = a[0] * cof[0] + a[1] * cof[1] + a[2] * cof[2]
    inv = torch.stack([cof[3 * j + i] for i in range(3) for j in range(3)]) / det
    return inv.T.reshape(n, 3, 3), det


def random_su3(n: int, eps: float, rng: np.random.Generator, chunk: int = 1 << 20, device="cpu") -> torch.Tensor:
    """n matrices exp(i*eps*H), H = sum_a h_a lambda_a / 2 with h_a ~ N(0, 1).

    The draws are taken as one [n, 8] block (row = matrix), so the result does
    not depend on ``chunk``.
    """
    h = torch.from_numpy(rng.standard_normal((n, 8)))
    lam = (gell_mann() / 2).to(device)
    out = torch.empty((n, 3, 3), dtype=CDT, device=device)
    for s in range(0, n, chunk):
        hs = torch.einsum("na,aij->nij", h[s:s + chunk].to(device=device, dtype=CDT), lam)
        out[s:s + chunk] = _expi_hermitian(hs, eps)
    return out


def gauge_random(dims, eps: float = 0.5, seed: int = 0, device="cpu") -> torch.Tensor:
    """Links U_mu(x) = exp(i*eps*H) with independent Gaussian traceless Hermitian H.

    Draw order: the [4*V, 8] block of N(0,1) numbers is indexed (mu, site, a).
    """
    lx, ly, lz, lt = _check_dims(dims)
    n = 4 * lx * ly * lz * lt
    rng = np.random.Generator(np.random.PCG64(seed))
    return random_su3(n, eps, rng, device=device).reshape(4, lt, lz, ly, lx, 3, 3)


def _shift(f: torch.Tensor, mu: int, step: int) -> torch.Tensor:
    """f(x + step*mu-hat) on a periodic block whose axes 0..3 are (t, z, y, x)."""
    return torch.roll(f, shifts=-step, dims=3 - mu)


def su3_project(v: torch.Tensor, iters: int = 30, tol: float = 1e-15) -> torch.Tensor:
    """Nearest SU(3) matrix: unitary polar factor, then the determinant phase removed.

    The polar factor W = V (V^+ V)^(-1/2) is computed with Newton's iteration
    W <- (zeta W + (zeta W)^{-+}) / 2 with determinant scaling
    zeta = |det W|^(-1/3) (Higham 1986, "Computing the polar decomposition with
    applications"). W is then divided by det(W)^(1/3) on the principal branch
    (argument in (-pi/3, pi/3]), the cube root nearest 1, giving det = 1.
    """
    shape = v.shape
    w = v.reshape(-1, 3, 3).clone()
    eye = torch.eye(3, dtype=CDT, device=v.device)
    for it in range(iters):
        inv, det = _inverse_and_det(w)
        zeta = det.abs().pow(-1.0 / 3.0).to(CDT)[:, None, None]
        w = 0.5 * (zeta * w + _dagger(inv) / zeta)
        if it >= 4:
            dev = (_dagger(w) @ w - eye).abs().amax().item()
            if dev < tol:
                break
    _, d = _inverse_and_det(w)
    w = w * torch.exp(-1j * torch.angle(d) / 3.0)[:, None, None]
    return w.reshape(shape)


def ape_smear(u: torch.Tensor, alpha: float = 0.5, steps: int = 3) -> torch.Tensor:
    """APE smearing: V = (1 - alpha) U + (alpha / 6) * (sum of the 6 staples), then SU(3).

    The gauge field is periodic in all four directions. Staples of U_mu(x):
    U_nu(x) U_mu(x+nu) U_nu(x+mu)^+  and  U_nu(x-nu)^+ U_mu(x-nu) U_nu(x-nu+mu).
    """
    for _ in range(steps):
        new = torch.empty_like(u)
        for mu in range(4):
            st = torch.zeros_like(u[mu])
            for nu in range(4):
                if nu == mu:
                    continue
                u_nu_xpmu = _shift(u[nu], mu, +1)
                st += u[nu] @ _shift(u[mu], nu, +1) @ _dagger(u_nu_xpmu)
                u_nu_xmnu = _shift(u[nu], nu, -1)
                st += _dagger(u_nu_xmnu) @ _shift(u[mu], nu, -1) @ _shift(u_nu_xpmu, nu, -1)
            new[mu] = su3_project((1.0 - alpha) * u[mu] + (alpha / 6.0) * st)
        u = new
    return u


def gauge_smeared(dims, seed: int, eps: float = 0.5, alpha: float = 0.5, steps: int = 3, device="cpu") -> torch.Tensor:
    """Random exp(i*eps*H) links followed by ``steps`` APE steps with SU(3) reprojection."""
    return ape_smear(gauge_random(dims, eps, seed, device=device), alpha, steps)


def gauge_unit(dims) -> torch.Tensor:
    """All links equal to the identity (free field)."""
    lx, ly, lz, lt = _check_dims(dims)
    eye = torch.eye(3, dtype=CDT)
    return eye.expand(4, lt, lz, ly, lx, 3, 3).clone()


def gauge_transform_field(dims, seed: int) -> torch.Tensor:
    """Random SU(3) matrix g(x) per site, shape [Lt, Lz, Ly, Lx, 3, 3] (eps = 1.0)."""
    lx, ly, lz, lt = _check_dims(dims)
    rng = np.random.Generator(np.random.PCG64(seed))
    return random_su3(lx * ly * lz * lt, 1.0, rng).reshape(lt, lz, ly, lx, 3, 3)


def gaussian_source(dims, seed: int) -> torch.Tensor:
    """Quark field with independent N(0, 1) real and imaginary parts (24 reals per site).

    Draw order: [V, 4, 3, 2] in lexicographic site order.
    """
    lx, ly, lz, lt = _check_dims(dims)
    rng = np.random.Generator(np.random.PCG64(seed))
    a = rng.standard_normal((lt, lz, ly, lx, 4, 3, 2))
    return torch.view_as_complex(torch.from_numpy(a))


def point_source(dims, spin: int, colour: int, site: int = 0) -> torch.Tensor:
    """Unit real entry at lexicographic ``site``, given spin and colour."""
    lx, ly, lz, lt = _check_dims(dims)
    f = torch.zeros((lt * lz * ly * lx, 4, 3), dtype=CDT)
    f[site, spin, colour] = 1.0
    return f.reshape(lt, lz, ly, lx, 4, 3)


def to_host_layout(f: torch.Tensor) -> torch.Tensor:
    """Complex field -> contiguous float64 tensor in the library's host layout."""
    return torch.view_as_real(f.contiguous()).contiguous()


def from_host_layout(a: torch.Tensor, dims) -> torch.Tensor:
    """Inverse of :func:`to_host_layout` for a quark field."""
    lx, ly, lz, lt = _check_dims(dims)
    return torch.view_as_complex(a.reshape(lt, lz, ly, lx, 4, 3, 2).contiguous())
