"""The hopping term of Eq. 1 evaluated in FP16 arithmetic, emulated in float64
-- test infrastructure only.

The paper's build (Sec. 5) declares its FP16 vectors and links as _Float16,
so the stencil's arithmetic is FP16 arithmetic; only the reductions are
widened. This module evaluates H_pq the way Sec. 2 describes one hop --
project the neighbour spinor onto two spin components, multiply both by the
link, rebuild the four components and accumulate over the eight directions
-- with every arithmetic operation rounded to FP16 (round to nearest even,
subnormals kept) and a product followed by an addition fused into one
rounding, as a compiler that contracts a*b + c does. Multiplications by 0,
+-1, +-2 and +-i are exact and need no rounding.

The paper fixes the arithmetic but not the order of evaluation. The order
below is a reading chosen to be the CUDA kernel's own, so that the two can be
compared bit for bit as a regression check of that kernel; it is not
independent evidence. The parity criterion of the FP16-arithmetic kernel is
its distance from the float64 Eq. 1 (relative L2 <= 2e-3), which holds for
any order.

Order of evaluation (the definition emulated here):
  * directions x, y, z, t; for each the forward hop, then the backward one;
  * half spinor: for the two leading nonzero rows k of the projector P,
    h_k = sum_s P[k, s] psi_s, one rounded addition per real part;
  * link product: chi_a = sum_b M_ab h_b for b = 0, 1, 2, the real part as
    Re(M_a0) Re(h_0) - Im(M_a0) Im(h_0) + Re(M_a1) Re(h_1) - ..., the imaginary
    part as Re(M_a0) Im(h_0) + Im(M_a0) Re(h_0) + ..., each term after the
    first fused into the running sum;
  * rebuild: row r of P is c_r times one of the two leading rows (c_r in
    {+-1, +-i}), and out_r += c_r chi, one rounded addition per real part.

The half spinor and the rebuild coefficients are read off the projector
matrices (1 -+ gamma_mu) of oracle.gamma.
"""

from __future__ import annotations

import numpy as np
import torch

from .gamma import projectors
from .wilson import _parity_tables, dims_of, restrict


def r16(a: np.ndarray) -> np.ndarray:
    """Round float64 values to FP16 (nearest even, subnormals kept) and back."""
    return a.astype(np.float16).astype(np.float64)


def fma16(a: np.ndarray, b: np.ndarray, c: np.ndarray) -> np.ndarray:
    """a * b + c rounded once to FP16 (exact in float64 for FP16 operands of similar size)."""
    return r16(a * b + c)


def split_projector(P: np.ndarray):
    """The two half-spinor rows of a rank-2 projector P and the rebuild of its
    nonzero rows: returns (terms, rebuild) with terms[j] the (spin, coefficient)
    pairs of row j and rebuild the (row r, j, c) with P[r] = c P[k_j]."""
    rows = [r for r in range(4) if np.any(P[r] != 0)]
    lead = rows[:2]
    terms = [[(s, complex(P[k, s])) for s in range(4) if P[k, s] != 0] for k in lead]
    rebuild = []
    for r in rows:
        for j, k in enumerate(lead):
            s0 = int(np.nonzero(P[k])[0][0])
            c = P[r, s0] / P[k, s0]
            if np.allclose(P[r], c * P[k], atol=0):
                rebuild.append((r, j, complex(c)))
                break
        else:
            raise ValueError("projector row is not a multiple of a leading row")
    return terms, rebuild


def _cscale(c: complex, xr: np.ndarray, xi: np.ndarray):
    """c x for c in {+-1, +-2, +-i}: exact."""
    return c.real * xr - c.imag * xi, c.real * xi + c.imag * xr


def rebuild_third_row(m_r: np.ndarray, m_i: np.ndarray) -> None:
    """Row 2 of SU(3) matrices [..., 3, 3] from rows 0 and 1 in FP16
    arithmetic, in place: row2_b = conj(r0_b1 r1_b2 - r0_b2 r1_b1) with
    (b1, b2) = (b+1, b+2) mod 3. Each complex product is formed real part of
    the left factor first, the second product fused into the first:
    re = Re(a) Re(c) - Im(a) Im(c) - Re(a') Re(c') + Im(a') Im(c'),
    im = Re(a) Im(c) + Im(a) Re(c) - Re(a') Im(c') - Im(a') Re(c'),
    a = r0_b1, c = r1_b2, a' = r0_b2, c' = r1_b1, one rounding per term."""
    for b in range(3):
        b1, b2 = (b + 1) % 3, (b + 2) % 3
        ar, ai = m_r[..., 0, b1], m_i[..., 0, b1]
        cr, ci = m_r[..., 1, b2], m_i[..., 1, b2]
        a2r, a2i = m_r[..., 0, b2], m_i[..., 0, b2]
        c2r, c2i = m_r[..., 1, b1], m_i[..., 1, b1]
        re = r16(ar * cr)
        re = fma16(ai, -ci, re)
        re = fma16(-a2r, c2r, re)
        re = fma16(-a2i, -c2i, re)
        im = r16(ar * ci)
        im = fma16(ai, cr, im)
        im = fma16(-a2r, c2i, im)
        im = fma16(-a2i, c2r, im)
        m_r[..., 2, b] = re
        m_i[..., 2, b] = -im


def hop_pq_fp16(U: torch.Tensor, psi: torch.Tensor, p: int, bc=(1, 1, 1, -1), recon: int = 18) -> torch.Tensor:
    """H restricted to outputs on parity p (Eq. 1), in FP16 arithmetic.

    U and psi are rounded to FP16 first (they are normally FP16 values
    already); with recon = 12 only the first two rows of each link matrix as
    it is applied (U_mu(x), or U_mu(x - mu)^+ for the backward hop) are
    kept and the third is rebuilt by rebuild_third_row, which assumes SU(3).
    The result is a full-lattice complex128 field of FP16 values, zero off
    parity p."""
    if recon not in (12, 18):
        raise ValueError("recon must be 12 or 18")
    dims = dims_of(psi)
    sites, per_mu = _parity_tables(dims, p, bc)
    pm, pp = projectors()
    uf = torch.view_as_real(U.reshape(4, -1, 3, 3).contiguous()).numpy()
    uf = r16(uf)
    pf = r16(torch.view_as_real(psi.reshape(-1, 4, 3).contiguous()).numpy())
    site_idx = sites.numpy()
    n = len(site_idx)
    acc_r = np.zeros((n, 4, 3))
    acc_i = np.zeros((n, 4, 3))
    for mu in range(4):
        up, dn, ph_up, ph_dn = per_mu[mu]
        up, dn = up.numpy(), dn.numpy()
        fu = ph_up.real.numpy().reshape(-1, 1)      # +-1 per site
        fd = ph_dn.real.numpy().reshape(-1, 1)
        # forward: U_mu(x); backward: U_mu(x - mu)^+ (conjugate transpose)
        mf_r, mf_i = uf[mu, site_idx, :, :, 0].copy(), uf[mu, site_idx, :, :, 1].copy()
        mb_r = np.swapaxes(uf[mu, dn, :, :, 0], -1, -2).copy()
        mb_i = -np.swapaxes(uf[mu, dn, :, :, 1], -1, -2)
        if recon == 12:
            rebuild_third_row(mf_r, mf_i)
            rebuild_third_row(mb_r, mb_i)
        for P, nb, f, m_r, m_i in ((pm[mu].numpy(), up, fu, mf_r, mf_i), (pp[mu].numpy(), dn, fd, mb_r, mb_i)):
            src_r, src_i = pf[nb, :, :, 0] * f[:, :, None], pf[nb, :, :, 1] * f[:, :, None]   # exact phase
            terms, rebuild = split_projector(P)
            h = []
            for row in terms:
                hr, hi = None, None
                for s, c in row:
                    tr, ti = _cscale(c, src_r[:, s], src_i[:, s])
                    hr, hi = (tr, ti) if hr is None else (r16(hr + tr), r16(hi + ti))
                h.append((hr, hi))
            chi = []
            for hr, hi in h:
                cr = np.empty((n, 3))
                ci = np.empty((n, 3))
                for a in range(3):
                    re = r16(m_r[:, a, 0] * hr[:, 0])
                    re = fma16(-m_i[:, a, 0], hi[:, 0], re)
                    im = r16(m_r[:, a, 0] * hi[:, 0])
                    im = fma16(m_i[:, a, 0], hr[:, 0], im)
                    for b in (1, 2):
                        re = fma16(m_r[:, a, b], hr[:, b], re)
                        re = fma16(-m_i[:, a, b], hi[:, b], re)
                        im = fma16(m_r[:, a, b], hi[:, b], im)
                        im = fma16(m_i[:, a, b], hr[:, b], im)
                    cr[:, a], ci[:, a] = re, im
                chi.append((cr, ci))
            for r, j, c in rebuild:
                tr, ti = _cscale(c, *chi[j])
                acc_r[:, r] = r16(acc_r[:, r] + tr)
                acc_i[:, r] = r16(acc_i[:, r] + ti)
    out = np.zeros(pf.shape)
    out[site_idx, :, :, 0] = acc_r
    out[site_idx, :, :, 1] = acc_i
    return torch.view_as_complex(torch.from_numpy(out).contiguous()).reshape(psi.shape)


def eo_operator_fp16(U16: torch.Tensor, psi_e: torch.Tensor, kappa: float, store, bc=(1, 1, 1, -1)) -> torch.Tensor:
    """A psi_e = psi_e - kappa^2 H_eo H_oe psi_e (Eq. 4) with both hops in FP16
    arithmetic; the odd intermediate and the result are stored with ``store``,
    the axpy is formed in float64 before that rounding."""
    tmp = store(hop_pq_fp16(U16, psi_e, 1, bc))
    return store(restrict(psi_e, 0) - kappa * kappa * hop_pq_fp16(U16, tmp, 0, bc))
