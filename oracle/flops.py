"""The hopping term of Eq. 1 in Sec. 2's three steps, on numbers that count
their own floating-point operations -- test infrastructure only.

Sec. 2 splits one nearest-neighbour hop into
  1. four-to-two: the projector (1 -+ gamma_mu) keeps two independent spin
     components of the neighbour spinor, six complex numbers over colour;
  2. three-to-three: each of the two colour vectors is multiplied by the
     link U_mu(x) (forward) or U_mu(x - mu)^+ (backward);
  3. two-to-four: the four spin components are rebuilt from the two by
     permutations and sign changes and accumulated into the output, twelve
     complex additions;
and counts 168 real operations for it, against 12 * 12 * 8 = 1152 for a
dense 12 x 12 complex block applied to a vector and accumulated.

Here every complex value is a ``Num`` that adds to a shared counter on each
real operation it performs: an addition of two complex numbers is 2, a
product of two complex numbers 6 (four real products, two real sums), a
product with a real factor other than +-1 is 2. A product with +-1 or +-i
exchanges real and imaginary parts and flips signs; it is not a
floating-point operation (Sec. 2: "permutation and sign modification").
The counts below are therefore those of the operations actually performed,
not constants. The half spinor and the rebuild coefficients are read off the
projector matrices of oracle.gamma; with the Dirac basis of oracle.gamma the
t projectors are diagonal (2 on two spin rows, 0 on the others), so a t hop
scales instead of adding in step 1 and accumulates only six complex numbers
in step 3.

Plain Python loops over sites: for lattices of a few hundred sites.
"""

from __future__ import annotations

import torch

from .gamma import projectors
from .wilson import _parity_tables, dims_of


class Counter:
    def __init__(self):
        self.n = 0


class Num:
    """A complex number whose arithmetic adds its real operations to ``ctr.n``."""

    __slots__ = ("re", "im", "ctr")

    def __init__(self, re, im, ctr):
        self.re, self.im, self.ctr = float(re), float(im), ctr

    def __add__(self, o):
        self.ctr.n += 2
        return Num(self.re + o.re, self.im + o.im, self.ctr)

    def __mul__(self, o):
        self.ctr.n += 6
        return Num(self.re * o.re - self.im * o.im, self.re * o.im + self.im * o.re, self.ctr)

    def times_const(self, c: complex):
        """c * self for a constant c of the projector or boundary phase."""
        if c in (1, -1):
            return Num(c.real * self.re, c.real * self.im, self.ctr)
        if c in (1j, -1j):                      # +-i: swap the parts, one sign change
            s = c.imag
            return Num(-s * self.im, s * self.re, self.ctr)
        if c.imag == 0:
            self.ctr.n += 2
            return Num(c.real * self.re, c.real * self.im, self.ctr)
        raise ValueError(f"unexpected constant {c}")


def half_spinor_rows(P: torch.Tensor):
    """Two linearly independent nonzero rows (k0, k1) of a rank-2 projector P,
    and for every nonzero row r the pair (j, c) with P[r] = c P[k_j]."""
    P = P.numpy()
    rows = [r for r in range(4) if abs(P[r]).sum() > 0]
    lead = rows[:2]
    rebuild = {}
    for r in rows:
        for j, k in enumerate(lead):
            s0 = next(s for s in range(4) if P[k, s] != 0)
            c = P[r, s0] / P[k, s0]
            if all(P[r, s] == c * P[k, s] for s in range(4)):
                rebuild[r] = (j, complex(c))
                break
        else:
            raise ValueError("projector rows are not multiples of two leading rows")
    return lead, rebuild


def one_hop(P: torch.Tensor, M, src, out, ctr: Counter) -> int:
    """out[s][a] += ((P (x) M) src)[s][a] for a spin projector P and a 3x3 colour
    matrix M (Nums), in Sec. 2's three steps; returns the real operations used."""
    n0 = ctr.n
    lead, rebuild = half_spinor_rows(P)
    Pn = P.numpy()
    # 1. four-to-two: h_j = sum_s P[k_j, s] src_s, for each colour
    h = []
    for k in lead:
        terms = [(s, complex(Pn[k, s])) for s in range(4) if Pn[k, s] != 0]
        hj = []
        for a in range(3):
            acc = src[terms[0][0]][a].times_const(terms[0][1])
            for s, c in terms[1:]:
                acc = acc + src[s][a].times_const(c)
            hj.append(acc)
        h.append(hj)
    # 2. three-to-three: chi_j = M h_j
    chi = []
    for hj in h:
        chi.append([M[a][0] * hj[0] + M[a][1] * hj[1] + M[a][2] * hj[2] for a in range(3)])
    # 3. two-to-four: out_r += c_r chi_j(r)
    for r, (j, c) in rebuild.items():
        for a in range(3):
            out[r][a] = out[r][a] + chi[j][a].times_const(c)
    return ctr.n - n0


def hop_pq_counted(U: torch.Tensor, psi: torch.Tensor, p: int, bc=(1, 1, 1, -1)):
    """H restricted to outputs on parity p (Eq. 1) through ``one_hop``.

    Returns (result as a full-lattice complex128 field, zero off parity p,
    and a dict (mu, +1 forward / -1 backward) -> set of operation counts
    seen for that hop over all sites)."""
    dims = dims_of(psi)
    sites, per_mu = _parity_tables(dims, p, bc)
    pm, pp = projectors()
    uf = U.reshape(4, -1, 3, 3)
    pf = psi.reshape(-1, 4, 3)
    ctr = Counter()
    counts = {}
    res = torch.zeros_like(pf)

    def num(z, phase=1.0):
        return Num(z.real * phase, z.imag * phase, ctr)   # the phase is +-1: a sign, not counted

    for i, x in enumerate(sites.tolist()):
        out = [[Num(0.0, 0.0, ctr) for _ in range(3)] for _ in range(4)]
        for mu in range(4):
            up, dn, ph_up, ph_dn = per_mu[mu]
            for sign, P, nb, ph in ((+1, pm[mu], up[i].item(), ph_up[i].item().real),
                                    (-1, pp[mu], dn[i].item(), ph_dn[i].item().real)):
                if sign > 0:
                    m = uf[mu, x]
                    M = [[num(m[a, b].item()) for b in range(3)] for a in range(3)]
                else:                                  # U_mu(x - mu)^+
                    m = uf[mu, nb]
                    M = [[num(m[b, a].item().conjugate()) for b in range(3)] for a in range(3)]
                src = [[num(pf[nb, s, a].item(), ph) for a in range(3)] for s in range(4)]
                counts.setdefault((mu, sign), set()).add(one_hop(P, M, src, out, ctr))
        for s in range(4):
            for a in range(3):
                res[x, s, a] = complex(out[s][a].re, out[s][a].im)
    return res.reshape(psi.shape), counts


def dense_block_flops(block: torch.Tensor, vec: torch.Tensor, out: torch.Tensor):
    """out += block @ vec for a 12 x 12 complex block on Nums; returns
    (the new out as complex128, the real operations used)."""
    ctr = Counter()
    o = [Num(z.real, z.imag, ctr) for z in out.tolist()]
    v = [Num(z.real, z.imag, ctr) for z in vec.tolist()]
    for r in range(12):
        for c in range(12):
            o[r] = o[r] + Num(block[r, c].real.item(), block[r, c].imag.item(), ctr) * v[c]
    return torch.tensor([complex(z.re, z.im) for z in o], dtype=torch.complex128), ctr.n
