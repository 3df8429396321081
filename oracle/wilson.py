"""Wilson-Dirac matrix and its even-odd form, float64, explicit spin matrices.

Fields are complex128 tensors: links ``U[mu, t, z, y, x, a, b]`` and quark
fields ``psi[t, z, y, x, spin, colour]`` (see ``paper_2602_14450_gb300.synth``).
Even-odd vectors are kept as full-lattice fields that vanish on the other
parity, so every function here is a direct transcription of a formula.

Boundary conditions: ``bc[mu]`` in {+1, -1} multiplies a hop that wraps
around the lattice in direction mu (fermion boundary phase); the links
themselves are never modified.
"""

from __future__ import annotations

import torch

from .gamma import projectors

CDT = torch.complex128


def dims_of(psi: torch.Tensor):
    lt, lz, ly, lx = psi.shape[:4]
    return (lx, ly, lz, lt)


def _neighbour(f: torch.Tensor, mu: int, step: int, phase: float) -> torch.Tensor:
    """f(x + step*mu-hat) with ``phase`` on the sites whose hop wraps around."""
    ax = 3 - mu
    g = torch.roll(f, shifts=-step, dims=ax)
    if phase != 1:
        edge = f.shape[ax] - 1 if step > 0 else 0
        idx = [slice(None)] * g.dim()
        idx[ax] = edge
        g[tuple(idx)] *= phase
    return g


def hop(U: torch.Tensor, psi: torch.Tensor, bc=(1, 1, 1, -1)) -> torch.Tensor:
    """Hopping term H of Eq. 1, so that D_W = 1 - kappa * H:

    (H psi)(x) = sum_mu [ (1 - gamma_mu) U_mu(x) psi(x + mu)
                        + (1 + gamma_mu) U_mu(x - mu)^+ psi(x - mu) ].

    Colour: (U psi_s)_a = sum_b U_ab psi_sb is ``psi @ U^T``; (U^+ psi)_a =
    sum_b conj(U_ba) psi_b is ``psi @ conj(U)``. Spin: a 4x4 matrix on the
    spin axis.
    """
    pm, pp = projectors()
    out = torch.zeros_like(psi)
    for mu in range(4):
        fwd = _neighbour(psi, mu, +1, bc[mu]) @ U[mu].transpose(-1, -2)
        out += pm[mu] @ fwd
        u_back = _neighbour(U[mu], mu, -1, 1)
        bwd = _neighbour(psi, mu, -1, bc[mu]) @ u_back.conj()
        out += pp[mu] @ bwd
    return out


def dirac(U, psi, kappa: float, bc=(1, 1, 1, -1)) -> torch.Tensor:
    """D_W psi = psi - kappa * H psi (Eq. 1)."""
    return psi - kappa * hop(U, psi, bc)


def parity(dims) -> torch.Tensor:
    """Site parity (x + y + z + t) mod 2 as an int tensor [Lt, Lz, Ly, Lx]; 0 is even."""
    lx, ly, lz, lt = dims
    t = torch.arange(lt).view(lt, 1, 1, 1)
    z = torch.arange(lz).view(1, lz, 1, 1)
    y = torch.arange(ly).view(1, 1, ly, 1)
    x = torch.arange(lx).view(1, 1, 1, lx)
    return (x + y + z + t) % 2


def restrict(psi: torch.Tensor, p: int) -> torch.Tensor:
    """Keep the sites of parity p, zero the others."""
    m = (parity(dims_of(psi)) == p).to(psi.dtype)
    return psi * m[..., None, None]


def hop_pq_full(U, psi, p: int, bc=(1, 1, 1, -1)) -> torch.Tensor:
    """H restricted to outputs on parity p and inputs on parity 1 - p, via the full-lattice hop."""
    return restrict(hop(U, restrict(psi, 1 - p), bc), p)


_TABLES = {}


def _parity_tables(dims, p: int, bc):
    """Lexicographic sites of parity p and, per direction, their neighbours and boundary phases."""
    key = (tuple(dims), p, tuple(bc))
    if key not in _TABLES:
        lx, ly, lz, lt = dims
        ext = (lx, ly, lz, lt)
        sites = torch.nonzero(parity(dims).reshape(-1) == p).reshape(-1)
        c = list(site_coords(dims, sites))
        lex = lambda cc: cc[0] + lx * (cc[1] + ly * (cc[2] + lz * cc[3]))
        per_mu = []
        for mu in range(4):
            up = [v.clone() for v in c]
            up[mu] = (c[mu] + 1) % ext[mu]
            dn = [v.clone() for v in c]
            dn[mu] = (c[mu] - 1) % ext[mu]
            ph_up = torch.where(c[mu] == ext[mu] - 1, float(bc[mu]), 1.0).to(CDT)[:, None, None]
            ph_dn = torch.where(c[mu] == 0, float(bc[mu]), 1.0).to(CDT)[:, None, None]
            per_mu.append((lex(up), lex(dn), ph_up, ph_dn))
        _TABLES[key] = (sites, per_mu)
    return _TABLES[key]


def hop_pq(U, psi, p: int, bc=(1, 1, 1, -1)) -> torch.Tensor:
    """H restricted to outputs on parity p and inputs on parity 1 - p (H_eo for p = 0).

    Eq. 1 evaluated only at the sites of parity p: their neighbours all lie on
    parity 1 - p, so only that part of psi is read. Same formula as ``hop``.
    """
    dims = dims_of(psi)
    sites, per_mu = _parity_tables(dims, p, bc)
    pm, pp = projectors()
    uf = U.reshape(4, -1, 3, 3)
    pf = psi.reshape(-1, 4, 3)
    acc = torch.zeros((len(sites), 4, 3), dtype=psi.dtype)
    for mu in range(4):
        up, dn, ph_up, ph_dn = per_mu[mu]
        fwd = (ph_up * pf[up]) @ uf[mu, sites].transpose(-1, -2)
        bwd = (ph_dn * pf[dn]) @ uf[mu, dn].conj()
        acc += pm[mu] @ fwd + pp[mu] @ bwd
    out = torch.zeros_like(pf)
    out[sites] = acc
    return out.reshape(psi.shape)


def eo_operator(U, psi_e, kappa: float, bc=(1, 1, 1, -1)) -> torch.Tensor:
    """A psi_e = psi_e - kappa^2 H_eo H_oe psi_e: the bracket of Eq. 4 with D_ee = D_oo = 1."""
    return restrict(psi_e, 0) - kappa * kappa * hop_pq(U, hop_pq(U, psi_e, 1, bc), 0, bc)


def eo_source(U, eta, kappa: float, bc=(1, 1, 1, -1)) -> torch.Tensor:
    """Right-hand side of Eq. 4: eta_e - D_eo eta_o = eta_e + kappa H_eo eta_o."""
    return restrict(eta, 0) + kappa * hop_pq(U, eta, 0, bc)


def eo_reconstruct(U, xi_e, eta, kappa: float, bc=(1, 1, 1, -1)) -> torch.Tensor:
    """Full solution from Eq. 5: xi_o = eta_o - D_oe xi_e = eta_o + kappa H_oe xi_e."""
    xi_o = restrict(eta, 1) + kappa * hop_pq(U, xi_e, 1, bc)
    return restrict(xi_e, 0) + xi_o


# --- sampled sites (for lattices too large to hold a dense check) -------------

def site_coords(dims, sites: torch.Tensor):
    lx, ly, lz, lt = dims
    s = sites.clone()
    x = s % lx
    s //= lx
    y = s % ly
    s //= ly
    z = s % lz
    t = s // lz
    return x, y, z, t


def hop_at_sites(U, psi, sites: torch.Tensor, bc=(1, 1, 1, -1)) -> torch.Tensor:
    """(H psi)(x) of Eq. 1 at the given lexicographic sites only; returns [n, 4, 3]."""
    dims = dims_of(psi)
    lx, ly, lz, lt = dims
    ext = (lx, ly, lz, lt)
    pm, pp = projectors()
    uf = U.reshape(4, -1, 3, 3)
    pf = psi.reshape(-1, 4, 3)
    c = list(site_coords(dims, sites))

    def lex(cc):
        return cc[0] + lx * (cc[1] + ly * (cc[2] + lz * cc[3]))

    out = torch.zeros((len(sites), 4, 3), dtype=CDT)
    for mu in range(4):
        up = [v.clone() for v in c]
        up[mu] = (c[mu] + 1) % ext[mu]
        ph_up = torch.where(c[mu] == ext[mu] - 1, float(bc[mu]), 1.0).to(CDT)[:, None, None]
        dn = [v.clone() for v in c]
        dn[mu] = (c[mu] - 1) % ext[mu]
        ph_dn = torch.where(c[mu] == 0, float(bc[mu]), 1.0).to(CDT)[:, None, None]
        fwd = (ph_up * pf[lex(up)]) @ uf[mu, lex(c)].transpose(-1, -2)
        bwd = (ph_dn * pf[lex(dn)]) @ uf[mu, lex(dn)].conj()
        out += pm[mu] @ fwd + pp[mu] @ bwd
    return out


# --- dense forms (tiny lattices only) -----------------------------------------

def dense_by_columns(U, kappa: float, bc=(1, 1, 1, -1)) -> torch.Tensor:
    """12V x 12V matrix whose column j is D_W applied to the j-th unit vector.

    Row/column index = site * 12 + spin * 3 + colour, site lexicographic.
    """
    lt, lz, ly, lx = U.shape[1:5]
    n = 12 * lx * ly * lz * lt
    e = torch.eye(n, dtype=CDT).reshape(n, lt, lz, ly, lx, 4, 3)
    cols = [dirac(U, e[j], kappa, bc).reshape(-1) for j in range(n)]
    return torch.stack(cols, dim=1)


def dense_by_blocks(U, kappa: float, bc=(1, 1, 1, -1)) -> torch.Tensor:
    """The same matrix written out block by block from Eq. 1.

    For every site x and direction mu, the 12x12 block coupling x to x+mu is
    -kappa * phase * kron(1 - gamma_mu, U_mu(x)) and the block coupling x to
    x-mu is -kappa * phase * kron(1 + gamma_mu, U_mu(x-mu)^+). Blocks landing on
    the same (x, y) pair (extent-2 directions) are added.
    """
    lt, lz, ly, lx = U.shape[1:5]
    ext = (lx, ly, lz, lt)
    v = lx * ly * lz * lt
    pm, pp = projectors()
    d = torch.eye(12 * v, dtype=CDT)
    uf = U.reshape(4, v, 3, 3)
    for s in range(v):
        c = [s % lx, (s // lx) % ly, (s // (lx * ly)) % lz, s // (lx * ly * lz)]
        for mu in range(4):
            up = list(c)
            up[mu] = (c[mu] + 1) % ext[mu]
            ph = bc[mu] if c[mu] == ext[mu] - 1 else 1
            j = up[0] + lx * (up[1] + ly * (up[2] + lz * up[3]))
            d[12 * s:12 * s + 12, 12 * j:12 * j + 12] -= kappa * ph * torch.kron(pm[mu], uf[mu, s])
            dn = list(c)
            dn[mu] = (c[mu] - 1) % ext[mu]
            ph = bc[mu] if c[mu] == 0 else 1
            j = dn[0] + lx * (dn[1] + ly * (dn[2] + lz * dn[3]))
            d[12 * s:12 * s + 12, 12 * j:12 * j + 12] -= kappa * ph * torch.kron(pp[mu], uf[mu, j].conj().T.contiguous())
    return d
