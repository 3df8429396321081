"""The hopping term of Eq. 1 on one sub-lattice of a split lattice, float64,
for checking the domain-decomposition logic on CPU processes -- test
infrastructure only.

A sub-lattice sees its own links and quark field. A hop whose neighbour lies
outside it (x_mu = L_mu - 1 forward, x_mu = 0 backward, in a split direction)
needs data of the neighbouring process: here the neighbour sends, for its
face x_mu = 0, the projected spinors (1 - gamma_mu) psi (the receiver's
forward hop multiplies them by its own U_mu(x)), and for its face
x_mu = L_mu - 1 the projected, transported spinors (1 + gamma_mu) U_mu(x)^+ psi
(the link of a backward hop belongs to the sender), each with the boundary
phase when the hop wraps around the global lattice. Faces are whole 3-d
slabs [.., 4, 3] of the local field (the sites of the other parity are zero).

This is Eq. 1 restated term by term on the local block, with explicit 4x4
spin projectors and 3x3 colour matrices; it shares nothing with the CUDA
path's face format or kernels.
"""

from __future__ import annotations

import torch

from .gamma import projectors
from .wilson import dims_of, parity, restrict


def _slab(f: torch.Tensor, mu: int, i: int) -> torch.Tensor:
    return f.select(3 - mu, i)


class SubDomain:
    """One sub-lattice: local links ``u`` [4, lt, lz, ly, lx, 3, 3] and the split.

    ``grid``/``coords`` place it in the process grid; ``bc`` are the global
    boundary phases. Vectors are local complex128 fields [lt, lz, ly, lx, 4, 3]
    that vanish off the parity they live on."""

    def __init__(self, u: torch.Tensor, kappa: float, grid, coords, bc=(1, 1, 1, -1)):
        self.u, self.kappa = u, float(kappa)
        self.grid, self.coords, self.bc = tuple(grid), tuple(coords), tuple(bc)
        self.dims = (u.shape[4], u.shape[3], u.shape[2], u.shape[1])
        self.pm, self.pp = projectors()

    def split(self, mu):
        return self.grid[mu] > 1

    # --- the backend protocol of paper_2602_14450_gb300.dd -------------------
    def new_vector(self):
        lx, ly, lz, lt = self.dims
        return torch.zeros((lt, lz, ly, lx, 4, 3), dtype=torch.complex128)

    def copy_(self, dst, src):
        dst.copy_(src)

    def face_buffers(self):
        send, recv = [None] * 8, [None] * 8
        lx, ly, lz, lt = self.dims
        full = (lt, lz, ly, lx)
        for mu in range(4):
            if self.split(mu):
                shape = tuple(full[i] for i in range(4) if i != 3 - mu) + (4, 3)
                for side in range(2):
                    send[2 * mu + side] = torch.zeros(shape, dtype=torch.complex128)
                    recv[2 * mu + side] = torch.zeros(shape, dtype=torch.complex128)
        return send, recv

    def pack(self, p: int, x: torch.Tensor, send):
        """Faces of x (parity 1 - p) for the neighbours' hops onto parity p."""
        xin = restrict(x, 1 - p)
        L = self.dims
        for mu in range(4):
            if not self.split(mu):
                continue
            lower = _slab(xin, mu, 0)                                   # to the neighbour below
            ph = self.bc[mu] if self.coords[mu] == 0 else 1
            send[2 * mu].copy_(ph * (self.pm[mu] @ lower))             # (1 - gamma_mu) on spin
            upper = _slab(xin, mu, L[mu] - 1)                           # to the neighbour above
            link = _slab(self.u[mu], mu, L[mu] - 1)                     # U_mu(x) at that face
            ph = self.bc[mu] if self.coords[mu] == self.grid[mu] - 1 else 1
            # (1 + gamma_mu) on spin, U^+ on colour: psi_a -> sum_b conj(U_ba) psi_b
            send[2 * mu + 1].copy_(ph * ((self.pp[mu] @ upper) @ link.conj()))

    def hop_interior(self, p: int, x: torch.Tensor, out: torch.Tensor, a=1.0, b=0.0, y=None):
        """out = a (hops of Eq. 1 inside the block) x + b y, on parity p."""
        xin = restrict(x, 1 - p)
        L = self.dims
        acc = torch.zeros_like(xin)
        for mu in range(4):
            ax = 3 - mu
            fwd = torch.roll(xin, shifts=-1, dims=ax)                   # x(site + mu)
            bwd = torch.roll(xin, shifts=+1, dims=ax)                   # x(site - mu)
            ub = torch.roll(self.u[mu], shifts=+1, dims=ax)             # U_mu(site - mu)
            idx_f = [slice(None)] * fwd.dim()
            idx_f[ax] = L[mu] - 1
            idx_b = [slice(None)] * bwd.dim()
            idx_b[ax] = 0
            if self.split(mu):                                          # these neighbours are remote
                fwd[tuple(idx_f)] = 0
                bwd[tuple(idx_b)] = 0
            else:                                                       # wrap of the global lattice
                fwd[tuple(idx_f)] *= self.bc[mu]
                bwd[tuple(idx_b)] *= self.bc[mu]
            acc += self.pm[mu] @ (fwd @ self.u[mu].transpose(-1, -2))
            acc += self.pp[mu] @ (bwd @ ub.conj())
        res = a * restrict(acc, p)
        if b != 0:
            res = res + b * restrict(y, p)
        out.copy_(res)

    def hop_faces(self, p: int, recv, out: torch.Tensor, a=1.0):
        """out += a (hops entering through the faces), on parity p."""
        L = self.dims
        m = (parity(self.dims) == p).to(torch.complex128)[..., None, None]
        add = torch.zeros_like(out)
        for mu in range(4):
            if not self.split(mu):
                continue
            link = _slab(self.u[mu], mu, L[mu] - 1)
            _slab(add, mu, L[mu] - 1).add_(recv[2 * mu] @ link.transpose(-1, -2))   # forward: U_mu(x) here
            _slab(add, mu, 0).add_(recv[2 * mu + 1])                                # backward: link applied
        out.add_(a * add * m)

    def dot(self, a, b) -> complex:
        return complex(torch.vdot(a.reshape(-1), b.reshape(-1)).item())

    def axpby(self, a, x, b, y):
        y.copy_(a * x + b * y)
