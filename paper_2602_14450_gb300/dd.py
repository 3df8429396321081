"""Domain decomposition of the even-odd Wilson operator over a grid of processes.

The paper runs its solver on 64 MPI processes (Sec. 6) with every global sum
taken in FP64 across them (Sec. 5, Fig. 3). This module is the host side of
that split for the library:

* ``Partition``  -- the process grid: global and local extents, a rank's
                    coordinates and origin, its neighbours, ``choose_grid``
                    (split t first, then z, y, x) and the slices that scatter
                    global fields to sub-lattices and gather them back.
* ``DistComm``   -- one sub-lattice per process: the face exchange with
                    ``torch.distributed`` point-to-point messages (gloo for
                    host buffers, NCCL for device buffers) and the FP64
                    allreduce of dot products.
* ``LocalComm``  -- every sub-lattice in this process (copies instead of
                    messages, the sum in rank order instead of an allreduce).
* ``GpuDomain``  -- one sub-lattice on the GPU through the C ABI
                    (``wd_dd_pack``, ``wd_dd_hop_interior``, ``wd_dd_hop_faces``,
                    ``wd_vec_dot``, ``wd_vec_axpby``).
* ``hop``, ``eo_operator``, ``dot``, ``bicgstab`` -- the operator and an FP64
                    BiCGStab on a set of sub-lattices. Each hop packs the
                    faces, starts the exchange, runs the interior kernel while
                    the faces travel, waits, and adds the face terms.

A domain object ("backend") offers: ``face_buffers()`` -> (send, recv) lists
of 8 (None for directions that are not split), ``pack``, ``hop_interior``,
``hop_faces``, ``dot`` (local FP64 part), ``axpby``, ``new_vector``,
``copy_``. Only ``GpuDomain`` is part of the library; tests supply a float64
CPU domain to check the split logic without a GPU.
"""

from __future__ import annotations

from dataclasses import dataclass

import torch

from . import wd


# --------------------------------------------------------------------------- grid

@dataclass(frozen=True)
class Partition:
    global_dims: tuple
    grid: tuple
    rank: int

    def __post_init__(self):
        gd, gr = tuple(int(d) for d in self.global_dims), tuple(int(p) for p in self.grid)
        object.__setattr__(self, "global_dims", gd)
        object.__setattr__(self, "grid", gr)
        if len(gd) != 4 or len(gr) != 4:
            raise ValueError("dims and grid need 4 entries (x, y, z, t)")
        for mu in range(4):
            if gr[mu] < 1 or gd[mu] % gr[mu]:
                raise ValueError(f"extent {gd[mu]} in direction {mu} does not split into {gr[mu]} parts")
            loc = gd[mu] // gr[mu]
            if loc < 2 or loc % 2:
                raise ValueError(f"local extent {loc} in direction {mu} must be even and >= 2")
        if not 0 <= self.rank < self.size:
            raise ValueError(f"rank {self.rank} outside a grid of {self.size}")

    @property
    def size(self) -> int:
        return self.grid[0] * self.grid[1] * self.grid[2] * self.grid[3]

    @property
    def local_dims(self) -> tuple:
        return tuple(self.global_dims[mu] // self.grid[mu] for mu in range(4))

    @staticmethod
    def coords_of(grid, rank) -> tuple:
        """Grid coordinates of a rank; x fastest: rank = cx + Px (cy + Py (cz + Pz ct))."""
        c = []
        for mu in range(4):
            c.append(rank % grid[mu])
            rank //= grid[mu]
        return tuple(c)

    @staticmethod
    def rank_of(grid, coords) -> int:
        r = 0
        for mu in (3, 2, 1, 0):
            r = r * grid[mu] + coords[mu] % grid[mu]
        return r

    @property
    def coords(self) -> tuple:
        return self.coords_of(self.grid, self.rank)

    @property
    def origin(self) -> tuple:
        return tuple(self.coords[mu] * self.local_dims[mu] for mu in range(4))

    def split(self, mu: int) -> bool:
        return self.grid[mu] > 1

    def neighbour(self, mu: int, step: int) -> int:
        """Rank of the sub-lattice `step` (+1 / -1) places away in direction mu (periodic)."""
        c = list(self.coords)
        c[mu] = (c[mu] + step) % self.grid[mu]
        return self.rank_of(self.grid, c)

    def face_sites(self, mu: int) -> int:
        """Face sites of one parity in direction mu (a face buffer's length in sites)."""
        ld = self.local_dims
        return ld[0] * ld[1] * ld[2] * ld[3] // (2 * ld[mu])

    def block(self):
        """Slices of this sub-lattice in a [Lt, Lz, Ly, Lx, ...] field."""
        o, ld = self.origin, self.local_dims
        return tuple(slice(o[mu], o[mu] + ld[mu]) for mu in (3, 2, 1, 0))

    def scatter_field(self, f: torch.Tensor) -> torch.Tensor:
        """This rank's block of a global quark field [Lt, Lz, Ly, Lx, 4, 3]."""
        return f[self.block()].contiguous()

    def scatter_gauge(self, u: torch.Tensor) -> torch.Tensor:
        """This rank's links of a global gauge field [4, Lt, Lz, Ly, Lx, 3, 3]."""
        return u[(slice(None),) + self.block()].contiguous()

    @staticmethod
    def gather_field(parts, blocks) -> torch.Tensor:
        """Assemble the global field from every rank's block (lists in rank order)."""
        p0 = parts[0]
        shape = [max(b[i].stop for b in blocks) for i in range(4)] + list(p0.shape[4:])
        out = torch.zeros(shape, dtype=p0.dtype, device=p0.device)
        for f, b in zip(parts, blocks):
            out[b] = f
        return out


def choose_grid(global_dims, nranks: int) -> tuple:
    """A process grid for nranks processes: factors of 2 (then 3, 5, ...) go to
    t first, then z, y, x, each time to the first direction whose local extent
    stays even after the split (the surface per site stays small and the
    innermost x direction, the one the kernels stream along, stays whole)."""
    grid = [1, 1, 1, 1]
    n = int(nranks)
    f = 2
    while n > 1:
        while n % f:
            f += 1
        for mu in (3, 2, 1, 0):
            loc = global_dims[mu] // grid[mu]
            if loc % f == 0 and (loc // f) % 2 == 0 and loc // f >= 2:
                grid[mu] *= f
                break
        else:
            raise ValueError(f"cannot split {tuple(global_dims)} over {nranks} processes")
        n //= f
    return tuple(grid)


# ----------------------------------------------------------------- communication

class LocalComm:
    """Every sub-lattice in this process: domains[r] is rank r of one Partition grid."""

    def __init__(self, parts):
        self.parts = list(parts)

    def start_exchange(self, sends, recvs):
        for r, p in enumerate(self.parts):
            for mu in range(4):
                if not p.split(mu):
                    continue
                recvs[p.neighbour(mu, -1)][2 * mu].copy_(sends[r][2 * mu])          # my lower face, down
                recvs[p.neighbour(mu, +1)][2 * mu + 1].copy_(sends[r][2 * mu + 1])  # my upper face, up
        return None

    def wait(self, handle):
        return None

    def allreduce(self, local_sums):
        """local_sums: per local domain a list of complex numbers; summed in rank order."""
        n = len(local_sums[0])
        return [sum((ls[i] for ls in local_sums), 0j) for i in range(n)]


class DistComm:
    """One sub-lattice per process over torch.distributed (gloo or NCCL)."""

    def __init__(self, part: Partition):
        import torch.distributed as dist
        self.dist = dist
        self.parts = [part]
        if dist.get_world_size() != part.size or dist.get_rank() != part.rank:
            raise ValueError("the process group must match the partition")

    def start_exchange(self, sends, recvs):
        dist, p = self.dist, self.parts[0]
        (send,), (recv,) = sends, recvs
        ops = []
        for mu in range(4):
            if not p.split(mu):
                continue
            # tags keep the two faces apart when both neighbours are the same process (gloo);
            # NCCL pairs messages in posting order, which is the same on every process
            ops.append(dist.P2POp(dist.isend, send[2 * mu], p.neighbour(mu, -1), tag=2 * mu))
            ops.append(dist.P2POp(dist.isend, send[2 * mu + 1], p.neighbour(mu, +1), tag=2 * mu + 1))
            ops.append(dist.P2POp(dist.irecv, recv[2 * mu], p.neighbour(mu, +1), tag=2 * mu))
            ops.append(dist.P2POp(dist.irecv, recv[2 * mu + 1], p.neighbour(mu, -1), tag=2 * mu + 1))
        return dist.batch_isend_irecv(ops) if ops else []

    def wait(self, handle):
        for op in handle or ():
            op.wait()

    def allreduce(self, local_sums):
        (ls,) = local_sums
        t = torch.tensor([[z.real, z.imag] for z in ls], dtype=torch.float64)
        self.dist.all_reduce(t)
        return [complex(a, b) for a, b in t.tolist()]


# -------------------------------------------------------------- the GPU sub-lattice

class GpuDomain:
    """One sub-lattice on the GPU: a library handle with its local links and the split.

    Vectors are packed parity vectors (uint8 device tensors of
    ``wd_vector_bytes``); face buffers are uint8 device tensors of
    ``wd_dd_face_bytes``."""

    def __init__(self, part: Partition, kappa: float, u_local_host: torch.Tensor, prec="fp64", recon=18,
                 bc=(1, 1, 1, -1), arith=32, stream=None):
        self.part, self.kappa, self.prec, self.recon = part, float(kappa), wd.PREC.get(prec, prec), int(recon)
        self.lat = wd.Lattice(part.local_dims, kappa, bc)
        self.lat.set_gauge(u_local_host)
        self.lat.set_arith(arith)
        self.lat.dd_set_partition(part.grid, part.coords)
        self.stream = stream

    def _s(self):
        return wd._stream(self.stream)

    def new_vector(self):
        return torch.zeros(self.lat.vector_bytes(self.prec), dtype=torch.uint8, device="cuda")

    def copy_(self, dst, src):
        dst.copy_(src)

    def face_buffers(self):
        send, recv = [None] * 8, [None] * 8
        for mu in range(4):
            if self.part.split(mu):
                nb = self.lat.dd_face_bytes(self.prec, mu)
                for side in range(2):
                    send[2 * mu + side] = torch.empty(nb, dtype=torch.uint8, device="cuda")
                    recv[2 * mu + side] = torch.empty(nb, dtype=torch.uint8, device="cuda")
        return send, recv

    def pack(self, parity, x, send):
        self.lat.dd_pack(self.prec, parity, x, send, self.stream)

    def hop_interior(self, parity, x, out, a=1.0, b=0.0, y=None):
        self.lat.dd_hop_interior(self.prec, self.recon, parity, x, y, a, b, out, self.stream)

    def hop_faces(self, parity, recv, out, a=1.0):
        self.lat.dd_hop_faces(self.prec, parity, recv, a, out, self.stream)

    def dot(self, a, b) -> complex:
        return self.lat.vec_dot(self.prec, a, b, self.stream)

    def axpby(self, a, x, b, y):
        self.lat.vec_axpby(self.prec, a, x, b, y, self.stream)

    def pack_field(self, parity, lex_dev, out):
        """Packed parity vector of a local FP64 host-layout device field."""
        self.lat.pack(self.prec, parity, lex_dev, out, self.stream)

    def unpack_field(self, parity, packed, lex_dev):
        self.lat.unpack(self.prec, parity, packed, lex_dev, self.stream)


# ------------------------------------------------------------- split operations

class DomainSet:
    """The sub-lattices this process holds (one, or all of them) and their communicator."""

    def __init__(self, domains, comm):
        self.domains = list(domains)
        self.comm = comm
        self.bufs = [d.face_buffers() for d in self.domains]
        self.kappa = self.domains[0].kappa

    def new_vectors(self):
        return [d.new_vector() for d in self.domains]


def hop(ds: DomainSet, parity, xs, outs, a=1.0, b=0.0, ys=None):
    """outs = a H_pq xs + b ys on every sub-lattice (H_pq of Eq. 1 onto parity `parity`)."""
    sends = [bf[0] for bf in ds.bufs]
    recvs = [bf[1] for bf in ds.bufs]
    for d, x, send in zip(ds.domains, xs, sends):
        d.pack(parity, x, send)
    handle = ds.comm.start_exchange(sends, recvs)
    for i, (d, x, out) in enumerate(zip(ds.domains, xs, outs)):   # overlaps the exchange
        d.hop_interior(parity, x, out, a, b, None if ys is None else ys[i])
    ds.comm.wait(handle)
    for d, recv, out in zip(ds.domains, recvs, outs):
        d.hop_faces(parity, recv, out, a)


def eo_operator(ds: DomainSet, xs, outs, tmps):
    """outs = xs - kappa^2 H_eo H_oe xs (Eq. 4) on even-site vectors."""
    k = ds.kappa
    hop(ds, 1, xs, tmps)
    hop(ds, 0, tmps, outs, a=-k * k, b=1.0, ys=xs)


def dot(ds: DomainSet, pairs):
    """Global FP64 dot products (a, b) = sum conj(a) b for a list of (as, bs) pairs:
    local FP64 sums on each sub-lattice, then one allreduce."""
    local = [[d.dot(a[i], b[i]) for a, b in pairs] for i, d in enumerate(ds.domains)]
    return ds.comm.allreduce(local)


def axpby(ds: DomainSet, a, xs, b, ys):
    """ys = a xs + b ys on every sub-lattice."""
    for d, x, y in zip(ds.domains, xs, ys):
        d.axpby(a, x, b, y)


def bicgstab(ds: DomainSet, bs, xs, tol: float, maxiter: int = 100000):
    """BiCGStab (van der Vorst) for A x = b with A the even-odd operator of Eq. 4
    on the split lattice, every scalar in FP64 and every dot product a global
    FP64 sum. Stops when the recursive |r| <= tol |b|. xs must be zero on entry.
    Returns (iterations, |r| / |b|)."""
    r = ds.new_vectors()
    rhat = ds.new_vectors()
    p = ds.new_vectors()
    v = ds.new_vectors()
    s = ds.new_vectors()
    t = ds.new_vectors()
    tmp = ds.new_vectors()
    for d, ri, rh, bi in zip(ds.domains, r, rhat, bs):
        d.copy_(ri, bi)
        d.copy_(rh, bi)
    (bb,) = dot(ds, [(bs, bs)])
    bnorm = abs(bb.real) ** 0.5
    rho_old = alpha = omega = 1.0 + 0j
    it = 0
    rn = bnorm
    while it < maxiter:
        (rr,) = dot(ds, [(r, r)])
        rn = abs(rr.real) ** 0.5
        if rn <= tol * bnorm or not rn == rn:
            break
        (rho,) = dot(ds, [(rhat, r)])
        beta = (rho / rho_old) * (alpha / omega)
        axpby(ds, -omega, v, 1.0, p)           # p = p - omega v
        axpby(ds, 1.0, r, beta, p)             # p = r + beta (p - omega v)
        eo_operator(ds, p, v, tmp)
        (rv,) = dot(ds, [(rhat, v)])
        alpha = rho / rv
        for d, si, ri in zip(ds.domains, s, r):
            d.copy_(si, ri)
        axpby(ds, -alpha, v, 1.0, s)           # s = r - alpha v
        eo_operator(ds, s, t, tmp)
        ts, tt = dot(ds, [(t, s), (t, t)])
        omega = ts / tt
        axpby(ds, alpha, p, 1.0, xs)           # x += alpha p + omega s
        axpby(ds, omega, s, 1.0, xs)
        for d, ri, si in zip(ds.domains, r, s):
            d.copy_(ri, si)
        axpby(ds, -omega, t, 1.0, r)           # r = s - omega t
        rho_old = rho
        it += 1
    return it, rn / bnorm
