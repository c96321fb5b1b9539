"""Decomposition of one domain into z-slabs with a halo exchange per step.

A domain of nz planes is split into contiguous z ranges, one per slab.  Each slab is a
context (lbve_create) holding its planes plus one ghost plane on each side that mirrors
the neighbouring slab's boundary plane; only its own planes are computed
(lbve_set_z_range).  One step of the domain (lbve_step_phase):

    stream-collide on every slab; exchange the PDFs that crossed each face and u;
    stress update on every slab; exchange tau.

The exchange packs a slab's face data into a device buffer (lbve_halo_pack) and unpacks
it into the neighbour (lbve_halo_unpack): here between slabs on one device
(``SlabDomain``), or between ranks with torch.distributed point-to-point messages
(``exchange_with_neighbours``, NCCL on GPUs).  All physics runs in the CUDA library; this
module only partitions, orders and moves buffers.
"""
from __future__ import annotations

import numpy as np

from . import lbve

NOSLIP = 1
FIELDS = (lbve.HALO_F, lbve.HALO_U, lbve.HALO_TAU)


def split_planes(nz: int, nslabs: int):
    """Contiguous z ranges [z0, z1) of nslabs slabs covering nz planes, sizes differing by
    at most one plane."""
    if not 1 <= nslabs <= nz:
        raise ValueError("need 1 <= nslabs <= nz")
    base, extra = divmod(nz, nslabs)
    out, z = [], 0
    for k in range(nslabs):
        n = base + (1 if k < extra else 0)
        out.append((z, z + n))
        z += n
    return out


def neighbours(k: int, nslabs: int, periodic_z: bool):
    """(lower, upper) slab indices of slab k, None beyond a closed domain."""
    lo = k - 1 if k > 0 else (nslabs - 1 if periodic_z else None)
    hi = k + 1 if k < nslabs - 1 else (0 if periodic_z else None)
    return lo, hi


def ghost_planes(z0: int, z1: int, nz: int, periodic_z: bool):
    """Global plane index of each local plane of the slab [z0, z1) with its two ghost
    planes (None: beyond a closed domain, a solid plane)."""
    out = []
    for z in range(z0 - 1, z1 + 1):
        if 0 <= z < nz:
            out.append(z)
        else:
            out.append(z % nz if periodic_z else None)
    return out


def slab_array(field, planes, axis, fill=0):
    """Local copy of a global array (..., nz, ny, nx) with the slab's planes on `axis`."""
    shape = list(field.shape)
    shape[axis] = len(planes)
    out = np.empty(shape, dtype=field.dtype)
    for k, z in enumerate(planes):
        idx = [slice(None)] * field.ndim
        idx[axis] = k
        if z is None:
            out[tuple(idx)] = fill
        else:
            src = [slice(None)] * field.ndim
            src[axis] = z
            out[tuple(idx)] = field[tuple(src)]
    return out


class SlabDomain:
    """A domain split into z-slabs on the current device; behaves like one Solver."""

    def __init__(self, shape, nslabs, *, periodic=(1, 1, 1), flags=None, wall_vel=(), **params):
        import torch

        nx, ny, nz = (int(v) for v in shape)
        self.shape = (nx, ny, nz)
        self.periodic_z = bool(periodic[2])
        self.ranges = split_planes(nz, nslabs)
        self.planes = [ghost_planes(z0, z1, nz, self.periodic_z) for z0, z1 in self.ranges]
        fl = np.zeros((nz, ny, nx), np.uint8) if flags is None else np.asarray(flags, np.uint8).reshape(nz, ny, nx)
        self.flags = fl
        self.slabs = []
        for (z0, z1), planes in zip(self.ranges, self.planes):
            s = lbve.Solver((nx, ny, z1 - z0 + 2), periodic=(periodic[0], periodic[1], 0), **params)
            s.set_z_range(1, z1 - z0 + 1, z0)
            s.set_geometry(slab_array(fl, planes, 0, fill=NOSLIP), wall_vel)
            self.slabs.append(s)
        self._buf = {w: [torch.empty(self.slabs[0].halo_bytes(w), dtype=torch.uint8, device="cuda") for _ in range(2)]
                     for w in FIELDS}

    @property
    def time(self) -> int:
        return self.slabs[0].time

    def init_fields(self, rho=None, u=None, tau=None):
        for s, planes in zip(self.slabs, self.planes):
            s.init_fields(rho=None if rho is None else slab_array(np.asarray(rho), planes, 0, fill=1.0),
                          u=None if u is None else slab_array(np.asarray(u), planes, 1),
                          tau=None if tau is None else slab_array(np.asarray(tau), planes, 1))

    def exchange(self, what):
        """Halo exchange of one field between every pair of neighbouring slabs."""
        n = len(self.slabs)
        for k in range(n):
            _, hi = neighbours(k, n, self.periodic_z)
            if hi is None:
                continue
            a, b = self.slabs[k], self.slabs[hi]
            up, down = self._buf[what]
            a.halo_pack(what, 1, up.data_ptr())
            b.halo_pack(what, 0, down.data_ptr())
            b.halo_unpack(what, 0, up.data_ptr())
            a.halo_unpack(what, 1, down.data_ptr())

    def step(self, n: int = 1):
        for _ in range(int(n)):
            for s in self.slabs:
                s.step_phase(0)
            self.exchange(lbve.HALO_F)
            self.exchange(lbve.HALO_U)
            for s in self.slabs:
                s.step_phase(1)
            self.exchange(lbve.HALO_TAU)

    def read_fields(self):
        """rho, u, tau, flags of the whole domain (ghost planes left out)."""
        parts = [s.read_fields() for s in self.slabs]
        rho = np.concatenate([p[0][1:-1] for p in parts], axis=0)
        u = np.concatenate([p[1][:, 1:-1] for p in parts], axis=1)
        tau = np.concatenate([p[2][:, 1:-1] for p in parts], axis=1)
        fl = np.concatenate([p[3][1:-1] for p in parts], axis=0)
        return rho, u, tau, fl

    def read_pdfs(self):
        return np.concatenate([s.read_pdfs()[:, 1:-1] for s in self.slabs], axis=1)

    def body_forces(self):
        return sum(s.body_forces() for s in self.slabs)

    def close(self):
        for s in self.slabs:
            s.close()
        self.slabs = []


def exchange_with_neighbours(what, rank, world, periodic_z, pack, unpack, send_bufs, recv_bufs, group=None):
    """One halo exchange of a field between the ranks of a z-decomposed domain, one slab
    per rank in z order.  pack(what, side, buf) fills a buffer from this rank's slab,
    unpack(what, side, buf) applies a received one (side 0: low z, 1: high z);
    send_bufs / recv_bufs hold two tensors each (index = side).  Every rank posts its sends
    (up, then down) before its receives (from below, then from above), so that messages
    between a pair of ranks match in order also where tags are not used (NCCL) and where
    both neighbours are one rank (two ranks, periodic); the tags keep them apart where
    they are (gloo)."""
    import torch.distributed as dist

    lo, hi = neighbours(rank, world, periodic_z)
    ops = []
    if hi is not None:
        pack(what, 1, send_bufs[1])
        ops.append(dist.P2POp(dist.isend, send_bufs[1], hi, group, tag=2 * what))
    if lo is not None:
        pack(what, 0, send_bufs[0])
        ops.append(dist.P2POp(dist.isend, send_bufs[0], lo, group, tag=2 * what + 1))
    if lo is not None:
        ops.append(dist.P2POp(dist.irecv, recv_bufs[0], lo, group, tag=2 * what))
    if hi is not None:
        ops.append(dist.P2POp(dist.irecv, recv_bufs[1], hi, group, tag=2 * what + 1))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    if hi is not None:
        unpack(what, 1, recv_bufs[1])
    if lo is not None:
        unpack(what, 0, recv_bufs[0])
