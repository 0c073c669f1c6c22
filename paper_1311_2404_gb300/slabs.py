"""Slab decomposition across processes (Sec. 3.6): one slab per rank.

The domain is cut into `world` slabs of whole rows of its slowest axis (z on
the 3-D lattices, y on D2Q9); rank r holds slab r as a rank handle of the
library (lbm_multi_create_rank).  Every time step
  1. lbm_multi_step_begin updates the slab's two boundary rows, packs the
     populations that leave through each face into the send buffers (only
     the directions with a component toward that face, Sec. 3.6's
     direction-limited exchange) and starts the bulk rows;
  2. exchange_faces moves the send buffers to the neighbouring ranks'
     receive buffers (periodic: rank world - 1's upper neighbour is rank 0);
  3. lbm_multi_step_end unpacks the received faces into the ghost rows.
The bulk rows update while the faces travel (Sec. 3.6's bulk/boundary
overlap).  With the NCCL backend the transfer is enqueued on the handle's
exchange stream straight from device memory; with gloo (CPU transport) the
faces are staged through pinned host memory.  All arithmetic runs in the
library's kernels; this module only moves buffers.
"""
from __future__ import annotations

import numpy as np

# message tags: faces travelling toward higher ranks, and toward lower ranks
TAG_UP, TAG_DOWN = 0, 1


def exchange_faces(send_up, send_down, recv_below, recv_above, rank, world, group=None):
    """Move one step's faces between the ranks of a periodic slab
    decomposition: send_up (leaving through the upper face) to rank + 1,
    where it arrives in recv_below; send_down to rank - 1, where it arrives
    in recv_above.  Tensors on the device of the group's backend (CUDA for
    NCCL, CPU for gloo), all of one size.  With world = 1 the rank is its own
    neighbour.  For two ranks both faces go to the same peer; the sends and
    receives are posted in the same order on both sides (and tagged), which
    pairs each face with the right receive buffer."""
    if world == 1:
        recv_below.copy_(send_up)
        recv_above.copy_(send_down)
        return
    import torch.distributed as dist
    up, down = (rank + 1) % world, (rank - 1) % world
    ops = [dist.P2POp(dist.isend, send_up, up, group, TAG_UP),
           dist.P2POp(dist.isend, send_down, down, group, TAG_DOWN),
           dist.P2POp(dist.irecv, recv_below, down, group, TAG_UP),
           dist.P2POp(dist.irecv, recv_above, up, group, TAG_DOWN)]
    for w in dist.batch_isend_irecv(ops):
        w.wait()


class _DeviceBytes:
    """A byte range of device memory owned by the library, seen by torch
    through the CUDA array interface (no copy, no ownership)."""

    def __init__(self, ptr: int, nbytes: int):
        self.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1",
                                         "data": (ptr, False), "version": 3, "strides": None}


class RankSlab:
    """Slab `rank` of a `world`-slab decomposition of an nx x ny x nz domain,
    stepped with its faces exchanged through torch.distributed.

    Setters take whole-domain arrays (each rank uses its rows); macro()
    returns whole-domain arrays holding this rank's rows (zeros elsewhere),
    so that a sum over ranks assembles the field."""

    def __init__(self, nx, ny, nz, lattice, model, tau, dtype, rank, world, group=None,
                 stream=None, overlap=True, host_staged=None):
        import torch
        import torch.distributed as dist
        from . import lbm
        self.lbm = lbm
        self.rank, self.world, self.group = rank, world, group
        self.D = 2 if lattice == lbm.LBM_D2Q9 else 3
        self.shape = (nz, ny, nx)
        self.m = lbm.lbm_multi_create_rank(nx, ny, nz, lattice, model, tau, dtype, world, rank)
        s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        lbm.lbm_multi_set_stream(self.m, s)
        lbm.lbm_multi_set_overlap(self.m, overlap)
        if host_staged is None:
            host_staged = world > 1 and dist.get_backend(group) != "nccl"
        self.host_staged = host_staged
        send, recv, nb = lbm.lbm_multi_face_buffers(self.m)
        self.face_bytes = nb
        self._send = torch.as_tensor(_DeviceBytes(send, 2 * nb), device="cuda")
        self._recv = torch.as_tensor(_DeviceBytes(recv, 2 * nb), device="cuda")
        self.exchange_stream = torch.cuda.ExternalStream(lbm.lbm_multi_exchange_stream(self.m))
        if host_staged:
            self._hsend = torch.empty(2 * nb, dtype=torch.uint8).pin_memory()
            self._hrecv = torch.empty(2 * nb, dtype=torch.uint8).pin_memory()
        self.rows = lbm.lbm_multi_rows(self.m)

    def close(self):
        """Free the handle.  The torch-side buffers go first: a pinned host
        buffer copied asynchronously on the exchange stream makes torch record
        an event on that stream when the buffer is freed, so the stream (the
        handle's) must still exist then."""
        if self.m:
            self.exchange_stream.synchronize()
            for name in ("_hsend", "_hrecv", "_send", "_recv"):
                if hasattr(self, name):
                    delattr(self, name)
            self.lbm.lbm_multi_destroy(self.m)
            self.m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_geometry(self, mask):
        self.lbm.lbm_multi_set_geometry(self.m, np.ascontiguousarray(mask, dtype=np.uint8))

    def set_force(self, fx, fy, fz=0.0):
        self.lbm.lbm_multi_set_force(self.m, fx, fy, fz)

    def set_rounding(self, mode):
        self.lbm.lbm_multi_set_rounding(self.m, mode)

    def set_boundary(self, cid, kind, method, normal, value):
        self.lbm.lbm_multi_set_boundary(self.m, cid, kind, method, normal, value)

    def init(self, rho, u):
        if isinstance(rho, np.ndarray):
            rho = np.ascontiguousarray(rho)
            u = np.ascontiguousarray(u, dtype=rho.dtype)
        self.lbm.lbm_multi_init_equilibrium(self.m, rho, u)

    def _transfer(self):
        import torch
        nb = self.face_bytes
        if self.host_staged:
            self.exchange_stream.synchronize()          # the faces are packed
            self._hsend.copy_(self._send)
            hs, hr = self._hsend, self._hrecv
            exchange_faces(hs[:nb], hs[nb:], hr[:nb], hr[nb:], self.rank, self.world,
                           self.group)
            with torch.cuda.stream(self.exchange_stream):
                self._recv.copy_(hr, non_blocking=True)
        else:
            s, r = self._send, self._recv
            with torch.cuda.stream(self.exchange_stream):
                exchange_faces(s[:nb], s[nb:], r[:nb], r[nb:], self.rank, self.world,
                               self.group)

    def step(self, n=1):
        """n time steps; the last writes rho and v."""
        for k in range(n):
            self.lbm.lbm_multi_step_begin(self.m, k == n - 1)
            self._transfer()
            self.lbm.lbm_multi_step_end(self.m)

    def macro(self, dtype=np.float64):
        rho = np.zeros(self.shape, dtype=dtype)
        u = np.zeros((self.D,) + self.shape, dtype=dtype)
        self.lbm.lbm_multi_get_macro(self.m, rho, u)
        return rho, u

    def halo_bytes(self):
        return self.lbm.lbm_multi_halo_bytes(self.m)
