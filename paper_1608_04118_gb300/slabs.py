"""One cavity split into row slabs across processes (one slab per rank).

Each rank advances its slab with the library's slab handle
(``ltne_create_slab``); after every step the values that stream across the
cuts -- five populations per column and direction, 5 x nx values per
message (see include/ltne.h) -- move between neighbouring ranks through
torch.distributed point-to-point operations: directly between device
buffers with NCCL, or staged through host memory with gloo.  The
observables are the FP64 accumulators of every slab, combined in rank order
on every rank.  Kernels of different ranks never wait on one another: the
exchange happens on the host side between steps.
"""
from __future__ import annotations

import numpy as np

from . import ltne as L


class HaloExchange:
    """Swap of the halo messages of one rank with its neighbours.

    ``send_lo`` / ``recv_lo`` face rank - 1, ``send_hi`` / ``recv_hi`` rank
    + 1 (None where there is no neighbour).  With ``host_staged`` the
    tensors may live on a device and are moved through host copies (gloo);
    otherwise the communicator moves them where they are (NCCL)."""

    def __init__(self, rank, world, send_lo, send_hi, recv_lo, recv_hi, host_staged, group=None):
        self.rank, self.world, self.group = rank, world, group
        self.dev = (send_lo, send_hi, recv_lo, recv_hi)
        self.host_staged = host_staged
        if host_staged:
            self.host = tuple(None if t is None else t.new_empty(t.shape, device="cpu")
                              for t in self.dev)
        else:
            self.host = self.dev

    def peers(self):
        """(peer rank, send index, receive index) for each neighbour."""
        out = []
        if self.rank > 0:
            out.append((self.rank - 1, 0, 2))
        if self.rank < self.world - 1:
            out.append((self.rank + 1, 1, 3))
        return out

    def exchange(self, stream=None):
        """Send both messages and receive both halos.  ``stream``: the CUDA
        stream the device buffers are produced and consumed on."""
        import torch
        import torch.distributed as dist

        peers = self.peers()
        if not peers:
            return
        if not self.host_staged:
            ops = []
            for peer, si, ri in peers:
                ops.append(dist.P2POp(dist.isend, self.dev[si], peer, group=self.group))
                ops.append(dist.P2POp(dist.irecv, self.dev[ri], peer, group=self.group))
            with torch.cuda.stream(stream):  # ordered after the pack, before the unpack
                for r in dist.batch_isend_irecv(ops):
                    r.wait()
            return
        if stream is not None:
            stream.synchronize()  # the pack kernels have written the messages
        for _, si, _ in peers:
            self.host[si].copy_(self.dev[si])
        reqs = []
        for peer, si, ri in peers:
            reqs.append(dist.isend(self.host[si], peer, group=self.group))
            reqs.append(dist.irecv(self.host[ri], peer, group=self.group))
        for r in reqs:
            r.wait()
        for _, _, ri in peers:
            if stream is not None:
                with torch.cuda.stream(stream):  # before the unpack on the same stream
                    self.dev[ri].copy_(self.host[ri])
            else:
                self.dev[ri].copy_(self.host[ri])


def combine_accumulators(parts):
    """The slabs' accumulator vectors combined in slab order (the same bits
    on every rank)."""
    acc = np.array(parts[0], dtype=np.float64)
    for p in parts[1:]:
        acc = L.ltne_accumulators_combine(acc, p)
    return acc


def all_accumulators(acc, group=None):
    """Every rank's accumulator vector, in rank order (gathered on CPU)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor(np.asarray(acc, dtype=np.float64))
    world = dist.get_world_size(group)
    out = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(out, t, group=group)
    return [o.numpy() for o in out]


class DistributedCavity:
    """The whole cavity, one row slab per rank of the default process group.

    ``DistributedCavity(nx, ny, **params)`` takes the whole cavity's size and
    any ltne_params field; every rank constructs it with the same arguments
    on its own CUDA device.  With an Ergun permeability and a porosity field
    pass ``d_p`` (``ltne_ergun_diameter`` of the whole field)."""

    def __init__(self, nx, ny, stream=None, device=None, group=None, **params):
        import torch
        import torch.distributed as dist

        self.group = group
        self.rank, self.world = dist.get_rank(group), dist.get_world_size(group)
        self.slab = L.SlabCavity(nx, ny, self.world, self.rank, stream=stream, device=device,
                                 **params)
        ws = self.slab.workspace
        base = ws.data_ptr()
        *ptrs, nbytes = self.slab.buffers
        dt = torch.float64 if int(self.slab.params.storage) == L.LTNE_F64 else torch.float32
        views = []
        for ptr in ptrs:
            if ptr is None:
                views.append(None)
            else:
                off = int(ptr) - base
                views.append(ws[off:off + nbytes].view(dt))
        backend = dist.get_backend(group)
        self.halo = HaloExchange(self.rank, self.world, *views, host_staged=backend != "nccl",
                                 group=group)
        self.steps = 0
        self.have_prev = False

    @property
    def params(self):
        return self.slab.params

    def set_fields(self, porosity=None, rho=None, ux=None, uy=None, T_f=None, T_s=None):
        """Initial fields of the WHOLE cavity (the same arrays on every rank;
        any may be None).  The halo rows start from the same values as the
        neighbours' own rows, so no exchange is needed before the first step."""
        self.slab.set_fields(porosity, rho, ux, uy, T_f, T_s)
        self.steps = 0
        self.have_prev = False
        return self

    def step(self, n):
        """n time steps, each followed by the halo exchange; the last one
        stores the macroscopic fields."""
        for k in range(int(n)):
            self.slab.step(1 if k == n - 1 else 0)
            self.halo.exchange(self.slab.stream)
            self.slab.unpack()
            self.steps += 1
        return self

    def observables(self, allow_nonfinite=False):
        """Observables of the whole cavity (every rank gets the same)."""
        parts = all_accumulators(self.slab.accumulators(), self.group)
        acc = combine_accumulators(parts)
        ob = L.ltne_observables_from_accumulators(self.params, self.steps, self.have_prev, acc,
                                                  allow_nonfinite)
        self.have_prev = True
        return ob

    def gather_fields(self):
        """The whole cavity's fields (ny x nx) on every rank."""
        import torch
        import torch.distributed as dist

        f = self.slab.fields()
        out = {}
        for k, v in f.items():
            t = torch.from_numpy(np.ascontiguousarray(v))
            rows = [torch.empty((L.ltne_slab_rows(self.slab.ny_global, self.world, r)[1],
                                 self.slab.nx), dtype=torch.float64)
                    for r in range(self.world)]
            # all_gather needs equal shapes: pad to the largest slab
            mx = max(r.shape[0] for r in rows)
            pad = torch.zeros((mx, self.slab.nx), dtype=torch.float64)
            pad[:t.shape[0]] = t
            bufs = [torch.empty_like(pad) for _ in range(self.world)]
            dist.all_gather(bufs, pad, group=self.group)
            out[k] = torch.cat([b[:r.shape[0]] for b, r in zip(bufs, rows)]).numpy()
        return out

    def close(self):
        self.slab.close()
