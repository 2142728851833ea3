"""One signal solved by several processes (include/csc_shard.h).

``solve`` runs DICOD's protocol (Sec. 2.2, Alg. 2) over ranks that each own
a contiguous run of segments: per phase every rank runs its segments, then
hands the changes it made to its halo to the neighbours; a sweep in which no
rank applied an update ends a CD round; the round ends with the neighbours'
border Z exchanged, an exact resync on every rank and the largest remaining
|Delta Z| reduced over ranks.  The objective is the sum of the ranks' parts.

The protocol only talks to two objects:

* a backend with the csc_shard_* calls of one rank (``CapiShard`` wraps the
  C ABI; the tests also drive a numpy backend through the same steps), and
* a communicator with ``exchange`` (blocks to/from the two neighbours),
  ``sum`` and ``max`` over ranks (``TorchComm`` uses torch.distributed:
  gloo with host buffers, or NCCL with device buffers).

Every step of the solve itself runs in the backend: this module only orders
the calls and moves the [K][L-1] halo blocks.
"""
from __future__ import annotations

import numpy as np

DRIFT_SWEEPS = 32  # a CD round still running after this many sweeps is resynced


class TorchComm:
    """Neighbour exchange and reductions over a torch.distributed process group."""

    def __init__(self, dist, device="cpu", group=None):
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.device = device

    def exchange(self, to_left, to_right, from_left, from_right):
        """Send to_left to rank-1 and to_right to rank+1; receive from_left from
        rank-1 and from_right from rank+1 (None where there is no neighbour)."""
        d = self.dist
        reqs = []
        if self.rank > 0:
            reqs.append(d.isend(to_left, self.rank - 1, group=self.group))
            reqs.append(d.irecv(from_left, self.rank - 1, group=self.group))
        if self.rank < self.world - 1:
            reqs.append(d.isend(to_right, self.rank + 1, group=self.group))
            reqs.append(d.irecv(from_right, self.rank + 1, group=self.group))
        for r in reqs:
            r.wait()

    def _reduce(self, v, op):
        import torch
        t = torch.tensor([float(v)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=op, group=self.group)
        return float(t.item())

    def sum(self, v):
        return self._reduce(v, self.dist.ReduceOp.SUM)

    def max(self, v):
        return self._reduce(v, self.dist.ReduceOp.MAX)


class CapiShard:
    """The csc_shard_* calls of one rank on a library handle."""

    def __init__(self, capi, h, plan):
        self.capi, self.h, self.plan = capi, h, plan

    def phase(self, p, tol):
        self.capi.csc_shard_phase(self.h, p, tol)

    def halo_out(self, to_left, to_right):
        self.capi.csc_shard_halo_out(self.h, to_left, to_right)

    def halo_in(self, from_left, from_right):
        self.capi.csc_shard_halo_in(self.h, from_left, from_right)

    def z_out(self, to_left, to_right):
        self.capi.csc_shard_z_out(self.h, to_left, to_right)

    def z_in(self, from_left, from_right):
        self.capi.csc_shard_z_in(self.h, from_left, from_right)

    def updates(self):
        return self.capi.csc_shard_updates(self.h)

    def resync(self, tol):
        return self.capi.csc_shard_resync(self.h, tol)

    def objective(self):
        return self.capi.csc_shard_objective(self.h)

    def get_z(self, out):
        self.capi.csc_shard_get_z(self.h, out)
        return out


def halo_buffers(K, plan, make):
    """(to_left, to_right, from_left, from_right) of shapes [K][halo]; None for
    a side without a neighbour.  make(shape) allocates one float32 buffer."""
    hl, hr = int(plan["halo_left"]), int(plan["halo_right"])
    left = (make((K, hl)), make((K, hl))) if hl > 0 else (None, None)
    right = (make((K, hr)), make((K, hr))) if hr > 0 else (None, None)
    return left[0], right[0], left[1], right[1]


def solve(backend, comm, K, plan, tol, max_resyncs=3, max_sweeps=1_000_000, make=None):
    """Run the sharded solve to tol (rules of csc_solve: CD to tol/2, exact
    resyncs, the last one allowed decides).  Returns a dict with the global
    objective E, convergence, the global update count, sweeps and resyncs;
    this rank's Z is then read with backend.get_z.  make(shape) allocates
    exchange buffers (numpy float32 by default; device tensors for NCCL)."""
    if make is None:
        make = lambda shape: np.zeros(shape, np.float32)  # noqa: E731
    c = int(plan["phases"])
    tl, tr, fl, fr = halo_buffers(K, plan, make)
    ztl, ztr, zfl, zfr = halo_buffers(K, plan, make)

    def border_z():
        backend.z_out(ztl, ztr)
        comm.exchange(ztl, ztr, zfl, zfr)
        backend.z_in(zfl, zfr)

    # CD runs to tol/2 and the exact check accepts at tol (as csc_solve)
    tol_inner = 0.5 * tol if max_resyncs > 0 else tol
    resyncs, drift_resyncs, sweeps = 0, 0, 0
    converged = False
    last = 0
    while True:
        round_sweeps = 0
        settled = False
        while True:
            for p in range(c):
                backend.phase(p, tol_inner)
                backend.halo_out(tl, tr)
                comm.exchange(tl, tr, fl, fr)
                backend.halo_in(fl, fr)
            sweeps += 1
            round_sweeps += 1
            total = backend.updates()
            applied = comm.sum(total - last)
            last = total
            if applied == 0:
                settled = True
                break
            if sweeps >= max_sweeps or (max_resyncs > 0 and round_sweeps >= DRIFT_SWEEPS):
                break
        if not settled and sweeps >= max_sweeps:
            break
        border_z()
        if max_resyncs == 0:
            converged = settled
            break
        dz = comm.max(backend.resync(tol))
        if settled:
            resyncs += 1
        else:
            drift_resyncs += 1
        if dz < tol:
            converged = True
            break
        if settled and resyncs > max_resyncs:
            break
    border_z()  # the objective needs the neighbours' Z within L-1 of the borders
    E = comm.sum(backend.objective())
    return {"E": E, "converged": converged, "updates": int(comm.sum(backend.updates())),
            "sweeps": sweeps, "resyncs": resyncs, "drift_resyncs": drift_resyncs}


def plan_dict(p) -> dict:
    """A csc_shard_plan (ctypes) as a dict."""
    return {name: getattr(p, name) for name, _ in p._fields_}
