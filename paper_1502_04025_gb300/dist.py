"""The lattice sharded over ranks in the time direction (arXiv:1502.04025,
Sec. 3.6: the lattice is distributed over processors; here in slabs of whole
Schwarz domains), with torch.distributed as the communication library.

This module only partitions fields and moves bytes: the hooks of
qdd_create_gauge_field_slab (a sum over ranks and a cyclic shift along the
rank ring) are implemented with torch.distributed (gloo on CPU tensors, NCCL
through CUDA tensors), and whole fields are sliced into and assembled from
the ranks' slabs.  Every step of the computation runs in libqdd.
"""
from __future__ import annotations

import ctypes
import sys
import traceback

import numpy as np

from paper_1502_04025_gb300 import qdd


def slab_partition(Lt: int, dom_t: int, size: int):
    """[(t0, lt)] of each rank: equal slabs of whole domains, each an even
    number of domain blocks (so the local colouring of the domains is the
    global one).  Raises ValueError when Lt cannot be split that way."""
    if size < 1 or Lt % size:
        raise ValueError(f"Lt = {Lt} does not split into {size} equal slabs")
    lt = Lt // size
    if lt % dom_t or (lt // dom_t) % 2 or lt // dom_t < 2:
        raise ValueError(f"a slab of {lt} planes is not an even number (>= 2) of {dom_t}-plane domain blocks")
    return [(r * lt, lt) for r in range(size)]


def _planes(field: np.ndarray, L, t_lo: int, t_hi: int) -> np.ndarray:
    """Planes t_lo .. t_hi-1 (periodic in t) of a field in the host layout
    (sites first, t slowest)."""
    Ls = int(L[0]) * int(L[1]) * int(L[2])
    Lt = int(L[3])
    f = field.reshape((Lt, Ls) + field.shape[1:])
    idx = np.arange(t_lo, t_hi) % Lt
    return np.ascontiguousarray(f[idx].reshape((-1,) + field.shape[1:]))


def extended_links(U: np.ndarray, L, dom, t0: int, lt: int) -> np.ndarray:
    """Links of the extended local lattice: planes t0 - dom_t .. t0 + lt + dom_t - 1."""
    return _planes(U, L, t0 - dom[3], t0 + lt + dom[3])


def local_field(x: np.ndarray, L, t0: int, lt: int) -> np.ndarray:
    """This rank's planes t0 .. t0+lt-1 of a spinor field (V, 4, 3) or (nrhs, V, 4, 3)."""
    if x.ndim == 4:
        return np.ascontiguousarray(np.stack([_planes(xi, L, t0, t0 + lt) for xi in x]))
    return _planes(x, L, t0, t0 + lt)


def local_lattice(L, lt: int):
    return (int(L[0]), int(L[1]), int(L[2]), int(lt))


class TorchComm:
    """The communication hooks of a sharded gauge field over torch.distributed.

    allreduce_sum sums host doubles over the ranks; shift sends to_up to
    rank+1 and to_dn to rank-1 (periodic) and receives the neighbours' into
    from_dn and from_up.  With the NCCL backend the bytes go through CUDA
    tensors on `device`.  A hook that raises returns 1, which the library
    turns into QDD_ECOMM."""

    def __init__(self, group=None, device=None):
        import torch
        import torch.distributed as dist

        self._torch, self._dist, self.group = torch, dist, group
        self.rank = dist.get_rank(group) if dist.is_initialized() else 0
        self.size = dist.get_world_size(group) if dist.is_initialized() else 1
        self.cuda = dist.is_initialized() and dist.get_backend(group) == "nccl"
        self.device = device
        self._ar = qdd.ALLREDUCE_FN(self._allreduce)
        self._sh = qdd.SHIFT_FN(self._shift)
        self.struct = qdd.qdd_comm(None, self.rank, self.size, self._ar, self._sh)

    def _host(self, ptr, nbytes):
        buf = (ctypes.c_uint8 * nbytes).from_address(ptr)
        return self._torch.from_numpy(np.frombuffer(buf, dtype=np.uint8))

    def _allreduce(self, user, buf, n):
        try:
            if self.size > 1:
                t = self._torch.from_numpy(np.ctypeslib.as_array(buf, shape=(n,)))
                if self.cuda:
                    tc = t.to(self.device)
                    self._dist.all_reduce(tc, group=self.group)
                    t.copy_(tc.cpu())
                else:
                    self._dist.all_reduce(t, group=self.group)
            return 0
        except Exception:
            traceback.print_exc(file=sys.stderr)
            return 1

    def _shift(self, user, to_up, from_dn, to_dn, from_up, nbytes):
        try:
            up, dn = self._host(to_up, nbytes), self._host(to_dn, nbytes)
            got_dn, got_up = self._host(from_dn, nbytes), self._host(from_up, nbytes)
            if self.size == 1:
                got_dn.copy_(up)
                got_up.copy_(dn)
                return 0
            dist = self._dist
            nxt, prv = (self.rank + 1) % self.size, (self.rank - 1) % self.size
            if self.group is not None:
                nxt = dist.get_global_rank(self.group, nxt)
                prv = dist.get_global_rank(self.group, prv)
            if self.cuda:
                b = [x.to(self.device) for x in (up, dn, got_dn, got_up)]
                ops = [dist.P2POp(dist.isend, b[0], nxt, self.group), dist.P2POp(dist.irecv, b[2], prv, self.group),
                       dist.P2POp(dist.isend, b[1], prv, self.group), dist.P2POp(dist.irecv, b[3], nxt, self.group)]
                for r in dist.batch_isend_irecv(ops):
                    r.wait()
                got_dn.copy_(b[2].cpu())
                got_up.copy_(b[3].cpu())
            else:
                reqs = [dist.isend(up, nxt, group=self.group, tag=1), dist.irecv(got_dn, prv, group=self.group, tag=1),
                        dist.isend(dn, prv, group=self.group, tag=2), dist.irecv(got_up, nxt, group=self.group, tag=2)]
                for r in reqs:
                    r.wait()
            return 0
        except Exception:
            traceback.print_exc(file=sys.stderr)
            return 1
