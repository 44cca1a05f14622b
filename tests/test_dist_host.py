"""The sharded lattice's host logic on CPU ranks (gloo, no GPU).

* slab_partition and extended_links slice a lattice into t-slabs of whole
  domains with one domain block of halo;
* the torch.distributed hooks (TorchComm) sum over the ranks and shift
  along the rank ring, called through their C function pointers;
* the exchange maps every slot to its true neighbour: for every face slot
  of the regions qdd_slab_regions names, the sending rank computes which
  site pushed into it under its local periodic wrap (global coordinates),
  ships that through the shift hook, and the receiving rank checks it is
  the true neighbour, in the global lattice, of the site the slot feeds;
  likewise for the two boundary planes of the operator.
"""
import os
import socket

import numpy as np
import pytest

from paper_1502_04025_gb300 import inputs

L, DOM = (8, 4, 4, 16), (4, 2, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_slab_partition_and_halo():
    from paper_1502_04025_gb300 import dist

    assert dist.slab_partition(16, 2, 2) == [(0, 8), (8, 8)]
    assert dist.slab_partition(96, 4, 4) == [(0, 24), (24, 24), (48, 24), (72, 24)]
    for bad in ((96, 4, 8), (16, 2, 3), (8, 4, 2)):  # odd block counts, unequal or too thin slabs
        with pytest.raises(ValueError):
            dist.slab_partition(*bad)
    U = inputs.gauge_field(L, 0.5, 1001)
    Ls = L[0] * L[1] * L[2]
    for t0, lt in dist.slab_partition(L[3], DOM[3], 2):
        e = dist.extended_links(U, L, DOM, t0, lt)
        assert e.shape == ((lt + 2 * DOM[3]) * Ls, 4, 3, 3)
        for k in range(lt + 2 * DOM[3]):
            t = (t0 - DOM[3] + k) % L[3]
            assert np.array_equal(e[k * Ls:(k + 1) * Ls], U[t * Ls:(t + 1) * Ls])
        x = inputs.gaussian_source(L, 7, nrhs=2)
        xl = dist.local_field(x, L, t0, lt)
        assert np.array_equal(xl, x[:, t0 * Ls:(t0 + lt) * Ls])


def _coords(Lc, n):
    return np.stack([n % Lc[0], (n // Lc[0]) % Lc[1], (n // (Lc[0] * Lc[1])) % Lc[2],
                     n // (Lc[0] * Lc[1] * Lc[2])], -1)


def _region_sites(q, Lloc, region):
    """Local host-site index of the site each slot of a region feeds, slot by
    slot in storage order (domain, then the slot index within the direction)."""
    d0, ndom, direction = region
    site_of, _, _ = q.qdd_layout(Lloc, DOM)
    foff, fcoord = q.qdd_layout_faces(Lloc, DOM)
    Vd = int(np.prod(DOM))
    mu = direction // 2
    count = Vd // DOM[mu]
    out = np.empty((ndom, count), dtype=np.int64)
    for k in range(ndom):
        d = d0 + k
        sites = site_of[d * Vd:(d + 1) * Vd]
        dt = _coords(Lloc, sites)[:, 3] % DOM[3]
        face = dt == (0 if direction == 7 else DOM[3] - 1)  # fed from below / from above
        for s in np.nonzero(face)[0]:
            out[k, (fcoord[s] >> (8 * mu)) & 255] = sites[s]
    return out.ravel()


def _rank_main(rank, size, port, errors):
    import torch.distributed as tdist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=size)
    try:
        import ctypes

        from paper_1502_04025_gb300 import dist, qdd

        comm = dist.TorchComm()
        assert (comm.rank, comm.size) == (rank, size)
        # allreduce through the C function pointer
        buf = np.arange(5, dtype=np.float64) + 10 * rank
        assert comm.struct.allreduce_sum(None, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 5) == 0
        assert np.array_equal(buf, np.arange(5) * size + 10 * sum(range(size)))
        # shift: up goes to rank+1, down to rank-1
        up = np.full(16, rank, dtype=np.uint8)
        dn = np.full(16, 100 + rank, dtype=np.uint8)
        got_dn, got_up = np.zeros(16, np.uint8), np.zeros(16, np.uint8)
        assert comm.struct.shift(None, up.ctypes.data, got_dn.ctypes.data, dn.ctypes.data, got_up.ctypes.data, 16) == 0
        assert (got_dn == (rank - 1) % size).all() and (got_up == 100 + (rank + 1) % size).all()

        # face-slot regions and operator planes: global coordinates through the shift
        t0, lt = dist.slab_partition(L[3], DOM[3], size)[rank]
        Lloc = dist.local_lattice(L, lt)
        Ls = L[0] * L[1] * L[2]
        for colour in (0, 1):
            reg_up, reg_dn = qdd.qdd_slab_regions(Lloc, DOM, colour)
            # receiving domains have the other colour; the regions lie in the first / last t-block
            sites_up, sites_dn = _region_sites(qdd, Lloc, reg_up), _region_sites(qdd, Lloc, reg_dn)
            c_up, c_dn = _coords(Lloc, sites_up), _coords(Lloc, sites_dn)
            assert (c_up[:, 3] == 0).all() and (c_dn[:, 3] == lt - 1).all()
            for c in (c_up, c_dn):
                # exactly the domains of the receiving colour (global block coordinates) in that t-block
                blocks = c // np.array(DOM)
                blocks[:, 3] += t0 // DOM[3]
                assert (blocks.sum(1) % 2 == 1 - colour).all()
                assert len({tuple(b[:3]) for b in blocks}) == np.prod(np.array(Lloc[:3]) // DOM[:3]) // 2
                assert len(set(map(tuple, c))) == len(c)  # every fed site once
            # who pushed under the local wrap: the far plane of this slab, in global coordinates
            push_up = c_up.copy()
            push_up[:, 3] = (t0 + lt - 1) % L[3]
            push_dn = c_dn.copy()
            push_dn[:, 3] = t0
            # who should have: the true neighbours of the fed sites
            true_up = c_up.copy()
            true_up[:, 3] = (t0 - 1) % L[3]
            true_dn = c_dn.copy()
            true_dn[:, 3] = (t0 + lt) % L[3]
            a_up = np.ascontiguousarray(push_up, dtype=np.int32)
            a_dn = np.ascontiguousarray(push_dn, dtype=np.int32)
            r_dn, r_up = np.zeros_like(a_up), np.zeros_like(a_dn)
            assert a_up.nbytes == a_dn.nbytes
            assert comm.struct.shift(None, a_up.ctypes.data, r_dn.ctypes.data, a_dn.ctypes.data, r_up.ctypes.data,
                                     a_up.nbytes) == 0
            assert np.array_equal(r_dn, true_up), f"colour {colour}: slots fed from below"
            assert np.array_equal(r_up, true_dn), f"colour {colour}: slots fed from above"
        # operator planes: plane lt-1 sends its backward hops up, plane 0 its forward hops down
        j = np.arange(Ls)
        last = np.stack([j % L[0], (j // L[0]) % L[1], j // (L[0] * L[1]), np.full(Ls, (t0 + lt - 1) % L[3])], -1)
        first = last.copy()
        first[:, 3] = t0
        a_up, a_dn = np.ascontiguousarray(last, np.int32), np.ascontiguousarray(first, np.int32)
        r_dn, r_up = np.zeros_like(a_up), np.zeros_like(a_dn)
        assert comm.struct.shift(None, a_up.ctypes.data, r_dn.ctypes.data, a_dn.ctypes.data, r_up.ctypes.data,
                                 a_up.nbytes) == 0
        exp_dn, exp_up = first.copy(), first.copy()
        exp_dn[:, 3] = (t0 - 1) % L[3]
        exp_up[:, 3] = (t0 + lt) % L[3]
        assert np.array_equal(r_dn, exp_dn) and np.array_equal(r_up, exp_up)
    except Exception as e:  # reported to the parent
        import traceback

        errors.put(f"rank {rank}: {e!r}\n{traceback.format_exc()}")
    finally:
        tdist.destroy_process_group()


@pytest.mark.parametrize("size", [1, 2, 4])
def test_exchange_maps_every_slot_to_its_true_neighbour(size):
    import torch.multiprocessing as mp

    from paper_1502_04025_gb300 import build

    build.build()
    ctx = mp.get_context("spawn")
    errors = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, size, port, errors)) for r in range(size)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    msgs = []
    while not errors.empty():
        msgs.append(errors.get())
    assert not msgs, "\n".join(msgs)
    assert all(p.exitcode == 0 for p in procs)
