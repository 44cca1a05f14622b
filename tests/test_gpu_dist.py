"""The lattice sharded in t over ranks, on one GPU: each rank is a process
with its own CUDA context on cuda:0 and its own slab gauge field, and the
ranks exchange through torch.distributed (gloo) on the host, between
launches: no kernel of one rank waits for another's.

Against the same computation on the whole lattice (one gauge field, one
process), assembled slab by slab:
  * clover blocks: bit for bit (built on the extended lattice from the same
    links);
  * the Schwarz method (FP32 and FP64, one and two right-hand sides, the
    maintained residual too): bit for bit, since every face slot has one
    writer and is summed in a fixed order on either side of a slab boundary;
  * the operator: to rounding (the boundary planes swap the wrapped hops for
    the neighbours');
  * the solve: the same iteration count and the solution to 1e-9, with a
    true FP64 residual below 1e-10 through the oracle (the dot products are
    summed over the ranks in another order).
A shift hook that fails is reported as QDD_ECOMM.
"""
import os
import socket

import numpy as np
import pytest

from paper_1502_04025_gb300 import inputs

pytestmark = pytest.mark.gpu

L, DOM, KAPPA = (8, 8, 8, 16), (4, 4, 4, 4), 0.12


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _compute(q, g, x, x2, V):
    out = {}
    out["clover"] = q.qdd_get_clover(g, V, 0)
    out["sclover"] = q.qdd_get_clover(g, V, 1)
    for p in ("f64", "df64", "f32"):
        out["D_" + p] = q.qdd_apply_D(g, x, p)
    out["psi32"], out["rho32"] = q.qdd_sap_apply(g, x, 4, 8, "f32", want_rho=True)
    out["psi64"] = q.qdd_sap_apply(g, x, 4, 5, "f64")
    out["psi2"] = q.qdd_sap_apply(g, x2, 4, 8, "f32", nrhs=2)
    xs, rep = q.qdd_solve(g, x, tol=1e-10, sap_prec="f32", arnoldi_prec="df64", relax_eta=1e-6, reorth=0)
    out["x"], out["iters"], out["res"] = xs, np.array(rep["iters"]), np.array(rep["true_rel_res"])
    xs2, rep2 = q.qdd_solve(g, x2, tol=1e-10, sap_prec="f16", nrhs=2)
    out["x2"], out["iters2"] = xs2, np.array(rep2["iters"])
    return out


def _rank_main(rank, size, port, tmpdir, errors):
    import torch
    import torch.distributed as tdist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=size)
    try:
        torch.cuda.set_device(0)
        from paper_1502_04025_gb300 import dist, qdd

        U = inputs.gauge_field(L, 0.5, 1001)
        t0, lt = dist.slab_partition(L[3], DOM[3], size)[rank]
        comm = dist.TorchComm()
        ctx = qdd.qdd_create(0, 0)
        g = qdd.qdd_create_gauge_field_slab(ctx, dist.local_lattice(L, lt), DOM,
                                            dist.extended_links(U, L, DOM, t0, lt), comm)
        qdd.qdd_set_clover(g, 1.0, KAPPA)
        x = dist.local_field(inputs.gaussian_source(L, 3004), L, t0, lt)
        x2 = dist.local_field(inputs.gaussian_source(L, 3005, nrhs=2), L, t0, lt)
        out = _compute(qdd, g, x, x2, L[0] * L[1] * L[2] * lt)
        np.savez(os.path.join(tmpdir, f"rank{rank}.npz"), **out)
        qdd.qdd_destroy_gauge(g)
        qdd.qdd_destroy(ctx)
    except Exception as e:
        import traceback

        errors.put(f"rank {rank}: {e!r}\n{traceback.format_exc()}")
    finally:
        tdist.destroy_process_group()


def _run_ranks(size, tmpdir):
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    errors = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, size, port, str(tmpdir), errors)) for r in range(size)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=600)
    msgs = []
    while not errors.empty():
        msgs.append(errors.get())
    assert not msgs, "\n".join(msgs)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    return [dict(np.load(os.path.join(tmpdir, f"rank{r}.npz"))) for r in range(size)]


@pytest.fixture(scope="module")
def whole(ora):
    from paper_1502_04025_gb300 import build

    build.build()
    from paper_1502_04025_gb300 import qdd

    U = inputs.gauge_field(L, 0.5, 1001)
    ctx = qdd.qdd_create(0, 0)
    g = qdd.qdd_create_gauge_field(ctx, L, DOM, U)
    qdd.qdd_set_clover(g, 1.0, KAPPA)
    x = inputs.gaussian_source(L, 3004)
    x2 = np.ascontiguousarray(inputs.gaussian_source(L, 3005, nrhs=2))
    out = _compute(qdd, g, x, x2, inputs.volume(L))
    qdd.qdd_destroy_gauge(g)
    qdd.qdd_destroy(ctx)
    return out, U, x, x2


def _assemble(parts, key):
    a = [p[key] for p in parts]
    if key in ("psi2", "x2"):  # (nrhs, V_local, 4, 3): sites on axis 1
        return np.concatenate(a, axis=1)
    return np.concatenate(a, axis=0)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("size", [1, 2])
def test_sharded_equals_whole_lattice(whole, ora, size, tmp_path):
    ref, U, x, x2 = whole
    parts = _run_ranks(size, tmp_path)
    for key in ("clover", "sclover", "psi32", "rho32", "psi64", "psi2"):
        assert np.array_equal(_assemble(parts, key), ref[key]), key
    for p, tol in (("f64", 1e-14), ("df64", 1e-13), ("f32", 1e-6)):
        got = _assemble(parts, "D_" + p)
        err = np.abs(got - ref["D_" + p]).reshape(-1, 12).max(1) / np.abs(ref["D_" + p]).reshape(-1, 12).max(1)
        print(f"DIST {size} ranks D {p}: max site error against the whole lattice {err.max():.2e}")
        assert err.max() <= tol, p
    xg = _assemble(parts, "x")
    A = ora.clover(L, U, 1.0, KAPPA)
    res = np.linalg.norm(x - ora.apply_D(L, U, A, KAPPA, xg)) / np.linalg.norm(x)
    iters = [int(p["iters"]) for p in parts]
    print(f"DIST {size} ranks solve: iterations {iters} (whole lattice {int(ref['iters'])}), "
          f"|x - x_whole|/|x_whole| {_rel(xg, ref['x']):.2e}, true residual {res:.2e}")
    assert len(set(iters)) == 1 and abs(iters[0] - int(ref["iters"])) <= 1
    assert _rel(xg, ref["x"]) <= 1e-9 and res <= 1e-10
    x2g = _assemble(parts, "x2")
    assert _rel(x2g, ref["x2"]) <= 1e-9
    for r in range(2):
        res2 = np.linalg.norm(x2[r] - ora.apply_D(L, U, A, KAPPA, x2g[r])) / np.linalg.norm(x2[r])
        assert res2 <= 1e-10


def test_failing_hook_is_reported():
    """A shift hook that fails (on the host) aborts the collective call with
    QDD_ECOMM; nothing on the GPU waits for it."""
    from paper_1502_04025_gb300 import build

    build.build()
    from paper_1502_04025_gb300 import dist, qdd

    class Broken(dist.TorchComm):
        def _shift(self, *a):
            return 1

    U = inputs.gauge_field(L, 0.5, 1001)
    ctx = qdd.qdd_create(0, 0)
    comm = Broken()
    assert comm.size == 1
    g = qdd.qdd_create_gauge_field_slab(ctx, L, DOM, dist.extended_links(U, L, DOM, 0, L[3]), comm)
    try:
        qdd.qdd_set_clover(g, 1.0, KAPPA)
        with pytest.raises(qdd.QddError) as e:
            qdd.qdd_sap_apply(g, inputs.gaussian_source(L, 3004), 4, 4, "f32")
        assert e.value.status == qdd.QDD_ECOMM
        with pytest.raises(qdd.QddError) as e:
            qdd.qdd_apply_D(g, inputs.gaussian_source(L, 3004), "f64")
        assert e.value.status == qdd.QDD_ECOMM
    finally:
        qdd.qdd_destroy_gauge(g)
        qdd.qdd_destroy(ctx)
