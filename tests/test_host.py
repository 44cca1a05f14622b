"""Host-side checks that need no GPU: the C-ABI library loads and exports
every entry point its header declares, and the pure host functions match
the numbers the paper prints."""
import ctypes
import json
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qdd.h")


@pytest.fixture(scope="session")
def qdd():
    from paper_1502_04025_gb300 import build

    build.build()
    from paper_1502_04025_gb300 import qdd as q

    return q


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(qdd_[A-Za-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["qdd_create", "qdd_create_gauge_field", "qdd_set_clover", "qdd_apply_D", "qdd_sap_apply",
                 "qdd_solve", "qdd_submit", "qdd_poll", "qdd_destroy", "qdd_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol(qdd):
    lib = ctypes.CDLL(qdd.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


C_CLIENT = r"""
#include <stdio.h>
#include <stdlib.h>
#include "qdd.h"
int main(void)
{
    qdd_mg_params p;
    qdd_mg_default_params(&p);
    const int L[4] = {8, 8, 8, 8}, dom[4] = {4, 4, 4, 4};
    int *site_of = malloc(4096 * sizeof(int));
    uint16_t *nbl = malloc(256 * 8 * sizeof(uint16_t));
    int *nbd = malloc(16 * 8 * sizeof(int));
    qdd_status st = qdd_layout(L, dom, site_of, nbl, nbd);
    const int bad[4] = {3, 8, 8, 8};
    qdd_status st2 = qdd_layout(bad, dom, site_of, nbl, nbd);
    unsigned long long hits = 1;
    qdd_status st3 = qdd_check_hits(&hits);
    printf("%d %d %.6f %d %d %d %llu\n", p.nv, p.bootstrap, qdd_load_model(8.0, 60.0), st, st2 == QDD_EINVAL,
           st3 == QDD_EINVAL, hits);
    free(site_of); free(nbl); free(nbd);
    return 0;
}
"""


def test_plain_c_client_links_and_calls_host_entry_points(qdd, tmp_path):
    """The header is plain C (C99, -pedantic) and a C program links against
    libqdd.so and calls its host-only entry points (no GPU needed)."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    libdir = os.path.dirname(qdd.LIB_PATH)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-o", str(exe), "-L", libdir, "-l:" + os.path.basename(qdd.LIB_PATH),
                        "-Wl,-rpath," + libdir], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    nv, boot, load, st, bad, nocheck, hits = out.stdout.split()
    assert (nv, boot, st, bad, nocheck, hits) == ("8", "0", "0", "1", "1", "0")
    assert abs(float(load) - qdd.qdd_load_model(8.0, 60.0)) < 1e-6


def test_binding_covers_every_symbol(qdd):
    for n in declared_functions():
        assert hasattr(qdd, n), n


GOLDEN = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_values.json")))


def test_load_model_pins(qdd):
    """Sec. 3.5: 64^3x128 on 1024 KNCs with 8x4^3 domains gives N_d = 64
    domains per KNC and 60 usable cores, load x/ceil(x) = 53%; the
    non-uniform split 128 = 4*28+16 gives (4*56+32)/(5*60) = 85%
    (tests/golden/paper_values.json)."""
    u, nu = GOLDEN["load_model"]["uniform"], GOLDEN["load_model"]["non_uniform"]
    assert qdd.qdd_load_model(u["domains_per_colour"], u["slots"]) == pytest.approx(32 / 60)
    assert round(100 * qdd.qdd_load_model(u["domains_per_colour"], u["slots"])) == u["load_percent"]
    # t-slices of 28 and 16 sites hold 56 and 32 domains per colour pair
    loads = [qdd.qdd_load_model(n, nu["slots"]) for n in nu["busy_per_knc"]]
    assert round(100 * sum(nu["busy_per_knc"]) / (len(nu["busy_per_knc"]) * nu["slots"])) == nu["load_percent"]
    assert all(0 < l <= 1 for l in loads)
    assert qdd.qdd_load_model(120, 60) == 1.0
    assert qdd.qdd_load_model(0, 60) == 0.0


def test_working_set_pins(qdd):
    """Sec. 3.3: an 8x4^3 domain needs 456 kB in single precision and 312 kB
    with half-precision links and clover (two full spinors plus three
    even-site spinors of the MR iteration; tests/golden/paper_values.json)."""
    w = GOLDEN["working_set"]
    dom = tuple(w["domain"])
    assert qdd.qdd_domain_working_set(dom, 4, 2, 3) == w["single_precision_kB"] * 1024
    assert qdd.qdd_domain_working_set(dom, 2, 2, 3) == w["half_links_clover_kB"] * 1024


def test_no_gpu_needed_for_errors(qdd):
    # a null context is rejected without touching the device
    assert qdd._lib.qdd_set_profiling(None, 1) == qdd.QDD_EINVAL
    # the normal build has no range checks to report
    with pytest.raises(qdd.QddError):
        qdd.qdd_check_hits()
    # nor a wait limit to lower
    with pytest.raises(qdd.QddError) as e:
        qdd.qdd_check_set_wait_limit(0, 0)
    assert e.value.status == qdd.QDD_EINVAL


def _coords(L, n):
    n = np.asarray(n)
    return np.stack([n % L[0], (n // L[0]) % L[1], (n // (L[0] * L[1])) % L[2], n // (L[0] * L[1] * L[2])], -1)


@pytest.mark.parametrize("L,dom", [((8, 8, 8, 8), (4, 4, 4, 4)), ((4, 4, 4, 4), (2, 2, 2, 2)),
                                   ((8, 4, 4, 12), (4, 2, 2, 2)), ((16, 8, 8, 8), (8, 4, 4, 4)),
                                   ((16, 16, 16, 32), (8, 4, 4, 4)), ((12, 8, 4, 4), (6, 4, 2, 2))])
def test_device_layout_tables(qdd, L, dom):
    """The neighbour tables the kernels use reproduce the periodic lattice
    neighbours, slots are colour-major and parity-split, and the
    internal-to-host map is a permutation."""
    site_of, nbl, nbd = qdd.qdd_layout(L, dom)
    V, Vd = int(np.prod(L)), int(np.prod(dom))
    Nd, Vh = V // Vd, Vd // 2
    assert np.array_equal(np.sort(site_of), np.arange(V))
    c = _coords(L, site_of)
    gi = np.arange(V)
    d, s = gi // Vd, gi % Vd
    # parity split inside every domain, colour-major domain slots
    assert np.array_equal(c.sum(1) % 2, (s >= Vh).astype(int))
    blk = c // np.array(dom)
    assert np.array_equal(blk.sum(1) % 2, (d >= Nd // 2).astype(int))
    # every site of a slot lies in one block
    for dd in (0, Nd // 2, Nd - 1):
        b = blk[d == dd]
        assert (b == b[0]).all()
    for k in range(8):
        mu, back = k // 2, k % 2
        e = nbl[s, k].astype(np.int64)
        cross = (e & 0x8000) != 0
        ns = e & 0x7FFF
        nd = np.where(cross, nbd[d, k], d)
        got = site_of[nd * Vd + ns]
        cc = c.copy()
        cc[:, mu] = (cc[:, mu] + (-1 if back else 1)) % L[mu]
        want = cc[:, 0] + L[0] * (cc[:, 1] + L[1] * (cc[:, 2] + L[2] * cc[:, 3]))
        assert np.array_equal(got, want), (k,)
        # a hop leaves the domain exactly when the block coordinate changes
        assert np.array_equal(cross, (cc[:, mu] // dom[mu]) != blk[:, mu])


def test_layout_rejects_bad_geometry(qdd):
    with pytest.raises(qdd.QddError):
        qdd.qdd_layout((8, 8, 8, 8), (8, 4, 4, 4))   # one block in x
    with pytest.raises(qdd.QddError):
        qdd.qdd_layout((12, 8, 8, 8), (4, 4, 4, 4))  # three blocks in x
    with pytest.raises(qdd.QddError):
        qdd.qdd_layout((8, 8, 8, 8), (3, 4, 4, 4))   # odd extent
    with pytest.raises(qdd.QddError):
        qdd.qdd_layout((32, 16, 16, 16), (16, 8, 4, 4))  # domain above 512 sites


ADMIT_DRIVER = r"""
#include <cstdio>
#include "admission.h"
using namespace qdd;
struct R { int id, g, nrhs; long bytes; int bypassed; };
static std::shared_ptr<R> req(int id, int g, int nrhs, long bytes) { return std::make_shared<R>(R{id, g, nrhs, bytes, 0}); }
static void show(const char *name, const AdmitResult<R> &res, const std::deque<std::shared_ptr<R>> &q)
{
    std::printf("%s %s", name, res.what == Admit::kBatch ? "batch" : res.what == Admit::kWait ? "wait" : "reject");
    for (auto &r : res.batch) std::printf(" %d", r->id);
    if (res.rejected) std::printf(" rejected=%d status=%d", res.rejected->id, (int)res.status);
    std::printf(" | left");
    for (auto &r : q) std::printf(" %d", r->id);
    std::printf("\n");
}
int main()
{
    long budget = 0;
    int err_id = -1;
    auto nrhs = [](const R &r) { return r.nrhs; };
    auto same = [](const R &a, const R &b) { return a.g == b.g; };
    auto prepare = [&](const R &lead, int total) {
        if (lead.id == err_id) return QDD_ENOMEM;
        return lead.bytes * total <= budget ? QDD_OK : QDD_EBUDGET;
    };
    {   // same gauge merges up to 12 right-hand sides, in queue order
        std::deque<std::shared_ptr<R>> q{req(0, 1, 4, 1), req(1, 2, 4, 1), req(2, 1, 4, 1), req(3, 1, 6, 1)};
        budget = 100;
        auto res = admit(q, true, 12, 8, nrhs, same, prepare);
        show("merge", res, q);
    }
    {   // the merged batch does not fit, its lead alone does
        std::deque<std::shared_ptr<R>> q{req(0, 1, 6, 10), req(1, 1, 6, 10)};
        budget = 60;
        auto res = admit(q, true, 12, 8, nrhs, same, prepare);
        show("shrink", res, q);
    }
    {   // a head that does not fit lets a later request that fits go first
        std::deque<std::shared_ptr<R>> q{req(0, 1, 1, 100), req(1, 2, 1, 10), req(2, 3, 1, 10)};
        budget = 50;
        auto res = admit(q, true, 12, 8, nrhs, same, prepare);
        show("bypass", res, q);
        std::printf("bypassed %d\n", q.front()->bypassed);
        q.front()->bypassed = 8;  // the bound reached: wait for the head
        auto res2 = admit(q, true, 12, 8, nrhs, same, prepare);
        show("bound", res2, q);
    }
    {   // nothing running: a head that does not fit is rejected
        std::deque<std::shared_ptr<R>> q{req(0, 1, 1, 100), req(1, 2, 1, 100)};
        budget = 50;
        auto res = admit(q, false, 12, 8, nrhs, same, prepare);
        show("reject", res, q);
    }
    {   // another preparation error fails the request it belongs to
        std::deque<std::shared_ptr<R>> q{req(0, 1, 1, 100), req(1, 2, 1, 10)};
        budget = 50;
        err_id = 1;
        auto res = admit(q, true, 12, 8, nrhs, same, prepare);
        show("error", res, q);
    }
    return 0;
}
"""


def test_serving_admission_policy(tmp_path):
    """The serving loop's admission rules (csrc/admission.h), compiled on the
    host with a fake memory budget: batching, shrinking to the lead, bounded
    bypass of a head that does not fit, rejection with nothing running, and
    error attribution."""
    import shutil
    import subprocess

    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    src = tmp_path / "admit.cpp"
    src.write_text(ADMIT_DRIVER)
    exe = tmp_path / "admit"
    r = subprocess.run([cxx, "-std=c++17", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                        "-I", os.path.join(ROOT, "paper_1502_04025_gb300", "csrc"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60).stdout.splitlines()
    assert out == [
        "merge batch 0 2 | left 1 3",
        "shrink batch 0 | left 1",
        "bypass batch 1 | left 0 2",
        "bypassed 1",
        "bound wait | left 0 2",
        "reject reject rejected=0 status=3 | left 1",
        "error reject rejected=1 status=2 | left 0",
    ], out


def test_multigrid_parameters_binding(qdd):
    """The C defaults reach Python field by field (no GPU involved), keyword
    overrides land in the struct, and a misspelt keyword is an error rather
    than a silently ignored attribute."""
    p = qdd.qdd_mg_default_params()
    assert (p.nv, p.setup_iters, p.setup_ncy, p.nmr, p.post_ncy, p.coarse_iters, p.sap_prec, p.bootstrap) == \
        (8, 3, 2, 4, 2, 12, qdd.QDD_PREC_F32, 0)
    p = qdd.qdd_mg_default_params(nv=12, bootstrap=2, sap_prec="f64")
    assert (p.nv, p.bootstrap, p.sap_prec) == (12, 2, qdd.QDD_PREC_F64)
    with pytest.raises(TypeError):
        qdd.qdd_mg_default_params(boot_strap=1)
