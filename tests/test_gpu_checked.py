"""The range-checked build (libqdd_check.so, -DQDD_CHECK) runs the hot paths
on every test geometry and reports no out-of-range index: the Schwarz
kernel's stencil, face-slot and reduction accesses in every storage
precision (whole and partial warps, staged and unstaged fields), the
full-lattice operators with whole and two-row links, a mixed-precision
solve and a multigrid setup.  It also makes the Schwarz kernel's first
bounded wait give up (its poll limit set to 0), which must come back as
QDD_ETIMEOUT and leave the gauge object usable.  The checked build runs in a
child process, since one process loads one build of the library."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import numpy as np
from paper_1502_04025_gb300 import inputs, qdd
assert qdd.LIB_PATH.endswith("libqdd_check.so")
ctx = qdd.qdd_create(0, 0)
geoms = [((8, 8, 8, 8), (4, 4, 4, 4)), ((4, 4, 4, 4), (2, 2, 2, 2)), ((8, 4, 4, 12), (4, 2, 2, 2)),
         ((16, 8, 8, 8), (8, 4, 4, 4)), ((12, 8, 4, 4), (6, 4, 2, 2))]
for L, dom in geoms:
    g = qdd.qdd_create_gauge_field(ctx, L, dom, inputs.gauge_field(L, 0.5, 1001))
    qdd.qdd_set_clover(g, 1.0, 0.12)
    x = inputs.gaussian_source(L, 2001)
    for two in (True, False):
        qdd.qdd_set_link_compression(g, two)
        for prec in ("f64", "df64", "f32", "h16", "f16", "bf16"):
            qdd.qdd_apply_D(g, x, prec)
    for prec in ("f64", "f32", "h16", "f16", "bf16"):
        qdd.qdd_sap_apply(g, x, 4, 4, prec, want_rho=True)
    xs = np.ascontiguousarray(inputs.gaussian_source(L, 2002, nrhs=2))
    qdd.qdd_sap_apply(g, xs, 2, 3, "f32", nrhs=2)
    _, rep = qdd.qdd_solve(g, x, tol=1e-8, sap_prec="f32", arnoldi_prec="df64")
    assert rep["converged"]
    qdd.qdd_destroy_gauge(g)
L, dom = (4, 4, 4, 4), (2, 2, 2, 2)
g = qdd.qdd_create_gauge_field(ctx, L, dom, inputs.gauge_field(L, 0.5, 1001))
qdd.qdd_set_clover(g, 1.0, 0.13)
qdd.qdd_mg_setup(g, np.ascontiguousarray(inputs.gaussian_source(L, 4001, nrhs=4)), nv=4, bootstrap=1)
qdd.qdd_mg_vcycle(g, np.ascontiguousarray(inputs.gaussian_source(L, 4006)))
qdd.qdd_destroy_gauge(g)
print("HITS", qdd.qdd_check_hits())
'''


def test_range_checked_build_sees_no_out_of_range_index():
    from paper_1502_04025_gb300 import build

    build.build(check=True)
    env = dict(os.environ, QDD_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr
    hits = [line for line in r.stdout.splitlines() if line.startswith("HITS")]
    assert hits == ["HITS 0"], r.stdout + r.stderr


CHILD_TIMEOUT = r'''
import numpy as np
from paper_1502_04025_gb300 import inputs, qdd
assert qdd.LIB_PATH.endswith("libqdd_check.so")
ctx = qdd.qdd_create(0, 0)
L, dom = (8, 8, 8, 8), (4, 4, 4, 4)
g = qdd.qdd_create_gauge_field(ctx, L, dom, inputs.gauge_field(L, 0.5, 1001))
qdd.qdd_set_clover(g, 1.0, 0.12)
eta = inputs.gaussian_source(L, 2001)
ref = qdd.qdd_sap_apply(g, eta, 4, 4, "f32")
qdd.qdd_check_set_wait_limit(0, 0)
try:
    qdd.qdd_sap_apply(g, eta, 4, 4, "f32")
    print("STATUS", qdd.QDD_OK)
except qdd.QddError as e:
    print("STATUS", e.status)
qdd.qdd_check_set_wait_limit(0, 1 << 22)
again = qdd.qdd_sap_apply(g, eta, 4, 4, "f32")
print("SAME", bool(np.array_equal(again, ref)))
x, rep = qdd.qdd_solve(g, eta, tol=1e-10, sap_prec="f32")
print("CONVERGED", bool(rep["converged"]))
'''


def test_device_wait_that_runs_out_is_reported_and_the_gauge_stays_usable():
    """The first bounded wait of every Schwarz CTA gives up at once (poll
    limit 0): each CTA flags the timeout, waits with the drain wait's own
    limit until its staging copies have landed, and leaves.  qdd_sap_apply
    reports QDD_ETIMEOUT; with the default limit back, the same call gives
    the same bits as before and a solve on the same gauge object converges."""
    from paper_1502_04025_gb300 import build

    build.build(check=True)
    env = dict(os.environ, QDD_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", CHILD_TIMEOUT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    out = dict(line.split(" ", 1) for line in r.stdout.splitlines() if " " in line)
    assert out.get("STATUS") == "6", r.stdout + r.stderr  # QDD_ETIMEOUT
    assert out.get("SAME") == "True" and out.get("CONVERGED") == "True", r.stdout + r.stderr
