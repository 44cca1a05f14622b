"""The bench's roofline accounting on the host: hops that leave a domain
(against a brute-force count over the domain's sites), the Schwarz flop
count per site, the operator's algorithmic bytes per site, and the DRAM
traffic record, which is reported only while the kernel's sources match."""
import itertools
import json
import os

import pytest

import bench


def _leaving_hops_brute(dom):
    total = 0
    for c in itertools.product(*[range(d) for d in dom]):
        for mu in range(4):
            total += (c[mu] + 1 >= dom[mu]) + (c[mu] - 1 < 0)
    return total / float(dom[0] * dom[1] * dom[2] * dom[3])


@pytest.mark.parametrize("dom", [(8, 4, 4, 4), (4, 4, 4, 4), (2, 2, 2, 2), (6, 4, 2, 2)])
def test_crossing_hops_per_site(dom):
    assert bench.crossing_hops_per_site(dom) == pytest.approx(_leaving_hops_brute(dom), rel=1e-15)


def test_operator_flop_decomposition():
    """Sec. 3.7 prints 1848 flop/site for Wilson-clover; the bench's count is
    hops 1320 + two Hermitian 6x6 clover blocks 504 + the final combination 24
    (tests/golden/paper_values.json)."""
    golden = json.load(open(os.path.join(bench.ROOT, "tests", "golden", "paper_values.json")))
    f = bench.SAP_FLOP
    assert f["hop"] + f["clover"] + f["combine"] == golden["flops_per_site"]["wilson_clover"]
    # eight spin-projected hops: per hop the projection (6 complex adds, 12 flop) and two 3x3 complex
    # matrix-vector products (9 complex multiplies at 6 and 6 complex adds at 2: 66 each); the 12
    # complex components of the 8 results are summed with 7 adds each (24 flop per add of a spinor)
    assert 8 * (12 + 2 * 66) + 7 * 24 == f["hop"]
    # a Hermitian 6x6 block times a complex 6-vector: 6 real diagonal entries times complex (12), the
    # 15 off-diagonal entries used twice (30 complex multiplies, 180), 5 complex adds per row (60)
    assert 2 * (12 + 30 * 6 + 6 * 5 * 2) == f["clover"]


def test_sap_flop_per_site():
    # inside a domain only the hops that stay in it are computed (Dirichlet boundary): an 8x4^3 domain
    # loses 1.75 of its 8 hops per site, a 4^4 domain 2; each hop is 144 flop and their sum takes one
    # spinor add (24) fewer than there are hops
    assert 8 * 144 + 7 * 24 == bench.SAP_FLOP["hop"]
    for dom, c in (((8, 4, 4, 4), 1.75), ((4, 4, 4, 4), 2.0)):
        hops = (8 - c) * 144 + (7 - c) * 24
        full = hops + 504 + 24
        # per even/odd pair: setup (odd clover; even hops + combine), nmr MR steps of two in-domain applies
        # plus the MR vector algebra, the reconstruction; then the inflow's entering hops
        pair = (504 + hops + 24) + 4 * (2 * full + 336) + full
        assert bench.sap_flop_per_site(dom, 4) == pytest.approx(pair / 2 + c * 168)
    assert bench.sap_flop_per_site((8, 4, 4, 4), 4) == pytest.approx(8736.0)
    assert bench.sap_flop_per_site((4, 4, 4, 4), 4) == pytest.approx(8568.0)
    # one launch sweeps half the sites: the 16^3x32 workload's flop per launch
    assert 16 * 16 * 16 * 32 // 2 * bench.sap_flop_per_site((8, 4, 4, 4), 4) == pytest.approx(572522496.0)


def test_operator_bytes_per_site():
    got = {p: (bench.op_bytes_per_site(p, True), bench.op_bytes_per_site(p, False))
           for p in ("f64", "df64", "f32", "h16", "f16", "bf16")}
    assert got == {"f64": (1536, 1536), "df64": (1536, 1536), "f32": (768, 672), "h16": (484, 436),
                   "f16": (396, 348), "bf16": (396, 348)}


def test_traffic_record_only_while_sources_match(tmp_path, monkeypatch):
    """A DRAM-traffic record names the sources of its kernel with their
    SHA-256; the bench reports it only while those files are unchanged."""
    import hashlib

    src = tmp_path / "csrc" / "kernel.cu"
    src.parent.mkdir(parents=True)
    src.write_text("__global__ void k() {}\n")
    (tmp_path / "profiles").mkdir()
    rec = {"k_example": {"sources": ["csrc/kernel.cu"], "sha256": hashlib.sha256(src.read_bytes()).hexdigest(),
                         "dram_bytes_per_launch": 12345}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("k_example") == 12345
    with open(src, "a") as f:
        f.write("\n")
    assert bench.ncu_traffic("k_example") is None
    assert bench.ncu_traffic("no_such_kernel") is None


def test_threaded_oracle_sample_evaluates_every_site(ora):
    """The all-cores CPU baseline splits the sampled sites over host threads
    that call the oracle's per-site routine concurrently: the pieces, put
    together, are the single-thread result bit for bit, and the timed helper
    runs."""
    from concurrent.futures import ThreadPoolExecutor

    import numpy as np

    from paper_1502_04025_gb300 import inputs

    W = dict(bench.CONFIGS[1])
    U = inputs.gauge_field(W["L"], W["eps"], W["gauge_seed"])
    b = bench.make_sources(W)
    sites = np.arange(int(np.prod(W["L"])))
    whole = ora.apply_D_sites(W["L"], U, W["csw"], W["kappa"], b, sites)
    with ThreadPoolExecutor(4) as ex:
        parts = list(ex.map(lambda c: ora.apply_D_sites(W["L"], U, W["csw"], W["kappa"], b, c),
                            np.array_split(sites, 7)))
    assert np.array_equal(np.concatenate(parts), whole)
    assert bench.oracle_sample_threads(W, U, b, 512, 3) > 0


def test_reference_arm_line(tmp_path):
    """bench.py --impl reference (the FP64 oracle timed on the host) prints
    one JSON line with the contract's keys: its measured value, a
    cpu_baseline describing this run with the same value, and an e2e object
    without host-device traffic."""
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--config", "1",
                        "--steps", "2", "--warmup", "1"], cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "ms"
    assert d["value"] > 0 and d["ms_per_step"] == d["value"] and d["steps"] == 2 and d["warmup"] == 1
    assert d["higher_is_better"] is False
    c = d["cpu_baseline"]
    assert c["kind"] == "oracle" and c["cores"] == 1 and c["value"] == d["value"] and c["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
