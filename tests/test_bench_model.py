"""Host-side logic of bench.py's roofline: the committed ncu traffic capture is used only while the stencil
sources it was taken on are unchanged, and its per-site / per-site-and-rhs bytes scale with the launches."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_capture_is_well_formed():
    d = json.load(open(os.path.join(ROOT, "profiles", "bri_stencil_traffic.txt")))
    assert len(d["stencil_source_sha256_16"]) == 16
    # the capture is at least the compulsory bytes: links 2880 + clover 288 per site, spinors 192 per site and rhs
    assert d["links_clover_bytes_per_site"] >= 2880 + 288
    assert d["spinor_bytes_per_site_rhs"] >= 192
    # bench.py uses it only while it matches the current stencil sources (else reports traffic null)
    t = bench.stencil_traffic()
    assert t is None or t["stencil_source_sha256_16"] == bench.stencil_source_hash()


def test_traffic_model_scales_with_sites_and_rhs():
    t = {"links_clover_bytes_per_site": 3000.0, "spinor_bytes_per_site_rhs": 200.0}
    vol = 1000
    # 10 launches carrying 25 rhs-applications in total: 2.5 rhs per launch on average
    got = bench.stencil_traffic_per_launch(t, vol, 10, 25 * vol, 1)
    assert got == int(vol * 3000.0 + 2.5 * vol * 200.0)
    assert bench.stencil_traffic_per_launch(None, vol, 10, 25 * vol, 1) is None
    assert bench.stencil_traffic_per_launch(t, vol, 10, 25 * vol, 2) is None  # BF16 links: not captured
    assert bench.stencil_traffic_per_launch(t, vol, 0, 0, 1) is None


def test_stale_capture_is_ignored(tmp_path, monkeypatch):
    d = json.load(open(os.path.join(ROOT, "profiles", "bri_stencil_traffic.txt")))
    d["stencil_source_sha256_16"] = "0" * 16
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "bri_stencil_traffic.txt").write_text(json.dumps(d))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "stencil_source_hash", lambda: "1" * 16)
    assert bench.stencil_traffic() is None


def test_both_arms_share_the_workload_config():
    a = bench.workload_config(4, 1, "gpu arithmetic")
    b = bench.workload_config(4, 1, "oracle arithmetic")
    assert {k: v for k, v in a.items() if k != "inner"} == {k: v for k, v in b.items() if k != "inner"}
    assert a["lattice"] == list(bench.DIMS) and a["kl_order"] == bench.KL_ORDER and a["tol"] == bench.TOL
