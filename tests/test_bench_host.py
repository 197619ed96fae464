"""Host-side pieces of the benchmark's roofline: the captured DRAM traffic is
scaled to a launch by the units it processes, and only reported while the
captured source is unchanged (a stale capture gives no number)."""
import hashlib
import os

import bench


def test_traffic_scales_by_units_and_goes_stale(tmp_path, monkeypatch):
    src = tmp_path / "kernel.cu"
    src.write_text("// a kernel\n")
    rel = os.path.relpath(src, bench.ROOT)
    sha = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    monkeypatch.setattr(bench, "TRAFFIC", {
        "k": dict(bytes=1000, units=100, unit="gaussians", tile=8, layers=1, src=rel, sha=sha)})
    units = dict(gaussians=400, pairs=7, curves=3)
    assert bench.traffic_per_launch("k", units, 8, 1) == 4000
    assert bench.traffic_per_launch("k", units, 16, 1) is None      # captured at another tile size
    assert bench.traffic_per_launch("k", units, 8, 0) is None       # captured with fill layers
    assert bench.traffic_per_launch("other", units, 8, 1) is None   # never captured
    src.write_text("// the kernel, changed since the capture\n")
    assert bench.traffic_per_launch("k", units, 8, 1) is None


def test_traffic_table_names_kernel_sources():
    for name, t in bench.TRAFFIC.items():
        assert os.path.exists(os.path.join(bench.ROOT, t["src"])), name
        assert t["bytes"] > 0 and t["units"] > 0 and len(t["sha"]) == 16, name
