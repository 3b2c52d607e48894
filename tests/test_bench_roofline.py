"""Roofline arithmetic of bench.py (CPU): the algorithmic bytes of each pass, and the rule that a
measured DRAM-traffic figure is reported only for the kernel sources it was captured from."""
import bench


def test_algorithmic_bytes_of_the_default_workload():
    # 512 x 512 x 10, complex64 half spectra of 512 x 257 bins:
    #   column pass: read q, xb (M planes each) and the packed factor (M(M+1)/2 planes), write x
    #   prior pass: read x, write q (M planes each); read and write u (M real planes)
    b = bench.algorithmic_bytes(512, 10, "dct8")
    bins = 512 * 257
    assert b["column_pass"] == (3 * 10 + 55) * bins * 8 == 89_477_120
    assert b["prior_pass"] == 2 * 10 * bins * 8 + 2 * 10 * 512 * 512 * 4 == 42_024_960
    # TV carries two components of u
    tv = bench.algorithmic_bytes(512, 10, "tv")
    assert tv["prior_pass"] - b["prior_pass"] == 2 * 10 * 512 * 512 * 4


def test_traffic_is_reported_only_for_the_captured_sources(monkeypatch):
    cur = bench.kernel_sources_hash()
    assert len(cur) == 16
    monkeypatch.setattr(bench, "TRAFFIC_CAPTURE", {"sources": cur, "bytes": {"column_pass": 1.5e6}})
    assert bench.measured_traffic("column_pass") == 1.5e6
    assert bench.measured_traffic("prior_pass") is None
    monkeypatch.setattr(bench, "TRAFFIC_CAPTURE", {"sources": "0" * 16, "bytes": {"column_pass": 1.5e6}})
    assert bench.measured_traffic("column_pass") is None


def test_committed_capture_matches_the_committed_kernels():
    """The DRAM traffic in bench.py was captured from the kernels as they are (a kernel change without
    a new capture turns the reported traffic into null; this test makes that visible)."""
    assert bench.TRAFFIC_CAPTURE["sources"] == bench.kernel_sources_hash()
    by = bench.TRAFFIC_CAPTURE["bytes"]
    alg = bench.algorithmic_bytes(512, 10, "dct8")
    # measured traffic must not exceed the algorithmic bytes by more than a few percent (no re-reads)
    assert 0.5 * alg["column_pass"] < by["column_pass"] < 1.05 * alg["column_pass"]
