"""Host-side pieces of the benchmark and of the reduced-precision option (CPU only).

- The DRAM traffic figure is reported only while the timed kernel's sources and launch shape are
  the ones the ncu capture saw (sha256 of the sources, tuning keys).
- The binary16 SH option is graded against the oracle given coefficients rounded by numpy; that
  reference rests on numpy's float16 conversion being IEEE round-to-nearest-even (the device's
  conversion), which is pinned here on values whose rounding the rule fixes exactly."""
import hashlib
import json
import os

import numpy as np
import pytest

import bench


def _write_traffic(root, sources, sha, tuning):
    os.makedirs(os.path.join(root, "profiles"), exist_ok=True)
    entry = {"dram_bytes_per_launch": 1234, "kernel": "k", "sources": sources, "sha256": sha, "tuning": tuning}
    with open(os.path.join(root, "profiles", "traffic.json"), "w") as f:
        json.dump({"room": {"blend": entry}}, f)


def test_traffic_reported_only_for_the_captured_kernel(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("kernel v1")
    sha = hashlib.sha256(b"kernel v1").hexdigest()
    _write_traffic(str(tmp_path), ["k.cu"], sha, {"blend_variant": 1})
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_for("room", "blend", {"blend_variant": 1}) == 1234
    assert bench.traffic_for("room", "blend", {"blend_variant": 4}) is None      # another launch shape
    assert bench.traffic_for("room", "sort", {"blend_variant": 1}) is None       # no capture of that stage
    assert bench.traffic_for("city", "blend", {"blend_variant": 1}) is None
    src.write_text("kernel v2")                                                   # the kernel changed
    assert bench.traffic_for("room", "blend", {"blend_variant": 1}) is None


def test_committed_traffic_matches_the_sources():
    """The committed figure belongs to the committed blend sources."""
    e = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))["room"]["blend"]
    h = hashlib.sha256()
    for f in e["sources"]:
        h.update(open(os.path.join(bench.ROOT, f), "rb").read())
    assert h.hexdigest() == e["sha256"]
    assert e["dram_bytes_per_launch"] > 0


@pytest.mark.parametrize("x,expect", [
    (1.0 + 2.0 ** -11, 1.0),                      # tie between 1 and 1 + 2^-10: to the even one
    (1.0 + 3 * 2.0 ** -11, 1.0 + 2.0 ** -9),      # tie between 1 + 2^-10 and 1 + 2^-9: to the even one
    (1.0 + 2.0 ** -11 + 2.0 ** -20, 1.0 + 2.0 ** -10),   # above the tie: up
    (-(1.0 + 2.0 ** -11), -1.0),
    (2.0 ** -24, 2.0 ** -24),                     # smallest subnormal is exact
    (2.0 ** -25, 0.0),                            # half of it: tie to even (zero)
    (3 * 2.0 ** -26, 2.0 ** -24),                 # above that tie: up to the smallest subnormal
    (65504.0, 65504.0),                           # largest finite
    (65520.0, np.inf),                            # the midpoint to the next binade rounds to infinity
])
def test_numpy_float16_is_round_to_nearest_even(x, expect):
    with np.errstate(over="ignore"):
        assert float(np.float32(x).astype(np.float16)) == expect


def test_clock_summary_counts_only_samples_inside_the_timed_region():
    """Samples taken before the timed region (the idle GPU while nvidia-smi starts) are left out;
    throttle reasons are reported when active in any counted sample; bad lines are skipped."""
    idle = "0, 120, 2070, 120.5, 0x1, Not Active, Not Active, Not Active, Not Active"
    load = "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active"
    capped = "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active"
    lines = [(0.0, idle), (0.5, idle), (1.0, load), (1.1, "garbage"), (1.2, load), (1.3, capped)]
    r = bench.summarize_clock_lines(lines, 1.0)
    assert r["samples"] == 3 and r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]
    r = bench.summarize_clock_lines(lines, 2.0)      # nothing inside the region
    assert r["samples"] == 0 and r["sm_mhz"] is None
