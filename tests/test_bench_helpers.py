"""bench.py's helpers without a GPU: the algorithmic-bytes model, the peak
source, and the rule that recorded DRAM traffic is used only for the kernel
sources it was measured on."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_algorithmic_bytes_model():
    st = {"m": 10, "triangles": 3, "wedges_up": 7, "scanned": 25, "dmin_sum": 40, "walked": 31,
          "compacted_slots": 12, "support_walked": 5, "support_hub_probes": 2}
    sup, peel = bench.algorithmic_bytes(st, n=6)
    # support: 32 B per edge, 8 B per vertex, 4 B per N+(v) entry read, 32 B
    # per hub-bitmap probe, 12 B per triangle
    assert sup == 32 * 10 + 8 * 6 + 4 * 5 + 32 * 2 + 12 * 3
    # peel: Scans 16 B per entry visited less 8 B per edge of the first
    # Scan, 36 B per edge, 4 B per shorter-row entry walked (as the rows
    # stood), 28 B per triangle, 24 B per row entry a compaction visited
    assert peel == (16 * 25 - 8 * 10) + 36 * 10 + 4 * 31 + 28 * 3 + 24 * 12
    # without compaction the walk is the static sum of min(d(u), d(v))
    st2 = {k: v for k, v in st.items() if k not in ("walked", "compacted_slots", "support_walked",
                                                    "support_hub_probes")}
    assert bench.algorithmic_bytes(st2, n=6)[1] == (16 * 25 - 8 * 10) + 36 * 10 + 4 * 40 + 28 * 3
    # without the support counts, W+ entries
    assert bench.algorithmic_bytes(st2, n=6)[0] == 32 * 10 + 8 * 6 + 4 * 7 + 12 * 3


def test_peak_comes_from_the_measured_file_when_present():
    peak, kind = bench.peaks()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        assert kind == "measured" and peak == pytest.approx(json.load(open(path))["hbm_gbs"])
    else:
        assert kind == "fallback" and peak == 6800.0


def test_recorded_traffic_is_keyed_to_the_kernel_sources(monkeypatch):
    rec = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))
    ent = rec[bench.WORKLOAD]["k_persistent"]
    if ent["source_hash"] == bench.kernel_source_hash("k_persistent"):
        assert bench.recorded_traffic("k_persistent", bench.WORKLOAD) == ent["bytes_per_step"]
    # any change to the sources makes the record stale
    monkeypatch.setattr(bench, "kernel_source_hash", lambda kernel="k_persistent": "0" * 16)
    assert bench.recorded_traffic("k_persistent", bench.WORKLOAD) is None
    assert bench.recorded_traffic("k_persistent", "no_such_workload") is None


def test_source_hash_depends_on_the_kernels_own_file():
    # the peel kernels hash peel.cu, the support kernel support.cu; both
    # include the shared headers
    assert bench.kernel_source_hash("k_persistent") == bench.kernel_source_hash("k_gprocess")
    assert bench.kernel_source_hash("k_persistent") != bench.kernel_source_hash("k_support_warp")
