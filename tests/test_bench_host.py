"""Host logic of bench.py (no GPU): the per-kernel roofline arithmetic, the
choice of the binding resource, the DRAM-traffic lookup guarded by the
kernel source hash, and the mapping of profiled kernels to the library's
work-counter slots."""
import json
import os
import re
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _counters(**slots):
    base = dict(closest_rays=0, shadow_rays=0, nodes=0, tris=0)
    return {k: dict(base, **v) for k, v in slots.items()}


def test_kernel_roofline_arithmetic():
    # 20 steps, two launches per step of 5 ms each: 200 ms over 40 launches
    prof = {"render_bounce": (200.0, 40), "sort_hist": (3.0, 140)}
    cnt = _counters(render_bounce=dict(nodes=2_000_000, tris=300_000))
    peak_ops, peak_l2 = 40e12, 12e12
    kr = bench.kernel_rooflines(prof, cnt, 20, peak_ops, peak_l2)
    assert set(kr) == {"render_bounce"}  # kernels without counted work are left out
    k = kr["render_bounce"]
    assert k["launches_per_step"] == 2
    assert k["avg_launch_ms"] == pytest.approx(5.0)
    # the counted step's work is spread over its launches
    assert k["node_visits_per_launch"] == pytest.approx(1_000_000)
    assert k["tri_tests_per_launch"] == pytest.approx(150_000)
    ops = bench.OPS_PER_BOX * bench.BOXES_PER_NODE * 1_000_000 + bench.OPS_PER_TRI * 150_000
    nbytes = bench.BYTES_PER_NODE * 1_000_000 + bench.BYTES_PER_TRI * 150_000
    assert k["alu"]["achieved"] == pytest.approx(ops / 5e-3 / 1e12)
    assert k["alu"]["frac"] == pytest.approx(ops / 5e-3 / peak_ops)
    assert k["l2"]["achieved"] == pytest.approx(nbytes / 5e-3 / 1e9)
    assert k["l2"]["frac"] == pytest.approx(nbytes / 5e-3 / peak_l2)


def test_work_unit_constants_follow_the_stated_counts():
    # a slab test is 6 FMA + 6 min/max, a binary node visit tests two boxes,
    # a watertight test is the shear and three edge functions
    assert bench.OPS_PER_BOX == 12 and bench.BOXES_PER_NODE == 2 and bench.OPS_PER_TRI == 26
    assert bench.BYTES_PER_NODE == 64 and bench.BYTES_PER_TRI == 48


def test_roofline_of_picks_the_dominant_kernel_and_the_binding_resource(monkeypatch):
    prof = {"backward_primary_first": (300.0, 20), "render_first": (150.0, 20), "sort_scatter": (400.0, 140)}
    cnt = _counters(backward_primary_edges=dict(nodes=1_500_000_000, tris=100_000_000),
                    render=dict(nodes=500_000_000, tris=40_000_000))
    res = {"prof": prof, "counters": cnt, "ms_per_step": 60.0}
    peaks = {"alu_ops": 39e12, "l2_bytes": 12e12}
    monkeypatch.setattr(bench, "ncu_traffic", lambda workload, kernel: None)
    # the ray kernel with the most event time (a sort's event time, which
    # includes waiting on the second stream, does not count)
    roof, kr = bench.roofline_of(res, 20, peaks, bench.PROCEDURAL)
    assert roof["kernel"] == "backward_primary_first"
    assert bench.roofline_of({"prof": {"sort_hist": (1.0, 7)}, "counters": {}, "ms_per_step": 1.0}, 1, peaks,
                             bench.PROCEDURAL)[0] is None
    k = kr["backward_primary_first"]
    binding = "alu" if k["alu"]["frac"] >= k["l2"]["frac"] else "l2"
    assert roof["bound"] == binding
    assert roof["frac"] == pytest.approx(k[binding]["frac"])
    assert roof["achieved"] / roof["peak"] == pytest.approx(roof["frac"])
    assert roof["share_of_step"] == pytest.approx(300.0 / 20 / 60.0)
    assert roof["algorithmic_bytes_per_launch"] == pytest.approx(
        bench.BYTES_PER_NODE * 1_500_000_000 + bench.BYTES_PER_TRI * 100_000_000)


def test_traffic_is_reported_only_for_the_captured_sources(monkeypatch):
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
        stored = json.load(f)
    workload = next(iter(stored))
    kernel = next(iter(stored[workload]))
    ent = stored[workload][kernel]
    assert ent["dram_bytes_per_launch"] > 0 and "--clock-control none" in ent["command"]
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: ent["source_hash"])
    assert bench.ncu_traffic(workload, kernel) == ent["dram_bytes_per_launch"]
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.ncu_traffic(workload, kernel) is None
    assert bench.ncu_traffic("no such workload", kernel) is None


def test_profiled_kernels_map_to_counter_slots_of_the_library():
    from paper_1904_12228_gb300 import drt
    slots = drt.Context.COUNTER_SLOTS
    assert set(bench.COUNTER_OF.values()) <= set(slots)
    # the binding's slot order is the library's enum of counter slots
    with open(os.path.join(ROOT, "paper_1904_12228_gb300", "csrc", "drt_internal.h")) as f:
        src = f.read()
    enum = dict((m.group(1), int(m.group(2))) for m in re.finditer(r"(kSlot\w+)\s*=\s*(\d+)", src))
    n = int(re.search(r"kKernelSlots\s*=\s*(\d+)", src).group(1))
    assert n == len(slots)
    expect = {"kSlotRender": "render", "kSlotBwdInterior": "backward_interior",
              "kSlotBwdPrimary": "backward_primary_edges", "kSlotDebug": "debug",
              "kSlotBwdSecondary": "backward_secondary_edges", "kSlotBwdSecSides": "backward_secondary_sides",
              "kSlotBwdSecBounce": "backward_secondary_bounce", "kSlotBwdPrimBounce": "backward_primary_bounce",
              "kSlotRenderBounce": "render_bounce"}
    assert set(enum) == set(expect)
    for name, slot in expect.items():
        assert slots[enum[name]] == slot, name
