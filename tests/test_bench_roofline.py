"""The bench's roofline arithmetic for its sub-workloads, on the CPU: each
score-pass kernel against the ALU-pipe peak of its form (maxima at the
measured DPX rate, adds at the measured integer-add rate, 32 lanes per
warp instruction, 2 cells per instruction for the packed kernels), with a
fake device and fake measured rates."""
import os
import sys
import types

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

RATES = {0: 1.98, 3: 3.907, 6: 2.0}   # probe forms: s16x2 maxima, integer add, s32 maxima


class FakeCtx:
    def probe_issue_rate(self, form):
        return RATES[form]


@pytest.fixture
def fake_device(monkeypatch):
    import torch
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    monkeypatch.setattr(torch.cuda, "get_device_properties",
                        lambda d: types.SimpleNamespace(multi_processor_count=152))


def test_every_roofline_entry_is_a_sub_workload():
    assert set(bench.SUB_KERNELS) <= set(bench.SUB_WORKLOADS)
    for name, (phase, kernel, packed, n_max, n_add) in bench.SUB_KERNELS.items():
        assert phase in ("inter16", "intra16") and kernel.startswith("k_")
        assert n_max >= 5 and n_add in (0, 1), name


@pytest.mark.parametrize("name,n_max,n_add", [("reads_vs_windows", 5, 1),
                                              ("long_pairs_global", 5, 1),
                                              ("long_pairs_local", 5.5, 0),
                                              ("protein_search_global", 5, 1)])
def test_peak_from_the_kernel_op_count(fake_device, name, n_max, n_add):
    clk = {"sm_mhz": 2070.0}
    phase = bench.SUB_KERNELS[name][0]
    r = bench.sub_roofline(name, FakeCtx(), clk, {phase: 4000.0})
    cycles = n_max / RATES[0] + n_add / RATES[3]
    peak = 152 * 2070e6 * 32 * 2 / cycles / 1e9
    assert r["bound"] == "alu" and r["unit"] == "GCUPS"
    assert r["peak"] == pytest.approx(peak, abs=0.1)
    assert r["frac"] == pytest.approx(4000.0 / peak, abs=1e-4)
    assert r["achieved"] == 4000.0
    # the two packed forms land within 0.1% of each other: 5.5 maxima cost
    # what 5 maxima and one add do at these rates
    assert 7230 < r["peak"] < 7260


def test_no_roofline_without_clocks_or_phase(fake_device):
    assert bench.sub_roofline("long_pairs_global", FakeCtx(), {}, {"intra16": 1.0}) is None
    assert bench.sub_roofline("long_pairs_global", FakeCtx(), {"sm_mhz": 2070.0}, {}) is None
    assert bench.sub_roofline("serving", FakeCtx(), {"sm_mhz": 2070.0}, {"inter16": 1.0}) is None
