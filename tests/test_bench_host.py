"""Host helpers of bench.py (no GPU): the cost-model constants derived from
per-stage times, the lookup of profiled DRAM traffic, the O1 cut-off of the
error statements, the ensemble's sampled systems and the compact legs."""
import json
import math

import bench
from paper_1712_04718_gb300 import systems


def test_cost_model_units():
    st = {"bin": 10.0, "scatter": 0.0, "spread": 20.0, "fft_fwd": 15.0, "scale": 5.0,
          "fft_inv": 15.0, "gather": 30.0}   # ms summed over 100 evaluations
    cm = bench.cost_model(st, 100, 1000, 32, 8, 3)
    # 0.6 ms per evaluation over N P^3 = 512 000 spread/gather terms
    assert math.isclose(cm["c_spread_gather_s"], 0.6e-3 / 512000.0, rel_tol=1e-12)
    assert math.isclose(cm["c_fft_s"], 0.3e-3 / (16384.0 * math.log2(16384.0)), rel_tol=1e-12)
    assert math.isclose(cm["c_solve_s"], 0.05e-3 / 32768.0, rel_tol=1e-12)
    assert cm["paper_i7_3770_1core_fp64"]["c_spread_gather_s"] == 5e-9


def test_profiled_traffic_needs_matching_sources():
    assert bench.profiled_traffic("k_gather", "no-such-workload") == (None, None)
    assert bench.profiled_traffic("no_such_kernel", bench.DEFAULT_WORKLOAD) == (None, None)


def test_o1_cutoff_is_far_below_each_target():
    for name, w in systems.WORKLOADS.items():
        tol = bench.o1_tolerance(w["target_rel_force_err"])
        assert 1e-16 <= tol <= 1e-6
        assert tol <= 1e-3 * w["target_rel_force_err"] or tol == 1e-16, name


def test_headline_meets_its_stated_error_by_construction():
    w = systems.WORKLOADS[bench.DEFAULT_WORKLOAD]
    assert w["target_source"] == "stated" and w["P"] == 8 and w["M"] == 52
    assert bench.DEFAULT_WORKLOAD not in bench.LEG_WORKLOADS
    for leg in bench.LEG_WORKLOADS:
        assert leg in systems.WORKLOADS


def test_ensemble_sample_spans_box_sizes():
    ens = [dict(L=L) for L in (5.0, 3.1, 6.9, 4.0, 3.5, 6.0, 4.5, 5.5, 3.0, 7.0, 6.5)]
    s = bench.ensemble_sample(ens)
    assert len(s) == bench.ENS_SAMPLE_SYSTEMS
    Ls = [ens[i]["L"] for i in s]
    assert min(Ls) == 3.0 and max(Ls) == 7.0


def test_compact_leg_stays_short():
    res = {"workload": "water-L10-M84-P8-fp32comp", "value": 7045.123456, "ms_step": 0.1419,
           "N": 100200, "roofline": {"frac": 0.0661234, "kernel": "k_fgather"},
           "clocks": {"sm_mhz": 2070.0, "reasons": []},
           "autograd": {"forward": 9035.0, "forward_backward": 5042.0, "unit": "evals/s"}}
    acc = {"rel_rms_force_err": 2.9e-4, "target": 5e-4, "target_met": True}
    eq = {"P": 8, "value": 3000.0, "ms": 0.33, "err": 2.8e-4, "equal": True}
    leg = bench.compact_leg(res, acc, eq)
    assert len(json.dumps(leg)) < 480
    assert leg["met"] and leg["fp64_eq"]["P"] == 8
    assert bench.r4(0.0661234) == 0.06612


def test_tile_gather_rule_names_the_kernel():
    """The bench names the gather kernel by the library's rule: dense tiles
    (the 100k-atom box, tile edge 8) use the tile gather, the 21.6k-atom box
    at tile edge 6 and an automatic tile do not; a region past 64 KB never."""
    assert bench.tile_gather_selected(100200, 84, 8, 8)
    assert not bench.tile_gather_selected(21642, 52, 6, 6)
    assert not bench.tile_gather_selected(21642, 52, 6, 0)
    assert not bench.tile_gather_selected(10 ** 7, 128, 24, 16)
    w = {"P": 8, "M": 84}
    assert bench.stage_work(w, "fp32comp", 100200, 3, 8)["gather"][2] == "k_fgather"
    assert bench.stage_work(w, "fp32comp", 100200, 4, 8)["gather"][2] == "k_gather"
