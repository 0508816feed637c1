"""Host helpers of bench.py (no GPU): the cost-model constants derived from
per-stage times, and the lookup of profiled DRAM traffic."""
import math

import bench


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
    assert bench.profiled_traffic("k_gather", "no-such-workload") is None
    assert bench.profiled_traffic("no_such_kernel", "water-L6-M52-P6-fp32comp") is None


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
