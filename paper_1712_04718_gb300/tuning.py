"""Autotuning of the spreading variant and tile edge, with a JSON cache.

For a single system the choice is between the sorted single-precision
pipeline with a tile edge, which trades the particles each spreading block
handles (and its shared-memory region) against the number of blocks and the
region flushes, with its own gather (variant 3) or with the gather fused into
the inverse transform (variant 5), and the unsorted one (variant 4), which
skips the sort and adds straight into the grid with global reductions.  The best
choice depends on the grid, the support, the particle count and the GPU.
tune_plan / tune_batch time a few candidates with CUDA events on the caller's
inputs and remember the winner in a JSON file (SE_TUNE_CACHE, else
~/.cache/se_gb300/tiles.json), keyed by the problem shape and the GPU name.
"""
import json
import os

import torch

DEFAULT_CANDIDATES = (4, 6, 8)


def cache_path():
    return os.environ.get("SE_TUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "se_gb300", "tiles.json")


def _load():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(key, value):
    data = _load()
    data[key] = value
    path = cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp.%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def _gpu():
    return torch.cuda.get_device_name().replace(" ", "_")


def _time(fn, reps):
    for _ in range(3):
        fn()
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        fn()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps


def default_configs(plan, unsorted=False):
    """(spread variant, tile edge) candidates for a plan: the sorted
    single-precision pipeline's tile edges, with its own gather (variant 3)
    and with the gather fused into the inverse transform (variant 5), and,
    with unsorted=True, the unsorted variant 4 too."""
    if plan.prec != 0 and plan.M <= 128:
        return ((4, 0),) * bool(unsorted) + tuple((v, t) for v in (3, 5)
                                                  for t in DEFAULT_CANDIDATES)
    return tuple((0, t) for t in DEFAULT_CANDIDATES)


def tune_plan(plan, xyz, q, configs=None, reps=50, use_cache=True):
    """Pick the spread variant and tile edge of a single-system plan and set
    them; returns (variant, tile, ms, cached)."""
    configs = tuple(configs) if configs is not None else default_configs(plan)
    key = "plan3:P%d:M%d:N%dk:prec%d:%s:%s" % (plan.P, plan.M, plan.N // 1000, plan.prec, _gpu(),
                                              "-".join("%d.%d" % c for c in configs))
    if use_cache:
        hit = _load().get(key)
        if hit:
            plan.set_tuning(hit["variant"], hit["tile"])
            return hit["variant"], hit["tile"], hit["ms"], True
    F = torch.empty((plan.N, 3), dtype=plan.dtype, device=xyz.device)
    phi = torch.empty((plan.N,), dtype=plan.dtype, device=xyz.device)
    best = None
    for v, t in configs:
        plan.set_tuning(v, t)
        ms = _time(lambda: plan.evaluate(xyz, q, F, phi), reps)
        if best is None or ms < best[2]:
            best = (v, t, ms)
    plan.set_tuning(best[0], best[1])
    _store(key, {"variant": best[0], "tile": best[1], "ms": best[2]})
    return best[0], best[1], best[2], False


def tune_batch(batch, xyz, q, candidates=(6, 8, 10, 12, 16), reps=10, use_cache=True):
    """Pick the tile edge of an ensemble (se_batch_autotune); returns (tile, ms, cached)."""
    key = "batch:P%d:S%d:M%d-%d:N%dk:%s" % (batch.P, batch.S, int(batch.Ms.min()),
                                             int(batch.Ms.max()), batch.Ntot // 1000, _gpu())
    if use_cache:
        hit = _load().get(key)
        if hit:
            batch.set_tile(hit["tile"])
            return hit["tile"], hit["ms"], True
    tile, ms = batch.autotune(xyz, q, candidates=candidates, reps=reps)
    _store(key, {"tile": tile, "ms": ms})
    return tile, ms, False


def tune_ewald(xyz, q, L, tol, quantity="force", rc_candidates=None, precision="fp32", reps=20):
    """Measured balance of the real-space and Fourier-space parts of the whole
    Ewald sum.  The fastest splitting parameter xi for a tolerance balances
    the costs of the two parts and depends on the implementation and the
    hardware (arXiv:1712.04718, Sec. 6.2).  For each real-space cut-off rc
    (default: six values from 0.5 to min(1.6, L/3)), the parameters
    se_select_params gives for the absolute rms tolerance tol (xi from rc, M,
    P), and the whole evaluation -- the k-space plan, then the real-space sum
    accumulated into the same outputs -- are timed on the caller's system
    (CUDA device tensors xyz [N, 3], q [N] of the precision's dtype).
    Returns (best, table): dicts with rc, xi, M, P and the milliseconds of the
    k-space part, the real-space part and the whole evaluation."""
    import numpy as np
    from . import se
    N = int(q.shape[0])
    Q = float((q.double() ** 2).sum())
    if rc_candidates is None:
        rc_candidates = [round(float(r), 3) for r in np.linspace(0.5, min(1.6, L / 3.0), 6)]
    table = []
    for rc in rc_candidates:
        s = se.select_params(quantity, tol, rc, L, Q)
        if not s["supported"] or rc > L / 3.0:
            continue
        plan = se.Plan(N, L, s["xi"], s["M"], s["P"], precision=precision)
        rs = se.RealSpace(N, L, s["xi"], rc, precision=precision)
        F = torch.empty((N, 3), dtype=plan.dtype, device=xyz.device)
        phi = torch.empty((N,), dtype=plan.dtype, device=xyz.device)
        E = torch.zeros(1, dtype=torch.float64, device=xyz.device)
        ms_k = _time(lambda: plan.evaluate(xyz, q, F, phi, E), reps)
        ms_r = _time(lambda: rs.evaluate(xyz, q, F, phi, E, accumulate=True), reps)

        def whole():
            plan.evaluate(xyz, q, F, phi, E)
            rs.evaluate(xyz, q, F, phi, E, accumulate=True)
        ms_t = _time(whole, reps)
        table.append({"rc": rc, "xi": s["xi"], "M": s["M"], "P": s["P"], "ms_kspace": ms_k,
                      "ms_real": ms_r, "ms_total": ms_t})
        plan.close()
        rs.close()
    if not table:
        raise ValueError("no cut-off in %s gives supported parameters for tol %g"
                         % (list(rc_candidates), tol))
    return min(table, key=lambda r: r["ms_total"]), table
