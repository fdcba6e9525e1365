"""Launch-shape autotuner for the hydro library.

Searches the handle's tunable launch parameters (``hydro_set_param``) on the
caller's own workload, timing what a time step runs: one SSP-RK3 step of the
multi-step graph (``hydro_rk3_run_cfl``: the three stage launches and, in mixed
precision, their coarse-fine correction passes), with CUDA events on the
launching stream after a warm-up replay.  The space:
  stage_ctas_per_sm  persistent stage CTAs per SM (sub-grids in flight per SM);
  prefetch_pass      the direction pass (0 x, 1 y, 2 z) in which a stage pulls
                     the rows its update reads into L2 (the prefetch distance);
  reflux_shape       threads per CTA and items per thread of the mixed
                     correction pass (mixed handles only);
  fused_rk3          the step as three stage launches (0) or one persistent
                     launch with per-sub-grid completion counters (1).
Results do not depend on any of them (the kernels' arithmetic and order are
fixed; only the launch shape changes), which a GPU test checks point by point.
The best point is cached in a JSON file (``$HYDRO_TUNE_CACHE``, else
``~/.cache/gb300_hydro_tune.json``) under the GPU name, the precision and the
sub-grid count rounded up to a power of two.
"""
from __future__ import annotations

import itertools
import json
import math
import os
import time
from typing import Callable, Dict, Iterable, List, Optional, Sequence, Tuple

from . import hydro as HY

PARAMS = {
    "stage_ctas_per_sm": HY.PARAM_STAGE_CTAS_PER_SM,
    "prefetch_pass": HY.PARAM_PREFETCH_PASS,
    "reflux_shape": HY.PARAM_REFLUX_SHAPE,
    "fused_rk3": HY.PARAM_FUSED_RK3,
}

SPACE_FP64 = {
    "stage_ctas_per_sm": (1,),      # the FP64 stage fits one CTA per SM
    "prefetch_pass": (0, 1, 2),
    "fused_rk3": (0, 1),
}
SPACE_MIXED = {
    "stage_ctas_per_sm": (1, 2),
    "prefetch_pass": (0, 1, 2),
    "reflux_shape": (0, 1, 2, 3),
    "fused_rk3": (0, 1),
}


def space_for(precision: str) -> Dict[str, Sequence[int]]:
    return SPACE_MIXED if precision == "mixed" else SPACE_FP64


def cache_path() -> str:
    return os.environ.get("HYDRO_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache",
                                                            "gb300_hydro_tune.json"))


def cache_key(gpu: str, precision: str, n_subgrids: int) -> str:
    bucket = 1 << max(0, math.ceil(math.log2(max(1, n_subgrids))))
    return "%s|%s|%d" % (gpu, precision, bucket)


def load_cache(path: Optional[str] = None) -> Dict[str, dict]:
    path = path or cache_path()
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def store_cache(key: str, entry: dict, path: Optional[str] = None) -> None:
    path = path or cache_path()
    d = load_cache(path)
    d[key] = entry
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def candidates(space: Dict[str, Sequence[int]]) -> List[Dict[str, int]]:
    names = sorted(space)
    return [dict(zip(names, vals)) for vals in itertools.product(*(space[n] for n in names))]


def search(measure: Callable[[Dict[str, int]], float], cands: Iterable[Dict[str, int]]) -> Tuple[Dict[str, int], list]:
    """Return the candidate with the smallest measured time and the full table.
    Candidates whose measurement raises are skipped."""
    table = []
    best, best_t = None, math.inf
    for c in cands:
        try:
            t = float(measure(c))
        except Exception as e:  # an invalid launch shape for this device
            table.append((c, None, repr(e)))
            continue
        table.append((c, t, None))
        if t < best_t:
            best, best_t = c, t
    if best is None:
        raise RuntimeError("no tuning candidate could be measured")
    return best, table


def apply(grid: "HY.HydroGrid", params: Dict[str, int]) -> None:
    for name, value in params.items():
        grid.set_param(PARAMS[name], int(value))


def tune(grid: "HY.HydroGrid", U, scratch1, scratch2, ids=None, batch_offsets=None, reps: int = 3,
         use_cache: bool = True, space: Optional[Dict[str, Sequence[int]]] = None) -> Dict[str, int]:
    """Tune ``grid`` (a HydroGrid whose batches list every sub-grid) on the
    state U (device), using scratch1/scratch2 as the RK3 scratch; U is restored
    afterwards.  Applies and returns the best parameters."""
    import torch
    space = space or space_for(grid.precision)
    key = cache_key(torch.cuda.get_device_name(), grid.precision, grid.n)
    if use_cache:
        hit = load_cache().get(key)
        if hit and set(hit.get("params", {})) == set(space):
            apply(grid, hit["params"])
            return dict(hit["params"])
    stream = torch.cuda.current_stream()
    backup = U.clone()
    ms = torch.zeros(2, dtype=torch.float64, device=U.device)
    grid.step(U, 0.0, U_out=scratch1, ids=ids, batch_offsets=batch_offsets, max_speed=ms)   # a CFL speed

    def measure(params):
        apply(grid, params)          # drops the captured graphs
        U.copy_(backup)
        ms0 = ms.clone()
        grid.rk3_run_cfl(U, 0.4, scratch1, scratch2, ms0, 1, ids=ids, batch_offsets=batch_offsets)
        torch.cuda.synchronize()
        times = []
        for _ in range(reps):
            U.copy_(backup)
            m = ms.clone()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            grid.rk3_run_cfl(U, 0.4, scratch1, scratch2, m, 1, ids=ids, batch_offsets=batch_offsets)
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
        grid.sync()
        return sorted(times)[len(times) // 2]

    try:
        best, table = search(measure, candidates(space))
    finally:
        U.copy_(backup)
        del backup
    apply(grid, best)
    store_cache(key, {"params": best, "ms": min(t for _, t, _ in table if t is not None),
                      "table": [[c, t] for c, t, _ in table], "when": time.strftime("%Y-%m-%dT%H:%M:%S")})
    return best
