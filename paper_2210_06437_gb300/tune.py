"""Launch-shape autotuner for the hydro library.

Searches the handle's tunable launch parameters (``hydro_set_param``) on the
caller's own batch: every candidate runs a few RK stages, timed with CUDA events
on the launching stream after warm-up, and the fastest is kept.  Results are
cached in a JSON file (``$HYDRO_TUNE_CACHE``, else ``~/.cache/gb300_hydro_tune.json``)
under a key made of the GPU name, the precision and the batch size rounded up
to a power of two, so a later run with a similar batch reuses them.
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
    "ghost_threads": HY.PARAM_GHOST_THREADS,
}

# candidate values per parameter (0 = the library's occupancy-derived default)
SPACE = {
    "stage_ctas_per_sm": (0, 1, 2),
    "ghost_threads": (128, 256, 512),
}


def cache_path() -> str:
    return os.environ.get("HYDRO_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache",
                                                            "gb300_hydro_tune.json"))


def cache_key(gpu: str, precision: str, n_items: int) -> str:
    bucket = 1 << max(0, math.ceil(math.log2(max(1, n_items))))
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


def candidates(space: Dict[str, Sequence[int]] = SPACE) -> List[Dict[str, int]]:
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


def tune(grid: "HY.HydroGrid", U, scratch, ids=None, batch_offsets=None, reps: int = 3, use_cache: bool = True,
         space: Dict[str, Sequence[int]] = SPACE) -> Dict[str, int]:
    """Tune ``grid`` (a HydroGrid) on the state U (device, ghosts as for
    hydro_step) writing into ``scratch``; applies and returns the best parameters."""
    import torch
    n_items = grid.n if ids is None else len(ids)
    key = cache_key(torch.cuda.get_device_name(), grid.precision, n_items)
    if use_cache:
        hit = load_cache().get(key)
        if hit and set(hit.get("params", {})) == set(space):
            apply(grid, hit["params"])
            return dict(hit["params"])
    stream = torch.cuda.current_stream()
    ms = torch.zeros(2, dtype=torch.float64, device=U.device)

    def measure(params):
        apply(grid, params)
        for _ in range(2):
            grid.step(U, 1e-9, U_out=scratch, ids=ids, batch_offsets=batch_offsets, max_speed=ms)
            grid.fill_ghosts(scratch)
        torch.cuda.synchronize()
        times = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            grid.step(U, 1e-9, U_out=scratch, ids=ids, batch_offsets=batch_offsets, max_speed=ms)
            grid.fill_ghosts(scratch)
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
        grid.sync()
        return sorted(times)[len(times) // 2]

    best, table = search(measure, candidates(space))
    apply(grid, best)
    store_cache(key, {"params": best, "ms": min(t for _, t, _ in table if t is not None),
                      "table": [[c, t] for c, t, _ in table], "when": time.strftime("%Y-%m-%dT%H:%M:%S")})
    return best
