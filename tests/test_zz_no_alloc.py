"""Allocation-free grid totals, hydro_totals_noalloc, against hydro_totals.

Some callers cannot allocate device memory (no cudaMalloc available to them:
an allocator callback, a framework that owns all device memory, a process with
its memory reserved up front).  hydro_totals_noalloc serves them with a fixed
scratch array inside the library.  This test calls it through the C ABI twice
in a row, on states of different sizes so that the second call runs over the
first call's leftovers in the shared array, and checks each result against the
handle-based hydro_totals bit for bit (both run the same deterministic passes
without atomics).  The file name makes pytest collect it last; it also passes
alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_totals_match_handle_totals():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_06437_gb300 import build
    from paper_2210_06437_gb300 import hydro as HY
    from paper_2210_06437_gb300 import workloads as W
    build.build()
    L = HY.load_library()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for cfg in (3, 2):   # 4096 sub-grids, then 512
        w = W.config(cfg)
        host = w.state()
        U = torch.from_numpy(host).cuda()
        dx = torch.as_tensor(w.grid.dx, dtype=torch.float64, device="cuda")
        g = HY.HydroGrid(w.grid)
        ref = g.totals(U).cpu().numpy()
        g.sync()
        out = torch.full((11,), float("nan"), dtype=torch.float64, device="cuda")
        rc = L.hydro_totals_noalloc(ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(dx.data_ptr()), w.grid.n,
                                    ctypes.c_void_p(out.data_ptr()), stream)
        assert rc == 0
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        # both run the same deterministic, atomic-free passes: identical bits,
        # so a stale partial or a wrong offset in the shared array would show
        assert np.array_equal(got.view(np.uint64), ref.view(np.uint64)), (got, ref)
        g.close()
    # sizes beyond the fixed scratch are refused before any launch
    big = HY.TOTALS_NOALLOC_MAX_SUBGRIDS + 1
    assert L.hydro_totals_noalloc(ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(dx.data_ptr()), big,
                                  ctypes.c_void_p(out.data_ptr()), stream) == -1
