"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, exports
every function include/hydro.h declares, and rejects bad grid descriptors on
the host before touching CUDA."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2210_06437_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2210_06437_gb300 import build, hydro
    build.build()
    return hydro.load_library(), hydro


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hydro.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hydro_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("hydro_create", "hydro_step", "hydro_totals", "hydro_fill_ghosts", "hydro_rk3_step", "hydro_sync",
              "hydro_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    L, hydro = lib
    names = declared_functions()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert set(hydro.EXPORTS) == set(names)


def _desc(hydro, w, **over):
    g = w.grid
    keep = dict(dx=np.ascontiguousarray(g.dx), nb=np.ascontiguousarray(g.neighbor, np.int32),
                rel=np.ascontiguousarray(g.neighbor_rel, np.int8), oc=np.ascontiguousarray(g.octant, np.int8))
    for k, v in over.items():
        if k in keep:
            keep[k] = v
    d = hydro.GridDesc(over.get("n", g.n), over.get("nf", 11), over.get("nx", 8), over.get("ghost", 3),
                       over.get("gamma", 5 / 3), over.get("eta", 1e-3), over.get("prec", 0), over.get("form", 0),
                       keep["dx"].ctypes.data, keep["nb"].ctypes.data, keep["rel"].ctypes.data, keep["oc"].ctypes.data)
    return d, keep


@pytest.mark.parametrize("over", [
    dict(nf=10), dict(nx=16), dict(ghost=2), dict(gamma=1.0), dict(gamma=float("nan")), dict(eta=1.0),
    dict(prec=2), dict(form=7), dict(n=0),
    dict(dx=np.full(8, -1.0)), dict(oc=np.full(8, 9, np.int8)),
    dict(rel=np.full((8, 6), 2, np.int8)),
    dict(nb=np.full((8, 6, 4), 8, np.int32)),
])
def test_create_rejects_bad_descriptors(lib, over):
    L, hydro = lib
    w = W.config(1)
    d, keep = _desc(hydro, w, **over)
    h = ctypes.c_void_p()
    assert L.hydro_create(ctypes.byref(d), ctypes.byref(h)) == -1
    assert not h.value


def test_null_arguments_are_rejected(lib):
    L, hydro = lib
    h = ctypes.c_void_p()
    assert L.hydro_create(None, ctypes.byref(h)) == -1
    assert L.hydro_create(None, None) == -1
    assert L.hydro_step(None, None, None, None, 1.0, 0.1, None, None, None) == -1
    assert L.hydro_totals(None, None, None, None) == -1
    assert L.hydro_sync(None) == -1
    L.hydro_destroy(None)


def test_new_entry_points_reject_null_handles(lib):
    L, hydro = lib
    assert L.hydro_tau_resync(None, None, None, None) == -1
    assert L.hydro_pack_interiors_range(None, None, None, 0, 1, None) == -1
    assert L.hydro_unpack_interiors_range(None, None, None, 0, 1, None) == -1
    assert L.hydro_diagnostics(None, None, None, None, None) == -1


def test_header_is_plain_c_and_links(lib, tmp_path):
    """The boundary is a C ABI: a C99 program includes the header with every
    warning an error, links against the library, and gets HYDRO_ERR_INVALID
    back from calls without a handle (no GPU needed)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    src = tmp_path / "abi.c"
    src.write_text(r'''
#include "hydro.h"
#include <stdio.h>
int main(void) {
  hydro_handle *h = NULL;
  int bad = 0;
  bad |= hydro_create(NULL, &h) != HYDRO_ERR_INVALID;
  bad |= hydro_sync(NULL) != HYDRO_ERR_INVALID;
  bad |= hydro_totals(NULL, NULL, NULL, NULL) != HYDRO_ERR_INVALID;
  bad |= hydro_tau_resync(NULL, NULL, NULL, NULL) != HYDRO_ERR_INVALID;
  bad |= hydro_launch_count(NULL) != 0;
  printf("%s\n", bad ? "FAIL" : "OK");
  return bad;
}
''')
    libdir = os.path.join(ROOT, "paper_2210_06437_gb300")
    exe = tmp_path / "abi"
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
           "-L", libdir, "-lhydro", "-Wl,-rpath," + libdir, "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "OK", (out.stdout, out.stderr)
