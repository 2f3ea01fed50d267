"""The C-ABI library builds, loads on a machine without a GPU, and exports
every entry point include/mgpbd.h declares (no compute call is made here)."""
import ctypes as C
import os
import re

import pytest

from paper_2505_13390_gb300 import build as B
from paper_2505_13390_gb300 import mgpbd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    txt = open(os.path.join(ROOT, "include", "mgpbd.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return set(re.findall(r"\b(mgpbd_\w+)\s*\(", txt))


def test_library_exports_every_declared_symbol():
    path = B.build()
    lib = C.CDLL(path)
    names = declared()
    assert len(names) >= 25
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert names == set(mgpbd.SIGNATURES), "binding and header disagree"


def test_default_params_and_host_only_calls():
    lib = mgpbd.load()
    p = mgpbd.Params()
    assert lib.mgpbd_default_params(C.byref(p)) == 0
    assert (p.theta_s, p.smooth_sweeps, p.lambda_min_est, p.coarse_max) == (0.1, 2, 0.1, 400)
    assert lib.mgpbd_default_params(None) == mgpbd.E_INVALID
    # argument checks that return before any CUDA call
    h = C.c_void_p()
    assert lib.mgpbd_create(None, C.byref(p), None, C.byref(h)) == mgpbd.E_INVALID
    assert not h.value
    assert lib.mgpbd_step(None, 1) == mgpbd.E_INVALID
    # a caller workspace that is NULL, misaligned or too small is refused on the host
    for ws, nbytes in ((None, 1 << 20), (0x1000 + 16, 1 << 20), (0x1000, 16)):
        h = C.c_void_p()
        assert lib.mgpbd_create_in_workspace(None, C.byref(p), ws, nbytes, None,
                                             C.byref(h)) == mgpbd.E_INVALID
        assert not h.value
    assert lib.mgpbd_create_in_workspace(None, C.byref(p), 0x1000, 1 << 20, None,
                                         None) == mgpbd.E_INVALID
    assert isinstance(lib.mgpbd_last_error(), bytes)


def test_workspace_size_is_host_only_and_grows_with_the_mesh():
    """mgpbd_workspace_size needs no device: it sizes an instance from its mesh."""
    from paper_2505_13390_gb300 import mgpbd
    from paper_2505_13390_gb300.meshgen import cloth, default_params, hex_block
    p = default_params()
    small = mgpbd.workspace_size(cloth(8, plane="xz"), p)
    big = mgpbd.workspace_size(cloth(32, plane="xz"), p)
    beam = mgpbd.workspace_size(hex_block(10, 4, 4, h=0.01), p)
    assert 0 < small < big and beam > big
    bad = cloth(8, plane="xz")
    bad.dist = bad.dist.copy()
    bad.dist[0, 0] = bad.n_verts  # out of range
    with pytest.raises(mgpbd.MgpbdError):
        mgpbd.workspace_size(bad, p)


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every ctypes mirror in the binding has the size and field offsets that
    a C compiler gives the header's struct (a mismatch would corrupt memory)."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    pairs = {"mgpbd_mesh_desc": mgpbd.MeshDesc, "mgpbd_params": mgpbd.Params,
             "mgpbd_solve_info": mgpbd.SolveInfo, "mgpbd_stats_t": mgpbd.Stats,
             "mgpbd_level_info": mgpbd.LevelInfo, "mgpbd_batch_config": mgpbd.BatchConfig,
             "mgpbd_step_request": mgpbd.StepRequest, "mgpbd_step_result": mgpbd.StepResult}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mgpbd.h"', 'int main(void) {']
    for cname, py in pairs.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True,
                               check=True).stdout.splitlines():
        cname, field, val = line.split()
        got[(cname, field)] = int(val)
    for cname, py in pairs.items():
        assert got[(cname, "sizeof")] == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_missing_library_fails_loudly():
    """No CPU fallback: without libmgpbd.so the binding raises on first use."""
    import subprocess
    import sys
    code = ("from paper_2505_13390_gb300 import mgpbd\n"
            "try:\n"
            "    mgpbd.load('/nonexistent/libmgpbd.so')\n"
            "except ImportError as e:\n"
            "    print('raised', e)\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("raised") and "missing" in r.stdout
