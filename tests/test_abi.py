"""CPU checks of the C-ABI library: it builds, loads and exports exactly the
entry points that include/*.h declare (no compute call: no GPU here)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in sorted(os.listdir(os.path.join(ROOT, "include")))
           if h.endswith(".h")]


def _declared():
    txt = "".join(open(h).read() for h in HEADERS)
    return sorted(set(re.findall(r"POT_API\s+[\w\s\*]+?\b(\w+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2601_17196_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    return b.LIB


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("aspot_solve", "sinkhorn_pot_solve", "pot_round", "pot_objective", "pot_workspace_size",
                 "pot_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    public = {s for s in exported if not s.startswith("_")}
    assert set(_declared()) == public


def test_library_loads_through_ctypes(libpath):
    import paper_2601_17196_gb300 as pkg
    L = pkg.lib()
    for name in _declared():
        assert hasattr(L, name)
    assert L.pot_last_error() in (b"",)


def test_argument_checks_run_before_any_launch(libpath):
    """Invalid problems are rejected on the host (no GPU needed)."""
    import ctypes as ct
    from paper_2601_17196_gb300 import binding as B
    L = B.lib()
    p = B._Problem()
    p.n, p.m, p.kind = 0, 5, 0
    b = ct.c_size_t(0)
    assert L.pot_workspace_size(ct.byref(p), None, ct.byref(b)) == 1
    assert b"n and m" in L.pot_last_error()
    p.n, p.m, p.kind, p.s = 4, 5, 0, 0.5
    p.r, p.c, p.C, p.ldc = 8, 8, 8, 3          # ldc < m
    assert L.pot_workspace_size(ct.byref(p), None, ct.byref(b)) == 1
    p.ldc = 5
    assert L.pot_workspace_size(ct.byref(p), None, ct.byref(b)) == 0 and b.value > 0
    p.kind = 7
    assert L.pot_workspace_size(ct.byref(p), None, ct.byref(b)) == 1


def test_binding_lists_every_declared_symbol():
    from paper_2601_17196_gb300 import binding as B
    assert sorted(B.EXPORTED) == _declared()


def test_warm_start_argument_checks(libpath):
    """The warm-start entry points reject bad arguments on the host."""
    import ctypes as ct
    import numpy as np
    from paper_2601_17196_gb300 import binding as B
    L = B.lib()
    n = ct.c_int64(0)
    assert L.pot_ws_param_count(0, ct.byref(n)) == 1
    assert L.pot_ws_param_count(2, ct.byref(n)) == 0
    H, F = 128, 7
    assert n.value == H * F + H + H * H + H * (H + 2) + H + H + 1
    s = B._WsSet()
    off = np.array([0, 5, 5], dtype=np.int64)          # second instance empty
    s.count, s.d, s.off, s.feats, s.extra = 2, 2, off.ctypes.data_as(ct.c_void_p), 8, 8
    b = ct.c_size_t(0)
    assert L.pot_ws_workspace_size(ct.byref(s), 4, ct.byref(b)) == 1
    assert b"no points" in L.pot_last_error()
    off[2] = 9
    assert L.pot_ws_workspace_size(ct.byref(s), 4, ct.byref(b)) == 0 and b.value > 0
    s.d = 7
    assert L.pot_ws_workspace_size(ct.byref(s), 4, ct.byref(b)) == 1
    s.d = 2
    idx = np.array([0, 2], dtype=np.int32)               # 2 is out of range
    assert L.pot_ws_forward(ct.byref(s), idx.ctypes.data_as(ct.c_void_p), 2, 8, 0, 8, 256, b.value, None) == 1
    assert b"out of range" in L.pot_last_error()
    idx[1] = 1
    assert L.pot_ws_forward(ct.byref(s), idx.ctypes.data_as(ct.c_void_p), 2, 8, 5, 8, 256, b.value, None) == 1
    assert b"mode" in L.pot_last_error()
    assert L.pot_ws_gradient(ct.byref(s), idx.ctypes.data_as(ct.c_void_p), 2, 8, 0, 8, 8, 256, b.value, None) == 1
    assert b"target" in L.pot_last_error()


def _fake_batch(B, sizes, kind=3, d=3):
    """Host-side problem structs (placeholder device pointers: the autotune
    cache calls only read sizes and validate arguments)."""
    import ctypes as ct
    arr = (B._Problem * len(sizes))()
    for k, (n, m) in enumerate(sizes):
        p = arr[k]
        p.n, p.m, p.kind, p.d, p.ldx, p.ldy, p.s = n, m, kind, d, d, d, 0.5
        p.X, p.Y, p.r, p.c = 16, 16, 16, 16
    return arr


def test_autotune_cache_calls(libpath, tmp_path):
    """Pin / look up / save / clear / load of the batched pass's tile shapes
    (host only), and the argument checks."""
    import ctypes as ct
    from paper_2601_17196_gb300 import binding as B
    L = B.lib()
    assert L.pot_autotune_clear() == 0
    a = _fake_batch(B, [(100, 120), (64, 2048)])
    b = _fake_batch(B, [(100, 121), (64, 2048)])
    h, w = ct.c_int32(-1), ct.c_int32(-1)
    assert L.pot_autotune_lookup(a, 2, ct.byref(h), ct.byref(w)) == 0 and (h.value, w.value) == (0, 0)
    assert L.pot_autotune_set(a, 2, 64, 128) == 0
    assert L.pot_autotune_set(b, 2, 256, 256) == 0
    assert L.pot_autotune_lookup(a, 2, ct.byref(h), ct.byref(w)) == 0 and (h.value, w.value) == (64, 128)
    assert L.pot_autotune_lookup(b, 2, ct.byref(h), ct.byref(w)) == 0 and (h.value, w.value) == (256, 256)
    for bad in ((48, 128), (64, 64), (0, 256), (512, 256)):
        assert L.pot_autotune_set(a, 2, *bad) == 1
    assert L.pot_autotune_set(_fake_batch(B, [(100, 120)], d=5), 1, 32, 256) == 1      # d > 4: not batched
    path = str(tmp_path / "tiles.txt")
    assert L.pot_autotune_save(path.encode()) == 0
    lines = open(path).read().split("\n")
    assert len([ln for ln in lines if ln]) == 2
    assert L.pot_autotune_clear() == 0
    assert L.pot_autotune_lookup(a, 2, ct.byref(h), ct.byref(w)) == 0 and h.value == 0
    assert L.pot_autotune_load(path.encode()) == 0
    assert L.pot_autotune_lookup(b, 2, ct.byref(h), ct.byref(w)) == 0 and (h.value, w.value) == (256, 256)
    bad = tmp_path / "bad.txt"
    bad.write_text("k3_d3_c1_N5_M5_n5_m5 48 256\n")
    assert L.pot_autotune_load(str(bad).encode()) == 1
    bad.write_text("k3_d3_c1_N5_M5_n5_m5 32\n")
    assert L.pot_autotune_load(str(bad).encode()) == 1
    assert L.pot_autotune_load(str(tmp_path / "missing.txt").encode()) == 1
    assert L.pot_autotune_lookup(a, 2, ct.byref(h), ct.byref(w)) == 0 and (h.value, w.value) == (64, 128)
    assert L.pot_autotune_clear() == 0


def test_headers_are_plain_c99():
    """Every public header compiles on its own as C99 (the boundary has no C++
    or CUDA types)."""
    import shutil
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    for h in HEADERS:
        r = subprocess.run([cc, "-fsyntax-only", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-x", "c",
                            "-I", os.path.join(ROOT, "include"), h], capture_output=True, text=True)
        assert r.returncode == 0 and not r.stderr.strip(), (h, r.stderr)


C_PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "aspot.h"
#include "registration.h"
#include "warmstart.h"
int main(void) {
  pot_problem p;
  size_t bytes = 0;
  int64_t np = 0;
  memset(&p, 0, sizeof(p));
  p.n = 0; p.m = 5;                                   /* invalid: rejected on the host */
  if (pot_workspace_size(&p, NULL, &bytes) != POT_EINVAL) return 1;
  if (strlen(pot_last_error()) == 0) return 2;
  if (pot_autotune_clear() != POT_OK) return 3;
  if (pot_ws_param_count(2, &np) != POT_OK || np <= 0) return 4;
  if (pot_rigid_workspace_size(4, &bytes) != POT_OK || bytes == 0) return 5;
  printf("ok %lld\n", (long long)np);
  return 0;
}
"""


def test_c_program_links_and_calls_the_library(libpath, tmp_path):
    """A plain C program includes the headers, links the shared library and
    calls host-side entry points (argument checks, the autotune cache, sizes)."""
    import shutil
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "probe.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "probe"
    libdir = os.path.dirname(libpath)
    name = os.path.basename(libpath)
    r = subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                        os.path.join(libdir, name), "-Wl,-rpath," + libdir], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.startswith("ok"), (r.returncode, r.stdout, r.stderr)
