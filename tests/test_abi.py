"""Host-side checks of the C ABI (no GPU needed).

- librosen.so builds for sm_103a and exports every function include/rosen.h
  declares;
- the ctypes structures of the binding have the C layout;
- argument validation returns ROSEN_EINVAL / ROSEN_ENOMEM before any CUDA
  call is made, so it is exercised here without a device.
"""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1704_04381_gb300 import build as pkg_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


@pytest.fixture(scope="module")
def rosen():
    pkg_build.build()
    from paper_1704_04381_gb300 import rosen as r
    r.load()
    return r


def declared_functions():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(rosen_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(rosen):
    names = declared_functions()
    assert "rosen_lattice_grow" in names and "rosen_reduce" in names
    out = subprocess.run(["nm", "-D", "--defined-only", rosen.library_path()],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (rosen_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    # Nothing but the ABI leaks out of the library.
    extra = [n for n in exported if n not in names]
    assert not extra, extra


def test_struct_layout_matches_c(rosen, tmp_path):
    structs = {
        "rosen_lattice_params": rosen.rosen_lattice_params,
        "rosen_lattice_out": rosen.rosen_lattice_out,
        "rosen_reduce_in": rosen.rosen_reduce_in,
        "rosen_offlattice_params": rosen.rosen_offlattice_params,
        "rosen_offlattice_out": rosen.rosen_offlattice_out,
        "rosen_ensemble": rosen.rosen_ensemble,
        "rosen_serve_config": rosen.rosen_serve_config,
        "rosen_request": rosen.rosen_request,
        "rosen_result": rosen.rosen_result,
        "rosen_serve_counters": rosen.rosen_serve_counters,
        "rosen_perm_params": rosen.rosen_perm_params,
        "rosen_perm_out": rosen.rosen_perm_out,
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rosen.h"', "int main(void){"]
    for name, cls in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for fname, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, fname, name, fname))
    lines.append('printf("rosen_stats %zu\\n", sizeof(rosen_stats));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert int(got["%s.%s" % (name, fname)]) == getattr(cls, fname).offset, (name, fname)
    assert int(got["rosen_stats"]) == 8 * len(rosen.STAT_KEYS)


def _grow(rosen, **kw):
    p = rosen.lattice_params(**{**dict(seed=1, N=16, C=10), **kw})
    o = rosen.rosen_lattice_out()
    return rosen.load().rosen_lattice_grow(ctypes.byref(p), ctypes.byref(o), None)


@pytest.mark.parametrize("kw", [
    dict(N=1), dict(N=513), dict(C=-1), dict(chain0=-5), dict(chain0=2 ** 32 - 5, C=10),
    dict(beta_eps=-0.1), dict(beta_eps=float("nan")), dict(beta_eps=float("inf")),
    dict(beta_eps=16.5),
    dict(flags=8), dict(flags=1), dict(flags=2), dict(lanes_per_chain=3),
    dict(max_attempts=-1), dict(max_attempts=65536),
])
def test_lattice_rejects_bad_parameters(rosen, kw):
    assert _grow(rosen, **kw) == rosen.ROSEN_EINVAL
    assert rosen.last_error() != ""


def test_long_lattice_validation(rosen):
    L = rosen.load()
    assert rosen.rosen_lattice_long_workspace_size(1, 10) == 0
    assert rosen.rosen_lattice_long_workspace_size(32769, 10) == 0
    assert rosen.rosen_lattice_long_workspace_size(1000, 0) == 0
    # A 256-byte header (the chain counter), then min(C, 131072) tables;
    # N + 1 = 1001 -> 1024 entries of 16 bytes per table.
    assert rosen.rosen_lattice_long_workspace_size(1000, 10) == 256 + 10 * 1024 * 16
    assert rosen.rosen_lattice_long_workspace_size(2, 10 ** 9) == 256 + (1 << 17) * 64 * 16

    def grow_long(ws, nbytes, **kw):
        p = rosen.lattice_params(**{**dict(seed=1, N=1000, C=10), **kw})
        o = rosen.rosen_lattice_out()
        return L.rosen_lattice_grow_long(ctypes.byref(p), ctypes.byref(o), ws, nbytes, None)

    assert grow_long(4096, 1 << 20, N=1) == rosen.ROSEN_EINVAL
    assert grow_long(4096, 1 << 20, N=32769) == rosen.ROSEN_EINVAL
    assert grow_long(4096, 1 << 20, beta_eps=-1.0) == rosen.ROSEN_EINVAL
    assert grow_long(None, 1 << 20) == rosen.ROSEN_EINVAL
    assert grow_long(4100, 1 << 20) == rosen.ROSEN_EINVAL
    assert grow_long(4104, 1 << 20) == rosen.ROSEN_EINVAL
    assert grow_long(4096, 1024 * 16 - 1) == rosen.ROSEN_ENOMEM
    assert "rosen_lattice_grow_long" in rosen.last_error()
    assert grow_long(4096, 1 << 20, C=0) == rosen.ROSEN_OK


def test_long_offlattice_validation(rosen):
    L = rosen.load()
    assert rosen.rosen_offlattice_long_workspace_size(1, 10) == 0
    assert rosen.rosen_offlattice_long_workspace_size(16385, 10) == 0
    assert rosen.rosen_offlattice_long_workspace_size(1000, 0) == 0
    # A 256-byte header (the chain counter), then min(C, 9728) slots.
    slot = rosen.rosen_offlattice_long_workspace_size(1000, 1) - 256
    assert slot % 16 == 0 and slot > 1000 * 4 * 16
    assert rosen.rosen_offlattice_long_workspace_size(1000, 10) == 256 + 10 * slot
    assert rosen.rosen_offlattice_long_workspace_size(1000, 10 ** 9) == 256 + 9728 * slot

    def grow_long(ws, nbytes, **kw):
        p = rosen.offlattice_params(**{**dict(seed=1, N=1000, C=10, k=32), **kw})
        o = rosen.rosen_offlattice_out()
        return L.rosen_offlattice_grow_long(ctypes.byref(p), ctypes.byref(o), ws, nbytes, None)

    assert grow_long(4096, 1 << 30, N=1) == rosen.ROSEN_EINVAL
    assert grow_long(4096, 1 << 30, N=16385) == rosen.ROSEN_EINVAL
    assert grow_long(4096, 1 << 30, k=0) == rosen.ROSEN_EINVAL
    assert grow_long(4096, 1 << 30, lanes_per_chain=8, k=8) == rosen.ROSEN_EINVAL
    assert "16 or 32" in rosen.last_error()
    assert grow_long(None, 1 << 30) == rosen.ROSEN_EINVAL
    assert grow_long(4104, 1 << 30) == rosen.ROSEN_EINVAL
    assert grow_long(4096, 1 << 30, C=0) == rosen.ROSEN_OK


def test_lattice_empty_launch_is_a_no_op(rosen):
    assert _grow(rosen, C=0) == rosen.ROSEN_OK


def test_misaligned_counts_rejected(rosen):
    p = rosen.lattice_params(seed=1, N=8, C=4)
    o = rosen.rosen_lattice_out(counts=8)
    assert rosen.load().rosen_lattice_grow(ctypes.byref(p), ctypes.byref(o), None) == \
        rosen.ROSEN_EINVAL


def test_reduce_validation(rosen):
    L = rosen.load()
    inp = rosen.rosen_reduce_in(kind=rosen.ROSEN_REDUCE_LATTICE, N=8, k=0, use_counts=0, C=0)
    assert L.rosen_reduce(ctypes.byref(inp), 1024, 2048, 1 << 20, None) == rosen.ROSEN_EINVAL
    inp.C = 100
    assert L.rosen_reduce(ctypes.byref(inp), 1024, 2048, 1 << 20, None) == rosen.ROSEN_EINVAL
    inp.logw, inp.r2_i, inp.n2rg2 = 4096, 8192, 16384
    need = rosen.rosen_reduce_workspace_size(100)
    assert need > 0
    assert L.rosen_reduce(ctypes.byref(inp), 1024, 2048, need - 1, None) == rosen.ROSEN_ENOMEM
    inp.kind = 7
    assert L.rosen_reduce(ctypes.byref(inp), 1024, 2048, need, None) == rosen.ROSEN_EINVAL
    assert rosen.rosen_reduce_workspace_size(10 ** 7) >= (10 ** 7 // 2048) * 96


def test_philox_validation(rosen):
    L = rosen.load()
    assert L.rosen_philox(1, 0, 0, 0, 2 ** 32 - 1, 2, 4096, None) == rosen.ROSEN_EINVAL
    assert L.rosen_philox(1, 0, 0, 0, 0, 4, 4100, None) == rosen.ROSEN_EINVAL
    assert L.rosen_philox(1, 0, 0, 0, 0, 0, None, None) == rosen.ROSEN_OK


def test_status_strings(rosen):
    assert rosen.status_string(rosen.ROSEN_OK) == "ROSEN_OK"
    assert rosen.status_string(rosen.ROSEN_ETIMEOUT) == "ROSEN_ETIMEOUT"
    assert "sm_103a" in rosen.version()


def _grow_off(rosen, **kw):
    p = rosen.offlattice_params(**{**dict(seed=1, N=16, C=10, k=32), **kw})
    o = rosen.rosen_offlattice_out()
    return rosen.load().rosen_offlattice_grow(ctypes.byref(p), ctypes.byref(o), None)


@pytest.mark.parametrize("kw", [
    dict(N=1), dict(N=1025), dict(k=0), dict(k=129), dict(C=-1), dict(chain0=2 ** 32),
    dict(potential=2), dict(sigma=-1.0), dict(sigma=float("nan")), dict(sigma=5.0),
    dict(potential=1, cutoff=0.0), dict(potential=1, cutoff=9.0), dict(potential=1, sigma=0.0),
    dict(beta_eps=-1.0), dict(beta_eps=float("inf")), dict(flags=4), dict(flags=1),
    dict(lanes_per_chain=7), dict(lanes_per_chain=8, k=33),
    dict(max_attempts=-1), dict(max_attempts=1 << 16),
])
def test_offlattice_rejects_bad_parameters(rosen, kw):
    assert _grow_off(rosen, **kw) == rosen.ROSEN_EINVAL
    assert rosen.last_error() != ""


def test_offlattice_empty_launch_is_a_no_op(rosen):
    assert _grow_off(rosen, C=0) == rosen.ROSEN_OK


@pytest.mark.parametrize("bad", [
    dict(model=2), dict(N=1), dict(C=0), dict(model=0, N=40000), dict(model=1, N=20000),
    dict(model=1, k=0),
    dict(model=1, potential=5), dict(beta_eps=-1.0), dict(max_attempts=-2),
    dict(model=0, max_attempts=70000),
])
def test_batch_rejects_bad_ensembles(rosen, bad):
    good = dict(model=1, N=16, C=100, seed=1, k=16, potential=1, beta_eps=0.5)
    ens = [rosen.ensemble(**good), rosen.ensemble(**{**good, **bad})]
    arr = (rosen.rosen_ensemble * 2)(*ens)
    h = ctypes.c_void_p()
    assert rosen.load().rosen_batch_create(arr, 2, ctypes.byref(h)) == rosen.ROSEN_EINVAL
    assert "ensemble 1" in rosen.last_error()


def _perm(rosen, ws=4096, nbytes=None, out=None, **kw):
    p = rosen.perm_params(**{**dict(seed=1, N=16, M0=100, max_population=400), **kw})
    o = out or rosen.rosen_perm_out(population=4096, logz=8192, final_n=12288)
    if nbytes is None:
        nbytes = rosen.load().rosen_perm_workspace_size(p.N, p.max_population)
    return rosen.load().rosen_perm_run(ctypes.byref(p), ctypes.byref(o), ws, nbytes, None)


@pytest.mark.parametrize("kw", [
    dict(N=1), dict(N=513), dict(M0=0), dict(max_population=50), dict(max_population=(1 << 24) + 1),
    dict(beta_eps=-0.5), dict(beta_eps=float("nan")), dict(mu=0.0), dict(mu=float("inf")),
    dict(c_hi=0.5, c_lo=0.5), dict(c_lo=-1.0), dict(c_lo=float("inf"), c_hi=float("inf")),
    dict(flags=1), dict(flags=2),
])
def test_perm_rejects_bad_parameters(rosen, kw):
    # Host-side validation before any CUDA call (flags=2 asks for coordinates
    # without an array).
    assert _perm(rosen, **kw) == rosen.ROSEN_EINVAL
    assert "rosen_perm_run" in rosen.last_error()


def test_perm_workspace_and_outputs(rosen):
    L = rosen.load()
    assert L.rosen_perm_workspace_size(1, 100) == 0
    assert L.rosen_perm_workspace_size(16, 0) == 0
    assert L.rosen_perm_workspace_size(16, (1 << 24) + 1) == 0
    n = L.rosen_perm_workspace_size(64, 10 ** 6)
    # one storage slot of keys (4 N bytes per chain) plus slot numbers,
    # weights, the free-slot stack and scans
    assert 4 * 64 * 10 ** 6 < n < (4 * 64 + 64) * 10 ** 6
    # an odd N rounds each half slot up to whole 16-byte words
    assert L.rosen_perm_workspace_size(65, 1024) >= 1024 * (4 * 2 * 36)
    assert _perm(rosen, nbytes=L.rosen_perm_workspace_size(16, 400) - 1) == rosen.ROSEN_ENOMEM
    assert _perm(rosen, ws=4096 + 16) == rosen.ROSEN_EINVAL          # 256-byte alignment
    missing = rosen.rosen_perm_out(population=4096, logz=None, final_n=12288)
    assert _perm(rosen, out=missing) == rosen.ROSEN_EINVAL
