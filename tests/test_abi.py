"""The C-ABI library builds, loads and exports every entry point that
include/csph.h declares; host-side argument checks reject bad calls before
any device work (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1805_05128_gb300 import build
    build.build()
    from paper_1805_05128_gb300 import abi
    return abi


def _declared():
    src = open(os.path.join(ROOT, "include", "csph.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^(?:int|void|const char\s*\*)\s*(\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("sph_init", "sph_build_cells", "sph_step", "voronoi_assign", "voronoi_balance",
                     "sph_conservation", "sph_read_status", "sph_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    L = lib.lib()
    for name in _declared():
        assert hasattr(L, name), name
    assert set(_declared()) == set(lib.EXPORTS)


def test_struct_layouts_match_header(lib, tmp_path):
    """The ctypes mirrors have the sizes and field offsets that a C compiler
    gives the structs of include/csph.h."""
    import subprocess
    prog = tmp_path / "layout.c"
    fields = {"sph_params": ["dim", "kappa", "cell_cap", "mat", "n_units", "pair_blocks_per_sm", "theta", "generators", "materials", "order", "solver", "load_measure", "list_cap", "unit_sched", "list_staging"],
              "sph_state": ["n", "x", "mat", "ax", "d", "id", "unit"],
              "sph_material": ["eos", "gamma", "s_a"]}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "csph.h"', "int main(void){"]
    for st, fs in fields.items():
        lines.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for f in fs:
            lines.append(f'printf("{st}.{f} %zu\\n", offsetof({st}, {f}));')
    lines.append("return 0;}")
    prog.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    out = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for st, fs in fields.items():
        cls = getattr(lib, st)
        assert C.sizeof(cls) == int(out[st]), st
        for f in fs:
            assert getattr(cls, f).offset == int(out[f"{st}.{f}"]), f"{st}.{f}"
    assert C.sizeof(lib.sph_balance_params) == 32


def _valid_params(lib):
    p = lib.sph_params()
    p.dim, p.kernel, p.precision, p.n_mat = 3, lib.SPH_KERNEL_CUBIC, lib.SPH_PREC_MIXED, 1
    p.kappa, p.eta, p.cfl, p.cell_beta, p.cell_cap = 2.0, 1.3, 0.3, 0.0, 1 << 20
    p.mat[0].eos, p.mat[0].gamma = lib.SPH_EOS_IDEAL, 1.4
    return p


def _fake_state(lib, n=10):
    s = lib.sph_state()
    s.n = n
    for k in lib.STATE_F64 + lib.STATE_RATES + lib.STATE_DERIVED:
        setattr(s, k, 0x1000)   # never dereferenced: the checks below fail first
    return s


@pytest.mark.parametrize("mutate,code", [
    (lambda p: setattr(p, "dim", 4), 1),
    (lambda p: setattr(p, "kernel", 7), 1),
    (lambda p: setattr(p, "precision", 3), 1),
    (lambda p: setattr(p, "n_mat", 0), 1),
    (lambda p: setattr(p, "eta", -1.0), 1),
    (lambda p: setattr(p, "n_units", 300), 1),
    (lambda p: setattr(p, "cell_cap", 0), 1),
    (lambda p: setattr(p, "solver", 2), 1),
    (lambda p: setattr(p, "load_measure", 2), 1),
    (lambda p: setattr(p, "order", 3), 1),
    (lambda p: setattr(p, "list_cap", 16), 1),
    (lambda p: setattr(p, "unit_sched", 3), 1),
    (lambda p: setattr(p, "list_staging", 2), 1),
    (lambda p: setattr(p.mat[0], "eos", 5), 1),
    (lambda p: (setattr(p.mat[0], "eos", 4), setattr(p.mat[0], "c0", 0.0)), 1),
])
def test_init_rejects_bad_parameters(lib, mutate, code):
    L = lib.lib()
    p = _valid_params(lib)
    mutate(p)
    h = C.c_void_p()
    offs = (C.c_int64 * 2)(0, 10)
    rc = L.sph_init(C.byref(h), C.byref(p), 1, offs, C.byref(_fake_state(lib)), None)
    assert rc == code and not h.value
    assert L.sph_last_error(None)


def test_init_rejects_bad_instances(lib):
    L = lib.lib()
    p = _valid_params(lib)
    h = C.c_void_p()
    offs = (C.c_int64 * 3)(0, 6, 6)          # empty second instance
    assert L.sph_init(C.byref(h), C.byref(p), 2, offs, C.byref(_fake_state(lib)), None) == lib.SPH_ERR_INVALID
    offs = (C.c_int64 * 2)(0, 9)             # does not end at n
    assert L.sph_init(C.byref(h), C.byref(p), 1, offs, C.byref(_fake_state(lib)), None) == lib.SPH_ERR_INVALID
    s = _fake_state(lib)
    s.vz = None                               # dim 3 needs z components
    offs = (C.c_int64 * 2)(0, 10)
    assert L.sph_init(C.byref(h), C.byref(p), 1, offs, C.byref(s), None) == lib.SPH_ERR_INVALID
    s = _fake_state(lib, n=1 << 26)
    offs = (C.c_int64 * 2)(0, 1 << 26)
    assert L.sph_init(C.byref(h), C.byref(p), 1, offs, C.byref(s), None) == lib.SPH_ERR_CAPACITY


def test_null_handle_calls_are_rejected(lib):
    L = lib.lib()
    st = C.c_int(0)
    assert L.sph_read_status(None, C.byref(st)) == lib.SPH_ERR_INVALID
    assert L.sph_step(None, None, 1, None, None) == lib.SPH_ERR_INVALID
    L.sph_destroy(None)
