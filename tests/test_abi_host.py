"""Host-side checks that need no GPU: the C-ABI library builds for sm_103a,
loads, and exports every entry point that include/lb.h declares; the
parameter rules of the workloads reproduce the paper's numbers."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for hdr in ("lb.h", "lb3.h"):
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(lb3?_[a-z_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared_symbols()
    for required in ("lb_create_grid", "lb_init", "lb_step_fv", "lb_step_st", "lb_moments",
                     "lb_nusselt", "lb_conservation", "lb_destroy", "lb_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_1505_03271_gb300 as lb
    L = lb.load()
    for name in _declared_symbols():
        assert hasattr(L, name), name
    assert set(lb.SYMBOLS) == set(_declared_symbols())
    from paper_1505_03271_gb300 import _build
    assert "arch=compute_103a,code=sm_103a" in _build.ARCH


def test_last_error_without_gpu_work():
    import paper_1505_03271_gb300 as lb
    lb.load()
    assert isinstance(lb.lb_last_error(), str)
    assert lb.lb_kernel_launches() >= 0


def test_struct_layouts_match_header():
    """ctypes mirrors of the C structs have the C sizes (int/double/pointer)."""
    import paper_1505_03271_gb300 as lb
    assert ctypes.sizeof(lb.lb_grid_desc) == 2 * 4 + 2 * 8 + 2 * 4 + 2 * 8 + 4 * 4 + 8
    assert ctypes.sizeof(lb.lb_params) == 10 * 8
    assert ctypes.sizeof(lb.lb_init_desc) == 2 * 4 + 2 * 8 + 8 + 4 * 8


def test_rb_parameter_rule_and_table():
    from paper_1505_03271_gb300 import configs as cfg
    for Ra, H in ((1e4, 64.0), (1e8, 1024.0)):
        p = cfg.rb_params(Ra, 1.0, H)
        assert abs(cfg.rayleigh(p, H) / Ra - 1) < 1e-12
        assert abs(np.sqrt(p.beta * p.grav * (p.T_bot - p.T_top) * H) - 0.1) < 1e-12
    # Table rb (Sec. IV): both rows give Ra = 2.5e6 with nu = tau c_s^2
    fv = cfg.RBParams(0.5, 0.5, 1.325e-4, 1.0, 1.0, 2.0, 0.0)
    st = cfg.RBParams(0.05, 0.05, 1.325e-3, 1.0, 1.0, 2.0, 0.0)
    assert abs(cfg.rayleigh(fv, 640.0) / 2.5e6 - 1) < 1e-3
    assert abs(cfg.rayleigh(st, 64.0) / 2.5e6 - 1) < 1e-3


def test_workload_rules():
    from paper_1505_03271_gb300 import configs as cfg
    w = cfg.channel()
    assert w.grid["nx"] == 256 and w.grid["ny"] == 512
    assert abs(w.params["tau"] - 0.2) < 1e-15
    assert abs(w.notes["Re"] - 10.0) < 1e-12
    dmin = cfg.min_cell(512, 512.0, 1, 2.0)
    assert 0.14 < dmin < 0.16
    assert abs(w.params["dt"] - 0.9 * dmin) < 1e-15
    t = cfg.tgv64("st")
    assert t.steps == 1000 and abs(t.params["tau"] - 0.3) < 1e-15
    assert cfg.bytes_per_cell(1, False) == 72 and cfg.bytes_per_cell(2, True) == 72
    assert cfg.bytes_per_cell(0, True) == 288


def test_serving_request_recipe():
    """The serving stream: seeded, sizes from the set, Ra in [1e4, 1e8],
    Poisson arrivals with the requested mean rate."""
    from paper_1505_03271_gb300 import serving
    a = serving.make_requests(400, 20.0)
    b = serving.make_requests(400, 20.0)
    assert [(r.n, r.Ra, r.nsteps, r.arrival) for r in a] == [(r.n, r.Ra, r.nsteps, r.arrival) for r in b]
    assert {r.n for r in a} <= set(serving.SIZES)
    assert all(1e4 <= r.Ra <= 1e8 and 50 <= r.nsteps <= 1000 for r in a)
    gaps = np.diff([0.0] + [r.arrival for r in a])
    assert abs(gaps.mean() * 20.0 - 1.0) < 0.15
    for r in a[:20]:
        assert r.params["dt"] <= 0.9 * min(np.diff(__import__("paper_1505_03271_gb300.configs",
                                                               fromlist=["x"]).faces(r.n, r.n, 1, 2.0)).min(),
                                           8 * min(r.params["tau"], r.params["tau_g"])) + 1e-15


C_CALLER = r"""
#include <stdio.h>
#include <string.h>
#include "lb.h"
#include "lb3.h"

int main(void) {
    lb_grid* g = NULL;
    lb3_grid* g3 = NULL;
    int n = -1;
    if (lb_create_grid(NULL, &g) != LB_ERR_ARG || g != NULL) return 1;
    if (strstr(lb_last_error(), "NULL") == NULL) return 2;
    if (lb3_create_grid(NULL, &g3) != LB_ERR_ARG) return 3;
    if (lb_step_fv(NULL, 1) == LB_OK || lb_step_st(NULL, 1) == LB_OK) return 4;
    if (lb_set_graph_steps(NULL, 32) != LB_ERR_ARG) return 5;
    if (lb_get_graph_steps(NULL, &n, NULL) != LB_ERR_ARG || n != -1) return 6;
    if (lb_destroy(NULL) != LB_OK) return 7;
    printf("launches %llu\n", lb_kernel_launches());
    return 0;
}
"""


def test_c_caller_links_and_runs(tmp_path):
    """A C99 program includes both headers, links the library and calls its
    argument checks (no device work): the boundary is usable from C."""
    import subprocess
    import paper_1505_03271_gb300 as lb
    lib = lb.library_path()
    lb.load()
    src = tmp_path / "caller.c"
    src.write_text(C_CALLER)
    exe = tmp_path / "caller"
    libdir = os.path.dirname(lib)
    name = os.path.basename(lib)[3:-3]  # libNAME.so -> NAME
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                    str(src), "-L", libdir, "-l" + name, "-Wl,-rpath," + libdir, "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stderr)
    assert r.stdout.strip() == "launches 0"


def test_product_and_oracle_share_no_code():
    """The CUDA path and the oracle are independent: no file of the package
    imports or includes anything of oracle/, and no oracle file includes a
    header or source of the package or include/."""
    pkg = os.path.join(ROOT, "paper_1505_03271_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_lib" in dirpath or "__pycache__" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), f
                assert not re.search(r"#\s*include\s*[<\"][^>\"]*(oracle|lbref)", text), f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".c", ".h", ".py")):
            text = open(os.path.join(ROOT, "oracle", f)).read()
            assert not re.search(r"#\s*include\s*[<\"][^>\"]*(lb\.h|lb3\.h|\.cuh|csrc)", text), f
            assert not re.search(r"^\s*(import|from)\s+paper_1505_03271_gb300\b", text, re.M), f


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """With the CUDA library absent the binding raises: there is no CPU path."""
    import paper_1505_03271_gb300 as lb
    from paper_1505_03271_gb300 import _build
    monkeypatch.setattr(lb, "_lib", None)
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "libmissing.so"))
    with pytest.raises(RuntimeError, match="CUDA library missing"):
        lb.load(build=False)


def _desc2(lb, **kw):
    d = dict(nx=16, ny=16, lx=16.0, ly=16.0, sx=0, sy=0, stretch_x=0.0, stretch_y=0.0, bcx=0, bcy=0,
             thermal=0, store=1, cuda_stream=None)
    d.update(kw)
    return lb.lb_grid_desc(**d)


def _desc3(lb, **kw):
    d = dict(nx=8, ny=8, nz=8, lx=8.0, ly=8.0, lz=8.0, sx=0, sy=0, sz=0, stretch_x=0.0, stretch_y=0.0,
             stretch_z=0.0, bcx=0, bcy=0, bcz=0, thermal=0, store=1, cuda_stream=None)
    d.update(kw)
    return lb.lb3_grid_desc(**d)


BAD_2D = {
    "empty axis": dict(nx=0),
    "too many cells": dict(nx=1 << 16, ny=(1 << 15) + 1),
    "unknown boundary": dict(bcy=7),
    "wall axis of one cell": dict(ny=1, bcy=1),
    "thermal with x walls": dict(thermal=1, bcx=1, bcy=1),
    "thermal with a density axis": dict(thermal=1, bcy=2),
    "unknown storage": dict(store=9),
    "unknown spacing": dict(sy=9),
    "zero length": dict(ly=0.0),
    "tanh without stretch": dict(sy=1, bcy=1),
    "sinh on an odd count": dict(ny=15, sy=2, stretch_y=2.0, bcy=1),
}

BAD_3D = {
    "empty axis": dict(nz=0),
    "density axis": dict(bcz=2),
    "wall axis of one cell": dict(nz=1, bcz=1),
    "16-bit storage": dict(store=2),
    "thermal with side walls": dict(thermal=1, bcx=1, bcz=1),
    "sinh on an odd count": dict(nz=9, sz=2, stretch_z=2.0, bcz=1),
    "zero length": dict(lx=0.0),
    "nz too large": dict(nx=1, ny=1, nz=70000),
}


@pytest.mark.parametrize("case", sorted(BAD_2D))
def test_create_grid_rejects_bad_descriptions(case):
    """Grid descriptions the method or the kernels cannot take are refused
    with LB_ERR_ARG and a message, before any device work."""
    import paper_1505_03271_gb300 as lb
    L = lb.load()
    h = ctypes.c_void_p()
    L.lb_set_graph_steps(None, 2)  # leaves "grid is NULL" as the last message
    assert L.lb_create_grid(ctypes.byref(_desc2(lb, **BAD_2D[case])), ctypes.byref(h)) == lb.LB_ERR_ARG
    assert not h.value and lb.lb_last_error() not in ("", "grid is NULL")


@pytest.mark.parametrize("case", sorted(BAD_3D))
def test_create_grid3_rejects_bad_descriptions(case):
    import paper_1505_03271_gb300 as lb
    L = lb.load()
    h = ctypes.c_void_p()
    L.lb_set_graph_steps(None, 2)
    assert L.lb3_create_grid(ctypes.byref(_desc3(lb, **BAD_3D[case])), ctypes.byref(h)) == lb.LB_ERR_ARG
    assert not h.value and lb.lb_last_error() not in ("", "grid is NULL")


def _declared_arities():
    out = {}
    for hdr in ("lb.h", "lb3.h"):
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for name, params in re.findall(r"\b(lb3?_[a-z_]+)\s*\(([^)]*)\)\s*;", text):
            params = params.strip()
            out[name] = 0 if params in ("", "void") else len(params.split(","))
    return out


def test_binding_signatures_match_headers():
    """The ctypes binding declares, for every entry point, as many argument
    types as the header has parameters (a mismatch would marshal garbage)."""
    import paper_1505_03271_gb300 as lb
    L = lb.load()
    arity = _declared_arities()
    assert set(arity) == set(lb.SYMBOLS)
    for name, n in arity.items():
        assert len(getattr(L, name).argtypes or []) == n, name


def _declared_param_types():
    out = {}
    for hdr in ("lb.h", "lb3.h"):
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for name, params in re.findall(r"\b(lb3?_[a-z_]+)\s*\(([^)]*)\)\s*;", text):
            ps = [p.strip() for p in params.split(",")]
            out[name] = [] if ps in ([""], ["void"]) else \
                [re.sub(r"\bconst\b", "", re.sub(r"\b[A-Za-z_0-9]+$", "", p)).replace(" ", "") for p in ps]
    return out


def _compatible(ctype_decl, ctype):
    """Whether a ctypes argument type marshals the C parameter type."""
    scalars = {"int": ctypes.c_int, "double": ctypes.c_double, "unsignedlonglong": ctypes.c_ulonglong}
    if ctype_decl in scalars:
        return ctype is scalars[ctype_decl]
    assert ctype_decl.endswith("*"), ctype_decl
    pointee = ctype_decl[:-1]
    if ctype is ctypes.c_void_p:
        return True  # opaque handles, device buffers
    if not hasattr(ctype, "_type_") or not issubclass(ctype, ctypes._Pointer):
        return False
    target = ctype._type_
    simple = {"double": ctypes.c_double, "float": ctypes.c_float, "int": ctypes.c_int,
              "unsignedlonglong": ctypes.c_ulonglong}
    if pointee in simple:
        return target is simple[pointee]
    if pointee.endswith("*"):  # handle out-parameter
        return target is ctypes.c_void_p
    return target.__name__ == pointee  # struct pointers: the mirror class of the same name


def test_binding_types_match_headers():
    """Each ctypes argument type marshals the header's parameter type:
    int/double/unsigned long long exactly, pointers to the same scalar or
    struct, opaque handles as void pointers."""
    import paper_1505_03271_gb300 as lb
    L = lb.load()
    for name, decl in _declared_param_types().items():
        for k, (cdecl, ct) in enumerate(zip(decl, getattr(L, name).argtypes or [])):
            assert _compatible(cdecl, ct), (name, k, cdecl, ct)
