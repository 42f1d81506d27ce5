"""Host-side checks of the C-ABI library (no GPU needed).

The shared library must load and export every function declared in
include/*.h; argument validation that happens before any device work must
return the documented error codes.
"""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from conftest import build_library
    build_library()
    import paper_2511_21640_gb300 as m
    return m


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            with open(os.path.join(ROOT, "include", fn)) as fh:
                txt = fh.read()
            names |= set(re.findall(r"\b(adc_[a-z0-9_]+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert {"adc_init", "adc_sigma", "adc_davidson", "adc_fns_density", "adc_free"} <= names
    raw = ctypes.CDLL(lib.LIB_PATH)
    for n in sorted(names):
        assert hasattr(raw, n), n


def test_error_strings_and_defaults(lib):
    for code in range(0, -9, -1):
        s = lib.lib.adc_strerror(code).decode()
        assert s.startswith("ADC_")
    o = lib.adc_opts()
    assert lib.lib.adc_opts_default(ctypes.byref(o)) == 0
    assert o.precision == 0 and abs(o.herm_tol - 1e-12) < 1e-30 and o.stream is None
    assert lib.lib.adc_dims(None, None, None) == -7
    assert lib.lib.adc_sigma(None, None, None, 1, 0) == -7
    assert lib.lib.adc_opts_default(None) == -1


@pytest.mark.parametrize("kind,order,nocc,nvir,code", [
    (2, 4, 3, 5, -1),   # EE, bad order
    (7, 3, 3, 5, -1),   # unknown kind
    (0, 4, 3, 5, -1),   # bad order
    (0, 3, 1, 5, -1),   # IP needs two occupied spinors
    (1, 2, 3, 1, -1),   # EA needs two virtual spinors
])
def test_init_rejects_bad_arguments_before_device_work(lib, kind, order, nocc, nvir, code):
    nmo = nocc + nvir
    B = np.zeros((2, nmo, nmo), np.complex128)
    eo = -np.ones(nocc)
    ev = np.ones(nvir)
    h = ctypes.c_void_p()
    rc = lib.lib.adc_init(ctypes.byref(h), B.ctypes.data, 2, eo.ctypes.data, nocc, ev.ctypes.data, nvir,
                          kind, order, 1.0, None)
    assert rc == code
    assert not h.value
    assert lib.lib.adc_last_error(None)


def test_binding_rejects_wrong_dtypes(lib):
    with pytest.raises(TypeError):
        lib._ptr(np.zeros(3, np.complex64), np.complex128)
    with pytest.raises(TypeError):
        lib._ptr(np.zeros((3, 3), np.complex128)[:, 0], np.complex128)


STRUCTS = ["adc_opts", "adc_stats", "adc_ssfns_root", "adc_batch_info", "adc_problem", "adc_batch_opts",
           "adc_kernel_stat"]


def test_python_struct_mirrors_match_the_headers(lib, tmp_path):
    """Size and field offsets of every public struct, as gcc lays it out from
    include/*.h, equal those of the ctypes mirrors of the Python binding."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "adc_gb300.h"', '#include "adc_gb300_diag.h"',
             "int main(void) {"]
    for st in STRUCTS:
        cls = getattr(lib, st)
        lines.append(f'  printf("{st} size %zu\\n", sizeof({st}));')
        for name, _ in cls._fields_:
            lines.append(f'  printf("{st} {name} %zu\\n", offsetof({st}, {name}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    c_layout = {tuple(ln.split()[:2]): int(ln.split()[2]) for ln in out if ln.strip()}
    for st in STRUCTS:
        cls = getattr(lib, st)
        assert c_layout[(st, "size")] == ctypes.sizeof(cls), st
        for name, _ in cls._fields_:
            assert c_layout[(st, name)] == getattr(cls, name).offset, (st, name)


@pytest.mark.parametrize("field,value", [("ee_vvvv", 2), ("ee_vvvv", -2), ("refine", 1), ("setup", 2)])
def test_init_rejects_bad_options_before_device_work(lib, field, value):
    o = lib.adc_opts()
    lib.lib.adc_opts_default(ctypes.byref(o))
    setattr(o, field, value)
    nocc, nvir = 3, 5
    nmo = nocc + nvir
    B = np.zeros((2, nmo, nmo), np.complex128)
    eo, ev = -np.ones(nocc), np.ones(nvir)
    h = ctypes.c_void_p()
    rc = lib.lib.adc_init(ctypes.byref(h), B.ctypes.data, 2, eo.ctypes.data, nocc, ev.ctypes.data, nvir,
                          2, 3, 1.0, ctypes.byref(o))
    assert rc == -1
    assert not h.value


def test_property_calls_need_a_context(lib):
    z = np.zeros(4, np.complex128)
    p = z.ctypes.data
    L = lib.lib
    assert L.adc_spectroscopic_amplitudes(None, p, 1, p) == -7
    assert L.adc_state_pair_density(None, p, p, 1, p) == -7
    assert L.adc_excited_density(None, p, 1, p) == -7
    assert L.adc_transition_density(None, p, 1, p) == -7
    assert L.adc_memory(None, p, p) == -7


def _prototypes():
    """name -> number of parameters of every function declared in include/*.h."""
    out = {}
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        with open(os.path.join(ROOT, "include", fn)) as fh:
            txt = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        for m in re.finditer(r"(const\s+char\s*\*|\bvoid\s|\bint64_t\s|\bint\s)\s*(adc_[a-z0-9_]+)\s*\(([^;{}]*?)\)\s*;",
                             txt):
            params = m.group(3).strip()
            ret = {"void": None, "int64_t": "i64", "int": "i"}.get(m.group(1).strip(), "p")
            out[m.group(2)] = (ret, [] if params in ("", "void") else [_c_kind(q) for q in params.split(",")])
    return out


def _c_kind(param):
    """Kind of a C parameter: pointer, int64, uint64, int or double."""
    if "*" in param:
        return "p"
    for c_t, kind in (("uint64_t", "u64"), ("int64_t", "i64"), ("double", "d"), ("int", "i")):
        if re.search(r"\b" + c_t + r"\b", param):
            return kind
    raise AssertionError(f"unknown parameter type: {param!r}")


def _ctypes_kind(t):
    if t in (ctypes.c_void_p, ctypes.c_char_p) or hasattr(t, "_type_") and isinstance(t._type_, type):
        return "p"
    return {ctypes.c_int64: "i64", ctypes.c_uint64: "u64", ctypes.c_int: "i", ctypes.c_double: "d"}[t]


def test_binding_signatures_match_the_header(lib):
    """Every function the binding declares to ctypes takes the arguments of its
    C prototype, in number and kind (pointer, 64-bit integer, int, double), and
    returns its kind: an argument added or retyped on one side only would pass
    garbage."""
    protos = _prototypes()
    checked = 0
    for name, (ret, kinds) in protos.items():
        f = getattr(lib.lib, name, None)
        if f is None or f.argtypes is None:
            continue
        assert [_ctypes_kind(t) for t in f.argtypes] == kinds, (name, f.argtypes, kinds)
        assert (None if f.restype is None else _ctypes_kind(f.restype)) == ret, (name, f.restype, ret)
        checked += 1
    assert checked == len(protos) == len(_declared()), (checked, len(protos))
