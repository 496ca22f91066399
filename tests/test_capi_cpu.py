"""The C ABI library builds, loads and exports every entry point of
include/inla_gpu.h; argument errors are reported without touching a GPU."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2204_04678_gb300 as pkg
from paper_2204_04678_gb300 import capi as C
from synth import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    pkg.build()
    return C.load()


def header_functions(header="inla_gpu.h"):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(inla_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_function_is_exported_and_bound(lib):
    names = header_functions()
    assert "inla_eval_batch" in names and "inla_model_create" in names
    for n in names:
        assert hasattr(lib, n), n
        assert n in C.SIGNATURES, n
    assert set(C.SIGNATURES) == set(names)


def test_probe_library_is_separate_and_complete(lib):
    # the benchmark's throughput probes live in their own library, not in the product
    probe = C.load_probe()
    names = header_functions("inla_probe.h")
    assert "inla_measure_fp64_peak" in names
    for n in names:
        assert hasattr(probe, n), n
        assert not hasattr(lib, n), n
    assert set(C.PROBE_SIGNATURES) == set(names)


def test_struct_layouts_match_the_c_compiler(tmp_path):
    # sizes and field offsets of the binding's structs equal those gcc gives the header
    structs = {"inla_model_desc": C.inla_model_desc, "inla_eval_opts": C.inla_eval_opts,
               "inla_eval_out": C.inla_eval_out, "inla_eval_out_host": C.inla_eval_out_host}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "inla_gpu.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    seen = 0
    for line in filter(None, out):
        name, field, val = line.split()
        cls = structs[name]
        expect = ctypes.sizeof(cls) if field == "size" else getattr(cls, field).offset
        assert int(val) == expect, (name, field)
        seen += 1
    assert seen == sum(len(c._fields_) + 1 for c in structs.values())


def _desc(mdl, keep):
    d = C.inla_model_desc()
    d.n_t, d.n_s, d.n_b, d.m = mdl.n_t, mdl.n_s, mdl.n_b, mdl.m
    d.lik = C.INLA_LIK_GAUSSIAN
    for name, arr, ct in (("C_diag", mdl.C_diag, ctypes.c_double), ("G_rowptr", mdl.G_rowptr, ctypes.c_int32),
                          ("G_col", mdl.G_col, ctypes.c_int32), ("G_val", mdl.G_val, ctypes.c_double),
                          ("A_rowptr", mdl.A_rowptr, ctypes.c_int64), ("A_col", mdl.A_col, ctypes.c_int32),
                          ("A_val", mdl.A_val, ctypes.c_double), ("y", mdl.y, ctypes.c_double)):
        keep.append(arr)
        setattr(d, name, arr.ctypes.data_as(ctypes.POINTER(ct)))
    d.tau_b = 1e-3
    for j in range(4):
        d.prior_mean[j] = 0.0
        d.prior_sd[j] = 10.0
    return d


def _binomial(d, m, trials=2.0, y=None):
    # a binomial description with N = trials everywhere (and y overridden)
    d.lik = C.INLA_LIK_BINOMIAL
    m.E = np.full(m.m, float(trials))
    m.y[:] = np.minimum(np.abs(np.round(m.y)), 2.0) if y is None else y
    d.E = m.E.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _split_row(m):
    # move the last spatial entry of a row into the next time block (columns stay sorted)
    r = int(np.nonzero(m.obs_t < m.n_t - 1)[0][0])
    k = int(m.A_rowptr[r]) + 2
    m.A_col[k] += m.n_s


@pytest.mark.parametrize("mutate,needle", [
    (lambda d, m: setattr(d, "n_t", 0), "n_t"),
    (lambda d, m: setattr(d, "n_b", 17), "n_b"),
    (lambda d, m: setattr(d, "tau_b", -1.0), "tau_b"),
    (lambda d, m: setattr(d, "y", None), "NULL"),
    (lambda d, m: m.A_col.__setitem__(0, 10 ** 6), "out of range"),
    (lambda d, m: m.C_diag.__setitem__(3, 0.0), "C_diag"),
    (lambda d, m: _split_row(m), "one time block"),
    (lambda d, m: setattr(d, "lik", 4), "unknown likelihood"),
    (lambda d, m: setattr(d, "lik", 3), "negative binomial size"),
    (lambda d, m: setattr(d, "lik", C.INLA_LIK_BINOMIAL), "trials"),
    (lambda d, m: _binomial(d, m, trials=2.5), "positive integers"),
    (lambda d, m: _binomial(d, m, y=3.0), "[0, N]"),
])
def test_invalid_descriptions_are_rejected_before_any_device_work(lib, mutate, needle):
    mdl = build("t", 3, 4, 2, 50)
    keep = []
    d = _desc(mdl, keep)
    mutate(d, mdl)
    h = ctypes.c_void_p()
    code = lib.inla_model_create(ctypes.byref(d), 0, ctypes.byref(h))
    assert code == C.INLA_ERR_ARG
    assert needle in lib.inla_last_error().decode()
    assert not h.value


def test_null_arguments(lib):
    assert lib.inla_model_create(None, 0, None) == C.INLA_ERR_ARG
    out = ctypes.c_size_t()
    o = C.inla_eval_opts()
    assert lib.inla_workspace_bytes(None, 1, ctypes.byref(o), ctypes.byref(out)) == C.INLA_ERR_ARG
    assert lib.inla_eval_batch(None, 1, None, None, None, None) == C.INLA_ERR_ARG
    v = ctypes.c_double()
    assert C.load_probe().inla_measure_fp64_peak(0, 0, None) == C.INLA_ERR_ARG
    assert lib.inla_set_wait_limit(0.0) == C.INLA_ERR_ARG
    assert lib.inla_set_time_partition(None, 2) == C.INLA_ERR_ARG
    assert lib.inla_set_point_groups(None, 2) == C.INLA_ERR_ARG
    lib.inla_model_destroy(None)
