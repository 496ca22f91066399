"""A plain C program (tests/c/host_api.c) against the library: it compiles as
C99 against include/inla_gpu.h and links to libinla_gpu.so with no Python or
PyTorch in the process (CPU); on a GPU its f and central-difference gradient
match the oracle's on the same workload."""
import os
import subprocess

import numpy as np
import pytest

import paper_2204_04678_gb300 as pkg
from synth import config_model, fd_stencil
from oracle import bta, fd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.dirname(pkg.__file__)


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    pkg.build()
    out = tmp_path_factory.mktemp("c_api") / "host_api"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c", "host_api.c"), "-o", str(out), "-L", PKG, "-linla_gpu",
                    "-Wl,-rpath," + PKG], check=True)
    return str(out)


def test_c_program_compiles_and_links(exe):
    assert os.access(exe, os.X_OK)


@pytest.mark.gpu
def test_c_program_matches_oracle(exe):
    theta = np.array([0.9, -1.1, 0.1, 1.4])
    r = subprocess.run([exe, *(f"{x:.17g}" for x in theta)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    v = r.stdout.split()
    f, g, status = float(v[0]), np.array([float(x) for x in v[1:5]]), int(v[5])
    assert status == 0
    mdl = config_model(1)
    ref_f = bta.gaussian(mdl, theta)["f"]
    assert abs(f - ref_f) <= 1e-10 * abs(ref_f)
    ref_g = fd.gradient_from_stencil([bta.gaussian(mdl, p)["f"] for p in fd_stencil(theta)])
    assert np.abs(g - ref_g).max() <= 4e-10 * abs(ref_f) / 1e-3
