"""The C-ABI library builds, loads and exports every entry point that
include/msf.h declares; argument checks run before any launch (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "msf.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(msf_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2008_01567_gb300 import build, msf
    build.build()
    msf._lib = None
    return msf.lib()


def test_header_declares_the_path(lib):
    names = _declared()
    for required in ("msf_project", "msf_backproject", "msf_prox_data", "msf_denoise",
                     "msf_train_step", "msf_mace_step"):
        assert required in names


@pytest.mark.parametrize("lang", ["c", "c++"])
def test_header_is_plain_c_and_cpp(tmp_path, lang):
    # the boundary is a C ABI: the header alone must compile as strict C99 and
    # as C++ (no torch or CUDA types in any signature)
    import shutil
    import subprocess
    cc = shutil.which("gcc" if lang == "c" else "g++")
    if cc is None:
        pytest.skip("no host compiler")
    src = tmp_path / "use_header.c"
    src.write_text('#include "msf.h"\nint main(void) { return 0; }\n')
    flags = ["-std=c99", "-pedantic"] if lang == "c" else ["-std=c++17", "-x", "c++"]
    r = subprocess.run([cc, *flags, "-Wall", "-Wextra", "-Werror", "-fsyntax-only", "-I",
                        os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


C_CALLER = r"""
#include <stdio.h>
#include <string.h>
#include "msf.h"
int main(void) {
    msf_projector* p = 0;
    msf_cnn* c = 0;
    if (strncmp(msf_version(), "msf-gb300", 9) != 0) return 1;
    /* argument errors come back as status codes before any device call */
    if (msf_projector_create(0, 0, &p) != MSF_ERR_ARG || p != 0) return 2;
    if (strstr(msf_last_error(), "NULL") == 0) return 3;
    if (msf_cnn_create(0, &c) != MSF_ERR_ARG || c != 0) return 4;
    printf("%s\n", msf_last_error());
    return 0;
}
"""


def test_library_links_and_runs_from_c(lib, tmp_path):
    # the boundary without Python: a C program linked against libmsf.so
    import shutil
    import subprocess
    from paper_2008_01567_gb300 import msf
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no host compiler")
    libdir = os.path.dirname(msf.LIB_PATH)
    src, exe = tmp_path / "caller.c", tmp_path / "caller"
    src.write_text(C_CALLER)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                        "-L", libdir, "-lmsf", "-Wl,-rpath," + libdir, "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, (run.returncode, run.stdout, run.stderr)
    assert "max_pixels" in run.stdout


def test_every_declared_symbol_is_exported(lib):
    from paper_2008_01567_gb300 import msf
    for name in _declared():
        assert hasattr(lib, name), name
        assert name in msf._SIGS, f"binding lacks {name}"


def test_argument_errors_before_launch(lib):
    from paper_2008_01567_gb300 import msf
    h = ctypes.c_void_p()
    st = lib.msf_projector_create(None, None, ctypes.byref(h))
    assert st == 1 and b"NULL" in lib.msf_last_error()
    ang = np.zeros(3)
    geom = msf.msf_geom(8, 8, 3, 0.1, 0.1, 0.3, 8.0, ang.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    vol = msf.msf_vol(8, 8, 8, 1, 1.0 / 8)
    # source inside the circumscribed cylinder
    assert lib.msf_projector_create(ctypes.byref(geom), ctypes.byref(vol), ctypes.byref(h)) == 1
    assert b"cylinder" in lib.msf_last_error()
    mrf = msf.msf_mrf(1.5, 1.2, 1.0, 0.1, 0.5)
    assert lib.msf_prox_qggmrf(ctypes.byref(vol), ctypes.byref(mrf), 1, 1, 0.1, 1, None) == 1
    assert b"p == 2" in lib.msf_last_error()
    assert lib.msf_weights(1, 1, 1, 10, -1.0, 1.0, None) == 1
    assert lib.msf_projector_set_tuning(None, 32, 4, 16) == 1
    assert lib.msf_mace_consensus(None, None, 2, 8, None, 0.5, None, None) == 1
    mu = (ctypes.c_double * 4)(0.5, 0.25, 0.25, 0.0)
    fake = ctypes.c_void_p(256)                    # never dereferenced: the checks come first
    assert lib.msf_mace_consensus(fake, fake, 3, 8, mu, 0.5, fake, None) == 1
    assert b"2 or 4" in lib.msf_last_error()
    assert lib.msf_version().startswith(b"msf-gb300")


def test_empty_and_negative_sizes_are_argument_errors(lib):
    """Empty volumes, detectors, view sets, CNN workspaces and batches are
    refused with MSF_ERR_ARG before any device call (so this runs without a GPU)."""
    from paper_2008_01567_gb300 import msf
    h = ctypes.c_void_p()

    def create(nx=8, nt=1, nu=8, nv=8, views=3):
        ang = np.zeros(max(views * nt, 1))
        geom = msf.msf_geom(nu, nv, views, 0.1, 0.1, 4.0, 8.0, ang.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        vol = msf.msf_vol(nx, nx, nx, nt, 1.0 / max(nx, 1))
        return lib.msf_projector_create(ctypes.byref(geom), ctypes.byref(vol), ctypes.byref(h))

    for bad in (dict(nx=0), dict(nx=-3), dict(nt=0), dict(nu=0), dict(nv=0), dict(views=0)):
        assert create(**bad) == 1, bad
        assert b"positive" in lib.msf_last_error(), (bad, lib.msf_last_error())
    assert lib.msf_cnn_create(0, ctypes.byref(h)) == 1
    assert lib.msf_cnn_create(-5, ctypes.byref(h)) == 1
    assert lib.msf_mace_batch_create(None, 0, ctypes.byref(h)) == 1
    for fn in ("msf_dataprox_create", "msf_map_create", "msf_fixcorr_create", "msf_mace_create"):
        assert getattr(lib, fn)(None, ctypes.byref(h)) == 1, fn
        assert b"NULL" in lib.msf_last_error(), fn


def test_static_projection_checks_every_column(lib):
    """msf_project_static checks on the host, before any device call, that the
    voxel planes of every (view, column) lie between source and detector; the
    geometry below fails on interior column 3 only (where the view's columns
    switch from x-major to y-major), so an end-columns check would pass it."""
    from paper_2008_01567_gb300 import msf
    from tests.test_zz_no_alloc import INTERIOR_FAIL as g
    ang = np.array([g["theta"]], dtype=np.float64)
    geom = msf.msf_geom(g["nu"], g["nv"], 1, g["du"], g["du"], g["dso"], g["dsd"],
                        ang.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    vol = msf.msf_vol(g["n"], g["n"], g["n"], 1, 1.0 / g["n"])
    fake = ctypes.c_void_p(256)                    # never dereferenced: the checks come first
    assert lib.msf_project_static(ctypes.byref(geom), ctypes.byref(vol), fake, fake, None) == 1
    assert b"column 3" in lib.msf_last_error(), lib.msf_last_error()


def test_binding_refuses_cpu_tensors(lib):
    torch = pytest.importorskip("torch")
    from paper_2008_01567_gb300 import msf
    with pytest.raises(ValueError):
        msf._ptr(torch.zeros(4))
