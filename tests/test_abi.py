"""Host-side checks of the C-ABI library: it loads, exports every symbol the
header declares, and rejects bad arguments before touching a GPU."""
import ctypes as ct
import os
import re
import subprocess

import numpy as np
import pytest

import __graft_entry__
from paper_1807_00699_gb300 import gda

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gda.h")


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.ensure_built()
    return gda.load_library()


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gda_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("gda_create", "gda_run", "gda_energy", "gda_best", "gda_get_state", "gda_set_state"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", gda.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (gda_\w+)", out))
    missing = [n for n in declared_symbols() if n not in exported]
    assert not missing, missing
    assert set(declared_symbols()) == set(gda.SIGNATURES), "binding and header disagree"


def test_default_params(lib):
    p = gda.default_params()
    assert (p.dt, p.eps, p.rho_th, p.beta0, p.eps_hat, p.noise_D) == (0.01, 0.1, 1.0, 1.0, 0.0, 0.0)
    assert p.integ == gda.EULER and p.prec == gda.FP32 and p.init_mode == 1
    assert ct.sizeof(gda.Params) == 136
    assert p.wait_s == 0.0 and p.withhold_flag == 0


def test_params_layout_matches_header(tmp_path):
    """The ctypes mirror of gda_params has the header's size and field offsets
    (checked by compiling the header with the host C compiler)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    names = [f[0] for f in gda.Params._fields_]
    src = ["#include <stddef.h>", "#include <stdio.h>", f'#include "{os.path.join(ROOT, "include", "gda.h")}"',
           "int main(void) {", '  printf("%zu\\n", sizeof(gda_params));']
    src += [f'  printf("%zu\\n", offsetof(gda_params, {n}));' for n in names]
    src += ["  return 0;", "}"]
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, str(c), "-o", str(exe)], check=True)
    out = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert out[0] == ct.sizeof(gda.Params)
    assert out[1:] == [getattr(gda.Params, n).offset for n in names]


def test_status_strings(lib):
    assert lib.gda_status_string(0) == b"ok"
    assert b"invalid" in lib.gda_status_string(1)


def _create(lib, J, N, model=0):
    h = ct.c_void_p()
    st = lib.gda_create(J.ctypes.data_as(ct.POINTER(ct.c_double)) if J is not None else None, None, N, model,
                        ct.byref(h))
    return st, h


def test_invalid_instances_rejected_on_host(lib):
    J = np.array([[0.0, 1.0], [2.0, 0.0]])
    st, h = _create(lib, J, 2)
    assert st == 1 and not h.value  # asymmetric
    J = np.array([[0.0, np.nan], [np.nan, 0.0]])
    assert _create(lib, J, 2)[0] == 1  # non-finite
    assert _create(lib, np.zeros((1, 1)), 0)[0] == 1  # N < 1
    assert _create(lib, None, 3)[0] == 1  # NULL J
    assert _create(lib, np.zeros((2, 2)), 2, model=7)[0] == 1  # unknown model


def test_null_context_calls(lib):
    assert lib.gda_run(None, None, 1, 1) == 1
    assert lib.gda_sync(None) == 1
    lib.gda_destroy(None)
    assert lib.gda_kernel_launches(None) == 0
