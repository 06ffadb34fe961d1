"""Host-side checks of the C ABI (no GPU): the library builds for sm_103a,
loads, exports every function include/cbdg.h declares, matches the header's
struct layout, and rejects invalid descriptors before touching a device."""
import ctypes
import os
import subprocess
import textwrap

import numpy as np
import pytest

from paper_1007_1609_gb300 import build as B
from paper_1007_1609_gb300 import cbdg
from paper_1007_1609_gb300 import workloads as wl


@pytest.fixture(scope="module")
def lib():
    B.build()
    return cbdg.load()


def test_exports_every_declared_function(lib):
    names = cbdg.header_functions()
    assert "cbdg_build_lattice" in names and "cbdg_scf_step" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert cbdg.cbdg_version().startswith("cbdg")


def test_descriptor_layout_matches_header(tmp_path):
    """Compile a probe against include/cbdg.h and compare offsets with ctypes."""
    src = tmp_path / "probe.c"
    fields = [f for f, _ in cbdg.cbdg_lattice_desc._fields_]
    body = "".join(f'  printf("{f} %zu\\n", offsetof(cbdg_lattice_desc, {f}));\n' for f in fields)
    src.write_text(textwrap.dedent("""
        #include <stddef.h>
        #include <stdio.h>
        #include "cbdg.h"
        int main(void) {
          printf("size %zu\\n", sizeof(cbdg_lattice_desc));
        """) + body + "  return 0;\n}\n")
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(B.ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    assert int(out["size"]) == ctypes.sizeof(cbdg.cbdg_lattice_desc)
    for f in fields:
        assert int(out[f]) == getattr(cbdg.cbdg_lattice_desc, f).offset, f


def _desc(p, **over):
    d = cbdg.cbdg_lattice_desc()
    keep = {}
    eps = np.ascontiguousarray(over.pop("eps", p.eps), dtype=np.float64)
    hop = np.ascontiguousarray(over.pop("hop", p.hop), dtype=np.complex128)
    delta = np.ascontiguousarray(over.pop("delta0", p.delta0), dtype=np.complex128)
    keep.update(eps=eps, hop=hop, delta=delta)
    d.Lx, d.Ly = p.Lx, p.Ly
    d.periodic_x, d.periodic_y = p.periodic_x, p.periodic_y
    d.eps, d.hop, d.delta0 = eps.ctypes.data, hop.ctypes.data, delta.ctypes.data
    d.mu, d.n_dirs, d.pairing, d.coupling = p.mu, hop.shape[1], p.pairing, p.coupling
    d.precision, d.complex_field = 0, 0
    for k, v in over.items():
        setattr(d, k, v)
    return d, keep


def _status(d):
    out = ctypes.c_void_p()
    st = cbdg.load().cbdg_build_lattice(ctypes.byref(d), None, ctypes.byref(out))
    return st, cbdg.cbdg_last_error()


@pytest.mark.parametrize("mutation,expect", [
    ("Lx0", cbdg.CBDG_ERR_INVALID_ARG),
    ("periodic2", cbdg.CBDG_ERR_INVALID_ARG),
    ("ndirs5", cbdg.CBDG_ERR_INVALID_ARG),
    ("nan_eps", cbdg.CBDG_ERR_INVALID_ARG),
    ("nonhermitian", cbdg.CBDG_ERR_INVALID_ARG),
    ("open_edge_hop", cbdg.CBDG_ERR_INVALID_ARG),
    ("complex_when_real", cbdg.CBDG_ERR_INVALID_ARG),
    ("bad_precision", cbdg.CBDG_ERR_INVALID_ARG),
    ("bad_pairing", cbdg.CBDG_ERR_INVALID_ARG),
    ("nan_mu", cbdg.CBDG_ERR_INVALID_ARG),
])
def test_invalid_descriptors_are_rejected(lib, mutation, expect):
    p = wl.random_swave(5, 16, seed=1, periodic=0)
    over = {}
    if mutation == "Lx0":
        over["Lx"] = 0
    elif mutation == "periodic2":
        p = wl.random_swave(2, 16, seed=1, periodic=0)
        over["periodic_x"] = 1
    elif mutation == "ndirs5":
        over["n_dirs"] = 5
    elif mutation == "nan_eps":
        e = p.eps.copy()
        e[3] = np.nan
        over["eps"] = e
    elif mutation == "nonhermitian":
        h = p.hop.copy()
        h[6, 0] = 0.9
        over["hop"] = h
    elif mutation == "open_edge_hop":
        h = p.hop.copy()
        h[4, 0] = 1.0  # site x = 4 has no +x neighbour on an open 5x5 lattice
        over["hop"] = h
    elif mutation == "complex_when_real":
        dl = p.delta0.copy()
        dl[0] = 0.5 + 0.1j
        over["delta0"] = dl
    elif mutation == "bad_precision":
        over["precision"] = 7
    elif mutation == "bad_pairing":
        over["pairing"] = 3
    elif mutation == "nan_mu":
        over["mu"] = float("nan")
    d, keep = _desc(p, **over)
    st, msg = _status(d)
    assert st == expect, msg
    assert msg


def test_null_arguments(lib):
    out = ctypes.c_void_p()
    assert lib.cbdg_build_lattice(None, None, ctypes.byref(out)) == cbdg.CBDG_ERR_INVALID_ARG
    assert lib.cbdg_moments(None, None, 0, 4, None, None) == cbdg.CBDG_ERR_INVALID_ARG
    assert lib.cbdg_scf_step(None, 0.01, 8, 0.5, None) == cbdg.CBDG_ERR_INVALID_ARG
    assert lib.cbdg_destroy(None) == cbdg.CBDG_OK
    assert lib.cbdg_set_option(None, 0, 1) == cbdg.CBDG_ERR_INVALID_ARG


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No fallback: without libcbdg.so the binding raises."""
    monkeypatch.setattr(cbdg, "_lib", None)
    monkeypatch.setattr(cbdg, "library_path", lambda: str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="not built"):
        cbdg.load()
