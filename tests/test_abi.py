"""The C ABI library loads and exports every entry point that include/*.h
declares (no GPU needed: nothing is called that touches the device)."""
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"\b(tdbem_\w+)\s*\(", txt):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("tdbem_create", "tdbem_history_eval", "tdbem_step", "tdbem_march", "tdbem_save", "tdbem_load",
              "tdbem_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    import paper_2303_05006_gb300 as pkg

    pkg.lib()  # loads the shared object
    out = subprocess.run(["nm", "-D", "--defined-only", pkg.library_path()], capture_output=True, text=True,
                         check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    missing = declared_symbols() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"


def test_package_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_2303_05006_gb300._binding as b

    monkeypatch.setattr(b, "_LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(b, "_lib", None)
    with pytest.raises(ImportError):
        b.lib()


def _c_layout(struct, fields):
    """sizeof and offsetof of the header's struct, from a C program built with gcc."""
    import tempfile

    src = ["#include <stddef.h>", "#include <stdio.h>", '#include "tdbem.h"', "int main(void) {",
           f'  printf("%zu\\n", sizeof({struct}));']
    src += [f'  printf("%zu\\n", offsetof({struct}, {f}));' for f in fields]
    src += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        c, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(c, "w").write("\n".join(src))
        subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    return int(out[0]), [int(x) for x in out[1:]]


@pytest.mark.parametrize("name", ["Params", "Info"])
def test_binding_structs_match_the_header(name):
    """Every field of the ctypes mirror sits at the header's offset, and the
    sizes agree (a field added to the header but not to the binding, or in
    another order, fails here)."""
    import paper_2303_05006_gb300._binding as b

    if not __import__("shutil").which("gcc"):
        pytest.skip("gcc not available")
    cls = getattr(b, name)
    struct = {"Params": "tdbem_params", "Info": "tdbem_info"}[name]
    fields = [f[0] for f in cls._fields_]
    size, offs = _c_layout(struct, fields)
    assert __import__("ctypes").sizeof(cls) == size
    assert [getattr(cls, f).offset for f in fields] == offs


def test_default_params_match_the_header():
    """tdbem_default_params (host only) fills the documented defaults."""
    import ctypes

    import paper_2303_05006_gb300._binding as b

    p = b.Params()
    b.lib().tdbem_default_params(ctypes.byref(p))
    assert (p.d, p.p_s, p.p_t, p.n_leaf, p.mode, p.m2l_prec, p.n_rhs, p.warm_start) == (2, 4, 4, 64, 0, 0, 1, 1)
    assert (p.theta, p.zeta, p.eps, p.mu, p.s_jump, p.chi) == (1.0, 1.0, 1.0, 1.0, 1.0, 1.0)
    assert (p.solve_tol, p.solve_maxit, p.precond, p.far_overlap) == (1e-13, 1000, 1, 1)
    assert p.p2p_prec == b.TDBEM_P_FP64 and p.max_device_bytes == 0 and p.solve_cluster == 0
