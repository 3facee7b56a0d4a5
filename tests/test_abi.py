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
