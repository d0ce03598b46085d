"""The C-ABI library loads on a machine without a GPU and exports every
function that include/ax.h declares; the Python binding uses the same names.
No compute call is made here."""
import ctypes
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_\s\*]*?\b([a-z][a-z0-9_]*)\s*\(", src, flags=re.M))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2504_07042_gb300 import build

    lib = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    declared = _declared()
    assert declared, "no declarations parsed"
    assert declared <= exported, sorted(declared - exported)
    L = ctypes.CDLL(lib)  # loads without a GPU
    for name in declared:
        assert hasattr(L, name)


def test_binding_names_follow_the_abi():
    from paper_2504_07042_gb300 import ax

    for name in ax.EXPORTS:
        assert name in _declared()
    assert ax._lib.ax_status_string(ax.AX_EINVERTED) == b"AX_EINVERTED"
