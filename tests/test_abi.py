"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/sdf.h declares (no compute calls here)."""
import os
import re
import subprocess

from paper_2606_17971_b300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(sdf_[A-Za-z0-9_]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_entry_point():
    lib = B.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\sT\s(sdf_[A-Za-z0-9_]+)", out))
    declared = declared_functions()
    assert declared, "no declarations parsed"
    assert declared <= exported, declared - exported


def test_binding_loads_and_names_match():
    B.build()
    from paper_2606_17971_b300 import sdf
    assert set(sdf.EXPORTED) <= declared_functions()
    o = sdf.default_opts()
    assert o.rtol == 1e-8 and o.tau == 1e-10 and o.tau_cond == 1e10 and o.max_outer == 30


def test_built_for_sm_103a_only():
    assert "arch=compute_103a,code=sm_103a" in " ".join(B.NVCC_FLAGS)
