"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/sdf.h declares, and the binding's ctypes signatures
agree with the header's prototypes (no compute calls here)."""
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


def _c_prototypes():
    """name -> (return kind, [parameter kinds]) from include/sdf.h, where a
    kind is 'ptr', 'i32', 'i64', 'u64', 'size', 'f64', 'f32' or 'void'."""
    import re
    hdr = open(os.path.join(ROOT, "include", "sdf.h")).read()
    hdr = re.sub(r"/\*.*?\*/", " ", hdr, flags=re.S)
    enums = set(re.findall(r"}\s*(\w+)\s*;", hdr)) & {"sdf_status", "sdf_dtype", "sdf_precision"}
    scalar = {"int": "i32", "int32_t": "i32", "int64_t": "i64", "uint64_t": "u64",
              "size_t": "size", "double": "f64", "float": "f32", "void": "void"}
    scalar.update({e: "i32" for e in enums})

    def kind(decl, is_param):
        decl = decl.strip()
        if "*" in decl:
            return "ptr"
        toks = [t for t in decl.replace("const", " ").split() if t]
        t = toks[0] if not is_param or len(toks) == 1 else toks[-2]
        return scalar[t]

    out = {}
    for ret, name, params in re.findall(r"\n([\w][\w \*]*?)\s*\b(sdf_\w+)\s*\(([^;{]*?)\)\s*;",
                                        hdr):
        ps = [p for p in (x.strip() for x in params.split(",")) if p and p != "void"]
        out[name] = (kind(ret, False), [kind(p, True) for p in ps])
    return out


def test_binding_signatures_match_the_header():
    # each ctypes signature of the binding against the header's prototype:
    # argument count and the kind of every argument (a double passed where
    # C expects an integer, or an int64 where it expects an int32, would
    # reach the library as garbage without any error)
    import ctypes
    from paper_2606_17971_b300 import sdf
    protos = _c_prototypes()
    ck = {ctypes.c_void_p: "ptr", ctypes.c_char_p: "ptr", ctypes.c_int: "i32",
          ctypes.c_int32: "i32", ctypes.c_int64: "i64", ctypes.c_uint64: "u64",
          ctypes.c_size_t: "size", ctypes.c_double: "f64", ctypes.c_float: "f32", None: "void"}

    def kind(t):
        if t in ck:
            return ck[t]
        if isinstance(t, type) and issubclass(t, ctypes._Pointer):
            return "ptr"
        raise AssertionError(t)

    assert set(sdf._sigs) <= set(protos), set(sdf._sigs) - set(protos)
    bad = []
    for name, (res, args) in sdf._sigs.items():
        cret, cargs = protos[name]
        got = (kind(res), [kind(a) for a in args])
        # on this ABI size_t is 64 bits wide, like int64_t
        norm = lambda ks: [("i64" if k == "size" else k) for k in ks]
        if got[0] != cret and not (cret == "ptr" and got[0] == "ptr") \
                or norm(got[1]) != norm(cargs):
            bad.append((name, (cret, cargs), got))
    assert not bad, bad
