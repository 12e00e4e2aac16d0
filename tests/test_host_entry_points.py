"""Host-only entry points of the library, exercised without a GPU: the DCT-II
temporal basis (App. E.2.1), the restricted eigensolve's defaults, the
argument checks of a problem given by its operator, which refuse a malformed
CSR before any device call, the solve options' defaults against the header's
documentation, and the layout of every struct the binding passes."""
import ctypes

import numpy as np
import pytest
import scipy.sparse as sp


@pytest.fixture(scope="module")
def sdf():
    from paper_2606_17971_b300 import sdf as S
    return S


def test_dct2_basis_matches_oracle_and_scipy(sdf):
    from scipy.fft import dct
    from oracle import spacetime_oracle as ST
    for n, r in ((8, 8), (16, 5), (1, 1), (13, 13)):
        w = sdf.dct2_basis(n, r)
        np.testing.assert_allclose(w, ST.dct2_basis(n, r), atol=1e-15)
        ref = dct(np.eye(n), type=2, norm="ortho", axis=0)[:r].T
        np.testing.assert_allclose(w, ref, atol=1e-14)
    # out-of-range requests leave the output untouched
    w = np.full((4, 5), 7.0, order="F")
    sdf._lib.sdf_dct2_basis(4, 5, w.ctypes.data)
    assert np.all(w == 7.0)


def test_restricted_eigensolve_defaults(sdf):
    o = sdf.EigOpts()
    sdf._lib.sdf_default_restricted_eig_opts(10, ctypes.byref(o))
    assert (o.degree, o.guard, o.tol) == (200, 32, 1e-8)
    sdf._lib.sdf_default_restricted_eig_opts(100, ctypes.byref(o))
    assert o.guard == 50


def _create(sdf, K, **kw):
    rp = np.ascontiguousarray(K.indptr, dtype=np.int32)
    ci = np.ascontiguousarray(K.indices, dtype=np.int32)
    v = np.ascontiguousarray(K.data, dtype=np.float64)
    h = ctypes.c_void_p()
    st = sdf._lib.sdf_problem_create_csr(K.shape[0], rp.ctypes.data, ci.ctypes.data,
                                         v.ctypes.data, kw.get("mass", 1.0),
                                         kw.get("alpha", 1e-4), kw.get("kscale", 1.0),
                                         ctypes.byref(h))
    if h.value:
        sdf._lib.sdf_problem_destroy(h)
    return st


def test_malformed_csr_operators_are_refused_on_the_host(sdf):
    K = sp.random(50, 50, density=0.1, format="csr", random_state=3) + sp.identity(50)
    K = K.tocsr()
    bad = K.copy()
    bad.indices[3] = 60  # a column outside [0, n)
    assert _create(sdf, bad) == 1
    bad = K.copy()
    bad.data[5] = np.nan  # a non-finite value
    assert _create(sdf, bad) == 1
    assert _create(sdf, K, alpha=0.0) == 1  # alpha must be positive
    assert _create(sdf, K, mass=-1.0) == 1


def test_solve_option_defaults_match_the_header(sdf):
    # every option the header documents with a bracketed default, read back
    # through the binding's struct: a field out of place in the ctypes
    # layout, or a default changed on one side only, fails here
    import os
    import re
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "include", "sdf.h")).read()
    block = hdr[hdr.index("/* Solve options"):hdr.index("} sdf_opts;")]
    doc = block[:block.index("*/")]
    # "name ... [value]" entries, the name at the start of a comment line
    entries = re.findall(r"\n \*   (\w+)(?:,\s*(\w+))?\s.*?\[([^\]]+)\]", doc, flags=re.S)
    o = sdf.default_opts()
    seen = set()
    consts = {"SDF_PREC_F64": sdf.PREC_F64}
    for name, name2, val in entries:
        vals = [v.strip() for v in val.split(",")]
        for nm, v in zip([name] + ([name2] if name2 else []), vals):
            v = v.split(":")[0].strip()
            want = consts[v] if v in consts else float(v)
            assert getattr(o, nm) == pytest.approx(want), (nm, getattr(o, nm), want)
            seen.add(nm)
    fields = {f[0] for f in sdf.Opts._fields_}
    assert seen == fields, fields - seen


def test_binding_structs_match_the_c_layout(sdf, tmp_path):
    # every struct the binding passes through the C ABI: size and the offset
    # of each field as the C compiler lays them out from include/sdf.h (the
    # header is plain C), against the ctypes declaration
    import os
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    pairs = [(sdf.ProblemDesc, "sdf_problem_desc"), (sdf.Opts, "sdf_opts"),
             (sdf.Stats, "sdf_stats"), (sdf.Profile, "sdf_profile"),
             (sdf.EigOpts, "sdf_eig_opts"), (sdf.EigStats, "sdf_eig_stats"),
             (sdf.MlpDesc, "sdf_mlp_desc"), (sdf.WarmModelDesc, "sdf_warm_model")]
    lines = ['#include "sdf.h"', "#include <stdio.h>", "#include <stddef.h>", "int main(void) {"]
    want = []
    for cls, cname in pairs:
        lines.append(f'  printf("%zu\\n", sizeof({cname}));')
        want.append((cname, "sizeof", ctypes.sizeof(cls)))
        for f in cls._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({cname}, {f[0]}));')
            want.append((cname, f[0], getattr(cls, f[0]).offset))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True,
                                          text=True).stdout.split()]
    assert len(got) == len(want)
    bad = [(c, f, w, g) for (c, f, w), g in zip(want, got) if w != g]
    assert not bad, bad
