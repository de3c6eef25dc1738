"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
entry point that include/mgx.h declares (no compute calls are made here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "mgx.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mgx_[a-zA-Z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    import paper_2011_14998_gb300 as mgx

    path = mgx.build()
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert "mgx_solve_J" in declared and "mgx_trace" in declared
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) <= set(mgx.ABI_SYMBOLS)


def test_rayset_npairs_host_only():
    import paper_2011_14998_gb300 as mgx

    mgx.build()
    assert mgx.mgx_rayset_npairs(1, 4) * 2 == 552
    assert mgx.mgx_rayset_npairs(4, 4) * 2 == 3072
    assert mgx.mgx_rayset_npairs(0, 3) == 69
    assert mgx.mgx_rayset_npairs(3, 2) == -1


def test_package_has_no_oracle_dependency():
    pkg = os.path.join(ROOT, "paper_2011_14998_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in src.lower(), f


def test_healpix_host_exports_match_oracle(orc):
    import numpy as np

    import paper_2011_14998_gb300 as mgx

    mgx.build()
    for l in range(5):
        for p in range(0, 12 * 4**l, max(1, (12 * 4**l) // 29)):
            assert mgx.mgx_antipode(l, p) == orc.antipode(l, p)
            assert np.array_equal(mgx.mgx_pix2vec(l, p), orc.pix2vec(l, p))
    import pytest

    with pytest.raises(ValueError):
        mgx.mgx_antipode(9, 0)
    with pytest.raises(ValueError):
        mgx.mgx_pix2vec(1, 48)


def test_every_declaration_cites_its_passage():
    # each entry point's comment (or its group's, within the last three comment
    # blocks) names the passage of the paper it implements, or says it has none
    import re

    txt = open(os.path.join(ROOT, "include", "mgx.h")).read()
    comments = [(m.end(), m.group(0)) for m in re.finditer(r"/\*.*?\*/", txt, flags=re.S)]
    cite = re.compile(r"Section|Eqs?\.|Fig\.|Table|no counterpart|paper does not|paper has no|Gorski")
    decl = re.compile(r"^(?:mgx_status|int64_t|int32_t|void|const char \*|double)\s+(mgx_\w+)\s*\(", re.M)
    names = []
    for m in decl.finditer(txt):
        before = [c for end, c in comments if end <= m.start()][-3:]
        if not any(cite.search(c) for c in before):
            names.append(m.group(1))
    assert names == [], names
