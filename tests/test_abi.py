"""C-ABI library: builds, loads and exports every symbol the headers declare
(no compute calls: this runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(hdr).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"(?:kq_status|void|const char\s*\*)\s*(\w+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    import paper_2308_00637_gb300 as kq
    return ctypes.CDLL(kq.LIB_PATH)


def test_headers_declare_the_boundary():
    names = declared_symbols()
    for required in ("qp_create", "ipm_solve", "kkt_pcg_solve", "qp_backward", "qp_destroy",
                     "qp_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_default_options_are_the_papers(lib):
    """Defaults equal the settings printed in sections 3.2 and 5.1."""
    import json
    import paper_2308_00637_gb300 as kq
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_settings.json")))
    o = kq.default_ipm_opts()
    assert o.gamma == gold["gamma"]["value"]
    assert o.mu_tol == gold["mu_tol"]["value"]
    assert o.pcg_tol == gold["pcg_tol"]["value"]
    assert o.pcg_maxit == gold["pcg_maxit"]["value"]
    assert o.mu0 == 1.0 and o.ipm_maxit == 200


def test_create_without_device_fails_loudly(lib):
    """On a machine without a GPU the product path raises; it never falls
    back to a CPU implementation."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import qpgen
    import paper_2308_00637_gb300 as kq
    with pytest.raises(kq.KQError):
        kq.create_from(qpgen.dense_qp(8, 4, seed=1))


def test_struct_layouts_match_header(tmp_path):
    """Every ctypes mirror of a header struct has the C compiler's size and
    field offsets (a field added on one side only would shift every field
    after it and be read as garbage)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    import paper_2308_00637_gb300 as m
    structs = {"kq_hop": m.KqHop, "kq_amat": m.KqAmat, "kq_ipm_opts": m.KqIpmOpts,
               "kq_ipm_iter": m.KqIpmIter, "kq_ipm_stats": m.KqIpmStats,
               "kq_pcg_opts": m.KqPcgOpts, "kq_pcg_stats": m.KqPcgStats,
               "kq_qp_desc": m.KqQpDesc, "kq_batch_stats": m.KqBatchStats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "kktqp.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f in py._fields_:
            lines.append(f'printf("{cname}.{f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                       text=True).stdout.splitlines())
    for cname, py in structs.items():
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for f in py._fields_:
            assert int(got[f"{cname}.{f[0]}"]) == getattr(py, f[0]).offset, (cname, f[0])
