"""The Python binding's ctypes structures and constants against the C headers (no GPU):
small C programs compiled with gcc from include/*.h print sizeof and every field's offset of
each struct of the interface, and the enum values; the binding must agree exactly (a field
added on one side only would silently shift every later field across the C interface)."""
import os
import shutil
import subprocess
import tempfile

import ctypes as C
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# C typedef name -> binding class name
PAIRS = {
    "igs_create_opts": "_CreateOpts",
    "igs_solve_opts": "_SolveOpts",
    "igs_result": "_Result",
    "igs_info": "_Info",
    "igs_profile": "_Profile",
    "igs_batch_opts": "_BatchOpts",
    "igs_batch_solve_opts": "_BatchSolveOpts",
    "igs_batch_result": "_BatchResult",
    "igs_batch_tune_entry": "_TuneEntry",
    "igs_batch_info": "_BatchInfo",
    "igs_server_opts": "_ServerOpts",
    "igs_request": "_Request",
    "igs_completion": "_Completion",
    "igs_server_stats": "_ServerStats",
}


def _c_layout(pkg):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "igs.h"', '#include "igs_batch.h"',
             '#include "igs_serve.h"', "int main(void) {"]
    for cname, pyname in PAIRS.items():
        cls = getattr(pkg, pyname)
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "layout.c")
        exe = os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines) + "\n")
        subprocess.run([gcc, "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    res = {}
    for ln in out.splitlines():
        cname, field, val = ln.split()
        res[(cname, field)] = int(val)
    return res


def test_ctypes_structs_match_the_headers():
    import paper_2205_07805_gb300 as pkg
    lay = _c_layout(pkg)
    for cname, pyname in PAIRS.items():
        cls = getattr(pkg, pyname)
        assert C.sizeof(cls) == lay[(cname, "sizeof")], (cname, C.sizeof(cls), lay[(cname, "sizeof")])
        for f, _ in cls._fields_:
            assert getattr(cls, f).offset == lay[(cname, f)], (cname, f)


def test_constants_match_the_headers():
    """Status codes, methods, precisions and kernel classes of the binding are the headers'."""
    import paper_2205_07805_gb300 as pkg
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    names = {"IGS_OK": pkg.OK, "IGS_NOT_CONVERGED": pkg.NOT_CONVERGED, "IGS_BREAKDOWN": pkg.BREAKDOWN,
             "IGS_EINVAL": pkg.EINVAL, "IGS_ENOMEM": pkg.ENOMEM, "IGS_ECUDA": pkg.ECUDA,
             "IGS_ENUMERIC": pkg.ENUMERIC, "IGS_ETIMEOUT": pkg.ETIMEOUT, "IGS_ENOTIMPL": pkg.ENOTIMPL,
             "IGS_METHOD_IGS": pkg.METHODS["igs"], "IGS_METHOD_ONE_REDUCE": pkg.METHODS["one_reduce"],
             "IGS_PREC_FP64": pkg.PRECISIONS["fp64"], "IGS_PREC_FP32_IR": pkg.PRECISIONS["fp32_ir"],
             "IGS_KCLASS_COUNT": len(pkg.KCLASS_NAMES)}
    body = "\n".join(f'  printf("{k} %d\\n", (int){k});' for k in names)
    src_text = ('#include <stdio.h>\n#include "igs.h"\n#include "igs_batch.h"\n#include "igs_serve.h"\n'
                "int main(void) {\n" + body + "\n  return 0;\n}\n")
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "consts.c"), os.path.join(d, "consts")
        open(src, "w").write(src_text)
        subprocess.run([gcc, "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    got = {k: int(v) for k, v in (ln.split() for ln in out.splitlines())}
    assert got == names
