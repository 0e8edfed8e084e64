"""CPU-side checks of the C ABI: the library builds, loads, exports every declared entry point,
the ctypes structures match the C layout, and argument validation answers without a GPU."""

import ctypes
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in ("sg.h", "sgnet.h")]


@pytest.fixture(scope="module")
def lib():
    from paper_1910_11505_gb300 import build as B
    B.build()
    from paper_1910_11505_gb300 import sg
    return sg.load_library()


def _declared():
    text = "".join(open(h).read() for h in HEADERS)
    return sorted(set(re.findall(r"^\s*(?:int|void|long long|const char\*)\s+(sg\w+)\s*\(", text, re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    from paper_1910_11505_gb300 import sg
    assert sorted(sg.EXPORTED) == names


def test_struct_layout_matches_c(tmp_path):
    from paper_1910_11505_gb300 import sg
    src = tmp_path / "lay.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "sg.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(sg_params),'
                   ' offsetof(sg_params, precision), offsetof(sg_params, inner_rtol),'
                   ' offsetof(sg_params, graphs),'
                   ' sizeof(sg_solve_info), offsetof(sg_solve_info, seconds)); return 0;}\n')
    exe = tmp_path / "lay"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    got = [ctypes.sizeof(sg.sg_params), sg.sg_params.precision.offset, sg.sg_params.inner_rtol.offset,
           sg.sg_params.graphs.offset, ctypes.sizeof(sg.sg_solve_info), sg.sg_solve_info.seconds.offset]
    assert [int(v) for v in out] == got


def test_defaults_and_argument_errors_without_gpu(lib):
    from paper_1910_11505_gb300 import sg
    p = sg.sg_default_params()
    assert (p.n, p.M, p.p, p.restart, p.precond) == (16, 2, 2, 30, sg.SG_PC_MEAN)
    assert p.rtol == 1e-10 and p.inner_rtol == 1e-4
    bad = [dict(n=1), dict(M=0), dict(M=9), dict(p=7), dict(ell=0.0), dict(sigma=-1.0),
           dict(restart=0), dict(restart=1025), dict(precond=9), dict(precision=3),
           dict(inner_iters=0), dict(max_iters=0), dict(n=1025),
           dict(n=770, precond=sg.SG_PC_MEAN), dict(n=770, precond=sg.SG_PC_FS_GS)]
    for kw in bad:
        with pytest.raises(sg.SGError) as ei:
            sg.sg_setup(sg.sg_default_params(**kw), stream=0)
        assert ei.value.code == sg.SG_ERR_ARG, kw
    out = ctypes.c_void_p()
    assert lib.sg_setup(None, 1, None, ctypes.byref(out)) == sg.SG_ERR_ARG
    assert lib.sg_dims(None, 0, None, None, None) == sg.SG_ERR_ARG
    assert b"handle" in lib.sg_last_error()
    lib.sg_free(None)
