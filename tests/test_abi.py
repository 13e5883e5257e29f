"""The C ABI library: it loads, exports what include/cs.h declares, its ctypes
mirror of cs_params matches the C layout, and host-side argument checks
answer without a GPU."""
import ctypes
import os
import re
import subprocess
import sys

import numpy as np
import pytest

from paper_2405_00366_gb300 import build, cs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return cs.lib()


def _declared_functions():
    names = set()
    for f in os.listdir(INCLUDE):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(INCLUDE, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(cs_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert "cs_solve" in names and "cs_problem_create" in names and "cs_result" in names
    out = subprocess.run(["nm", "-D", "--defined-only", cs.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(lib, n)


def test_params_layout_matches_c(tmp_path):
    fields = [f for f, _ in cs.cs_params._fields_]
    src = tmp_path / "layout.c"
    body = "\n".join(f'  printf("{f} %zu\\n", offsetof(cs_params, {f}));' for f in fields)
    src.write_text(f"""#include <stddef.h>
#include <stdio.h>
#include "cs.h"
int main(void) {{
  printf("size %zu\\n", sizeof(cs_params));
{body}
  return 0;
}}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", INCLUDE, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = dict(line.split() for line in out.splitlines())
    assert int(got["size"]) == ctypes.sizeof(cs.cs_params)
    for f in fields:
        assert int(got[f]) == getattr(cs.cs_params, f).offset, f


def test_defaults(lib):
    p = cs.cs_params_default()
    assert (p.n_outer, p.n_steps, p.dt, p.p0, p.p1, p.beta, p.tau) == (20, 1000, 0.01, 0.0, 1.5, 0.2, 1.0)
    assert p.precision == cs.CS_P_FP32 and p.field == cs.CS_FIELD_CN and p.refit == cs.CS_REFIT_EXACT
    q = cs.cs_params_default(precision="fp64", field="bn", n_steps=7)
    assert (q.precision, q.field, q.n_steps) == (cs.CS_P_FP64, cs.CS_FIELD_BN, 7)


def test_host_argument_checks_need_no_gpu(lib):
    h = ctypes.c_void_p()
    A = np.zeros((3, 4))
    y = np.zeros(3)
    P = ctypes.c_void_p
    assert lib.cs_problem_create(None, P(y.ctypes.data), 3, 4, 0.1, 0, None, ctypes.byref(h)) == cs.CS_EINVAL
    assert "NULL" in cs.cs_last_error()
    assert lib.cs_problem_create(P(A.ctypes.data), P(y.ctypes.data), 0, 4, 0.1, 0, None,
                                 ctypes.byref(h)) == cs.CS_EINVAL
    assert lib.cs_problem_create(P(A.ctypes.data), P(y.ctypes.data), 3, 4, -1.0, 0, None,
                                 ctypes.byref(h)) == cs.CS_EINVAL
    assert lib.cs_problem_create(P(A.ctypes.data), P(y.ctypes.data), 3, 4, float("nan"), 0, None,
                                 ctypes.byref(h)) == cs.CS_EINVAL
    p = cs.cs_params_default()
    assert lib.cs_solve(None, ctypes.byref(p), 1) == cs.CS_EINVAL
    assert lib.cs_result(None, None, None, None, None) == cs.CS_EINVAL
    lib.cs_problem_destroy(None)


def test_tune_info_reports_cache_path(lib, tmp_path):
    """cs_tune_info answers on the host: no tunings yet and the cache file named by
    CS_TUNE_CACHE (read in a fresh process, which loads the file on first use)."""
    cache = tmp_path / "sub" / "tune.txt"
    code = ("import sys; sys.path.insert(0, sys.argv[1]); from paper_2405_00366_gb300 import cs; "
            "print(cs.cs_tune_info())")
    env = dict(os.environ, CS_TUNE_CACHE=str(cache))
    r = subprocess.run([sys.executable, "-c", code, ROOT], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip().splitlines()[-1] == repr((0, 0, str(cache)))


def test_tune_cache_file_with_bad_lines_loads(lib, tmp_path):
    """A tuning-cache file with malformed lines (no tab, empty key or value,
    binary junk, an over-long line) loads without error on the host: the process
    reports no tunings and no hits, and the file is left as it was."""
    cache = tmp_path / "tune.txt"
    junk = (b"no tab on this line\n\tempty key\nkey only\t\n" + bytes(range(1, 9)) + b"\n" + b"x" * 10000 +
            b"\tlong\nbatch|cs-tune-1|fake|sm103|152|p3|T16\t1 4 0 0\n")
    cache.write_bytes(junk)
    code = ("import sys; sys.path.insert(0, sys.argv[1]); from paper_2405_00366_gb300 import cs; "
            "print(cs.cs_tune_info())")
    env = dict(os.environ, CS_TUNE_CACHE=str(cache))
    r = subprocess.run([sys.executable, "-c", code, ROOT], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip().splitlines()[-1] == repr((0, 0, str(cache)))
    assert cache.read_bytes() == junk
