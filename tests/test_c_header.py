"""The C ABI is usable from plain C: a C99 program that includes include/pod2g.h
compiles with gcc, links against libpod2g.so and makes host-only calls (options,
status strings, argument validation) without a GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_SRC = r"""
#include <stdio.h>
#include <string.h>
#include "pod2g.h"

int main(void) {
    pod2g_opts o;
    pod2g_default_opts(&o);
    pod2g_t h = 0;
    int bad = pod2g_create(NULL, NULL, 0, &o, &h);
    printf("%d %d %d %d %d %d|%s|%s\n", o.pre, o.post, o.chunk, o.method, o.smoother, bad,
           pod2g_strerror(POD2G_NOT_CONVERGED), pod2g_strerror(POD2G_TOO_LARGE));
    return (h == 0 && bad == POD2G_INVALID_ARG) ? 0 : 1;
}
"""


@pytest.fixture(scope="module")
def lib_path():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2207_02543_gb300 as pkg
    return pkg.LIB_PATH


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not available")
def test_c99_program_uses_the_abi(tmp_path, lib_path):
    src = tmp_path / "use_abi.c"
    src.write_text(C_SRC)
    exe = tmp_path / "use_abi"
    libdir = os.path.dirname(lib_path)
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                        "-o", str(exe), "-L", libdir, "-lpod2g", f"-Wl,-rpath,{libdir}"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    fields, s1, s2 = out.stdout.strip().split("|")
    assert fields.split() == ["1", "1", "8", "0", "0", "4"]
    assert s1.startswith("not converged") and "noalloc" in s2
