"""The boundary from plain C, without Python or a GPU: ``include/sf.h``
compiles as strict C99, and a C program linked against ``libsf_gb300.so``
calls the device-free entry points (the launch planner, argument
validation of ``sf_create``)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2501_19042_gb300")

PROGRAM = r"""
#include <stdio.h>
#include "sf.h"
int main(void) {
  int nr[1] = {16}, ns[1] = {1024}, out[4] = {0, 0, 0, 0};
  size_t smem = 0;
  sf_status st = sf_plan_launch(3, 100, 1, nr, ns, SF_PREC_FP32, 152, 232448, out, &smem);
  printf("%d %d %d %d %d %zu\n", (int)st, out[0], out[1], out[2], out[3], smem);
  sf_problem bad = {0};
  sf_handle *h = NULL;
  printf("%d %d\n", (int)sf_create(&bad, 0, &h), h == NULL);
  printf("%d\n", (int)sf_plan_launch(3, 100, 1, nr, ns, 7, 152, 232448, out, NULL));
  return 0;
}
"""


@pytest.fixture(scope="module")
def built():
    import paper_2501_19042_gb300 as P
    P.build()
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")


def test_header_is_strict_c99(built, tmp_path):
    src = tmp_path / "h.c"
    src.write_text('#include "sf.h"\nint main(void) { return (int)(sizeof(sf_problem) == 0); }\n')
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-I", os.path.join(ROOT, "include"), "-c", str(src), "-o", str(tmp_path / "h.o")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_c_program_calls_the_library(built, tmp_path):
    src = tmp_path / "consumer.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "consumer"
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-I", os.path.join(ROOT, "include"), str(src),
                        "-L", PKG, "-lsf_gb300", "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, LD_LIBRARY_PATH=PKG + os.pathsep + os.environ.get("LD_LIBRARY_PATH", ""))
    r = subprocess.run([str(exe)], capture_output=True, text=True, env=env, timeout=60)
    assert r.returncode == 0, r.stderr
    lines = r.stdout.split("\n")
    st, G, warps, tc, nq, smem = (int(x) for x in lines[0].split())
    assert (st, G, warps, tc, nq) == (0, 7, 11, 50, 3) and 0 < smem <= 232448
    assert lines[1].split() == ["1", "1"]     # SF_ERR_INVALID_ARG, no handle returned
    assert lines[2] == "1"                     # unknown precision rejected
