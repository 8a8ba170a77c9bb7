"""The C ABI from C: include/lfmm.h compiles as strict C99 and a C program links the
library and calls its host-only entry points (no GPU needed)."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "lfmm.h"

int main(void) {
    /* a unit square: four elements, chord midpoints, lengths and outward normals */
    const int32_t counts[1] = {4};
    const double verts[8] = {0, 0, 1, 0, 1, 1, 0, 1};
    double pts[8], w[4], nrm[8];
    const double yint[1] = {0.0};
    const double k_bad[4] = {4.0, 0.0, -1.0, 0.0};   /* k <= 0 in the second layer */
    const double k_ok[4] = {4.0, 0.0, 6.0, 0.0};
    const double eta[2] = {1.0, 2.0};
    lfmm_medium m = NULL;
    lfmm_status st;
    if (lfmm_polygon_elements(1, counts, verts, pts, w, nrm) != LFMM_OK) return 1;
    if (pts[0] != 0.5 || pts[1] != 0.0 || w[2] != 1.0 || nrm[1] != -1.0) return 2;
    st = lfmm_medium_create(2, yint, k_bad, eta, &m);
    if (st != LFMM_ERR_INVALID_ARG || m != NULL) return 3;
    if (strlen(lfmm_last_error()) == 0) return 4;
    st = lfmm_medium_create(2, yint, k_ok, eta, &m);
    if (st != LFMM_OK || m == NULL) return 5;
    if (lfmm_medium_destroy(m) != LFMM_OK) return 6;
    printf("ok %d\n", (int)LFMM_C64);
    return 0;
}
"""


@pytest.fixture(scope="module")
def libdir():
    from paper_2511_12450_gb300 import _build

    _build.build()
    d = os.path.join(ROOT, "paper_2511_12450_gb300", "_lib")
    assert os.path.exists(os.path.join(d, "liblfmm.so"))
    return d


def test_header_is_strict_c99_and_links(libdir):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    work = os.path.join(ROOT, "tests", "_build")   # git-ignored
    os.makedirs(work, exist_ok=True)
    src = os.path.join(work, "use_lfmm.c")
    with open(src, "w") as f:
        f.write(C_PROGRAM)
    exe = os.path.join(work, "use_lfmm")
    cmd = [cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
           str(src), "-o", str(exe), "-L", libdir, "-llfmm", "-Wl,-rpath," + libdir]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, (run.returncode, run.stdout, run.stderr)
    assert run.stdout.strip() == "ok 16"
