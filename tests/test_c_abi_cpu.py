"""The boundary as a C program sees it: include/pyronn.h compiles as strict C99, and a program linked
against libpyronn.so creates a geometry, queries its description, forward-projector and adjoint
configurations and sample count, reads the error state of a rejected call and releases the handle.
These are host calls only, so no GPU is needed."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "pyronn.h"

int main(void) {
    pyronn_vol_desc vol = {3, {16, 24, 32}, {0.5, 0.5, 0.5}, {0.0, 0.0, 0.0}};
    pyronn_det_desc det = {{20, 40}, {0.6, 0.6}, {0.0, 0.0}};
    pyronn_geom_t g = NULL;
    int fp[20], adj[8], n_views = 0, kind = -1, ndim = 0;
    int64_t samples = 0;
    if (pyronn_version() <= 0) return 2;
    if (pyronn_geom_create_cone_circular(&vol, &det, 12, 6.283185307179586, 750.0, 1200.0, 0.0, &g) != PYRONN_OK)
        return 3;
    if (pyronn_geom_info(g, &n_views, &kind, &ndim) != PYRONN_OK || n_views != 12 || kind != 1 || ndim != 3) return 4;
    if (pyronn_geom_fp_config(g, PYRONN_F32, fp) != PYRONN_OK) return 5;
    if (pyronn_geom_adjoint_config(g, adj) != PYRONN_OK) return 6;
    if (pyronn_geom_count_samples(g, &samples) != PYRONN_OK || samples <= 0) return 7;
    /* a rejected call (null geometry) returns an error code and leaves a message */
    if (pyronn_fp(NULL, NULL, NULL, PYRONN_F32, 1, NULL) != PYRONN_INVALID_ARG) return 8;
    if (strlen(pyronn_last_error()) == 0) return 9;
    printf("%d %d %d %d %lld\n", fp[0], fp[16], adj[0], adj[1], (long long)samples);
    if (pyronn_geom_destroy(g) != PYRONN_OK) return 10;
    return 0;
}
"""


@pytest.fixture(scope="module")
def libdir():
    from paper_2511_08427_gb300 import build
    return os.path.dirname(build.build())


def test_header_compiles_as_c99_and_links(libdir, tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "abi.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "abi"
    cmd = [cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"), str(src),
           "-L", libdir, "-lpyronn", "-Wl,-rpath," + libdir, "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    fp_kernel, xt, adj_kernel, adj_depth, samples = (int(v) for v in r.stdout.split())
    # nx = 32 and ny = 24 FP32 elements are multiples of 16 bytes: TMA projector with the y-fastest copy
    assert fp_kernel == 3 and xt == 1
    assert adj_kernel == 3 and adj_depth in (8, 6, 5, 4)
    assert samples > 0
