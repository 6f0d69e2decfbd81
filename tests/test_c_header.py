"""The boundary from C: include/nd.h compiles as C99 and as C++17 with every
warning an error, and a C program linked against libnd.so gets the
documented statuses from calls that need no GPU (argument checks made
before any CUDA call, the status strings, the process-wide limits).  The
Python tests go through ctypes; this one checks that a C caller, which sees
only the header, can use the library as it is."""
import os
import shutil
import subprocess

import pytest

from paper_1704_00386_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "nd.h"

#define EXPECT(call, want)                                                  \
    do {                                                                    \
        nd_status got_ = (call);                                            \
        if (got_ != (want)) {                                               \
            printf("FAIL line %d: %s gave %d (%s), want %d\n", __LINE__,    \
                   #call, (int)got_, nd_strerror(got_), (int)(want));       \
            return 1;                                                       \
        }                                                                   \
    } while (0)

int main(void) {
    static const int64_t rp[3] = {0, 1, 2};
    static const int32_t col[2] = {1, 0};
    nd_csr g;
    nd_incidence* h = NULL;
    int64_t a = 0, b = 0, nnz = 0;
    int q = 0;
    int32_t it = 0;
    int s;

    if (nd_abi_version() != 1) { printf("FAIL abi version\n"); return 1; }
    for (s = ND_OK; s <= ND_E_BUSY; ++s) {
        const char* msg = nd_strerror((nd_status)s);
        if (msg == NULL || msg[0] == '\0') { printf("FAIL strerror(%d)\n", s); return 1; }
    }
    if (strcmp(nd_strerror(ND_OK), "ok") != 0) { printf("FAIL strerror(ND_OK)\n"); return 1; }

    g.n = 2; g.nnz = 2; g.row_ptr = rp; g.col = col; g.on_device = 0;
    EXPECT(nd_build_incidence(NULL, 1, 2, NULL, &h), ND_E_INVAL);
    EXPECT(nd_build_incidence(&g, 1, 3, NULL, &h), ND_E_UNSUPPORTED_RS);
    EXPECT(nd_build_incidence(&g, 2, 2, NULL, &h), ND_E_INVAL);
    EXPECT(nd_build_incidence_ex(&g, 3, 4, ND_BUILD_ON_THE_FLY, NULL, &h), ND_E_UNSUPPORTED_RS);
    if (h != NULL) { printf("FAIL a refused build returned a handle\n"); return 1; }
    if (strlen(nd_last_error()) == 0) { printf("FAIL no message after a refusal\n"); return 1; }

    EXPECT(nd_incidence_info(NULL, &a, &b, &q), ND_E_INVAL);
    EXPECT(nd_snd(NULL, NULL, 0, 10, &it, NULL), ND_E_INVAL);
    EXPECT(nd_and(NULL, NULL, 0, 1, 10, &it, &a, NULL), ND_E_INVAL);
    EXPECT(nd_iterate_k(NULL, ND_SND, -1, NULL, 0, 0, &it, NULL), ND_E_INVAL);

    EXPECT(nd_normalize(NULL, NULL, -1, 4, 0, NULL, NULL, 0, &nnz, NULL), ND_E_INVAL);
    EXPECT(nd_normalize(NULL, NULL, 0, 4, 0, NULL, NULL, 0, NULL, NULL), ND_E_INVAL);
    EXPECT(nd_core_snd_noalloc(NULL, NULL, (int64_t)1 << 21, 0, NULL, 10, &it, NULL), ND_E_TOO_LARGE);
    EXPECT(nd_core_snd_noalloc(NULL, NULL, -1, 0, NULL, 10, &it, NULL), ND_E_INVAL);

    EXPECT(nd_set_wait_limit(0.0), ND_E_INVAL);
    EXPECT(nd_set_wait_limit(600.0), ND_OK);
    EXPECT(nd_set_handle_memory_limit(-1), ND_E_INVAL);
    EXPECT(nd_set_handle_memory_limit(0), ND_OK);
    nd_free(NULL);  /* a no-op */
    printf("ok\n");
    return 0;
}
"""


def _compile(tmp_path, compiler, std, src_name):
    src = tmp_path / src_name
    src.write_text(PROGRAM)
    exe = tmp_path / (src_name + ".bin")
    libdir = os.path.dirname(_build.build())
    cmd = [compiler, f"-std={std}", "-Wall", "-Wextra", "-Werror", "-pedantic",
           "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
           "-L", libdir, "-lnd", f"-Wl,-rpath,{libdir}"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    return exe


@pytest.mark.parametrize("compiler,std,src_name", [("gcc", "c99", "abi.c"), ("g++", "c++17", "abi.cc")])
def test_header_compiles_and_links_from_c(tmp_path, compiler, std, src_name):
    if shutil.which(compiler) is None:
        pytest.skip(f"{compiler} is not installed")
    exe = _compile(tmp_path, compiler, std, src_name)
    # run with no GPU visible, so every call above must decide before touching CUDA
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    res = subprocess.run([str(exe)], capture_output=True, text=True, env=env, timeout=120)
    assert res.returncode == 0, res.stdout + res.stderr
    assert res.stdout.strip().endswith("ok")
