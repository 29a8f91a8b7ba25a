"""The boundary is a C ABI: include/acs.h compiles as strict C99 without
warnings, and a C program linked against the library gets the documented
defaults and the host-side error codes (no device needed)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIBDIR = os.path.join(ROOT, "paper_2103_00736_gb300")

CLIENT = r"""
#include <stdio.h>
#include <string.h>
#include "acs.h"

int main(void) {
    acs_settings s;
    if (acs_settings_default(&s) != ACS_SOLVED) return 10;
    if (s.mu != 1.0 || s.t != 9.2 || s.cond_first != 300 || s.cond_period != 100) return 11;
    if (strstr(acs_version(), "sm_103a") == NULL) return 12;

    /* a row without entries: malformed CSR, refused before the device */
    int64_t row_ptr[3] = {0, 1, 1};
    int32_t col[1] = {0};
    double val[1] = {1.0}, b[2] = {1.0, 1.0}, c[2] = {1.0, 1.0};
    acs_problem* p = NULL;
    if (acs_problem_create(2, 2, row_ptr, col, val, b, c, 2, 0, NULL, &s, &p) != ACS_ERR_CSR || p) return 13;

    /* cone sizes that do not add up to n */
    int64_t rp2[3] = {0, 1, 2};
    int32_t col2[2] = {0, 1};
    double val2[2] = {1.0, 1.0};
    int32_t dims[1] = {3};
    if (acs_problem_create(2, 2, rp2, col2, val2, b, c, 0, 1, dims, &s, &p) != ACS_ERR_CONES || p) return 14;

    /* the team assignment of the serving loop, host only */
    double work[2] = {3.0 * 16384.0, 100.0};
    int32_t cta[3 * 8];
    if (acs_debug_assign_teams(2, work, 8, cta) != ACS_SOLVED) return 15;
    if (cta[0] != 0 || cta[1] != 0 || cta[2] != 1 || cta[2 * 8] != 2) return 16;

    acs_server_config cfg;
    if (acs_server_config_default(&cfg) != ACS_SOLVED || cfg.round_ms != 2.0) return 17;
    printf("ok %s\n", acs_status_string(ACS_ERR_CSR));
    return 0;
}
"""


@pytest.fixture(scope="module")
def lib_built():
    from paper_2103_00736_gb300 import capi, build
    if not os.path.exists(capi.LIB_PATH):
        build.build()
    return capi.LIB_PATH


def test_header_is_c99_and_a_c_client_runs(lib_built, tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "client.c"
    src.write_text(CLIENT)
    exe = tmp_path / "client"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        f"-I{os.path.join(ROOT, 'include')}", str(src), f"-L{LIBDIR}", "-lacs",
                        f"-Wl,-rpath,{LIBDIR}", "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert r.stdout.startswith("ok ")
