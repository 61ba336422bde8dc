"""The boundary from plain C: a C99 program includes include/ssvp.h (no C++), links libssvp.so and
calls it (no GPU needed: without one, ssvp_create reports SSVP_EDEVICE)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_SOURCE = r"""
#include <stdio.h>
#include <string.h>
#include "ssvp.h"

int main(void) {
    ssvp_params p;
    memset(&p, 0x5a, sizeof p);
    ssvp_params_default(&p);
    if (p.k != 7 || p.half_window != 15 || p.mode != SSVP_MODE_DENOISE || p.frame_end != -1) return 2;
    if (ssvp_sync(NULL) != SSVP_EINVAL) return 3;
    if (strlen(ssvp_trace_kind_name(SSVP_TRACE_GATHER)) == 0) return 4;
    ssvp_ctx *ctx = NULL;
    int rc = ssvp_create(&ctx, 0, NULL);
    if (rc == SSVP_OK) {
        ssvp_destroy(ctx);
        puts("create ok");
    } else {
        printf("create %d: %s\n", rc, ssvp_last_error(NULL));
        if (rc != SSVP_EDEVICE) return 5;
    }
    return 0;
}
"""


def test_a_c99_program_builds_against_the_header_and_runs(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    import paper_2102_03011_gb300 as ss  # the library is built
    lib_dir = os.path.dirname(ss.LIB_PATH)
    src = tmp_path / "client.c"
    src.write_text(C_SOURCE)
    exe = tmp_path / "client"
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    "-o", str(exe), "-L", lib_dir, "-lssvp", f"-Wl,-rpath,{lib_dir}"], check=True,
                   capture_output=True, text=True)
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, (run.returncode, run.stdout, run.stderr)
    assert run.stdout.startswith("create ")
