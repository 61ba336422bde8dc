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


def test_binding_structs_match_the_header_field_by_field(tmp_path):
    """Every field of the public structures sits at the same offset in the C header and in the
    ctypes binding, and the structures have the same size."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    import ctypes
    import paper_2102_03011_gb300 as ss
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "ssvp.h"', "int main(void) {"]
    structs = {"ssvp_params": ss.ssvp_params, "ssvp_plan_config": ss.ssvp_plan_config,
               "ssvp_train_config": ss.ssvp_train_config}
    for cname, py in structs.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        cname, field, value = line.split()
        got[(cname, field)] = int(value)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
