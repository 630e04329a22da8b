"""The boundary is a C ABI: a plain C99 program compiles against include/lbfmm.h, links
liblbfmm and calls its host-only entry points (options, workspace sizes, status strings;
no GPU needed)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include "lbfmm.h"
int main(void)
{
    lbf_options o;
    if (lbf_default_options(&o) != LBF_OK) return 1;
    const int64_t ptr[4] = {0, 300, 700, 1000};
    size_t plan = 0, batch = 0;
    if (lbf_workspace_size(3, ptr, &o, &plan) != LBF_OK) return 2;
    if (lbf_batch_workspace_size(3, ptr, &o, 16, &batch) != LBF_OK) return 3;
    o.restart = 0;
    const int bad = lbf_workspace_size(3, ptr, &o, &plan);
    printf("%d %zu %zu %d %s\n", o.p, plan, batch, bad, lbf_status_string(bad));
    return 0;
}
"""


def test_c_program_links_and_calls_the_host_entry_points(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    from paper_1306_0612_gb300.build import LIB, build

    build()
    src = tmp_path / "client.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "client"
    libdir = os.path.dirname(LIB)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe), "-L", libdir, "-llbfmm", "-Wl,-rpath," + libdir],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    p, plan, batch, bad = int(out[0]), int(out[1]), int(out[2]), int(out[3])
    assert p == 26 and plan > 0 and batch > plan
    assert bad < 0 and " ".join(out[4:]) == "invalid argument"
