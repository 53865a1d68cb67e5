"""include/fc.h is usable from plain C: a C99 program that includes it
compiles warning-free, links against libfc.so and calls the host-only entry
points (no GPU needed)."""
import os
import shutil
import subprocess

import pytest

from paper_2101_06192_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "fc.h"

int main(void) {
  /* Hoeffding tree count of Algorithm 1 (host arithmetic) */
  int64_t tau = fc_tau_for(0.1, 0.1, 0.5, 60);
  if (tau <= 0) return 1;
  if (fc_tau_for(0.0, 0.1, 0.5, 60) != -1) return 2;
  if (fc_mlp_param_count() != 769) return 3;
  if (strcmp(fc_status_str(FC_EINVAL), "") == 0) return 4;
  /* argument errors are reported without touching a device */
  if (fc_graph_info(NULL, NULL, NULL, NULL, NULL) != FC_EINVAL) return 5;
  if (fc_last_error_message()[0] == '\0') return 6;
  printf("%lld\n", (long long)tau);
  return 0;
}
"""


def test_c99_program_compiles_links_and_runs(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    lib = build.build()
    libdir = os.path.dirname(lib)
    src = tmp_path / "use_fc.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "use_fc"
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
           str(src), "-o", str(exe), "-L", libdir, "-l:" + os.path.basename(lib), "-Wl,-rpath," + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, (r.returncode, r.stderr)
    assert int(r.stdout.strip()) > 0
