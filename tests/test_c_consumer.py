"""The boundary from C: a C99 program compiled against include/rmips.h and
linked to librmips.so (no Python, no torch), calling the host-only entry
points -- no GPU needed."""
import os
import shutil
import subprocess

import pytest

from paper_2110_07131_gb300 import rmips

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_SOURCE = r"""
#include <stdio.h>
#include <string.h>
#include "rmips.h"

int main(void) {
  /* u.(a - b) = 1*(1 - 0) + 2*(0 - 1) = -1: negative */
  const float u[2] = {1.0f, 2.0f}, a[2] = {1.0f, 0.0f}, b[2] = {0.0f, 1.0f};
  if (rmips_exact_sign_host(u, a, b, 2) != -1) return 1;
  if (rmips_exact_sign_host(u, a, a, 2) != 0) return 2;       /* an exact tie */
  if (rmips_exact_sign_host(u, b, a, 2) != 1) return 3;
  if (strcmp(rmips_status_string(RMIPS_OK), "ok") != 0) return 4;
  if (strstr(rmips_status_string(RMIPS_ERR_CAPACITY), "capacity") == NULL) return 5;
  /* a null argument is refused with a status and a message, before any device call */
  rmips_index* idx = (rmips_index*)0;
  rmips_status s = rmips_build_index(NULL, 0, NULL, 0, 0, NULL, NULL, &idx);
  if (s != RMIPS_ERR_ARG || idx != NULL || strlen(rmips_last_error()) == 0) return 6;
  printf("c consumer ok\n");
  return 0;
}
"""


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not available")
def test_c_program_uses_the_library_through_its_header(tmp_path):
    lib = rmips.load_library()          # builds librmips.so if needed
    assert lib is not None
    libdir = os.path.dirname(rmips.LIB_PATH)
    src = tmp_path / "consumer.c"
    src.write_text(C_SOURCE)
    exe = tmp_path / "consumer"
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
           "-o", str(exe), "-L", libdir, "-l:librmips.so", f"-Wl,-rpath,{libdir}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60,
                       env={**os.environ, "CUDA_VISIBLE_DEVICES": ""})
    assert r.returncode == 0 and "c consumer ok" in r.stdout, (r.returncode, r.stdout, r.stderr)
