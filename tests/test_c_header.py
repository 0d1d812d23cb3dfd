"""include/fv.h is plain C: a C99 program that includes it compiles with
-Wall -Werror, links against libfv.so, and reaches the library's argument
checks (which run before any CUDA call, so no GPU is needed)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "fv.h"

int main(void) {
  double x = 0.0;
  int8_t f = 1;
  uint8_t st = 0;
  /* n < 0 and an unknown model are argument errors, reported before any launch */
  if (fv_implied_vol(FV_BLACK76, FV_LBR, &x, &x, &x, &x, &x, NULL, &f, -1, &x, &st, NULL) !=
      FV_ERR_ARG)
    return 1;
  if (strstr(fv_last_error(), "n = -1") == NULL) return 2;
  if (fv_price((fv_model)7, &f, &x, &x, &x, &x, NULL, &x, 1, &x, NULL) != FV_ERR_ARG) return 3;
  /* n = 0 touches nothing */
  if (fv_implied_vol(FV_BSM, FV_HALLEY, NULL, NULL, NULL, NULL, NULL, NULL, NULL, 0, NULL, NULL,
                     NULL) != FV_SUCCESS)
    return 4;
  if (fv_workspace_size(FV_LBR, 1000) != 0 || fv_workspace_size(FV_HALLEY, 1000) < 1000) return 5;
  /* the stream plan's transfer mode: a plan is required */
  int mode = -1;
  if (fv_stream_plan_set_transfer(NULL, FV_TRANSFER_DIRECT) != FV_ERR_ARG) return 6;
  if (fv_stream_plan_last_transfer(NULL, &mode) != FV_ERR_ARG || mode != -1) return 7;
  printf("%s\n", fv_status_string(FV_ERR_UNSUPPORTED));
  return 0;
}
"""


@pytest.fixture(scope="module")
def lib():
    from paper_2604_27210_gb300 import build
    return build.build()


def test_header_compiles_as_c_and_links(tmp_path, lib):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_fv.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "use_fv"
    libdir = os.path.dirname(lib)
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe), "-L", libdir, "-l:libfv.so",
                    "-Wl,-rpath," + libdir], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert "UNSUPPORTED" in r.stdout
