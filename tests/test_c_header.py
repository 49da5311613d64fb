"""The C ABI from C: include/apsp_fw.h compiles as strict C99 and C++17 with
warnings as errors, a C program links against libapspfw.so, and the calls that
need no GPU (argument checks, status strings, block size, variant table)
answer as the header documents.  CPU only."""
import os
import shutil
import subprocess

import pytest

from paper_2105_07298_gb300 import build as apsp_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "apsp_fw.h"

static int fails = 0;
#define EXPECT(cond) do { if (!(cond)) { printf("failed: %s\n", #cond); ++fails; } } while (0)

int main(void) {
  int32_t n[2] = {4, 1025};
  int64_t off[2] = {0, 16};
  int32_t block = 0, tr = 0, tc = 0, eager = 0;
  apsp_batched_plan *plan = NULL;
  EXPECT(apsp_version() >= 100);
  EXPECT(apsp_fw_block_size(4) == 128 && apsp_fw_block_size(8) == 128 && apsp_fw_block_size(2) == 0);
  EXPECT(strcmp(apsp_status_string(APSP_OK), "APSP_OK") == 0);
  EXPECT(strncmp(apsp_status_string(APSP_ENEGCYCLE), "APSP_ENEGCYCLE", 14) == 0);
  EXPECT(apsp_fw_f32(NULL, 0, 0, NULL, NULL) == APSP_OK);
  EXPECT(apsp_fw_f32(NULL, 5, 5, NULL, NULL) == APSP_EINVAL);
  EXPECT(apsp_fw_f64(NULL, 5, 4, NULL, NULL) == APSP_EINVAL);
  EXPECT(apsp_fw_i32(NULL, -1, 4, NULL, NULL) == APSP_EINVAL);
  EXPECT(apsp_fw_f32_host(NULL, NULL, NULL, 5, NULL, NULL, NULL) == APSP_EINVAL);
  EXPECT(apsp_batched_plan_create(n, off, 2, &plan) == APSP_EUNSUPPORTED && plan == NULL);
  EXPECT(apsp_fw_batched_f32(NULL, NULL, n, off, 2, NULL) == APSP_EUNSUPPORTED);
  EXPECT(apsp_fw_batched_f32_noalloc(NULL, NULL, n, off, -1, NULL) == APSP_EINVAL);
  EXPECT(apsp_batched_num_classes() == 4);
  EXPECT(apsp_batched_variant_info(2, &block, &tr, &tc, &eager) == APSP_OK);
  EXPECT(block == 128 && tr == 8 && tc == 4 && eager == 1);
  EXPECT(apsp_check_negative_cycle(NULL, 3, 4, 4, NULL) == APSP_EINVAL);
  EXPECT(apsp_wait_timeout_selftest(0, NULL) == APSP_EINVAL);
  printf("%s\n", fails ? "FAIL" : "OK");
  return fails != 0;
}
"""


def _need(tool):
    if shutil.which(tool) is None:
        pytest.skip(f"{tool} not found")


@pytest.mark.parametrize("compiler,std", [("gcc", "-std=c99"), ("g++", "-std=c++17")])
def test_header_compiles_cleanly(tmp_path, compiler, std):
    _need(compiler)
    src = tmp_path / ("h.c" if compiler == "gcc" else "h.cpp")
    src.write_text('#include "apsp_fw.h"\nint apsp_header_only_check(void) { return APSP_OK; }\n')
    subprocess.run([compiler, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                    f"-I{os.path.join(ROOT, 'include')}", str(src)], check=True)


def test_c_program_links_and_calls_the_library(tmp_path):
    _need("gcc")
    lib = apsp_build.build()
    src = tmp_path / "abi.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "abi"
    libdir = os.path.dirname(lib)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", f"-I{os.path.join(ROOT, 'include')}", str(src),
                    "-o", str(exe), lib, f"-Wl,-rpath,{libdir}"], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), r.stdout + r.stderr
