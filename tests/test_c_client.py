"""The boundary from plain C: include/sphere_poisson.h compiles as C99 with
warnings as errors, and a C program linked against the built library calls the
host-side entry points that touch no device (status strings, the plan's size and
argument checks, the null-handle checks).  No GPU is needed."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_CLIENT = r"""
#include <stdio.h>
#include <string.h>
#include "sphere_poisson.h"

int main(void) {
  sp_plan_t plan = (sp_plan_t)0;
  size_t ws = 0;
  int bad = 0;
  /* odd n_lambda, a prime factor above 31, a length above 12288 */
  if (sphere_poisson_plan(&plan, 8, 15, SP_FP64, 0, 0u, &ws) != SP_ERR_BAD_SIZE) bad |= 1;
  if (sphere_poisson_plan(&plan, 37, 74, SP_FP64, 0, 0u, &ws) != SP_ERR_BAD_SIZE) bad |= 2;
  if (sphere_poisson_plan(&plan, 12800, 64, SP_FP64, 0, 0u, &ws) != SP_ERR_BAD_SIZE) bad |= 4;
  if (plan != (sp_plan_t)0) bad |= 8;
  if (sphere_poisson_plan(&plan, 8, 16, 99, 0, 0u, &ws) != SP_ERR_UNSUPPORTED) bad |= 16;
  if (sphere_poisson_plan((sp_plan_t*)0, 8, 16, SP_FP64, 0, 0u, &ws) != SP_ERR_NULL) bad |= 32;
  if (sphere_poisson_solve((sp_plan_t)0, (const double*)0, (double*)0, (void*)0, 0, (void*)0,
                           (double*)0) != SP_ERR_BAD_PLAN) bad |= 64;
  if (strlen(sphere_poisson_status_string(SP_ERR_BAD_SIZE)) < 5) bad |= 128;
  printf("%s\n", sphere_poisson_status_string(SP_ERR_BAD_SIZE));
  return bad;
}
"""


def test_header_compiles_as_c99():
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-fsyntax-only",
                        "-I", os.path.join(ROOT, "include"), "-x", "c", "-"],
                       input="#include \"sphere_poisson.h\"\nint main(void) { return 0; }\n",
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_c_program_links_and_calls_the_host_checks(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_1510_08094_gb300 import _lib

    lib = _lib.load()
    so = lib._name
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                        so, "-Wl,-rpath," + os.path.dirname(so), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert "bad grid size" in r.stdout
