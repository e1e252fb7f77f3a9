"""The boundary is plain C: include/*.h compile as strict C99 and C++17, and
a C program linked against libbamg.so calls the host-side entry points
(defaults, status strings, argument checks, network parameter files) with
no Python and no GPU involved."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INC = os.path.join(ROOT, "include")

CLIENT = r"""
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include "bamg.h"
#include "bamg_steps.h"

int main(int argc, char** argv) {
  if (argc < 2) return 2;
  bamg_params p;
  if (bamg_params_default(&p) != BAMG_OK) return 3;
  printf("defaults %d %d %d %.2f %d\n", p.r, p.nu_pre, p.nu_post, p.omega, p.c_max);
  printf("status %s | %s\n", bamg_status_string(BAMG_ERR_IO), bamg_status_string(BAMG_ERR_ARG));
  bamg_hierarchy* h = NULL;
  printf("setup-null %d\n", (int)bamg_setup(NULL, &p, NULL, &h));
  int np = bamg_mlp_num_params();
  float* w = (float*)malloc(sizeof(float) * np);
  float* back = (float*)malloc(sizeof(float) * np);
  for (int i = 0; i < np; ++i) { w[i] = 0.5f * (float)i - 7.0f; back[i] = 0.0f; }
  int s1 = (int)bamg_mlp_save(argv[1], w, 0, NULL);
  int s2 = (int)bamg_mlp_load(argv[1], back, 0, NULL);
  int same = 1;
  for (int i = 0; i < np; ++i) same &= (back[i] == w[i]);
  printf("file %d %d %d %d\n", np, s1, s2, same);
  FILE* f = fopen(argv[1], "r+b");
  if (!f) return 4;
  fseek(f, 40, SEEK_SET);
  fputc(0x5a, f);
  fclose(f);
  back[0] = 42.0f;
  int s3 = (int)bamg_mlp_load(argv[1], back, 0, NULL);
  printf("corrupt %d %.1f %s\n", s3, back[0], bamg_last_error()[0] ? "msg" : "nomsg");
  free(w);
  free(back);
  return 0;
}
"""


def _gcc():
    g = shutil.which("gcc")
    if not g:
        pytest.skip("gcc not available")
    return g


@pytest.mark.parametrize("lang", [["-x", "c", "-std=c99", "-pedantic"], ["-x", "c++", "-std=c++17"]])
def test_headers_are_strict_c_and_cpp(tmp_path, lang):
    src = tmp_path / "h.c"
    src.write_text('#include "bamg.h"\n#include "bamg_steps.h"\nint main(void) { return 0; }\n')
    r = subprocess.run([_gcc()] + lang + ["-Wall", "-Wextra", "-Werror", "-fsyntax-only", "-I", INC, str(src)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_c_program_uses_the_library_without_python(tmp_path):
    import __graft_entry__ as g
    g.build()
    from paper_1402_4005_gb300 import _lib
    libdir = os.path.dirname(_lib.LIB_PATH)
    src = tmp_path / "client.c"
    src.write_text(CLIENT)
    exe = tmp_path / "client"
    r = subprocess.run([_gcc(), "-std=c99", "-Wall", "-Werror", "-I", INC, str(src), "-o", str(exe),
                        "-L", libdir, "-lbamg", f"-Wl,-rpath,{libdir}"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    cuda_lib = "/usr/local/cuda/lib64"
    env = dict(os.environ)
    env["LD_LIBRARY_PATH"] = cuda_lib + (":" + env["LD_LIBRARY_PATH"] if env.get("LD_LIBRARY_PATH") else "")
    r = subprocess.run([str(exe), str(tmp_path / "net.bin")], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    lines = r.stdout.splitlines()
    assert lines[0] == "defaults 8 3 3 0.70 4"
    assert lines[1] == "status file error | invalid argument"
    assert lines[2] == "setup-null 1"
    assert lines[3] == "file 9360 0 0 1"
    assert lines[4] == "corrupt 10 42.0 msg"
