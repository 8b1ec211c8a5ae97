"""The boundary from plain C: include/kd.h compiles as strict C99 on its own, and a C
program linked against libkd.so calls the host-only entry points (no GPU involved)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1902_00387_gb300")

PROGRAM = r"""
#include <math.h>
#include <stdio.h>
#include <string.h>
#include "kd.h"

int main(void) {
  kd_params p;
  kd_ctx* ctx = NULL;
  double h[2 * 4], eig[2 * 2];
  memset(&p, 0, sizeof(p));
  p.flow = KD_FLOW_GALLOWAY_PROCTOR;
  p.n = 15;                                     /* odd: rejected on the host */
  p.kz = 0.57; p.Rm = 100.0; p.dt_fine = 5e-3; p.n_coarse = 16; p.dt_coarse = 5e-3;
  if (kd_create(&p, NULL, &ctx) != KD_EINVAL || ctx != NULL) return 1;
  if (kd_destroy(NULL) != KD_OK) return 2;
  if (strcmp(kd_last_error(NULL), "NULL context") != 0) return 3;
  /* [[2, 1], [0, 3]]: eigenvalues 2 and 3 */
  memset(h, 0, sizeof(h));
  h[0] = 2.0; h[2] = 1.0; h[6] = 3.0;
  if (kd_hessenberg_eig(2, h, eig, NULL) != KD_OK) return 4;
  if (!((fabs(eig[0] - 2.0) < 1e-14 && fabs(eig[2] - 3.0) < 1e-14) ||
        (fabs(eig[0] - 3.0) < 1e-14 && fabs(eig[2] - 2.0) < 1e-14))) return 5;
  if (kd_hessenberg_eig(0, h, eig, NULL) != KD_EINVAL) return 6;
  {
    size_t held = 7, limit = 7;
    if (kd_set_alloc_limit(NULL, 1u << 20) != KD_EINVAL) return 7;
    if (kd_get_alloc_bytes(NULL, &held, &limit) != KD_EINVAL || held != 7 || limit != 7) return 8;
  }
  printf("%s\n", kd_version());
  return 0;
}
"""


@pytest.fixture(scope="module")
def lib_path():
    import __graft_entry__
    __graft_entry__.build()
    return os.path.join(PKG, "libkd.so")


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_header_is_strict_c99(tmp_path):
    src = tmp_path / "h.c"
    src.write_text('#include "kd.h"\nint kd_header_only;\n')
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I",
                        os.path.join(ROOT, "include"), "-c", str(src), "-o", str(tmp_path / "h.o")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_c_program_calls_the_host_entry_points(tmp_path, lib_path):
    src = tmp_path / "prog.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "prog"
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                        "-L", PKG, "-lkd", "-Wl,-rpath," + PKG, "-lm", "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, (r.returncode, r.stderr)
    assert r.stdout.startswith("kd ")


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_struct_layouts_match_the_binding(tmp_path):
    """sizeof and every field offset of the ABI structs, from the C compiler, equal those
    of the ctypes structures of the binding."""
    import paper_1902_00387_gb300.kd as K
    structs = [K.kd_params, K.kd_parareal_stats, K.kd_instance, K.kd_instance_result, K.kd_sweep_stats]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "kd.h"', "int main(void) {"]
    for st in structs:
        name = st.__name__
        lines.append('  printf("%s sizeof %%zu\\n", sizeof(%s));' % (name, name))
        for f in st._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, f[0], name, f[0]))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        s, f, v = line.split()
        got[(s, f)] = int(v)
    for st in structs:
        name = st.__name__
        assert got[(name, "sizeof")] == K.ctypes.sizeof(st), name
        for f in st._fields_:
            assert got[(name, f[0])] == getattr(st, f[0]).offset, (name, f[0])


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_readme_c_example_compiles(tmp_path):
    """The C calling sequence shown in README.md compiles as C99 against include/kd.h."""
    import re
    text = open(os.path.join(ROOT, "README.md")).read()
    blocks = re.findall(r"```c\n(.*?)```", text, flags=re.S)
    assert blocks, "README.md has no C example"
    src = tmp_path / "readme.c"
    src.write_text(blocks[0])
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-c", str(src),
                        "-o", str(tmp_path / "readme.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
