"""The C-ABI library builds, loads and exports every entry point that include/kd.h
declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "kd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kd_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1902_00387_gb300 as kd
    return kd.load()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ["kd_create", "kd_destroy", "kd_fine_batched", "kd_coarse", "kd_parareal_run", "kd_growth_rate"]:
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    for s in declared_symbols():
        assert hasattr(lib, s), s


def test_binding_names_match_header(lib):
    import paper_1902_00387_gb300 as kd
    for s in declared_symbols():
        assert callable(getattr(kd, s)), s


def test_version_and_argument_validation_without_gpu(lib):
    import paper_1902_00387_gb300 as kd
    assert "sm_103a" in kd.kd_version()
    out = ctypes.c_void_p()
    bad = kd.make_params(kd.KD_FLOW_ROBERTS, 49, 1.0, 8.0, 1e-2)        # odd n
    assert lib.kd_create(ctypes.byref(bad), None, ctypes.byref(out)) == kd.KD_EINVAL
    bad = kd.make_params(kd.KD_FLOW_ROBERTS, 32, 1.0, -8.0, 1e-2)       # Rm <= 0
    assert lib.kd_create(ctypes.byref(bad), None, ctypes.byref(out)) == kd.KD_EINVAL
    bad = kd.make_params(kd.KD_FLOW_ROBERTS, 32, 1.0, 8.0, 1e-2, n_coarse=64)
    assert lib.kd_create(ctypes.byref(bad), None, ctypes.byref(out)) == kd.KD_EINVAL
    assert lib.kd_destroy(None) == kd.KD_OK
    assert lib.kd_fine_batched(None, None, None, None, 1, 1) == kd.KD_EINVAL


def test_struct_layout_matches_header(lib, tmp_path):
    """Every ctypes mirror of a header struct has the C compiler's size and field offsets."""
    import shutil
    import subprocess
    import paper_1902_00387_gb300 as kd
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [kd.kd_params, kd.kd_parareal_stats, kd.kd_instance, kd.kd_instance_result, kd.kd_sweep_stats]
    exprs, want = [], []
    for st in structs:
        name = st.__name__
        exprs.append("sizeof(%s)" % name)
        want.append(ctypes.sizeof(st))
        for fname, _ in st._fields_:
            exprs.append("offsetof(%s, %s)" % (name, fname))
            want.append(getattr(st, fname).offset)
    probe = tmp_path / "probe.c"
    body = "".join('printf("%%zu\\n", (size_t)%s);' % e for e in exprs)
    probe.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "kd.h"\nint main(void){' + body +
                     ' return 0;}\n')
    exe = tmp_path / "probe"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(probe), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got == want, [(e, g, w) for e, g, w in zip(exprs, got, want) if g != w]


def declarations():
    """(return type, name, [parameter types]) of every function that include/kd.h declares."""
    src = open(os.path.join(ROOT, "include", "kd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"^\s*#.*$", "", src, flags=re.M)
    out = []
    for ret, name, args in re.findall(r"([A-Za-z_][\w \*]*?)\s*\b(kd_[a-z_0-9]+)\s*\(([^)]*)\)\s*;", src):
        params = [a.strip() for a in args.split(",")] if args.strip() not in ("", "void") else []
        # drop the parameter name, keep the type
        types = [re.sub(r"\b[A-Za-z_]\w*$", "", p).strip() if not p.endswith("*") else p for p in params]
        out.append((" ".join(ret.split()), name, types))
    return out


def c_kind(t):
    t = t.replace("const", "").strip()
    if "*" in t:
        return "ptr"
    return {"int": "int", "double": "double", "float": "float", "long long": "i64", "size_t": "size",
            "kd_status": "int"}[" ".join(t.split())]


def ctypes_kind(ct):
    if ct in (ctypes.c_void_p, ctypes.c_char_p) or (isinstance(ct, type) and issubclass(ct, ctypes._Pointer)):
        return "ptr"
    return {ctypes.c_int: "int", ctypes.c_double: "double", ctypes.c_float: "float", ctypes.c_longlong: "i64",
            ctypes.c_size_t: "size"}[ct]


def test_binding_signatures_match_header(lib):
    """Every entry point's ctypes argument and return types agree with its C declaration
    (count and kind), so the binding cannot pass an int where the ABI reads a double."""
    decls = declarations()
    assert len(decls) == len(declared_symbols())
    for ret, name, types in decls:
        fn = getattr(lib, name)
        assert fn.argtypes is not None, name
        assert [c_kind(t) for t in types] == [ctypes_kind(a) for a in fn.argtypes], name
        want = "ptr" if "*" in ret else c_kind(ret)
        assert want == ctypes_kind(fn.restype), (name, ret, fn.restype)
