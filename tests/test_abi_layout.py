"""The ctypes binding against the C header, on the CPU: every struct the
binding mirrors has the C compiler's size and field offsets (a small C
program including include/moma.h prints them), and every prototype in the
header has as many parameters as the binding's argtypes."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

import paper_2608_17844_b300 as m
from paper_2608_17844_b300 import moma as mb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "moma.h")
STRUCTS = [mb.moma_options, mb.moma_solve_opts, mb.moma_solve_info, mb.moma_server_opts, mb.moma_request,
           mb.moma_result, mb.moma_server_stats]


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    d = tmp_path_factory.mktemp("abi")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "moma.h"', "int main(void) {"]
    for s in STRUCTS:
        n = s.__name__
        lines.append(f'  printf("{n} %zu\\n", sizeof({n}));')
        for f, _ in s._fields_:
            lines.append(f'  printf("{n}.{f} %zu\\n", offsetof({n}, {f}));')
    lines += ["  return 0;", "}"]
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "layout"
    subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {k: int(v) for k, v in (l.split() for l in out.splitlines())}


@pytest.mark.parametrize("s", STRUCTS, ids=lambda s: s.__name__)
def test_struct_size_and_offsets_match_c(c_layout, s):
    n = s.__name__
    assert ctypes.sizeof(s) == c_layout[n]
    for f, _ in s._fields_:
        assert getattr(s, f).offset == c_layout[f"{n}.{f}"], f


def _prototypes():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    protos = {}
    for mt in re.finditer(r"\b(moma_\w+)\s*\(([^;{}]*?)\)\s*;", text):
        name, args = mt.group(1), " ".join(mt.group(2).split())
        protos[name] = 0 if args in ("", "void") else args.count(",") + 1
    return protos


def test_every_prototype_has_the_bindings_argument_count(moma_lib):
    protos = _prototypes()
    assert set(protos) == set(m.EXPORTS)
    L = m.lib()
    for name, nargs in protos.items():
        argtypes = getattr(L, name).argtypes
        if name == "moma_last_error":
            assert nargs == 0 and not argtypes
            continue
        assert argtypes is not None and len(argtypes) == nargs, name


@pytest.mark.parametrize("lang", ["c", "c++"])
def test_header_compiles_cleanly(tmp_path, lang):
    """The header stands alone in C11 and C++17 with warnings as errors."""
    cc = shutil.which("gcc" if lang == "c" else "g++")
    if cc is None:
        pytest.skip("no compiler")
    src = tmp_path / ("h.c" if lang == "c" else "h.cpp")
    src.write_text('#include "moma.h"\nint main(void) {\n  moma_status (*f)(moma_array *, int) = moma_profile;\n'
                   '  (void)f;\n  return sizeof(moma_request) == 0;\n}\n')
    std = "-std=c11" if lang == "c" else "-std=c++17"
    r = subprocess.run([cc, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.dirname(HEADER),
                        "-c", str(src), "-o", str(tmp_path / "h.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_enum_constants_match_the_header(tmp_path):
    """Every MOMA_* enumerator the binding defines (flags, precisions,
    operators, timing selectors, status codes) has the header's value, as
    the C compiler evaluates it."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    text = open(HEADER).read()
    names = sorted(n for n in set(re.findall(r"\b(MOMA_[A-Z0-9_]+)\s*=", text)) if hasattr(mb, n))
    assert any(n.startswith("MOMA_FLAG_") for n in names) and "MOMA_FLAG_SPLIT_ARNOLDI" in names
    lines = ['#include <stdio.h>', '#include "moma.h"', "int main(void) {"]
    lines += [f'  printf("{n} %lld\\n", (long long){n});' for n in names]
    lines += ["  return 0;", "}"]
    src = tmp_path / "enums.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "enums"
    subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = dict(l.split() for l in out if l.strip())
    for n in names:
        assert int(got[n]) == int(getattr(mb, n)), n
