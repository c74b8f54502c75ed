"""The C ABI library builds for sm_103a and exports what include/asci.h declares (CPU)."""
import ctypes as ct
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "asci.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(asci_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def built_lib():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2303_05688_gb300 import build
    return build.build()


def test_header_declares_the_search_boundary():
    names = _declared()
    for f in ("asci_search", "asci_excitations", "asci_diagonal", "asci_sort_accumulate",
              "asci_select_topn", "asci_default_opts", "asci_version", "asci_strerror"):
        assert f in names


def test_library_exports_every_declared_symbol(built_lib):
    out = subprocess.run(["nm", "-D", "--defined-only", built_lib], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (asci_\w+)", out))
    missing = [f for f in _declared() if f not in exported]
    assert not missing, missing


def test_library_loads_and_host_only_calls_work(built_lib):
    lib = ct.CDLL(built_lib)
    lib.asci_version.restype = ct.c_char_p
    assert b"sm_103a" in lib.asci_version()
    lib.asci_strerror.restype = ct.c_char_p
    assert lib.asci_strerror(-1) == b"invalid argument"
    import paper_2303_05688_gb300 as m
    o = m._Opts()
    m.load().asci_default_opts(ct.byref(o))
    assert o.eps_search == 0.0 and o.precision == 0 and o.max_batch_pairs == 0


def test_library_is_built_for_sm_103a(built_lib):
    from paper_2303_05688_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_2303_05688_gb300 as m
    monkeypatch.setattr(m, "_LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(m, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        m.load()


def test_header_compiles_as_c_and_links(built_lib, tmp_path):
    """include/asci.h is plain C99 (warning-free) and a C program links against
    the library and runs its host-only calls."""
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    src = tmp_path / "use.c"
    src.write_text(r"""
#include <stdio.h>
#include <string.h>
#include "asci.h"
int main(void) {
  asci_opts o; asci_davidson_opts d; asci_loop_opts l;
  asci_default_opts(&o); asci_default_davidson_opts(&d); asci_default_loop_opts(&l);
  if (o.precision != ASCI_FP64 || d.max_subspace != 16 || l.max_steps != 8) return 2;
  if (strstr(asci_version(), "sm_103a") == NULL) return 3;
  if (asci_launch_count() != 0) return 4;
  printf("%s\n", asci_strerror(ASCI_EINVAL));
  return 0;
}
""")
    exe = tmp_path / "use"
    libdir = os.path.dirname(built_lib)
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I",
                        os.path.join(ROOT, "include"), str(src), "-L", libdir, "-lasci",
                        f"-Wl,-rpath,{libdir}", "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "invalid argument"


def test_binding_structs_match_the_header(tmp_path):
    """Every struct the binding passes by pointer has the header's size and
    field offsets (a field added to asci.h without the binding, or in another
    place, would shift everything after it)."""
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    import ctypes as ct
    m = pytest.importorskip("paper_2303_05688_gb300")
    pairs = [("asci_det", m._Det), ("asci_ints", m._Ints), ("asci_opts", m._Opts),
             ("asci_select_state", m._SelectState), ("asci_problem", m._Problem),
             ("asci_stats", m._Stats), ("asci_davidson_opts", m._DavOpts),
             ("asci_loop_opts", m._LoopOpts), ("asci_loop_stats", m._LoopStats)]
    lines = []
    for cname, py in pairs:
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    src = tmp_path / "layout.c"
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"asci.h\"\n"
                   "int main(void) {\n" + "\n".join(lines) + "\n  return 0;\n}\n")
    exe = tmp_path / "layout"
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:-1]): int(l.split()[-1]) for l in out if l.strip()}
    for cname, py in pairs:
        assert got[(cname, "size")] == ct.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
