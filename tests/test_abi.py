"""The C-ABI library loads, exports every function include/hbaca.h declares,
and the ctypes structures match the C layout.  CPU only (no compute calls)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1901_06101_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include"))) if f.endswith(".h")]


def declared_functions(probe=False):
    """Functions the headers declare: those of libhbaca.so, or (probe) of
    libhbaca_probe.so (include/hbaca_probe.h)."""
    names = []
    for h in HEADERS:
        if (os.path.basename(h) == "hbaca_probe.h") != probe:
            continue
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(hbaca_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(B.LIB_PATH):
        pytest.skip("libhbaca.so not built")
    return B.lib()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "hbaca_compress" in names and "hbaca_workspace_size" in names
    for n in names:
        assert hasattr(lib, n), n
    bound = {s[0] for s in B.SIGNATURES}
    assert set(names) <= bound, set(names) - bound


def test_probe_library_exports_its_header():
    if not os.path.exists(B.PROBE_PATH):
        pytest.skip("libhbaca_probe.so not built")
    names = declared_functions(probe=True)
    assert names == ["hbaca_debug_fp64_probe"]
    L = B.probe_lib()
    for n in names:
        assert hasattr(L, n), n
    assert {s[0] for s in B.PROBE_SIGNATURES} == set(names)
    assert not hasattr(B.lib(), "hbaca_debug_fp64_probe")  # not in the compression library


def test_version_and_last_error(lib):
    assert b"sm_103a" in lib.hbaca_version()
    assert isinstance(lib.hbaca_last_error(), bytes)


def _c_layout():
    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "hbaca.h"
#define F(T, f) printf(#T "." #f " %zu\n", offsetof(T, f));
int main(void) {
  printf("hbaca_gen %zu\nhbaca_opts %zu\nhbaca_result %zu\nhbaca_leaf_trace %zu\n",
         sizeof(hbaca_gen), sizeof(hbaca_opts), sizeof(hbaca_result), sizeof(hbaca_leaf_trace));
  F(hbaca_gen, h) F(hbaca_gen, a) F(hbaca_gen, K) F(hbaca_gen, q2) F(hbaca_gen, r2)
  F(hbaca_opts, seed) F(hbaca_opts, flags) F(hbaca_opts, cluster) F(hbaca_opts, srrqr_f)
  F(hbaca_result, d_rank) F(hbaca_result, rank) F(hbaca_result, leaf_iters_max)
  F(hbaca_leaf_trace, I) F(hbaca_leaf_trace, mu)
  return 0;
}
'''
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "l.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "l")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    return dict(line.split() for line in out.strip().splitlines())


def test_struct_layout_matches_c():
    L = _c_layout()
    assert int(L["hbaca_gen"]) == ctypes.sizeof(B.Gen)
    assert int(L["hbaca_opts"]) == ctypes.sizeof(B.Opts)
    assert int(L["hbaca_result"]) == ctypes.sizeof(B.Result)
    assert int(L["hbaca_leaf_trace"]) == ctypes.sizeof(B.LeafTrace)
    for key, cls in [("hbaca_gen", B.Gen), ("hbaca_opts", B.Opts), ("hbaca_result", B.Result),
                     ("hbaca_leaf_trace", B.LeafTrace)]:
        for k, v in L.items():
            if k.startswith(key + "."):
                assert getattr(cls, k.split(".")[1]).offset == int(v), k


def test_workspace_size_and_argument_checks(lib):
    g = B.Gen(kind=B.GEN_GAUSSIAN, dtype=B.F64, m=2000, n=2000, x=8, y=8, dim=3, h=1.0)
    o = B.make_opts(1e-6, 8, 2, rank_cap=128, leaf_rank_cap=256)
    n = B.workspace_size(g, o)
    assert n > 0 and n % 256 == 0
    bad = B.make_opts(1e-6, 64, 2)  # d > 32
    with pytest.raises(B.HbacaError):
        B.workspace_size(g, bad)
    bad = B.make_opts(1e-6, 8, 11)  # 2^L > min(m, n)
    with pytest.raises(B.HbacaError):
        B.workspace_size(g, bad)
    g2 = B.Gen(kind=B.GEN_HELMHOLTZ, dtype=B.F64, m=10, n=10, x=8, y=8, dim=3)  # Helmholtz must be complex
    with pytest.raises(B.HbacaError):
        B.workspace_size(g2, o)


def test_library_has_no_torch_dependency(lib):
    out = subprocess.run(["ldd", B.LIB_PATH], capture_output=True, text=True).stdout
    assert "torch" not in out and "c10" not in out


def test_flag_and_status_constants_match_the_header():
    """Every HBACA_FLAG_* the header defines has the same value in the
    binding, and the status codes the binding maps agree with the enum."""
    src = open(os.path.join(ROOT, "include", "hbaca.h")).read()
    flags = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define HBACA_FLAG_([A-Z_]+) (\d+)u", src)}
    assert {"ASYNC", "PROFILE", "TAPE", "GRAPH", "SINGLE_CLUSTER"} <= set(flags)
    for name, v in flags.items():
        assert getattr(B, "FLAG_" + name) == v, name
    assert len(set(flags.values())) == len(flags)
    assert all(v & (v - 1) == 0 for v in flags.values())  # one bit each
    codes = {m.group(1): int(m.group(2)) for m in re.finditer(r"HBACA_([A-Z_]+) = (\d+),?", src)}
    assert codes["TIMEOUT"] == 4 and codes["RANK_CAPACITY"] == 2 and codes["NUMERICAL"] == 6
