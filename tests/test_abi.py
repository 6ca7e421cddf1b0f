"""The C-ABI library loads and exports what include/lev.h declares (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            with open(os.path.join(ROOT, "include", fn)) as f:
                txt = f.read()
            names |= set(re.findall(r"^(?:int|const char\*)\s+(lev_[a-z0-9_]+)\s*\(", txt, re.M))
    return names


@pytest.fixture(scope="module")
def lev():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2105_11004_gb300 as L
    return L


def test_library_exports_every_declared_symbol(lev):
    declared = _declared_symbols()
    assert {"lev_create", "lev_sketch_dense", "lev_rrqr", "lev_estimate_dense", "lev_final_dense"} <= declared
    out = subprocess.run(["nm", "-D", "--defined-only", lev.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (lev_[a-z0-9_]+)", out))
    assert declared <= exported, declared - exported
    for name in declared:
        assert hasattr(lev.lib, name)
        assert name in lev.SIGNATURES


def test_params_struct_layout_matches_header(lev, tmp_path):
    """Every field of the ctypes mirror sits at the offset the C compiler gives it in lev.h."""
    fields = [f for f, _ in lev.lev_params._fields_]
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "lev.h"\nint main(void) {\n'
                   '  printf("size %zu\\n", sizeof(lev_params));\n'
                   + "".join(f'  printf("{f} %zu\\n", offsetof(lev_params, {f}));\n' for f in fields)
                   + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    assert int(got["size"]) == ctypes.sizeof(lev.lev_params)
    for f in fields:
        assert int(got[f]) == getattr(lev.lev_params, f).offset, f
    p = lev.make_params()
    assert p.eps == 0.5 and abs(p.delta - 1 / 3) < 1e-15 and p.gamma == 2.0 and p.tau == 1e-5


def test_resolve_sizes_follow_the_paper(lev):
    # Alg. 3: s = ceil((d^2 + d) / ((2 eps - eps^2)^2 delta)), m = ceil(gamma d);
    # JL size k = ceil(4 ln n / (eps^2 / 2 - eps^3 / 3)).
    import math
    s, m, k = lev.lev_resolve_sizes(lev.make_params(), 10**6, 256)
    assert s == math.ceil((256 ** 2 + 256) / ((1 - 0.25) ** 2 / 3))
    assert m == 512
    assert k == math.ceil(4 * math.log(10**6) / (0.125 - 0.125 / 3))
    s, m, k = lev.lev_resolve_sizes(lev.make_params(s=65536, m=1024, k=256), 10**6, 256)
    assert (s, m, k) == (65536, 1024, 256)
    s, m, k = lev.lev_resolve_sizes(lev.make_params(sketch_identity=True, omega_identity=True), 500, 8)
    assert (s, m, k) == (500, 500, 8)


@pytest.mark.parametrize("n,d,kw", [(0, 8, {}), (10, 0, {}), (10, 5000, {}), (10, 8, {"k": 5000}),
                                    (70000, 8, {"sketch_identity": True})])
def test_resolve_sizes_rejects_bad_shapes(lev, n, d, kw):
    with pytest.raises(lev.LevError) as e:
        lev.lev_resolve_sizes(lev.make_params(**kw), n, d)
    assert e.value.code == lev.LEV_EINVAL


def test_null_handle_is_einval(lev):
    rc = lev.lib.lev_sketch_dense(None, None, 10, 4, 4, ctypes.byref(lev.make_params()), None, None)
    assert rc == lev.LEV_EINVAL
    assert b"handle" in lev.lib.lev_last_error()


def test_default_handle_is_per_thread(lev, monkeypatch):
    """A handle serves one host thread at a time: default_handle gives each thread its own, and
    the same one on every call from that thread (a stand-in Handle; no GPU)."""
    import threading

    made = []

    class FakeHandle:
        def __init__(self, device=0):
            self.device = device
            made.append(self)

    monkeypatch.setattr(lev, "Handle", FakeHandle)
    monkeypatch.setattr(lev, "_tls", threading.local())
    h0 = lev.default_handle(0)
    assert lev.default_handle(0) is h0 and lev.default_handle(1) is not h0
    got = {}

    def worker():
        got["a"] = lev.default_handle(0)
        got["b"] = lev.default_handle(0)

    t = threading.Thread(target=worker)
    t.start()
    t.join()
    assert got["a"] is got["b"] and got["a"] is not h0
    assert len(made) == 3


def test_binding_fails_loudly_without_the_library(tmp_path):
    """No CPU or library fallback: the binding without liblev.so refuses to import."""
    import shutil
    import sys
    shutil.copytree(os.path.join(ROOT, "paper_2105_11004_gb300"), tmp_path / "paper_2105_11004_gb300",
                    ignore=shutil.ignore_patterns("*.so", "__pycache__", "csrc"))
    r = subprocess.run([sys.executable, "-c", "import paper_2105_11004_gb300"], cwd=tmp_path, capture_output=True,
                       text=True, timeout=120)
    assert r.returncode != 0
    assert "ImportError" in r.stderr and "liblev.so is not built" in r.stderr


def test_binding_constants_match_header(lev):
    """Every status code, precision and flag the header defines has the same value in the binding."""
    with open(os.path.join(ROOT, "include", "lev.h")) as f:
        txt = f.read()
    defs = dict(re.findall(r"^#define (LEV_[A-Z0-9_]+)\s+(\d+)u?\b", txt, re.M))
    assert {"LEV_OK", "LEV_EINVAL", "LEV_BF16X3", "LEV_SKETCH_SRHT", "LEV_CSR_UNCHECKED"} <= set(defs)
    for name, value in defs.items():
        assert getattr(lev, name) == int(value), name
