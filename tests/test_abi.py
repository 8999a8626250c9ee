"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/*.h; the product path never links or imports the oracle.
No compute calls (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w \*]*?\b(music_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1610_10053_gb300 import build
    path = build.build()
    return ctypes.CDLL(path), path


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("music_create_grid", "music_residual", "music_jv", "music_precond_apply",
                     "music_newton_step", "music_destroy_grid", "music_spatial_operator"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    L, path = lib
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_1610_10053_gb300 import binding
    assert set(declared_functions()) <= set(binding.SIGNATURES)


def test_struct_layouts_match_binding(tmp_path):
    """Every struct of the C headers has the size and field offsets that the
    ctypes binding assumes (checked by compiling a C program against them)."""
    from paper_1610_10053_gb300 import binding as b
    structs = {"music_grid_desc": b.GridDesc, "music_step_stats": b.StepStats,
               "music_server_opts": b.ServerOpts, "music_solve_req": b.SolveReq,
               "music_solve_result": b.SolveResult, "music_tune_report": b.TuneReport, "music_dt_limits": b.DtLimits,
               "music_peaks": b.Peaks}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "music_server.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append('printf("%s sizeof %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln:
            parts = ln.split()
            got[(parts[0], parts[1])] = int(parts[2])
    for cname, cls in structs.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)


def test_library_does_not_contain_the_oracle(lib):
    L, path = lib
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    assert "or_spatial_operator" not in out and "or_newton_step" not in out


def test_product_never_imports_oracle():
    pkg = os.path.join(ROOT, "paper_1610_10053_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", txt, flags=re.M), f
                assert "liboracle" not in txt and "music_oracle" not in txt, f


def test_invalid_descriptor_is_rejected_without_gpu_work(lib):
    """Argument validation happens before any device call."""
    from paper_1610_10053_gb300 import binding
    L = binding.load()
    d = binding.GridDesc()
    d.ndim = 4
    h = ctypes.c_void_p()
    assert L.music_create_grid(ctypes.byref(d), ctypes.byref(h)) == 1
    assert "ndim" in binding.last_error()
    assert L.music_create_grid(None, ctypes.byref(h)) == 1
    assert L.music_destroy_grid(None) == 0
    assert L.music_state_size(None) == 0
    assert L.music_vanleer_slopes(None, None, None, -1, None) == 1
    assert L.music_vanleer_slopes(None, None, None, 5, None) == 1
    assert L.music_vanleer_slopes(None, None, None, 0, None) == 0
    assert L.music_stencil_quotients(None, None, None, -1, None) == 1
    assert L.music_stencil_quotients(None, None, None, 5, None) == 1
    assert L.music_stencil_quotients(None, None, None, 0, None) == 0


def test_binding_rejects_mis_sized_vectors_before_any_library_call(lib):
    """The binding checks the dtype, size and placement of every device
    vector it hands to the library, which would otherwise read or write the
    grid's full size through the caller's pointer.  A stand-in grid object
    (no device state) is enough: the checks come before any call."""
    torch = pytest.importorskip("torch")
    from paper_1610_10053_gb300 import binding as B
    from paper_1610_10053_gb300 import inputs as I
    p = I.kelvin_helmholtz(n=8)
    g = object.__new__(B.Grid)
    g.prob, g.precision, g.h = p, B.MIXED, None
    g.desc = B.desc_from_problem(p, B.MIXED)
    g.n = p.U.size
    U = torch.zeros(g.n, dtype=torch.float64)
    v32 = torch.zeros(g.n, dtype=torch.float32)
    cases = [
        (lambda: g.spatial_operator(U[:-1]), "entries"),
        (lambda: g.spatial_operator(U.float()), "float64"),
        (lambda: g.spatial_operator(U), "CUDA"),
        (lambda: g.residual(U, U[:5], 0.1), "entries"),
        (lambda: g.jv(U, U, 0.1), "float32"),          # a mixed grid's Krylov vectors are FP32
        (lambda: g.jv(U, v32[:-4], 0.1), "entries"),
        (lambda: g.precond(U, 0.1, U), "float32"),
        (lambda: g.set_state(np.zeros(g.n - 1)), "entries"),
    ]
    for call, word in cases:
        with pytest.raises(ValueError, match=word):
            call()
    g.precision = B.FP64
    with pytest.raises(ValueError, match="float64"):
        g.jv(U, v32, 0.1)
    with pytest.raises(ValueError, match="rate"):
        B.cfl_rate_noalloc(p, U, torch.zeros(2, dtype=torch.float64))
