"""The C-ABI library loads without a GPU and exports every function that
include/kry.h declares; the Python binding's signatures, structs and enums match the header."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "kry.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kry_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2012_13133_gb300.build import build_library
    return build_library()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["kry_embed_eigs", "kry_matvec", "kry_logdet", "kry_solve", "kry_profile_loglik", "kry_krige"]:
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (kry_[a-z_0-9]+)", out))
    assert set(declared_functions()) <= exported


def test_binding_signatures_cover_header(libpath):
    from paper_2012_13133_gb300 import kry
    assert set(kry.SIGNATURES) == set(declared_functions())


STRUCTS = {
    "kry_grid": ["n1", "n2", "dx1", "dx2"],
    "kry_cov": ["sigma2", "range", "nu", "tau2", "aniso_angle", "aniso_ratio"],
    "kry_opts": ["prec", "nprobe", "nsteps", "seed", "rtol", "maxit", "reorth", "precond"],
    "kry_request": ["kind", "n1", "n2", "mask", "y", "X", "ncov", "cov", "opts", "loglik", "logdet", "beta",
                    "target_cells", "target_X", "mean"],
}


def test_binding_structs_and_enums_match_the_header(libpath, tmp_path):
    """Compile a C program against include/kry.h that prints every struct's size and field offsets
    and every enum value; the ctypes binding must agree (same layout on this host's ABI)."""
    import shutil

    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    from paper_2012_13133_gb300 import kry

    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "kry.h"', "int main(void) {"]
    for s, fields in STRUCTS.items():
        lines.append(f'printf("{s} size %zu\\n", sizeof({s}));')
        for f in fields:
            lines.append(f'printf("{s} {f} %zu\\n", offsetof({s}, {f}));')
    enums = [n for n in kry.STATUS_NAMES] + ["KRY_F32", "KRY_F64", "KRY_AUTO"]
    for e in enums:
        lines.append(f'printf("enum {e} %d\\n", (int){e});')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        parts = line.split()
        got[tuple(parts[:-1])] = int(parts[-1])
    for s, fields in STRUCTS.items():
        cls = getattr(kry, s)
        assert [f[0] for f in cls._fields_] == fields, s
        assert got[(s, "size")] == ctypes.sizeof(cls), s
        for f in fields:
            assert got[(s, f)] == getattr(cls, f).offset, (s, f)
    for i, e in enumerate(kry.STATUS_NAMES):
        assert got[("enum", e)] == i, e
    assert got[("enum", "KRY_F32")] == kry.KRY_F32 and got[("enum", "KRY_F64")] == kry.KRY_F64
    assert got[("enum", "KRY_AUTO")] == kry.KRY_AUTO


def test_binding_refuses_host_and_strided_tensors(libpath):
    """Device-pointer arguments are checked in the binding before any library call."""
    torch = pytest.importorskip("torch")
    from paper_2012_13133_gb300 import kry

    assert kry._ptr(None) is None
    with pytest.raises(ValueError, match="CUDA tensor"):
        kry._ptr(torch.zeros(4, dtype=torch.float64))


def test_binding_checks_dtype_and_size_before_calling_the_library(libpath):
    """Every device buffer is checked against the dtype and element count the C ABI will read, so
    a wrong dtype or a short buffer raises in Python instead of being read out of bounds.  The
    context here is never created in the library: each call must raise before reaching it."""
    torch = pytest.importorskip("torch")
    import weakref

    from paper_2012_13133_gb300 import kry

    ctx = object.__new__(kry.Context)
    ctx.h, ctx.p, ctx.n1, ctx.n2, ctx.torch, ctx._embeds = None, 10, 4, 4, torch, weakref.WeakSet()
    emb = object.__new__(kry.Embed)
    emb.ctx, emb.handle, emb.min_over_max, emb.prec = ctx, None, 1.0, kry.KRY_F32
    f32 = lambda *s: torch.zeros(*s, dtype=torch.float32)  # noqa: E731
    f64 = lambda *s: torch.zeros(*s, dtype=torch.float64)  # noqa: E731
    opts = kry.Opts()
    cov = kry.kry_cov(1.0, 0.1, 0.5, 0.1, 0.0, 1.0)
    cases = [
        (lambda: ctx.matvec(emb, f64(10)), "dtype float32"),
        (lambda: ctx.matvec(emb, f32(9)), r"\(nvec, 10\)"),
        (lambda: ctx.matvec(emb, f32(2, 10), out=f32(1, 10)), "out: expected 20"),
        (lambda: ctx.matvec(emb, f32(2, 10)), "CUDA tensor"),
        (lambda: ctx.solve(emb, f32(2, 10)), "B: expected dtype float64"),
        (lambda: ctx.profile_loglik(f64(10), f64(3, 9), [cov], opts), "X: expected 30"),
        (lambda: ctx.profile_loglik(f64(10), f64(3, 10), [cov], opts), "CUDA tensor"),
        (lambda: ctx.krige(cov, opts, f64(10), f64(3, 10), cells=f64(5), Xc=f64(3, 5)), "cells: expected dtype int64"),
        (lambda: ctx.loglik_krige(cov, opts, f64(10), f64(3, 10), cells=torch.zeros(5, dtype=torch.int64),
                                  Xc=f64(3, 4)), "Xc: expected 15"),
        (lambda: ctx.genhybr(cov, f64(11), 5), "b: expected 10"),
        (lambda: ctx.sample(cov, 8, 8, f64(2, 8, 4)), "xi: expected 128"),
        (lambda: ctx.bootstrap_var(cov, opts, f64(3, 8, 8), f64(3, 10), torch.zeros(2, dtype=torch.int64)),
         r"\(nrep, 2, M1, M2\)"),
        (lambda: ctx.bootstrap_var(cov, opts, f64(3, 2, 8, 8), f64(3, 9), torch.zeros(2, dtype=torch.int64)),
         "eps: expected 30"),
        (lambda: ctx.set_mask(f32(4, 4)), "mask: expected dtype"),
        (lambda: ctx.set_mask(torch.zeros(4, 4, dtype=torch.uint8)), "CUDA tensor"),
    ]
    for call, msg in cases:
        with pytest.raises(ValueError, match=msg):
            call()


def test_server_requests_are_sized_against_their_mask(libpath):
    """The server reads p values of y and X and N - p kriging targets, counted from the mask alone;
    requests whose buffers disagree are refused in Python before any library call."""
    from paper_2012_13133_gb300 import kry

    srv = object.__new__(kry.Server)
    srv.h, srv._live = None, {}
    mask = np.zeros((4, 5), dtype=np.uint8)
    mask[:2] = 1                                   # p = 10, N - p = 10
    cov = kry.kry_cov(1.0, 0.1, 0.5, 0.1, 0.0, 1.0)
    opts = kry.Opts()
    with pytest.raises(ValueError, match="needs y"):
        srv.submit(kry.KRY_REQ_LOGLIK, mask, np.zeros(9), np.zeros((3, 10)), cov, opts)
    with pytest.raises(ValueError, match="needs y"):
        srv.submit(kry.KRY_REQ_LOGLIK, mask, np.zeros(10), np.zeros((3, 9)), cov, opts)
    with pytest.raises(ValueError, match="every unobserved cell"):
        srv.submit(kry.KRY_REQ_KRIGE, mask, np.zeros(10), np.zeros((3, 10)), cov, opts,
                   target_cells=np.arange(10, 19), target_X=np.zeros((3, 9)))
    with pytest.raises(ValueError, match="every unobserved cell"):
        srv.submit(kry.KRY_REQ_KRIGE, mask, np.zeros(10), np.zeros((3, 10)), cov, opts)
