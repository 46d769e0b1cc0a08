"""Allocation-free matvec (kry_matvec_noalloc).

Some callers cannot allocate device memory when they call the library: work
captured into a CUDA graph in global capture mode, hosts whose device memory
is all owned by their own pool, and loops that cannot absorb cudaMalloc's
device synchronisation.  kry_matvec_noalloc serves them with a static device
scratch array.  This file checks, through the C ABI, that two calls in a row
give the same result as kry_matvec (within the FP32 matvec tolerance of the
parity tests), that it takes no device memory, and that grids too large for
its scratch are refused.  It is named so that pytest collects it last."""
import ctypes as C

import numpy as np
import pytest

from paper_2012_13133_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2012_13133_gb300 import kry  # noqa: E402

DEV = torch.device("cuda:0")
TOL = 1e-5   # FP32 matvec relative l2 tolerance used by the parity tests


def _noalloc(ctx, emb, V, out):
    lib = kry.lib()
    return lib.kry_matvec_noalloc(ctx.h, emb.handle, C.c_void_p(V.data_ptr()), C.c_void_p(out.data_ptr()),
                                  V.shape[0], V.shape[1])


def test_noalloc_matches_matvec_twice():
    ctx = kry.Context(0)
    n1, n2 = 300, 260
    mask = I.mask_uniform(n1, n2, 0.5, 3)
    p = ctx.set_mask(torch.from_numpy(mask.astype(np.uint8)).to(DEV))
    emb = ctx.embed(I.Cov(1.0, 0.05, 1.5, 0.05), kry.KRY_F32)
    V = torch.tensor(I.normals((7, p), 21), dtype=torch.float32, device=DEV)
    ref = ctx.matvec(emb, V)
    torch.cuda.synchronize()
    for call in range(2):
        out = torch.full_like(V, float("nan"))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info(0)[0]
        st = _noalloc(ctx, emb, V, out)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info(0)[0]
        assert st == kry.KRY_OK, kry.lib().kry_last_error(ctx.h)
        for k in range(V.shape[0]):
            err = float(torch.linalg.norm(out[k].double() - ref[k].double()) / torch.linalg.norm(ref[k].double()))
            assert err <= TOL, (call, k, err)
        if call == 1:
            # the first call may load the module that holds the static array;
            # the second must not take any device memory
            assert free1 == free0
    emb.free()
    ctx.close()


def test_noalloc_refuses_grids_beyond_its_scratch():
    ctx = kry.Context(0)
    n1, n2 = 1024, 1024
    mask = I.mask_uniform(n1, n2, 0.5, 2)
    p = ctx.set_mask(torch.from_numpy(mask.astype(np.uint8)).to(DEV))
    emb = ctx.embed(I.Cov(1.0, 0.05, 1.5, 0.05), kry.KRY_F64)   # 1024 x 2048 x 16 B = 32 MiB
    V = torch.zeros((2, p), dtype=torch.float64, device=DEV)
    out = torch.zeros_like(V)
    st = _noalloc(ctx, emb, V, out)
    assert st == kry.KRY_EUNSUPPORTED
    assert b"16 MiB" in kry.lib().kry_last_error(ctx.h)
    emb.free()
    ctx.close()
