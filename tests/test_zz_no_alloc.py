"""Allocation-free matvec (kry_matvec_noalloc).

Some callers cannot allocate device memory when they call the library: hosts
whose device memory is all owned by their own pool or arena, and loops that
cannot absorb the device-wide synchronisation of cudaMalloc / cudaFree.
kry_matvec_noalloc serves them with a static device scratch array.  This file
checks, through the C ABI, on two calls in a row:

* that its result equals kry_matvec's (same passes, same schedule) and, within
  the parity tests' tolerances, the FP64 oracle's (1e-5 relative in FP32,
  1e-12 in FP64);
* at 1024 x 1024 in FP32, where one complex pair fills the scratch, that a
  five-vector call runs its three batches correctly;
* that the second call takes no device memory;
* that grids too large for the scratch are refused with a message.

It is named so that pytest collects it last."""
import ctypes as C

import numpy as np
import pytest

from oracle import kryoracle as O
from paper_2012_13133_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2012_13133_gb300 import kry  # noqa: E402

DEV = torch.device("cuda:0")
TOL = {kry.KRY_F32: 1e-5, kry.KRY_F64: 1e-12}   # matvec relative l2 tolerances of the parity tests


def _noalloc(ctx, emb, V, out):
    lib = kry.lib()
    return lib.kry_matvec_noalloc(ctx.h, emb.handle, C.c_void_p(V.data_ptr()), C.c_void_p(out.data_ptr()),
                                  V.shape[0], V.shape[1])


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("n1,n2,prec,nvec", [
    (300, 260, kry.KRY_F32, 7),      # several pairs in one batch
    (200, 170, kry.KRY_F64, 5),      # FP64 passes
    (1024, 1024, kry.KRY_F32, 5),    # one pair per batch: three batches
])
def test_noalloc_matches_matvec_and_oracle_twice(n1, n2, prec, nvec):
    ctx = kry.Context(0)
    mask = I.mask_uniform(n1, n2, 0.5, 3)
    cov = I.Cov(1.0, 0.05, 1.5, 0.05)
    p = ctx.set_mask(torch.from_numpy(mask.astype(np.uint8)).to(DEV))
    emb = ctx.embed(cov, prec)
    dt = torch.float32 if prec == kry.KRY_F32 else torch.float64
    Vh = I.normals((nvec, p), 21)
    V = torch.tensor(Vh, dtype=dt, device=DEV)
    ref_lib = ctx.matvec(emb, V)
    ref = O.FFTProblem(n1, n2, mask, cov).matvec(V.double().cpu().numpy())
    torch.cuda.synchronize()
    for call in range(2):
        out = torch.full_like(V, float("nan"))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info(0)[0]
        st = _noalloc(ctx, emb, V, out)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info(0)[0]
        assert st == kry.KRY_OK, kry.lib().kry_last_error(ctx.h)
        got = out.double().cpu().numpy()
        lib = ref_lib.double().cpu().numpy()
        for k in range(nvec):
            assert _rel(got[k], lib[k]) <= TOL[prec], (call, k)
            assert _rel(got[k], ref[k]) <= TOL[prec], (call, k, _rel(got[k], ref[k]))
        assert np.array_equal(got, lib), (call, np.abs(got - lib).max())
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
