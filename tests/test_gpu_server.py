"""Continuous-batching server: every request gives the same result alone and in
a concurrent mix of differently sized requests, memory admission serialises
what does not fit, and requests beyond the budget are refused."""
import numpy as np
import pytest

from oracle import kryoracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2012_13133_gb300 import kry  # noqa: E402
from paper_2012_13133_gb300 import serve  # noqa: E402


def specs():
    out = []
    for k, (n, miss, nu, rng, t2, kind) in enumerate([(48, 0.3, 0.5, 0.1, 0.1, "loglik"),
                                                      (64, 0.6, 1.5, 0.05, 0.05, "krige"),
                                                      (40, 0.2, 1.5, 0.15, 0.2, "loglik"),
                                                      (96, 0.5, 0.5, 0.08, 0.03, "krige"),
                                                      (72, 0.8, 0.5, 0.03, 0.1, "loglik"),
                                                      (33, 0.4, 1.5, 0.1, 0.1, "krige")]):
        out.append(dict(id=k, arrival=0.0, n=n, frac_missing=miss, nu=nu, range=rng, tau2=t2, kind=kind,
                        mask_seed=100 + k, data_seed=200 + k))
    return out


@pytest.fixture(scope="module")
def reqs():
    sp = specs()
    return serve.build_requests(sp, serve.make_masks(sp, 1), nprobe=8, nsteps=30, rtol=1e-8, maxit=5000)


def run(server, reqs):
    ts = [server.submit(r["kind"], r["mask"], r["y"], r["X"], r["cov"], r["opts"], r.get("target_cells"),
                        r.get("target_X")) for r in reqs]
    return [server.wait(t, 600.0) for t in ts]


def test_alone_equals_mix_and_matches_oracle(reqs):
    alone = []
    s = kry.Server(0, 1, 16 << 30)
    for r in reqs:
        alone += run(s, [r])
    s.close()
    mix_server = kry.Server(0, 4, 16 << 30)
    mixed = run(mix_server, reqs)
    mix_server.close()
    assert {m["slot"] for m in mixed} != {0}      # the mix really ran in several slots
    for r, a, m in zip(reqs, alone, mixed):
        assert a["status"] == kry.KRY_OK and m["status"] == kry.KRY_OK, (a["error"], m["error"])
        if r["kind"] == kry.KRY_REQ_LOGLIK:
            assert m["loglik"] == pytest.approx(a["loglik"], rel=1e-12)
        else:
            assert np.allclose(m["mean"], a["mean"], rtol=1e-12, atol=1e-14)
        assert np.allclose(m["beta"], a["beta"], rtol=1e-12, atol=1e-14)
    # and each result is the oracle's, within the parity tolerances
    for r, a in zip(reqs, alone):
        n = r["mask"].shape[0]
        P = O.FFTProblem(n, n, r["mask"], r["cov"])
        Xo = r["X"].T
        if r["kind"] == kry.KRY_REQ_LOGLIK:
            ref = P.profile_loglik(r["y"], Xo, r["opts"].nprobe, r["opts"].nsteps, r["opts"].seed, tol=1e-12)
            assert a["loglik"] == pytest.approx(ref["loglik"], rel=1e-3)
        else:
            dense = O.loglik_dense(O.dense_K(n, n, r["mask"], r["cov"]), r["y"], Xo)
            mu = P.krige_cells(r["y"], Xo, dense["beta"], r["target_cells"], r["target_X"].T, tol=1e-12)
            assert np.linalg.norm(a["mean"] - mu) <= 1e-4 * np.linalg.norm(mu)


def test_admission_by_memory_and_refusal(reqs):
    # a budget that holds about one request at a time still completes them all
    est_small = 600 << 20
    s = kry.Server(0, 4, est_small)
    out = run(s, reqs[:3])
    assert all(o["status"] == kry.KRY_OK for o in out)
    s.close()
    tiny = kry.Server(0, 2, 1 << 20)
    r = reqs[0]
    with pytest.raises(kry.KryError) as ei:
        tiny.submit(r["kind"], r["mask"], r["y"], r["X"], r["cov"], r["opts"])
    assert ei.value.status == kry.KRY_ENOMEM
    tiny.close()
