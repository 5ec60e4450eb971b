"""The serving runtime: the same results alone and in the mix, admission by HBM budget,
and the autotuner's plan cache."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_11168_gb300 import build, hs as _hs

    build.build()
    _hs.load()
    return _hs


def _requests(hs, serve):
    reqs = []
    specs = [((16, 16, 16), 5.0, hs.HS_FP32_REFINED, 6), ((24, 24, 24), 0.01, hs.HS_FP32, 2),
             ((16, 24, 12), 50.0, hs.HS_FP64, 3), ((32, 32, 32), 0.0, hs.HS_FP32_REFINED, 1),
             ((24, 18, 12), 1e6, hs.HS_FP32_REFINED, 2)]
    for i, (grid, contrast, prec, nl) in enumerate(specs):
        ids = synth.centred_sphere(grid, volume_fraction=0.2)
        table = synth.two_phase_table(1.0, 0.3, contrast, 0.3)
        reqs.append(serve.Request(ids=ids, table=table, loads=serve.unit_loads()[:nl], precision=prec, tol=1e-6,
                                  max_iter=400, fields=True, tag=i))
    return reqs


def test_same_alone_and_in_the_mix(hs):
    from paper_2405_11168_gb300 import serve

    alone = {}
    srv = serve.Server(budget_bytes=8 << 30, slots=1)
    try:
        for r in _requests(hs, serve):
            alone[r.tag] = srv.submit(r).result(timeout=300)
    finally:
        srv.close()
    srv = serve.Server(budget_bytes=8 << 30, slots=4)
    try:
        futs = [srv.submit(r) for r in _requests(hs, serve)]
        mix = {f.result(timeout=300).tag: f.result(timeout=300) for f in futs}
    finally:
        srv.close()
    assert srv.max_running >= 2
    for tag, a in alone.items():
        b = mix[tag]
        assert a.iters == b.iters and a.status == b.status
        np.testing.assert_array_equal(a.errs, b.errs)
        np.testing.assert_array_equal(a.sig_eff, b.sig_eff)
        np.testing.assert_array_equal(a.eps, b.eps)
        np.testing.assert_array_equal(a.sig, b.sig)


def test_admission_respects_the_budget(hs):
    from paper_2405_11168_gb300 import serve

    reqs = _requests(hs, serve)
    need = max(serve.request_bytes(r) for r in reqs)
    srv = serve.Server(budget_bytes=int(1.5 * need), slots=4)
    try:
        res = [f.result(timeout=300) for f in [srv.submit(r) for r in reqs]]
    finally:
        srv.close()
    assert srv.max_used <= int(1.5 * need)
    assert len(res) == len(reqs)
    small = serve.Server(budget_bytes=need // 2, slots=1)
    try:
        with pytest.raises(ValueError):
            small.submit(max(reqs, key=serve.request_bytes))
    finally:
        small.close()


def test_autotune_plan_cache(hs):
    ids = synth.random_phase_map((32, 32, 32), 2, seed=1)
    table = synth.two_phase_table(1.0, 0.3, 3.0, 0.3)
    opts, ms = hs.autotune(ids, table, precision=hs.HS_FP32, iters=4)
    assert ms > 0 and opts["ytile"] in (2, 4, 8) and opts["zchunk"] >= 1
    opts2, ms2 = hs.autotune(ids, table, precision=hs.HS_FP32, iters=4)
    assert ms2 == -1.0 and opts2 == opts
    # the tuned tiling gives the same result as the default one (up to rounding order)
    s1 = hs.Solver(ids, table, precision=hs.HS_FP64)
    s2 = hs.Solver(ids, table, precision=hs.HS_FP64, ytile=opts["ytile"], zchunk=opts["zchunk"])
    E = np.array([1e-3, 0, 0, 0, 0, 0])
    o1 = s1.solve(E, tol=1e-9, max_iter=500)
    o2 = s2.solve(E, tol=1e-9, max_iter=500)
    assert o1["iters"] == o2["iters"]
    np.testing.assert_allclose(o1["sig_eff"], o2["sig_eff"], rtol=1e-10, atol=1e-16)
    s1.close()
    s2.close()
