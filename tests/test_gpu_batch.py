"""Batched stepping (lbm_batch_*) and serving (lbm_server_*) on the GPU.

* every domain of a mixed batch ends equal to round-off to the same domain
  stepped alone with lbm_step: one launch per (lattice, model, storage) group
  runs the same per-cell code (the two kernels are compiled separately, so
  fused multiply-adds may be placed differently);
* the per-domain check-step residual equals the single-solver one;
* admission respects the byte budget; domains added or removed mid-run keep
  the others exact;
* the server's result for a request is the same alone and in a mix (bitwise
  for FP32; within the FP16 tolerance for FP16, whose stochastic rounding
  draws depend on the launch counter).
"""
import numpy as np
import pytest

from paper_1610_01388_gb300 import lbm
from paper_1610_01388_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GB = 1 << 30


def _cases():
    ch = W.channel_params(H=31, nu_p=0.1, u_newton=0.02, bn=1.0)
    du = W.duct_params(H=23, nu_p=0.1, u_newton=0.02, bn=2.0)
    por, _ = W.porous_mask(32, porosity=0.7, r_min=3, r_max=5, seed=3)
    return [
        ("D2Q9", W.channel_mask(4, 32), dict(model="PR", storage="F32", mu_p=0.1, sigma_y=ch["sigma_y"],
                                             m=1e5, g=(ch["g"], 0, 0))),
        ("D2Q9", W.channel_mask(4, 32), dict(model="IR", storage="F64", mu_p=0.1, sigma_y=ch["sigma_y"],
                                             g=(ch["g"], 0, 0))),
        ("D3Q19", W.duct_mask(20, 24, 24), dict(model="IR", storage="F32", mu_p=0.1,
                                                sigma_y=du["sigma_y"], g=(du["g"], 0, 0))),
        ("D3Q27", W.duct_mask(12, 24, 24), dict(model="PR", storage="F32", mu_p=0.1,
                                                sigma_y=du["sigma_y"], m=1e6, g=(du["g"], 0, 0))),
        ("D3Q27", por, dict(model="IR", storage="F32", mu_p=0.1, sigma_y=1e-6, g=(2e-5, 0, 0))),
        ("D3Q15", W.duct_mask(9, 10, 11), dict(model="PR", storage="F32", mu_p=0.05, sigma_y=1e-5,
                                               m=1e4, g=(1e-5, 2e-6, 0))),
        ("D3Q19", W.duct_mask(10, 16, 16), dict(model="PR", storage="F64", mu_p=0.1,
                                                sigma_y=du["sigma_y"], m=1e6, g=(du["g"], 0, 0),
                                                newton_iters=3)),
    ]


def test_mixed_batch_matches_single_domain_runs():
    k = 50
    b = lbm.Batch(4 * GB, check_every=k)
    ids = []
    for lat, mask, prm in _cases():
        ids.append(b.add(lat, mask, **prm))
    n = 333                                    # graphs + singles + 6 check steps
    b.step(n)
    for (lat, mask, prm), dom in zip(_cases(), ids):
        ref = lbm.Solver(lat, mask, check_every=k, **prm)
        ref.step(n)
        got = lbm.lbm_get_populations(b.solver(dom))
        want = ref.get_populations()
        _, w = lbm.lbm_lattice_info(lat)
        off = want - w.reshape((-1, 1, 1, 1))
        # the batched and the single-domain kernels are compiled separately, so
        # FMA contraction may differ: agreement to round-off, not bit for bit
        tol = 1e-12 if prm["storage"] == "F64" else 1e-5
        assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(off)), (lat, prm)
        if prm["model"] == "PR":
            t1, t2 = lbm.lbm_get_tau(b.solver(dom)), ref.get_tau()
            assert np.max(np.abs(t1 - t2) / t2) <= tol
        st = b.status(dom)
        r, at, qx = ref.residual()
        assert st.steps == n and at == 300
        assert abs(st.residual - r) <= max(tol, 1e-12) * 10 * abs(r)
        assert abs(st.flow[0] - qx) <= tol * abs(qx)
        ref.close()
    b.close()


def _run_mix(n, k=50):
    b = lbm.Batch(4 * GB, check_every=k)
    ids = [b.add(lat, mask, **prm) for lat, mask, prm in _cases()]
    b.step(n)
    out = [(lbm.lbm_get_populations(b.solver(d)), b.status(d)) for d in ids]
    b.close()
    return out


@pytest.mark.parametrize("ctas,concurrent", [(1, False), (3, False), (0, True), (2, True)])
def test_batch_schedule_does_not_change_results(ctas, concurrent):
    """A persistent grid (ctas_per_sm > 0) and concurrent group branches in
    the graphs change only the launch shape: populations, residuals and flow
    rates stay bit for bit those of the default schedule."""
    n = 333
    lbm.lbm_tuning_clear()
    ref = _run_mix(n)
    try:
        for lat, _, prm in _cases():
            lbm.lbm_tuning_set_batch(lat, prm["model"], prm["storage"], ctas)
        lbm.lbm_tuning_set_batch_concurrency(concurrent)
        got = _run_mix(n)
    finally:
        lbm.lbm_tuning_clear()
    for (fa, sa), (fb, sb) in zip(ref, got):
        assert np.array_equal(fa, fb)
        assert sa.steps == sb.steps and sa.checks == sb.checks
        assert sa.residual == sb.residual and list(sa.flow) == list(sb.flow)


def test_budget_and_add_remove_mid_run():
    lat, mask, prm = _cases()[2]
    need = lbm.lbm_workspace_bytes(lat, mask.shape[2], mask.shape[1], mask.shape[0],
                                   lbm.lbm_params_default(check_every=10, **prm))
    b = lbm.Batch(2 * need + need // 2, check_every=10)
    a1 = b.add(lat, mask, **prm)
    a2 = b.add(lat, mask, **prm)
    assert b.try_add(lat, mask, **prm) is None          # third does not fit
    used, ndom, _ = b.usage()
    assert ndom == 2 and used == 2 * need
    b.step(40)
    b.remove(a1)
    a3 = b.add(lat, mask, **prm)                        # admitted into the freed memory
    b.step(25)
    ref2 = lbm.Solver(lat, mask, check_every=10, **prm)
    ref2.step(65)
    ref3 = lbm.Solver(lat, mask, check_every=10, **prm)
    ref3.step(25)
    _, w = lbm.lbm_lattice_info(lat)
    for dom, ref in ((a2, ref2), (a3, ref3)):
        got, want = lbm.lbm_get_populations(b.solver(dom)), ref.get_populations()
        scale = np.max(np.abs(want - w.reshape((-1, 1, 1, 1))))
        assert np.max(np.abs(got - want)) <= 1e-5 * scale
    b.close()
    ref2.close()
    ref3.close()


def _serve(reqs, budget, k=100, chunk=200):
    srv = lbm.Server(budget, check_every=k)
    ids = [srv.submit(lat, mask, keep_fields=True, **kw) for lat, mask, kw in reqs]
    for _ in range(10000):
        srv.advance(chunk)
        q, r, _ = srv.pending()
        if q == 0 and r == 0:
            break
    out = []
    for rid, (lat, mask, kw) in zip(ids, reqs):
        res = srv.result(rid)
        rho, u = srv.fields(rid, mask.shape if mask.ndim == 3 else (1,) + mask.shape)
        out.append((res.state, res.steps, res.flow_x, u))
    srv.close()
    return out


def _requests():
    rq = []
    for i, (lat, mask, prm) in enumerate(_cases()):
        if prm["storage"] == "F64":
            continue
        rq.append((lat, mask, dict(tolerance=1e-4, max_steps=1400 + 200 * i, **prm)))
    por, _ = W.porous_mask(24, porosity=0.7, r_min=3, r_max=4, seed=9)
    # FP16: its stochastic-rounding draws differ between runs, so let it run to
    # its cap (a tolerance it cannot reach) to compare equal step counts
    rq.append(("D3Q27", por, dict(tolerance=1e-30, max_steps=1000, model="IR", storage="F16",
                                  mu_p=0.1, sigma_y=1e-6, g=(2e-5, 0, 0))))
    return rq


def test_server_results_same_alone_and_in_mix():
    reqs = _requests()
    mixed = _serve(reqs, budget=GB)
    # a budget that admits about two requests at a time forces queueing and
    # mid-flight admission
    need = []
    for lat, mask, kw in reqs:
        prm = {k: v for k, v in kw.items() if k not in ("tolerance", "max_steps")}
        m3 = mask if mask.ndim == 3 else mask[None]
        need.append(lbm.lbm_workspace_bytes(lat, m3.shape[2], m3.shape[1], m3.shape[0],
                                            lbm.lbm_params_default(check_every=100, **prm)))
    small = _serve(reqs, budget=2 * max(need))
    for i, req in enumerate(reqs):
        alone = _serve([req], budget=GB)[0]
        for other in (mixed[i], small[i]):
            assert other[0] == alone[0] and other[1] == alone[1]
            if req[2]["storage"] == "F16":
                du = np.linalg.norm(other[3] - alone[3]) / np.linalg.norm(alone[3])
                assert du < 1e-3
            else:
                assert np.array_equal(other[3], alone[3])
                assert other[2] == alone[2]
        assert alone[0] in (lbm.LBM_REQ_CONVERGED, lbm.LBM_REQ_CAPPED)
