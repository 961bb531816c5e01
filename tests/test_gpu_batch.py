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


@pytest.mark.parametrize("ctas,concurrent,tile", [
    (1, False, (256, 1)), (3, False, (256, 1)), (0, True, (256, 1)), (2, True, (256, 1)),
    (0, False, (128, 1)), (0, False, (512, 1)), (0, False, (128, 2)), (2, True, (256, 2)),
])
def test_batch_schedule_does_not_change_results(ctas, concurrent, tile):
    """A persistent grid (ctas_per_sm > 0), concurrent group branches in the
    graphs and the plain-step tile shape change only the launch shape:
    populations, residuals and flow rates stay bit for bit those of the
    default schedule."""
    n = 333
    lbm.lbm_tuning_clear()
    ref = _run_mix(n)
    try:
        for lat, mask, prm in _cases():
            lbm.lbm_tuning_set_batch(lat, prm["model"], prm["storage"], ctas)
            if prm["storage"] != "F64":
                for cls in range(0, 40):
                    lbm.lbm_tuning_set_batch_tile(lat, prm["model"], prm["storage"], cls, *tile)
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


# --- the batch and the server against the FP64 oracle ------------------------------

# relative L2 velocity error against the oracle at equal step count
ORACLE_BAR = {"F64": 1e-10, "F32": 1e-5, "F16": 1e-3}


def _oracle_for(lat, mask, prm):
    import oracle
    p = oracle.params(model=prm["model"], nu_p=prm["mu_p"], sigma_y=prm.get("sigma_y", 0.0),
                      m=prm.get("m", 0.0), g=prm["g"], newton=prm.get("newton_iters", 0))
    return oracle.State(lat, p, mask if mask.ndim == 3 else mask[None])


def _rel_l2(u_gpu, u_orc, mask):
    fl = (mask if mask.ndim == 3 else mask[None]) == 0
    a, b = u_gpu[:, fl], u_orc[:, fl]
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _oracle_cases():
    por, _ = W.porous_mask(32, porosity=0.7, r_min=3, r_max=5, seed=4)
    du = W.duct_params(H=23, nu_p=0.1, u_newton=0.02, bn=2.0)
    return _cases() + [
        ("D3Q27", W.duct_mask(12, 24, 24), dict(model="PR", storage="F16", mu_p=0.1,
                                                sigma_y=du["sigma_y"], m=1e6, g=(du["g"], 0, 0))),
        ("D3Q19", por, dict(model="IR", storage="F16", mu_p=0.1, sigma_y=1e-6, g=(2e-5, 0, 0))),
        ("D3Q19", por, dict(model="PR", storage="F32", mu_p=0.1, sigma_y=1e-6, m=1e6,
                            g=(2e-5, 0, 0))),
    ]


@pytest.mark.parametrize("tile", [(256, 1), (128, 2)])
def test_batched_domains_match_oracle(tile):
    """Every domain of a mixed batch (four lattices, both models, FP64, FP32
    and FP16 storage, the Newton-implicit PR step) after 1000 batched steps
    against the oracle stepped 1000 times: relative L2 of u_real within 1e-10
    (FP64), 1e-5 (FP32), 1e-3 (FP16); the last check step's flow rate too
    (a check step measures the populations it streams: the state after 999
    steps)."""
    n, k = 1000, 50
    lbm.lbm_tuning_clear()
    try:
        for lat, _, prm in _oracle_cases():
            if prm["storage"] != "F64":
                for cls in range(0, 40):
                    lbm.lbm_tuning_set_batch_tile(lat, prm["model"], prm["storage"], cls, *tile)
        b = lbm.Batch(4 * GB, check_every=k)
        ids = [b.add(lat, mask, **prm) for lat, mask, prm in _oracle_cases()]
        b.step(n)
        for (lat, mask, prm), dom in zip(_oracle_cases(), ids):
            o = _oracle_for(lat, mask, prm)
            o.step(n - 1)
            q_check = o.flowrate(0)
            o.step(1)
            _, uo = o.fields()
            _, ug = lbm.lbm_fields(b.solver(dom))
            err = _rel_l2(ug.reshape(uo.shape), uo, mask)
            assert err <= ORACLE_BAR[prm["storage"]], (lat, prm, err)
            st = b.status(dom)
            assert abs(st.flow[0] - q_check) <= 10 * ORACLE_BAR[prm["storage"]] * abs(q_check), (lat, prm)
        b.close()
    finally:
        lbm.lbm_tuning_clear()


def test_served_results_match_oracle():
    """Requests served in a mix, under a budget that admits about two at a
    time (queueing and mid-flight admission), each run to its 1000-step cap:
    the final u_real of every request against the oracle stepped 1000 times,
    within the same bars as the batch."""
    reqs = []
    for lat, mask, prm in _oracle_cases():
        if prm.get("newton_iters"):
            continue
        reqs.append((lat, mask, dict(tolerance=1e-30, max_steps=1000, **prm)))
    need = []
    for lat, mask, kw in reqs:
        prm = {k: v for k, v in kw.items() if k not in ("tolerance", "max_steps")}
        m3 = mask if mask.ndim == 3 else mask[None]
        need.append(lbm.lbm_workspace_bytes(lat, m3.shape[2], m3.shape[1], m3.shape[0],
                                            lbm.lbm_params_default(check_every=100, **prm)))
    served = _serve(reqs, budget=2 * max(need))
    for (lat, mask, kw), (state, steps, _, u) in zip(reqs, served):
        assert state == lbm.LBM_REQ_CAPPED and steps == 1000
        prm = {k: v for k, v in kw.items() if k not in ("tolerance", "max_steps")}
        o = _oracle_for(lat, mask, prm)
        o.step(1000)
        _, uo = o.fields()
        err = _rel_l2(u.reshape(uo.shape), uo, mask)
        assert err <= ORACLE_BAR[prm["storage"]], (lat, prm, err)


def test_flow_change_is_the_relative_change_of_the_mean_velocity():
    """lbm_domain_status.flow_change against the same quantity formed on the
    host from a single-domain solver's flow rates at two check steps k apart:
    |S - S_prev| / |S| with S_a = L_a Q_a, the sums of u_real."""
    lat, mask, prm = _cases()[3]
    k = 50
    b = lbm.Batch(GB, check_every=k)
    dom = b.add(lat, mask, **prm)
    b.step(k)
    assert b.status(dom).flow_change == -1.0        # one check step so far
    ref = lbm.Solver(lat, mask, check_every=k, **prm)
    L = np.array([mask.shape[2], mask.shape[1], mask.shape[0]], float)
    ref.step(k - 1)
    s0 = np.array([ref.flowrate(a) for a in range(3)]) * L
    b.step(k)
    ref.step(k)
    s1 = np.array([ref.flowrate(a) for a in range(3)]) * L
    want = np.linalg.norm(s1 - s0) / np.linalg.norm(s1)
    got = b.status(dom).flow_change
    assert want > 0 and abs(got - want) <= 1e-6 * want, (got, want)
    ref.close()
    b.close()


def test_server_steady_criteria():
    """A channel served to steady state under each criterion: the request is
    retired as converged at the first advance whose last check step shows a
    change below the tolerance, and not before."""
    ch = W.channel_params(H=15, nu_p=0.1, u_newton=0.02, bn=0.5)
    mask = W.channel_mask(4, 16)
    kw = dict(model="IR", storage="F32", mu_p=0.1, sigma_y=ch["sigma_y"], g=(ch["g"], 0, 0))
    for crit, tol in (("flow", 1e-7), ("residual", 1e-6)):
        srv = lbm.Server(GB, check_every=100)
        rid = srv.submit("D2Q9", mask, tolerance=tol, max_steps=200_000, criterion=crit, **kw)
        for _ in range(2000):
            srv.advance(200)
            if srv.pending()[:2] == (0, 0):
                break
        res = srv.result(rid)
        srv.close()
        assert res.state == lbm.LBM_REQ_CONVERGED, crit
        # replay alone: the change at the retiring advance is below tol, the one before is not
        b = lbm.Batch(GB, check_every=100)
        dom = b.add("D2Q9", mask, **kw)
        changes = []
        while b.status(dom).steps < res.steps:
            b.step(200)
            st = b.status(dom)
            changes.append(st.flow_change if crit == "flow" else st.residual)
        b.close()
        assert 0.0 <= changes[-1] < tol and not (0.0 <= changes[-2] < tol), (crit, changes[-3:])
