"""Bounded waits (lbm_set_wait_limit) on the GPU, without any fault: a tiny
limit against ~0.3 s of queued steps makes the waiting calls of a solver, a
batch and a server return LBM_ETIMEOUT while the work keeps running; with the
limit raised the same handles carry on and end exactly where an undisturbed
run ends."""
import numpy as np
import pytest

from paper_1610_01388_gb300 import lbm
from paper_1610_01388_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GB = 1 << 30
PRM = dict(model="IR", storage="F32", mu_p=0.1, sigma_y=1e-6, g=(1e-6, 0.0, 0.0))


def _timed_out(fn):
    with pytest.raises(lbm.LbmError) as e:
        fn()
    return e.value.status == lbm.LBM_ETIMEOUT


@pytest.fixture
def restore_limit():
    yield
    lbm.lbm_set_wait_limit(0.0)


def test_solver_waits_time_out_and_recover(restore_limit):
    mask = W.duct_mask(256, 128, 128)          # ~140 us per step: 2000 steps ~ 0.3 s
    ref = lbm.Solver("D3Q27", mask, check_every=100, **PRM)
    ref.step(2000)
    rho_ref, u_ref = ref.fields()
    ref.close()
    s = lbm.Solver("D3Q27", mask, check_every=100, **PRM)
    lbm.lbm_set_wait_limit(1e-6)
    s.step(2000)
    assert _timed_out(s.sync)
    assert _timed_out(s.fields)
    assert _timed_out(lambda: lbm.lbm_flowrate(s.h, 0))
    lbm.lbm_set_wait_limit(60.0)
    s.sync()
    rho, u = s.fields()
    assert np.array_equal(rho, rho_ref) and np.array_equal(u, u_ref)
    r, at, _ = s.residual()
    assert at == 2000 and r > 0
    s.close()


def test_batch_and_server_waits_time_out_and_recover(restore_limit):
    mask = W.duct_mask(256, 96, 96)
    b = lbm.Batch(8 * GB, check_every=100)
    dom = b.add("D3Q27", mask, **PRM)
    lbm.lbm_set_wait_limit(1e-6)
    b.step(2000)
    assert _timed_out(lambda: b.status(dom))
    lbm.lbm_set_wait_limit(60.0)
    st = b.status(dom)
    assert st.steps == 2000 and st.checks == 20
    b.close()

    srv = lbm.Server(8 * GB, check_every=100)
    rid = srv.submit("D3Q27", mask, tolerance=1e-30, max_steps=1200, **PRM)
    lbm.lbm_set_wait_limit(1e-6)
    assert _timed_out(lambda: srv.advance(400))     # steps queued, nothing judged
    assert srv.result(rid).state == lbm.LBM_REQ_RUNNING
    lbm.lbm_set_wait_limit(60.0)
    for _ in range(10):
        srv.advance(400)
        if srv.result(rid).state != lbm.LBM_REQ_RUNNING:
            break
    res = srv.result(rid)
    assert res.state == lbm.LBM_REQ_CAPPED and res.steps == 1200
    srv.close()
