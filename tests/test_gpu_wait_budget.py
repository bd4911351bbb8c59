"""Bounded dependency waits of the dataflow schedule.

A host-side hook makes one forward task's wait for its input words never
succeed: the wait must give up after its budget, the sweep must end,
the next synchronizing call must report STA_ERR_TIMEOUT once, and the handle and
the CUDA context must stay usable (the next analysis matches the oracle again).
No fault is injected on the device: the wait simply runs out.
"""
import time

import numpy as np
import pytest

import netgen
import oracle
from tests import _parity as tp

pytestmark = pytest.mark.gpu

STA_ERR_TIMEOUT = 5
STA_ERR_STATE = 6


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _engine(w, schedule="dataflow", use_graphs=True):
    import torch
    from paper_2603_28381_gb300 import StaEngine
    eng = StaEngine(w.netlist, w.library, use_graphs=use_graphs, schedule=schedule)
    eng.set_positions(torch.from_numpy(w.xy.astype(np.float32)).cuda())
    return eng


@pytest.mark.parametrize("use_graphs", [True, False])
def test_expired_wait_is_reported_and_handle_recovers(use_graphs):
    from paper_2603_28381_gb300 import StaError
    w = netgen.tiny_design(0)
    eng = _engine(w, use_graphs=use_graphs)
    eng.forward(lse=True, rat=True, gamma=10.0)
    ok = eng.summary()                       # a normal analysis first (no report pending)

    eng._debug_expire_wait()
    t0 = time.perf_counter()
    eng.forward(lse=True, rat=True, gamma=10.0)
    with pytest.raises(StaError) as ei:
        eng.summary()
    dt = time.perf_counter() - t0
    assert ei.value.status == STA_ERR_TIMEOUT
    assert 0.9 < dt < 30.0                   # the wait ran into its 1 s budget, then ended
    eng.synchronize()                        # reported once: nothing pending any more

    # the next analysis on the same handle is complete and right again
    eng.forward(lse=True, rat=True, gamma=10.0)
    assert eng.summary() == ok
    ora = oracle.sta(w.netlist, w.library, w.xy, 10.0, 1.0, 0.5)
    tp.assert_parity(tp.run_gpu(w.netlist, w.library, w.xy, 10.0, (1.0, 0.5), engine=eng), ora)


def test_expiry_reported_by_synchronize_and_gradient():
    from paper_2603_28381_gb300 import StaError
    w = netgen.tiny_design(1)
    eng = _engine(w)
    eng._debug_expire_wait()
    eng.forward(lse=True, rat=True, gamma=10.0)
    # device-side output: no report yet; the gradient sweep after it also ends
    import torch
    g = torch.empty(w.netlist.num_pins, 2, device="cuda")
    eng.backward_grad((1.0, 0.5), out=g)
    with pytest.raises(StaError) as ei:
        eng.synchronize()
    assert ei.value.status == STA_ERR_TIMEOUT
    eng.synchronize()
    eng.forward(lse=True, rat=True, gamma=10.0)
    gh = eng.backward_grad((1.0, 0.5), out=torch.empty(w.netlist.num_pins, 2))  # host output: checked
    ora = oracle.sta(w.netlist, w.library, w.xy, 10.0, 1.0, 0.5)
    scale = max(np.abs(ora["grad"]).max(), 1e-20)
    assert np.abs(gh.numpy() - ora["grad"]).max() <= tp.GRAD_RTOL * scale


def test_level_schedule_has_no_waits():
    from paper_2603_28381_gb300 import StaError
    eng = _engine(netgen.tiny_design(2), schedule="levels")
    with pytest.raises(StaError) as ei:
        eng._debug_expire_wait()
    assert ei.value.status == STA_ERR_STATE
