"""Bounded device-side waits: a pipeline wait whose barrier phase never completes gives up after its
budget, reports DR_ERR_TIMEOUT to the host, and leaves the device usable.

The failure is made without a fault: one thread waits on a fresh mbarrier that nothing arrives on,
through the same bounded wait the tensor-core pipelines use."""
import time

import numpy as np
import pytest

from oracle import reach as orc
from paper_2605_25346_b300 import _lib, api
from paper_2605_25346_b300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seconds", [0.02, 0.2])
def test_wait_gives_up_and_device_stays_usable(seconds):
    lib = _lib.load()
    t0 = time.perf_counter()
    rc = lib.dr_check_wait_expiry(seconds)
    dt = time.perf_counter() - t0
    assert rc == _lib.DR_ERR_TIMEOUT, lib.dr_last_error(None)
    # the budget is counted in SM cycles at the rated clock, and each test of the barrier may sleep
    # up to 100 us: the wait ends near its budget, never long after it
    assert dt < seconds * 3 + 1.0, dt
    # a normal pass on the same device afterwards
    p = wl.random_problem(71, [3, 16, 16, 2], D=8, H=3, eps=0.2)
    r = api.Reach(0).load(p)
    g = r.bounds(on_device=False)
    r.close()
    o = orc.reach(p)
    olo, ohi = o["lo"].numpy(), o["hi"].numpy()
    scale = np.maximum(np.maximum(np.abs(olo), np.abs(ohi)), ohi - olo)
    err = np.maximum(np.abs(g["lo"] - olo), np.abs(g["hi"] - ohi)) / scale
    assert err.max() <= 1e-5
