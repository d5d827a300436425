"""The step kernel's bounded waits: when its shared-memory copy stages never complete (the
test hook makes every stage wait for 16 bytes more than it copies), each CTA gives up after
about a second, flags the fault and returns; the host reports LBM_EDEVICE and the CUDA
context stays usable.  No GPU fault, trap or hang is involved."""
import time

import numpy as np
import pytest

import lbm_workloads as WL

pytestmark = pytest.mark.gpu


def test_copy_wait_timeout_reports_device_fault_and_recovers():
    from paper_2210_07501_gb300 import Lbm, LbmError, LBM_EDEVICE
    w = WL.channel(64, 32, 16, W=4.0)            # one strip, one segment: one CTA
    ref = Lbm(w["domain"], w["params"], precision="fp32")
    ref.lbm_init_fields()
    ref.lbm_step(20)
    expect = ref.lbm_fields()

    g = Lbm(w["domain"], w["params"], precision="fp32")
    g.lbm_init_fields()
    g.lbm_test_stall_copies(True)
    t0 = time.perf_counter()
    g.lbm_step(1)
    with pytest.raises(LbmError) as e:
        g.lbm_diag()
    waited = time.perf_counter() - t0
    assert e.value.status == LBM_EDEVICE
    assert 0.5 < waited < 30.0                   # the waits gave up, they did not hang
    with pytest.raises(LbmError) as e:
        g.lbm_fields()
    assert e.value.status == LBM_EDEVICE
    # a new state clears the fault; stepping is normal again on the same context
    g.lbm_test_stall_copies(False)
    g.lbm_init_fields()
    g.lbm_step(20)
    got = g.lbm_fields()
    for k in ("phi", "u", "v", "T", "dp"):
        assert np.array_equal(got[k], expect[k]), k
    g.close()
    ref.close()
