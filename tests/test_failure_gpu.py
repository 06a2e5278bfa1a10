"""Failure detection on the GPU without faulting it: the statuses
HYDRO_ETIMEOUT and HYDRO_ENOMEM are made to happen by the host, and the
context (or the device, after a failed hydro_init) stays usable.

* HYDRO_ETIMEOUT: hydro_set_wait_limit(0) makes every sweep warp give up at
  its first wait for a TMA copy.  The copies themselves are ordinary loads of
  the context's own state, so each warp still waits (with the default bound)
  for the copies it issued before it leaves the kernel: nothing is left in
  flight and nothing waits on a flag that no one sets forever.
* HYDRO_ENOMEM: a context whose first state buffer alone is larger than the
  device memory; cudaMalloc refuses it on the host side of the call.
"""
import numpy as np
import pytest

import oracle as O
from paper_2106_13465_gb300 import hydro as H
from paper_2106_13465_gb300 import problems as pr

pytestmark = pytest.mark.gpu

TOL64 = 1e-11


def _rel(a, b):
    """Relative error, floored at 1e-3 of the plane's scale for the momenta."""
    scale = np.abs(b).reshape(4, -1).max(axis=1)[:, None, None]
    floor = np.array([0.0, 1e-3, 1e-3, 0.0])[:, None, None] * scale
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), floor)))


@pytest.mark.parametrize("precision", [64, 32])
def test_timeout_status_then_context_still_steps_correctly(precision):
    pb = pr.random_modes(96, 64, seed=5)
    want, dts, _ = O.run(pb.U, pb.h, pb.bc, 4)
    with H.Context([(pb.nx, pb.ny, pb.h, pb.bc)], precision=precision) as c:
        c.set_state(0, pb.U)
        c.set_wait_limit(0)
        with pytest.raises(H.HydroError) as e:
            c.step(1)
        assert e.value.status == H.HYDRO_ETIMEOUT
        assert c.stats()["status_flags"] & 4
        # one more step (the counter is odd), then a CUDA graph of 20 steps
        # captured with the lowered limit
        with pytest.raises(H.HydroError) as e:
            c.step(21)
        assert e.value.status == H.HYDRO_ETIMEOUT
        # the default limit again (the graph is captured anew), a fresh state
        c.set_wait_limit(-1)
        c.set_state(0, pb.U)
        assert c.stats()["status_flags"] == 0
        if precision == 64:
            c.step(4)
            assert _rel(c.get_state(0), want) <= TOL64
        else:
            c.step(4, dt_override=dts)
            got = c.get_state(0)
            assert np.abs(got[0] - want[0]).sum() / np.abs(want[0]).sum() < 1e-6
        c.step(20)  # and through a graph with the default limit
        assert c.stats()["status_flags"] == 0


def test_wait_limit_argument_checked():
    pb = pr.sod(32, 4, 0)
    with H.Context([(pb.nx, pb.ny, pb.h, pb.bc)]) as c:
        assert H.hydro_set_wait_limit(c.ctx, 1 << 32) == H.HYDRO_EINVAL
        assert H.hydro_set_wait_limit(c.ctx, (1 << 32) - 1) == H.HYDRO_OK
        assert H.hydro_set_wait_limit(c.ctx, -1) == H.HYDRO_OK


def test_context_larger_than_device_memory_reports_enomem():
    import torch
    _free, total = torch.cuda.mem_get_info()
    n = 46000  # one FP64 plane of 46016 x 46000 cells: just below 2^31
    per_buffer = 4 * 8 * n * ((n + 31) // 32 * 32)
    k = int(total // per_buffer) + 1
    p, _arr = H.make_params([(n, n, 1.0 / n, (0, 0, 0, 0))] * k, precision=64)
    st, ctx = H.hydro_init(p)
    assert st == H.HYDRO_ENOMEM, H.hydro_last_error(None)
    assert not ctx.value
    assert "cudaMalloc" in H.hydro_last_error(None)
    # the device is still usable: an ordinary context runs and matches the oracle
    pb = pr.sedov(48)
    want, _, _ = O.run(pb.U, pb.h, pb.bc, 3)
    with H.Context([(pb.nx, pb.ny, pb.h, pb.bc)]) as c:
        c.set_state(0, pb.U)
        c.step(3)
        assert _rel(c.get_state(0), want) <= TOL64
