"""GPU check of hydro_conservation_noalloc, the entry point for callers that
cannot allocate device memory while they run (stream capture, hard latency
limits, host frameworks that own all GPU memory).  It must give the same
totals as hydro_conservation on a context holding the same state, call after
call, although every call reuses the same fixed device scratch array.  This
file is collected last so that a run stopping at the first failure has run
every other test first."""
import numpy as np
import pytest

from paper_2106_13465_gb300 import hydro as H
from paper_2106_13465_gb300 import problems as pr

pytestmark = pytest.mark.gpu


def _context_sums(pb):
    with H.Context([(pb.nx, pb.ny, pb.h, pb.bc)], precision=64) as c:
        c.set_state(0, pb.U)
        return c.conservation(0)


def test_noalloc_totals_match_the_context_entry_point_on_consecutive_calls():
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    sums = torch.zeros(4, dtype=torch.float64, device="cuda")
    # a taller grid first, then a shorter one: the second call must not pick
    # up rows the first left in the shared scratch array
    for pb in (pr.sedov(150, 300), pr.random_modes(96, 80, seed=8), pr.sod(37, 5, 0)):
        want = _context_sums(pb)
        U = torch.from_numpy(np.ascontiguousarray(pb.U)).cuda()
        st = H.hydro_conservation_noalloc(U.data_ptr(), pb.nx, pb.ny, pb.h, sums.data_ptr(), stream)
        assert st == H.HYDRO_OK
        torch.cuda.synchronize()
        got = sums.cpu().numpy()
        # the same summation order as the context's entry point: the same bits
        assert np.array_equal(got, want), (pb.name, got, want)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    U = torch.zeros(8, dtype=torch.float64, device="cuda")
    sums = torch.zeros(4, dtype=torch.float64, device="cuda")
    assert H.hydro_conservation_noalloc(U.data_ptr(), 1, 32769, 0.1, sums.data_ptr()) == H.HYDRO_EINVAL
    assert H.hydro_conservation_noalloc(0, 4, 4, 0.1, sums.data_ptr()) == H.HYDRO_EINVAL
    assert H.hydro_conservation_noalloc(U.data_ptr(), 2, 1, 0.0, sums.data_ptr()) == H.HYDRO_EINVAL
