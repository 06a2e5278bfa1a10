"""The -fopenmp build of the oracle (lines of a sweep shared among threads,
as the paper's Fine-Grain version shares its loop over lines, §2) gives the
same bits as the single-threaded build for every thread count: each line is
computed by the same code whichever thread takes it."""
import numpy as np
import pytest

import oracle as O
from paper_2106_13465_gb300 import problems as pr


@pytest.mark.parametrize("make", [
    lambda: pr.random_modes(67, 45, seed=3),
    lambda: pr.sedov(40, 33),
    lambda: pr.sod(50, 7, 0),
    lambda: pr.transpose(pr.sod(50, 7, 0)),
])
def test_openmp_build_bit_identical_to_single_thread(make):
    pb = make()
    want, wdts, _ = O.run(pb.U, pb.h, pb.bc, 7, step0=1)
    for n in (1, 3, 8):
        got, gdts, _ = O.run(pb.U, pb.h, pb.bc, 7, step0=1, threads=n)
        assert np.array_equal(got, want), n
        assert np.array_equal(gdts, wdts), n


def test_openmp_thread_count_is_taken():
    assert O.set_threads(3) == 3
    assert O.set_threads(1) == 1
