"""Error bounds of the FP64 arithmetic helpers the sweep kernels use in place
of IEEE division and powers (godunov.cuh): the refined FP32-seeded
reciprocal (within 1 ulp), the division through it (within 2 ulp) and the
7th root of the rarefaction power for gamma = 7/5 (within 3 ulp), checked
against references computed in extended precision on the host.  The helper
kernel is built here from the library's own header."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2106_13465_gb300", "csrc")


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    so = tmp_path_factory.mktemp("mathprobe") / "libmathprobe.so"
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-fmad=false", "-std=c++17",
                    "-shared", "-Xcompiler", "-fPIC", "-I", CSRC, "-o", str(so),
                    os.path.join(ROOT, "tests", "csrc", "math_probe.cu")], check=True)
    lib = ctypes.CDLL(str(so))
    lib.math_probe_eval.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_longlong]
    lib.math_probe_eval.restype = ctypes.c_int

    def run(fn, x, y=None):
        dx = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        dy = torch.from_numpy(np.ascontiguousarray(y if y is not None else x)).cuda()
        out = torch.empty_like(dx)
        assert lib.math_probe_eval(fn, dx.data_ptr(), dy.data_ptr(), out.data_ptr(), dx.numel()) == 0
        return out.cpu().numpy()
    return run


def inputs(n=1 << 20, emin=-1020, emax=1020, seed=7):
    rng = np.random.default_rng(seed)
    m = 1.0 + rng.random(n)
    e = rng.integers(emin, emax + 1, n)
    x = np.ldexp(m, e)
    edge = np.array([1.0, 2.0, 0.5, 1.0 + 2.0 ** -52, 2.0 - 2.0 ** -52, np.finfo(np.float64).tiny,
                     np.finfo(np.float64).max, 127.99999999999999, 128.0, 2.0 ** 7, 2.0 ** -7, 2.0 ** 70,
                     2.0 ** -70, 3.0, 7.0, 1e-300, 1e300])
    return np.concatenate([x, edge])


def ulp_err(got, ref_ld):
    ref = ref_ld.astype(np.float64)
    return np.abs(got.astype(np.longdouble) - ref_ld) / np.spacing(np.abs(ref)).astype(np.longdouble)


@pytest.mark.gpu
def test_reciprocal_within_one_ulp(probe):
    x = inputs()
    x = np.concatenate([x, -x])
    err = ulp_err(probe(0, x), 1.0 / x.astype(np.longdouble))
    assert float(err.max()) <= 1.0


@pytest.mark.gpu
def test_division_within_two_ulp(probe):
    a = inputs(emin=-500, emax=500, seed=3)
    a[::2] *= -1.0
    b = inputs(emin=-500, emax=500, seed=5)
    err = ulp_err(probe(2, a, b), a.astype(np.longdouble) / b.astype(np.longdouble))
    assert float(err.max()) <= 2.0


@pytest.mark.gpu
def test_seventh_root_within_three_ulp(probe):
    x = inputs()
    ref = np.power(x.astype(np.longdouble), np.longdouble(1) / np.longdouble(7))
    got = probe(1, x)
    assert float(ulp_err(got, ref).max()) <= 3.0
    # exact powers of 2^7 give exact roots
    e = np.arange(-1015, 1016, 7)
    assert np.array_equal(probe(1, np.ldexp(1.0, e)), np.ldexp(1.0, e // 7))
