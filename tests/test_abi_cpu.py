"""CPU checks of the C-ABI boundary: the library builds and loads, exports
every function include/hydro.h declares, and rejects invalid arguments before
touching a GPU.  No compute call runs here."""
import ctypes
import os
import re

import pytest

from paper_2106_13465_gb300 import build as B
from paper_2106_13465_gb300 import hydro as H

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hydro.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hydro_[a-z0-9_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    path = B.build()
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(lib, name), f"{name} declared in hydro.h but not exported"
    assert sorted(H.EXPORTS) == declared


def test_version():
    assert re.fullmatch(r"\d+\.\d+\.\d+", H.hydro_version())


def _params(**kw):
    grids = kw.pop("grids", [(16, 16, 1 / 16, (0, 0, 0, 0))])
    p, arr = H.make_params(grids, **kw)
    return p, arr


@pytest.mark.parametrize("kw,msg", [
    (dict(precision=16), "precision"),
    (dict(gamma=1.0), "gamma"),
    (dict(cfl=0.0), "cfl"),
    (dict(niter=-1), "niter"),
    (dict(rho_floor=0.0), "floor"),
    (dict(grids=[(1, 16, 0.1, (0, 0, 0, 0))]), "nx"),
    (dict(grids=[(16, 16, 0.0, (0, 0, 0, 0))]), "h must"),
    (dict(grids=[(65536, 32768, 0.1, (0, 0, 0, 0))]), "2^31"),
    (dict(grids=[(46337, 46337, 0.1, (0, 0, 0, 0))]), "2^31"),
    (dict(grids=[(16, 16, 0.1, (2, 0, 0, 0))]), "periodic"),
    (dict(grids=[(16, 16, 0.1, (0, 0, 7, 0))]), "boundary"),
])
def test_invalid_params_rejected_before_any_gpu_call(kw, msg):
    p, _arr = _params(**kw)
    st, ctx = H.hydro_init(p)
    assert st == H.HYDRO_EINVAL
    assert not ctx.value
    assert msg in H.hydro_last_error(None)


def test_null_arguments_rejected():
    L = H.load()
    assert L.hydro_init(None, None) == H.HYDRO_EINVAL
    assert H.hydro_step(None, 1) == H.HYDRO_EINVAL
    assert H.hydro_set_state(None, 0, 0, 0) == H.HYDRO_EINVAL
    assert H.hydro_get_stats(None)[0] == H.HYDRO_EINVAL
    H.hydro_destroy(None)


def test_no_gpu_reports_cuda_error_not_a_fallback():
    """Without a usable GPU the library refuses with HYDRO_ECUDA: there is no
    CPU path behind the ABI."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    p, _arr = _params()
    st, ctx = H.hydro_init(p)
    assert st == H.HYDRO_ECUDA
    assert not ctx.value


@pytest.mark.parametrize("kw,msg", [(dict(riemann=2), "riemann_solver"), (dict(slope=3), "slope_type"),
                                    (dict(trace=5), "trace_type")])
def test_invalid_scheme_variants_rejected(kw, msg):
    p, _arr = _params(**kw)
    st, ctx = H.hydro_init(p)
    assert st == H.HYDRO_EINVAL
    assert msg in H.hydro_last_error(None)
