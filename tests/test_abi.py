"""The C-ABI library on the host (no GPU needed): it loads, exports every
symbol include/sensei.h declares, sizes workspaces and rejects bad
arguments before any launch."""
import ctypes as C
import os
import re

import pytest

from paper_2305_18057_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sensei():
    libbuild.build()
    from paper_2305_18057_gb300 import sensei as s
    s.load()
    return s


def _declared():
    with open(os.path.join(ROOT, "include", "sensei.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"^(?:sensei_status|const char \*|double \*)\s*(sensei_\w+)\s*\(", text, re.M)))


def test_every_declared_symbol_is_exported(sensei):
    names = _declared()
    assert len(names) == len(sensei.EXPORTS)
    L = sensei.load()
    for n in names:
        assert hasattr(L, n), n
    assert sorted(sensei.EXPORTS) == names


def _scheme(sensei, **kw):
    d = dict(gamma=1.4, limiter=sensei.LIM_VANLEER, kappa=1 / 3, eps=1.0, entropy_fix=0.1, precision=sensei.FP64,
             reconstruct_conserved=0)
    d.update(kw)
    return sensei.Scheme(**d)


def test_workspace_size_grows_with_the_grid(sensei):
    s = _scheme(sensei)
    a = sensei.sensei_workspace_size([(32, 16, 8)], s)
    b = sensei.sensei_workspace_size([(64, 16, 8)], s)
    c = sensei.sensei_workspace_size([(32, 16, 8), (32, 16, 8)], s)
    assert 0 < a < b and c > a and a % 256 == 0
    # state stage buffers: two FP64 copies of 5 x (36 rounded) x 20 x 12 values at least
    assert a > 2 * 5 * 36 * 20 * 12 * 8
    # the FP32-flux form adds FP32 face metrics
    assert sensei.sensei_workspace_size([(32, 16, 8)], _scheme(sensei, precision=sensei.FP32_FLUX)) > a


def test_invalid_arguments_rejected_on_host(sensei):
    bad = [
        ([(0, 4, 4)], _scheme(sensei)),
        ([(1, 4, 4)], _scheme(sensei)),     # below the ghost depth
        ([(4, 1, 4)], _scheme(sensei)),
        ([(4, 4, 0)], _scheme(sensei)),
        ([(4, 4, 4)], _scheme(sensei, gamma=1.0)),
        ([(4, 4, 4)], _scheme(sensei, limiter=7)),
        ([(4, 4, 4)], _scheme(sensei, precision=9)),
        ([(4, 4, 4)], _scheme(sensei, eps=2.0)),
        ([(4, 4, 4)], _scheme(sensei, entropy_fix=-1.0)),
        ([(4, 4, 4)], _scheme(sensei, mu=-1.0, prandtl=0.72)),
        ([(4, 4, 4)], _scheme(sensei, mu=1e-3, prandtl=0.0)),
    ]
    for blocks, sch in bad:
        with pytest.raises(sensei.SenseiError) as e:
            sensei.sensei_workspace_size(blocks, sch)
        assert e.value.status == sensei.ERR_INVALID_ARG
        assert sensei.sensei_last_error() != ""
    # the viscous flux runs in the FP64 and double-float forms only
    for prec in (sensei.FP32_FLUX, sensei.FP32_STORE):
        with pytest.raises(sensei.SenseiError) as e:
            sensei.sensei_workspace_size([(4, 4, 4)], _scheme(sensei, mu=1e-3, prandtl=0.72, precision=prec))
        assert e.value.status == sensei.ERR_UNSUPPORTED
    assert sensei.sensei_workspace_size([(4, 4, 4)], _scheme(sensei, mu=1e-3, prandtl=0.72, precision=sensei.DF64)) > 0
    # its workspace adds the primitives and the viscous residual
    assert sensei.sensei_workspace_size([(32, 16, 8)], _scheme(sensei, mu=1e-3, prandtl=0.72)) > \
        sensei.sensei_workspace_size([(32, 16, 8)], _scheme(sensei))
    # the FP32-storage form fits its FP32 stage states in the FP64 stage buffers
    assert sensei.sensei_workspace_size([(32, 16, 8)], _scheme(sensei, precision=sensei.FP32_STORE)) > 0
    L = sensei.load()
    assert L.sensei_set_bc(None, 0, 0, 0, None, -1, -1, 0) == sensei.ERR_INVALID_ARG
    assert L.sensei_rk_step(None, None, 1, 0.5, 0.0, None, None) == sensei.ERR_INVALID_ARG
    assert L.sensei_norms(None, None, None, None, None) == sensei.ERR_INVALID_ARG
    assert L.sensei_destroy_grid(None) == sensei.ERR_INVALID_ARG
    assert L.sensei_debug_set(None, sensei.DEBUG_WAIT_LIMIT, 0) == sensei.ERR_INVALID_ARG
    lay = sensei.Layout()
    assert L.sensei_state_layout(None, 0, C.byref(lay)) == sensei.ERR_INVALID_ARG
    # a grid cannot be created without a workspace (checked before any CUDA call)
    blocks = (sensei.BlockDesc * 1)(sensei.BlockDesc(8, 8, 8))
    out = C.c_void_p()
    nodes = (C.c_void_p * 1)(1024)
    assert L.sensei_create_grid(blocks, 1, nodes, C.byref(_scheme(sensei)), None, 0, None,
                                C.byref(out)) == sensei.ERR_INVALID_ARG
    assert L.sensei_create_grid(blocks, 1, nodes, C.byref(_scheme(sensei)), C.c_void_p(4096), 16, None,
                                C.byref(out)) == sensei.ERR_INVALID_ARG
    assert "too small" in sensei.sensei_last_error()
