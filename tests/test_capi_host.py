"""CPU-only checks of the C-ABI library: it builds, loads, exports every
function include/pamd.h declares, and rejects bad arguments before touching
the GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import pamd_inputs as pi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    txt = open(os.path.join(ROOT, "include", "pamd.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pamd_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1806_06016_gb300 import build, pamd
    build.build()
    return pamd.load()


def test_library_exports_every_declared_function(lib):
    names = _header_functions()
    assert "pamd_init" in names and "pamd_resample" in names
    for n in names:
        assert hasattr(lib, n), n
    from paper_1806_06016_gb300 import pamd
    assert set(pamd.EXPORTS) >= set(names) - {"pamd_obs", "pamd_options", "pamd_topology", "pamd_ctx"}


def test_options_default(lib):
    from paper_1806_06016_gb300 import pamd
    o = pamd.pamd_options_default()
    assert o.gamma_per_ps == 1.0 and o.precision == 0 and o.lanes_per_replica == 0
    assert not o.stream


def _init_rc(top, R=4, T0=300.0, **opt):
    from paper_1806_06016_gb300 import pamd
    lib = pamd.load()
    o = pamd.pamd_options_default()
    for k, v in opt.items():
        setattr(o, k, v)
    ta = pamd._TopologyArgs(top)
    ctx = C.c_void_p()
    rc = lib.pamd_init(C.byref(ctx), C.byref(ta.s), R, T0, 1, C.byref(o))
    if rc == 0:
        lib.pamd_destroy(ctx)
    return rc, pamd.pamd_last_error()


def test_argument_validation_before_device_use(lib):
    from paper_1806_06016_gb300 import pamd
    top = pi.make_chain(10, 1)
    assert _init_rc(top, R=0)[0] == pamd.PAMD_EINVAL
    assert _init_rc(top, T0=-1.0)[0] == pamd.PAMD_EINVAL
    assert _init_rc(top, lanes_per_replica=33)[0] == pamd.PAMD_EINVAL
    assert _init_rc(top, lanes_per_replica=-1)[0] == pamd.PAMD_EINVAL
    assert _init_rc(top, lanes_per_replica=4, warps_per_block=9)[0] == pamd.PAMD_EINVAL
    assert _init_rc(top, precision=7)[0] == pamd.PAMD_EUNSUPPORTED
    bad = pi.make_chain(10, 1)
    bad.bond = bad.bond.copy(); bad.bond[3, 1] = 10
    rc, msg = _init_rc(bad)
    assert rc == pamd.PAMD_EINVAL and "bonds" in msg
    bad = pi.make_chain(10, 1)
    bad.mass = bad.mass.copy(); bad.mass[2] = 0.0
    assert _init_rc(bad)[0] == pamd.PAMD_EINVAL
    bad = pi.make_chain(10, 1)
    bad.dih_n = bad.dih_n.copy(); bad.dih_n[0] = 7
    assert _init_rc(bad)[0] == pamd.PAMD_EINVAL
    bad = pi.make_chain(10, 1)
    bad.angle = bad.angle.copy(); bad.angle[0] = [2, 2, 3]
    assert _init_rc(bad)[0] == pamd.PAMD_EINVAL
    big = pi.make_chain(257, 1)
    assert _init_rc(big)[0] == pamd.PAMD_EUNSUPPORTED
    # 8 atoms per lane at most: 75 atoms cannot run on 8 lanes
    assert _init_rc(pi.make_chain(75, 1), lanes_per_replica=8)[0] == pamd.PAMD_EINVAL


def test_null_context_calls_fail_cleanly(lib):
    from paper_1806_06016_gb300 import pamd
    assert lib.pamd_propagate(None, 1, 0.001, 300.0) == pamd.PAMD_EINVAL
    assert lib.pamd_sync(None) == pamd.PAMD_EINVAL
    assert lib.pamd_launch_count(None) == -1
    lib.pamd_destroy(None)
