"""CPU-only checks of the C-ABI library: it builds, loads, exports every
function the headers under include/ declare, and rejects bad
arguments before touching the GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import pamd_inputs as pi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"\b(pamd_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


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


def _header_range(field):
    """The 'a..b' range the header states for a pamd_options field."""
    txt = open(os.path.join(ROOT, "include", "pamd.h")).read()
    m = re.search(r"\b" + field + r";\s*/\*[^*]*?(\d+)\.\.(\d+)", txt)
    assert m, field
    return int(m.group(1)), int(m.group(2))


def test_header_ranges_match_validation(lib):
    """The ranges include/pamd.h states for the launch-shape options are the
    ones pamd_init accepts: both ends pass argument validation (without a GPU
    the call then fails at the device, never with PAMD_EINVAL) and one past
    either end is rejected."""
    from paper_1806_06016_gb300 import pamd
    top = pi.make_chain(10, 1)
    lo, hi = _header_range("lanes_per_replica")
    assert (lo, hi) == (1, 32)
    small = pi.make_chain(6, 1)  # one lane holds at most 8 atoms
    for lanes, t in ((lo, small), (2, top), (hi, top), (hi, pi.make_chain(256, 1))):
        assert _init_rc(t, lanes_per_replica=lanes)[0] != pamd.PAMD_EINVAL, lanes
    assert _init_rc(top, lanes_per_replica=hi + 1)[0] == pamd.PAMD_EINVAL
    assert _init_rc(top, lanes_per_replica=-1)[0] == pamd.PAMD_EINVAL
    lo, hi = _header_range("warps_per_block")
    assert (lo, hi) == (1, 8)
    for w in (0, lo, hi):
        assert _init_rc(top, warps_per_block=w)[0] != pamd.PAMD_EINVAL, w
    assert _init_rc(top, warps_per_block=hi + 1)[0] == pamd.PAMD_EINVAL
    for pa in (pamd.PAMD_PAIRS_AUTO, pamd.PAMD_PAIRS_SCALAR, pamd.PAMD_PAIRS_PACKED):
        assert _init_rc(top, pair_arith=pa)[0] != pamd.PAMD_EINVAL
    assert _init_rc(top, pair_arith=3)[0] == pamd.PAMD_EINVAL
    assert _init_rc(top, pair_arith=pamd.PAMD_PAIRS_PACKED, replicas_per_lane=2)[0] == pamd.PAMD_EINVAL


def test_null_context_calls_fail_cleanly(lib):
    from paper_1806_06016_gb300 import pamd
    assert lib.pamd_propagate(None, 1, 0.001, 300.0) == pamd.PAMD_EINVAL
    assert lib.pamd_sync(None) == pamd.PAMD_EINVAL
    assert lib.pamd_launch_count(None) == -1
    lib.pamd_destroy(None)


def test_surrogate_argument_validation(lib):
    """The surrogate's entry points reject bad shapes and null pointers
    before any device work."""
    from paper_1806_06016_gb300 import pamd
    h = C.c_void_p()
    for n_atoms, hidden in [(1, 128), (pamd.PAMD_MAX_ATOMS + 1, 128), (22, 0), (22, 100), (22, 2048)]:
        assert lib.pamd_mlp_create(C.byref(h), n_atoms, hidden, 0, None) == pamd.PAMD_EINVAL
        assert not h.value
    assert "n_atoms" in pamd.pamd_last_error() or "hidden" in pamd.pamd_last_error()
    assert lib.pamd_mlp_create(None, 22, 128, 0, None) == pamd.PAMD_EINVAL
    dummy = C.c_void_p(16)
    for M, N, K, lda, ldb, ldc in [(0, 8, 8, 8, 8, 8), (8, 8, 12, 16, 16, 8), (8, 8, 8, 4, 8, 8),
                                   (8, 16, 8, 8, 8, 8)]:
        assert lib.pamd_gemm_bf16(dummy, dummy, dummy, M, N, K, lda, ldb, ldc, None) == pamd.PAMD_EINVAL
    assert lib.pamd_gemm_bf16(None, dummy, dummy, 8, 8, 8, 8, 8, 8, None) == pamd.PAMD_EINVAL
    for fn in ("pamd_mlp_info", "pamd_mlp_sync", "pamd_mlp_get_params", "pamd_mlp_get_grads"):
        args = [None] * (4 if fn == "pamd_mlp_info" else (1 if fn == "pamd_mlp_sync" else 2))
        assert getattr(lib, fn)(*args) == pamd.PAMD_EINVAL
    assert lib.pamd_mlp_energy_forces(None, None, 4, None, None) == pamd.PAMD_EINVAL
    assert lib.pamd_mlp_loss_grads(None, None, None, None, None, 4, 1.0, None) == pamd.PAMD_EINVAL
    assert lib.pamd_mlp_launch_count(None) == 0
    lib.pamd_mlp_destroy(None)


def test_checkpoint_and_model_files_validation(lib, tmp_path):
    """File entry points reject null handles, missing and foreign files
    before any device work."""
    from paper_1806_06016_gb300 import pamd
    assert lib.pamd_checkpoint(None, b"x") == pamd.PAMD_EINVAL
    assert lib.pamd_restore(None, b"x") == pamd.PAMD_EINVAL
    assert lib.pamd_mlp_save(None, b"x") == pamd.PAMD_EINVAL
    h = C.c_void_p()
    assert lib.pamd_mlp_load(C.byref(h), str(tmp_path / "missing").encode(), None) == pamd.PAMD_EINVAL
    junk = tmp_path / "junk.bin"
    junk.write_bytes(b"not a model file at all")
    assert lib.pamd_mlp_load(C.byref(h), str(junk).encode(), None) == pamd.PAMD_EINVAL
    assert "not a model file" in pamd.pamd_last_error()
    assert not h.value


def test_wham_rejects_bad_arguments_before_touching_the_gpu(lib):
    from paper_1806_06016_gb300 import pamd
    T = np.array([300.0, 250.0])
    fake = 256  # never dereferenced: every case fails validation first

    def rc(**kw):
        args = dict(n_temps=2, R=10, T=T, n_bins=16, e_range=None, max_iter=5, tol=0.0, T_eval=None)
        args.update(kw)
        try:
            pamd.pamd_wham(fake, args.pop("n_temps"), args.pop("R"), args.pop("T"), args.pop("n_bins"), **args)
        except pamd.PamdError as e:
            return e.code
        return 0

    assert rc(n_bins=0) == pamd.PAMD_EINVAL
    assert rc(n_bins=65537) == pamd.PAMD_EINVAL
    assert rc(n_temps=0, T=np.zeros(0)) == pamd.PAMD_EINVAL
    assert rc(R=0) == pamd.PAMD_EINVAL
    assert rc(T=np.array([300.0, -1.0])) == pamd.PAMD_EINVAL
    assert rc(max_iter=-1) == pamd.PAMD_EINVAL
    assert rc(tol=-1.0) == pamd.PAMD_EINVAL
    assert rc(T_eval=[0.0]) == pamd.PAMD_EINVAL
    assert rc(e_range=(0.0, np.inf)) == pamd.PAMD_EINVAL
    assert rc(lnZ_init=[0.0, np.nan]) == pamd.PAMD_EINVAL
    with pytest.raises(pamd.PamdError):
        pamd.pamd_record_energies(None, 0, 0)


def test_adaptive_and_rule_arguments_rejected_before_touching_the_gpu(lib):
    from paper_1806_06016_gb300 import pamd
    fake = 256
    bad = [(10, 300.0, 300.0, 0.5), (10, 300.0, 400.0, 0.5), (0, 300.0, 200.0, 0.5),
           (10, 300.0, 200.0, 0.0), (10, 300.0, 200.0, 1.0), (10, -1.0, -2.0, 0.5)]
    for R, Tp, Tf, a in bad:
        with pytest.raises(pamd.PamdError) as ei:
            pamd.pamd_overlap_temperature(fake, R, Tp, Tf, a)
        assert ei.value.code == pamd.PAMD_EINVAL
    with pytest.raises(pamd.PamdError):
        pamd.pamd_next_temperature(None, 300.0, 200.0, 0.5)
    with pytest.raises(pamd.PamdError):
        pamd.pamd_anneal_adaptive(None, 300.0, 200.0, 0.5, 10, 0.001, 5)
    assert _init_rc(pi.make_chain(5, 1), resample_rule=4)[0] == pamd.PAMD_EINVAL
    assert _init_rc(pi.make_chain(5, 1), resample_rule=-1)[0] == pamd.PAMD_EINVAL
    # the variable-size rules: mixed precision and one replica per lane group only
    for rule in (pamd.PAMD_RESAMPLE_NEAREST, pamd.PAMD_RESAMPLE_POISSON):
        assert _init_rc(pi.make_chain(5, 1), resample_rule=rule, precision=1)[0] == pamd.PAMD_EUNSUPPORTED
        assert _init_rc(pi.make_chain(5, 1), resample_rule=rule, replicas_per_lane=2)[0] == \
            pamd.PAMD_EUNSUPPORTED
        assert _init_rc(pi.make_chain(5, 1), R=0x7fff0000, resample_rule=rule)[0] == pamd.PAMD_EINVAL
