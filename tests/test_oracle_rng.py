"""Pins of the oracle's random-number and exponential primitives.

* Philox4x32-10 is checked against an independent implementation: Triton's
  ``tl.philox`` run by Triton's CPU interpreter (a library routine).
* The Box-Muller normals are checked for their moments and by a KS test.
* exp_det is checked against the correctly rounded exponential from mpmath
  (error bound: 1 ulp) and against libm on a dense sweep.
"""
import math
import os

import numpy as np
import pytest


def _triton_philox(seed, ctrs):
    """Philox4x32-10 outputs from Triton's interpreter for a batch of counters."""
    os.environ["TRITON_INTERPRET"] = "1"
    triton = pytest.importorskip("triton")
    import torch
    import triton.language as tl

    n = ctrs.shape[0]
    blk = 1 << max(0, (n - 1).bit_length())

    @triton.jit
    def kern(out, c0p, c1p, c2p, c3p, seed, n, BLK: tl.constexpr):
        off = tl.arange(0, BLK)
        m = off < n
        c0 = tl.load(c0p + off, mask=m, other=0)
        c1 = tl.load(c1p + off, mask=m, other=0)
        c2 = tl.load(c2p + off, mask=m, other=0)
        c3 = tl.load(c3p + off, mask=m, other=0)
        a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
        tl.store(out + off * 4 + 0, a, mask=m)
        tl.store(out + off * 4 + 1, b, mask=m)
        tl.store(out + off * 4 + 2, c, mask=m)
        tl.store(out + off * 4 + 3, d, mask=m)

    cols = [torch.from_numpy(ctrs[:, q].astype(np.uint32).view(np.int32).copy()) for q in range(4)]
    out = torch.zeros(n * 4, dtype=torch.int32)
    kern[(1,)](out, *cols, seed, n, BLK=blk)
    return out.numpy().view(np.uint32).reshape(n, 4)


def test_philox_matches_triton_interpreter(orc):
    rng = np.random.default_rng(5)
    ctrs = rng.integers(0, 2**32, (64, 4), dtype=np.uint64).astype(np.uint32)
    ctrs[0] = 0
    ctrs[1] = [2**32 - 1] * 4
    for seed in (0, 12345, 0xDEADBEEF_01234567):
        ref = _triton_philox(seed, ctrs)
        key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
        got = np.stack([orc.philox4x32_10(c, key) for c in ctrs])
        np.testing.assert_array_equal(got, ref)


def test_normals_moments_and_ks(orc):
    scipy_stats = pytest.importorskip("scipy.stats")
    z = np.array([orc.normal3(777, a, s, 3, 0) for a in range(100) for s in range(200)]).ravel()
    n = len(z)
    assert abs(z.mean()) < 4.0 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 4.0 * math.sqrt(2.0 / n)
    kurt = np.mean(z**4) / np.mean(z**2) ** 2
    assert abs(kurt - 3.0) < 0.1
    assert scipy_stats.kstest(z, "norm").pvalue > 1e-4
    # the three components of one draw are uncorrelated
    zz = z.reshape(-1, 3)
    cc = np.corrcoef(zz.T)
    assert np.abs(cc - np.eye(3)).max() < 4.0 / math.sqrt(zz.shape[0])


def test_normals_differ_per_counter_field(orc):
    base = orc.normal3(1, 2, 3, 4, 0)
    for args in [(1, 3, 3, 4, 0), (1, 2, 4, 4, 0), (1, 2, 3, 5, 0), (1, 2, 3, 4, 1), (2, 2, 3, 4, 0)]:
        assert not np.allclose(orc.normal3(*args), base)


def test_exp_det_correctly_rounded_within_one_ulp(orc):
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 120
    rng = np.random.default_rng(11)
    xs = np.concatenate([rng.uniform(-700, 0, 400), rng.uniform(-1, 1, 200),
                         [0.0, -1e-300, -0.34657359, 0.34657359, -708.0, 5.0, 700.0]])
    got = orc.exp_det(xs)
    for x, g in zip(xs, got):
        exact = mp.exp(mp.mpf(float(x)))
        ulp = math.ulp(float(exact))
        assert abs(mp.mpf(float(g)) - exact) <= ulp, (x, g)


def test_exp_det_sweep_against_libm(orc):
    xs = np.linspace(-40.0, 0.0, 20001)
    got = orc.exp_det(xs)
    ref = np.exp(xs)
    ulps = np.abs(got - ref) / np.spacing(ref)
    assert ulps.max() <= 1.0
    assert orc.exp_det([-709.0])[0] == 0.0
