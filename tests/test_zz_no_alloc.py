"""The allocation-free resampling entry point against pamd_resample.

pamd_resample_counts_noalloc serves callers that cannot allocate device
memory (a framework that owns the device pool, code that must not trigger
cudaFree's implicit synchronisation, fixed memory budgets).  Its copy counts
must equal pamd_resample's bit for bit and its ln Q to 1e-12, on two calls in
a row (the second call must not see the first call's leftovers in the shared
scratch array).  This file sorts last so that a failure here does not hide
the other GPU tests.
"""
import numpy as np
import pytest

import pamd_inputs as pi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_06016_gb300 import build, pamd
    build.build()
    pamd.load()
    return torch, pamd


@pytest.mark.parametrize("R", [1, 3000, 262144])
def test_noalloc_counts_match_resample(env, R):
    torch, pamd = env
    top = pi.make_chain(12, 2)
    seed, dt = 77, 0.001
    temps = [900.0, 860.0, 820.0]
    ctx = pamd.pamd_init(top, R, temps[0], seed)
    try:
        pamd.pamd_propagate(ctx, 3, dt, temps[0])
        for i in (1, 2):  # two calls in a row
            _, _, E, _ = pamd.pamd_get_state(ctx, positions=False, velocities=False, families=False)
            ref_counts, ref_lnq = pamd.pamd_resample(ctx, temps[i - 1], temps[i])
            E_dev = torch.tensor(E, dtype=torch.float64, device="cuda")
            counts = torch.full((R,), -7, dtype=torch.int32, device="cuda")
            lnq = torch.zeros(1, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            pamd.pamd_resample_counts_noalloc(E_dev.data_ptr(), R, temps[i - 1], temps[i], seed, i,
                                              counts.data_ptr(), lnq.data_ptr())
            torch.cuda.synchronize()
            np.testing.assert_array_equal(counts.cpu().numpy(), ref_counts)
            assert abs(lnq.item() - ref_lnq) <= 1e-12 * max(1.0, abs(ref_lnq))
            pamd.pamd_propagate(ctx, 3, dt, temps[i])
    finally:
        pamd.pamd_destroy(ctx)


def test_noalloc_rejects_oversized_population(env):
    torch, pamd = env
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    counts = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(pamd.PamdError) as ei:
        pamd.pamd_resample_counts_noalloc(E.data_ptr(), 262145, 500.0, 450.0, 1, 1, counts.data_ptr())
    assert ei.value.code == pamd.PAMD_EINVAL and "262144" in str(ei.value)
