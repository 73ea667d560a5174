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


def test_noalloc_molecule_stream_and_optional_outputs(env):
    """mol_id > 0 selects that molecule's Philox stream: counts equal those of
    molecule 1 of a batch context; lnQ_dev and status_dev may be NULL."""
    torch, pamd = env
    tops = [pi.make_chain(12, 3), pi.make_chain(15, 4)]
    Rs, T0, T1, seed = [700, 900], 800.0, 760.0, 31
    ctx = pamd.pamd_init_batch(tops, Rs, [T0, T0], seed)
    try:
        pamd.pamd_propagate(ctx, 3, 0.001, T0)
        _, _, E1, _ = pamd.pamd_get_state(pamd.pamd_batch_sub(ctx, 1), positions=False,
                                          velocities=False, families=False)
        ref_counts, ref_lnq = pamd.pamd_resample(ctx, T0, T1)
        ref1 = ref_counts[Rs[0]:]
        E_dev = torch.tensor(E1, dtype=torch.float64, device="cuda")
        counts = torch.full((Rs[1],), -7, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        pamd.pamd_resample_counts_noalloc(E_dev.data_ptr(), Rs[1], T0, T1, seed, 1, counts.data_ptr(),
                                          0, mol_id=1)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(counts.cpu().numpy(), ref1)
        lnq = torch.zeros(1, dtype=torch.float64, device="cuda")
        status = torch.full((1,), 99, dtype=torch.int32, device="cuda")
        pamd.pamd_resample_counts_noalloc(E_dev.data_ptr(), Rs[1], T0, T1, seed, 1, counts.data_ptr(),
                                          lnq.data_ptr(), mol_id=1, status_dev=status.data_ptr())
        torch.cuda.synchronize()
        np.testing.assert_array_equal(counts.cpu().numpy(), ref1)
        assert abs(lnq.item() - ref_lnq[1]) <= 1e-12 * max(1.0, abs(ref_lnq[1]))
        assert status.item() == 0
    finally:
        pamd.pamd_destroy(ctx)


def test_noalloc_nonfinite_energy_gets_weight_zero(env, orc):
    """An infinite energy: status PAMD_ENONFINITE, that replica weight 0, and
    the counts equal the oracle's bit for bit (on cooling the oracle's weight
    of E = +inf is exactly 0 as well)."""
    torch, pamd = env
    R, Tp, Tn, seed, ridx = 5000, 700.0, 650.0, 1234, 3
    E = pi.random_energies(R, -80.0, 25.0, 4)
    E[17] = np.inf
    _, W = orc.resample_weights(E, Tp, Tn)
    assert W[17] == 0
    ref = orc.multinomial_counts(W, seed, ridx)
    E_dev = torch.tensor(E, dtype=torch.float64, device="cuda")
    counts = torch.zeros(R, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for _ in range(2):  # the second call starts from the first call's scratch
        pamd.pamd_resample_counts_noalloc(E_dev.data_ptr(), R, Tp, Tn, seed, ridx, counts.data_ptr(),
                                          status_dev=status.data_ptr())
        torch.cuda.synchronize()
        np.testing.assert_array_equal(counts.cpu().numpy(), ref)
        assert status.item() == pamd.PAMD_ENONFINITE
    # a finite population afterwards reports 0 again
    E_dev[17] = -80.0
    pamd.pamd_resample_counts_noalloc(E_dev.data_ptr(), R, Tp, Tn, seed, ridx, counts.data_ptr(),
                                      status_dev=status.data_ptr())
    torch.cuda.synchronize()
    assert status.item() == 0


def test_noalloc_rejects_oversized_population(env):
    torch, pamd = env
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    counts = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(pamd.PamdError) as ei:
        pamd.pamd_resample_counts_noalloc(E.data_ptr(), 262145, 500.0, 450.0, 1, 1, counts.data_ptr())
    assert ei.value.code == pamd.PAMD_EINVAL and "262144" in str(ei.value)
