"""Pins of the critical-mode subset in the oracle: the whole mode set gives Psi_N, and a brute
force over the subset (Eq. 4 then Eq. 7 with every index in the subset) agrees."""
import itertools

import numpy as np

import npf_synth as S
import oracle


def test_all_modes_is_psiN():
    sysm = S.config_small(0, orders=(3,))
    a = oracle.psiN_subset(sysm.tensors[3], 10, 3, sysm.U, sysm.V, sysm.lam, np.arange(10))
    b = oracle.psiN(sysm.tensors[3], 10, 3, sysm.U, sysm.V, sysm.lam, p1_block=10)
    np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-13 * np.abs(b).max())


def test_brute_force_subset():
    n, N = 6, 3
    sysm = S.modal_system(n, 3)
    A = S.random_packed_tensor_dense_fill(n, N, 7)
    modes = [4, 1, 2]
    got = oracle.psiN_subset(A, n, N, sysm.U, sysm.V, sysm.lam, modes)
    h = oracle.h_brute(oracle.unpack(A, n, N), sysm.U, sysm.V, sysm.lam)
    want = np.zeros((n, n), dtype=complex)
    for i in modes:
        for k in range(n):
            acc = 0
            for p in itertools.product(modes, repeat=N):
                acc += h[(i,) + p] * np.prod([sysm.V[q, k] for q in p])
            want[i, k] = -acc
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14)
