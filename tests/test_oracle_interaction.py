"""Pins of the mode-interaction NPFs (Eqs. 6-9) in the oracle: the reconstruction of the
excitation (Eq. 6) has the residual order that the corrected coordinates imply, a brute-force
evaluation of Eqs. 8-9 from Eq. 4 agrees, and the small-excitation limit is the linear PF."""
import itertools

import numpy as np

import npf_synth as S
import oracle


def _residual(sysm, order, delta):
    t = oracle.interaction_npfs(sysm, order, delta)
    return np.abs(delta - t.sum(axis=0).sum(axis=1)).max()   # x^k(0) = delta for every k


def _slope(sysm, order):
    r1, r2 = _residual(sysm, order, 0.02), _residual(sysm, order, 0.01)
    return np.log2(r1 / r2)


def test_reconstruction_residual_order():
    """x = Phi (z + h(z)) with z = zeta - h(zeta): for a single order N the residual is
    O(delta^(2N-1)) (it vanishes with the uncorrected zeta and is O(delta^N) with the wrong
    sign of the correction); with orders 2 and 3 together the h2-h2 cross term gives delta^3."""
    base = S.config_small(0, orders=(2, 3))
    only2 = S.ModalSystem(n=10, A1=base.A1, lam=base.lam, U=base.U, V=base.V, P=base.P,
                          tensors={2: base.tensors[2]})
    only3 = S.ModalSystem(n=10, A1=base.A1, lam=base.lam, U=base.U, V=base.V, P=base.P,
                          tensors={3: base.tensors[3]})
    assert 2.6 < _slope(only2, 2) < 3.4
    assert 4.5 < _slope(only3, 3) < 5.5
    assert 2.6 < _slope(base, 3) < 3.4
    assert _residual(only2, 2, 0.02) > 1e-12


def test_brute_force_eqs_8_9():
    n = 4
    sysm = S.modal_system(n, 11)
    for N in (2, 3):
        sysm.tensors[N] = S.random_packed_tensor_dense_fill(n, N, 20 + N)
    delta = 0.3
    h = {N: oracle.h_brute(oracle.unpack(sysm.tensors[N], n, N), sysm.U, sysm.V, sysm.lam)
         for N in (2, 3)}
    got = oracle.interaction_npfs(sysm, 3, delta)
    for k in range(n):
        zeta = delta * sysm.V[:, k]
        z = zeta.copy()
        for N in (2, 3):
            for p in itertools.product(range(n), repeat=N):
                z -= h[N][(slice(None),) + p] * np.prod(zeta[list(p)])
        np.testing.assert_allclose(got[0][k], sysm.U[k] * z, rtol=1e-12, atol=1e-14)
        for M in (2, 3):
            T = np.zeros(n, dtype=complex)
            for p in itertools.product(range(n), repeat=M):
                T += h[M][(slice(None),) + p] * np.prod(z[list(p)])
            np.testing.assert_allclose(got[M - 1][k], sysm.U[k] * T, rtol=1e-11, atol=1e-13)


def test_small_excitation_limit_is_linear_pf():
    """pN1 / delta -> the linear PF phi_ki psi_ik with an O(delta) error, and pNM = O(delta^M):
    a tenfold smaller excitation shrinks them by 10, 10^2 and 10^3."""
    sysm = S.config_small(1, orders=(2, 3))
    lin = sysm.U * sysm.V.T
    a, b = (oracle.interaction_npfs(sysm, 3, d) for d in (1e-4, 1e-5))
    ratio_lin = np.abs(a[0] / 1e-4 - lin).max() / np.abs(b[0] / 1e-5 - lin).max()
    assert 9.0 < ratio_lin < 11.0
    assert 90.0 < np.abs(a[1]).max() / np.abs(b[1]).max() < 110.0
    assert 900.0 < np.abs(a[2]).max() / np.abs(b[2]).max() < 1100.0
