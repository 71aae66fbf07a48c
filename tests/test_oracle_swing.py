"""Pins of the swing-model inputs and of the oracle's closed-form derivative tensors: central
finite differences of the model's right-hand side, the equilibrium, and the Jacobian."""
import numpy as np

import npf_synth as S
from oracle import swing


def test_equilibrium_and_jacobian():
    mod = S.swing_model(4, 2)
    x0 = np.concatenate([mod.delta, np.zeros(4)])
    assert np.abs(mod.f(x0)).max() < 1e-12
    h = 1e-6
    J = np.zeros((8, 8))
    for a in range(8):
        e = np.zeros(8)
        e[a] = h
        J[:, a] = (mod.f(x0 + e) - mod.f(x0 - e)) / (2 * h)
    np.testing.assert_allclose(mod.jacobian(), J, atol=1e-8)


def test_closed_form_tensors_match_finite_differences():
    mod = S.swing_model(3, 0)
    for N, tol in ((2, 1e-6), (3, 2e-5)):
        A = swing.packed_tensor(mod, N)
        F = swing.finite_difference_tensor(mod, N)
        assert np.abs(A - F).max() < tol * np.abs(A).max(), N
        assert np.count_nonzero(A[:3]) == 0            # angle equations are linear


def test_order4_closed_form_matches_richardson_differences():
    """Order 4: the central difference of step h has an O(h^2) error and an O(eps / h^4)
    rounding error, so one Richardson step, (4 D(h/2) - D(h)) / 3, removes the h^2 term and
    leaves ~1e-8 at h = 0.02."""
    for m, seed in ((2, 0), (3, 1)):
        mod = S.swing_model(m, seed)
        A = swing.packed_tensor(mod, 4)
        h = 2e-2
        F = (4 * swing.finite_difference_tensor(mod, 4, h / 2)
             - swing.finite_difference_tensor(mod, 4, h)) / 3
        assert np.count_nonzero(A) > 0
        assert np.abs(A - F).max() < 1e-6 * np.abs(A).max(), m


def test_zero_mode_of_the_rotational_symmetry():
    """Without reference-bus lines, shifting every angle by the same amount leaves f unchanged,
    so A1 has the eigenvector (1, .., 1, 0, .., 0) with eigenvalue 0; the lines remove it."""
    mod = S.swing_model(5, 3, bus=False)
    v = np.concatenate([np.ones(5), np.zeros(5)])
    assert np.abs(mod.jacobian() @ v).max() < 1e-12
    withbus = S.swing_model(5, 3)
    assert np.abs(np.linalg.eigvals(withbus.jacobian())).min() > 1e-3
