"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test targets a mistake the oracle could plausibly make (a dropped 1/N!, a flipped sign in
the resonance denominator, a transposed eigenvector, a wrong lower-index pairing, a wrong
Khatri-Rao orientation):

* the normal-form (homological) property of h, checked by evaluating the transformed dynamics;
* the scalar textbook normal form x' = lam x + c x^N  ->  h = c / ((N-1) lam);
* the linear participation factors (order 1) summing to 1 over states and over modes;
* the collapse identity with the divide disabled (a closed form at any size);
* invariance of the NPFs under eigenvector rescaling, and the matching scaling of h;
* symmetry of h in the lower indices; the identity-eigenvector case; the eps clamp;
* brute force (Eq. 4 and the Psi_N sum written out literally) against the factorised forms;
* the contraction chain run on A1 as an order-1 tensor with the divide off: Psi A1 Phi =
  diag(lambda), which the eigen-decomposition of the generator fixes.
"""
import itertools
import math

import numpy as np
import pytest

import npf_synth as S
import oracle


def dense_from_packed(packed, n, N):
    """Independent expansion: packed order is combinations_with_replacement order."""
    d = np.zeros((n,) + (n,) * N)
    for r, t in enumerate(itertools.combinations_with_replacement(range(n), N)):
        for perm in set(itertools.permutations(t)):
            d[(slice(None),) + perm] = packed[:, r]
    return d


def poly_eval(T, z, N):
    """T[i, p_1..p_N] contracted with z on every lower index."""
    out = T
    for _ in range(N):
        out = out @ z          # contracts the trailing axis
    return out


def test_packed_count_and_unpack_match_itertools():
    for n, N in [(3, 2), (4, 3), (5, 4)]:
        pk = S.random_packed_tensor(n, N, 7)
        assert oracle.packed_count(n, N) == pk.shape[1]
        np.testing.assert_array_equal(oracle.unpack(pk, n, N), dense_from_packed(pk, n, N))


@pytest.mark.parametrize("N", [2, 3, 4, 5])
def test_scalar_textbook_normal_form(N):
    # x' = lam x + c x^N. With x = z + h z^N and z' = lam z the z^N terms cancel when
    # N h lam = lam h + c, i.e. h = c / ((N-1) lam). The derivative tensor is A_N = N! c.
    lam = np.array([-0.7 + 0.3j])
    c = 1.9
    U = np.ones((1, 1), complex)
    V = np.ones((1, 1), complex)
    pk = np.array([[math.factorial(N) * c]])
    h = oracle.h_fact(pk, 1, N, U, V, lam)
    np.testing.assert_allclose(h.ravel()[0], c / ((N - 1) * lam[0]), rtol=1e-14)
    hb = oracle.h_brute(oracle.unpack(pk, 1, N), U, V, lam)
    np.testing.assert_allclose(hb.ravel()[0], c / ((N - 1) * lam[0]), rtol=1e-14)


@pytest.mark.parametrize("N,seed", [(2, 0), (3, 1), (4, 2)])
def test_homological_equation_residual(N, seed):
    """With x = Phi (z + h(z)), z' = Lambda z, the order-N terms of
    Psi f(x) - d/dt(z + h(z)) vanish for f(x) = A1 x + (1/N!) A_N[x,..,x]."""
    n = 4
    sysm = S.modal_system(n, seed)
    pk = S.random_packed_tensor_dense_fill(n, N, seed + 11)
    A = dense_from_packed(pk, n, N)
    h = oracle.h_brute(oracle.unpack(pk, n, N), sysm.U, sysm.V, sysm.lam)
    rng = np.random.default_rng(seed)
    z0 = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    # D_t of the lower-index polynomial multiplies h^i_p by sum_m lam_{p_m}
    lam_sum = np.zeros((n,) * N, complex)
    for m in range(N):
        shape = [1] * N
        shape[m] = n
        lam_sum = lam_sum + sysm.lam.reshape(shape)

    def residual(t, hh):
        z = t * z0
        hz = poly_eval(hh, z, N)
        x = sysm.U @ (z + hz)
        f = sysm.A1 @ x + poly_eval(A, x, N) / math.factorial(N)
        dz = sysm.lam * z + poly_eval(hh * lam_sum[None], z, N)
        return sysm.V @ f - dz

    for t in (1e-3, 1e-4):
        r = np.abs(residual(t, h)).max()
        r0 = np.abs(residual(t, np.zeros_like(h))).max()
        # without h the residual is O(t^N); with the oracle's h it must be O(t^(N+1))
        assert r0 > 1e-3 * t ** N
        assert r < 50 * t * r0, (t, r, r0)
    # and a plausible mistake (no 1/N!) breaks it
    bad = h * math.factorial(N)
    assert np.abs(residual(1e-4, bad)).max() > 0.1 * np.abs(residual(1e-4, np.zeros_like(h))).max()


def test_linear_participation_factors_sum_to_one():
    sysm = S.modal_system(10, 3)
    P = oracle.npf(sysm.U, sysm.V)
    np.testing.assert_allclose(P, sysm.U * sysm.V.T, rtol=1e-15, atol=1e-300)
    np.testing.assert_allclose(P.sum(axis=0), np.ones(10), atol=1e-12)
    np.testing.assert_allclose(P.sum(axis=1), np.ones(10), atol=1e-12)


@pytest.mark.parametrize("n,N", [(6, 2), (6, 3), (4, 4), (10, 3)])
def test_collapse_identity(n, N):
    """Divide disabled: sum_p C^i_p prod_m psi_{p_m k} = (1/N!) sum_j psi_ij A^j_{k..k}, because
    sum_p phi_{a p} psi_{p k} = delta_{a k}. So Psi_N[i,k] = -(1/N!) sum_j psi_ij A^j_{k..k}."""
    sysm = S.modal_system(n, n + N)
    pk = S.random_packed_tensor(n, N, 5 * n + N)
    diag_rank = {t: r for r, t in enumerate(itertools.combinations_with_replacement(range(n), N))}
    Akk = np.array([pk[:, diag_rank[(k,) * N]] for k in range(n)]).T      # [j, k]
    expect = -(sysm.V @ Akk) / math.factorial(N)
    got = oracle.psiN(pk, n, N, sysm.U, sysm.V, sysm.lam, divide=False)
    np.testing.assert_allclose(got, expect, rtol=0, atol=1e-12 * np.abs(expect).max())


@pytest.mark.parametrize("N", [2, 3])
def test_rescaling_invariance(N):
    n = 6
    sysm = S.modal_system(n, 4)
    pk = S.random_packed_tensor(n, N, 44)
    rng = np.random.default_rng(0)
    s = (0.5 + rng.random(n)) * np.exp(2j * np.pi * rng.random(n))
    U2 = sysm.U * s[None, :]
    V2 = sysm.V / s[:, None]
    P1 = oracle.npf(sysm.U, sysm.V,
                    oracle.psiN(pk, n, N, sysm.U, sysm.V, sysm.lam))
    P2 = oracle.npf(U2, V2, oracle.psiN(pk, n, N, U2, V2, sysm.lam))
    np.testing.assert_allclose(P2, P1, rtol=0, atol=1e-12 * np.abs(P1).max())
    h1 = oracle.h_fact(pk, n, N, sysm.U, sysm.V, sysm.lam)
    h2 = oracle.h_fact(pk, n, N, U2, V2, sysm.lam)
    scale = 1.0 / s
    for m in range(N):
        shape = [1] * (N + 1)
        shape[m + 1] = n
        scale = scale.reshape([n] + [1] * N) if m == 0 else scale
        scale = scale * s.reshape(shape)
    np.testing.assert_allclose(h2, h1 * scale, rtol=0, atol=1e-12 * np.abs(h1).max())


@pytest.mark.parametrize("N", [2, 3, 4])
def test_h_symmetric_in_lower_indices(N):
    n = 5 if N < 4 else 4
    sysm = S.modal_system(n if n % 2 == 0 else 6, 9)
    n = sysm.n
    pk = S.random_packed_tensor(n, N, 99)
    h = oracle.h_fact(pk, n, N, sysm.U, sysm.V, sysm.lam)
    for perm in itertools.permutations(range(1, N + 1)):
        np.testing.assert_allclose(np.transpose(h, (0,) + perm), h, rtol=0,
                                   atol=1e-13 * np.abs(h).max())


@pytest.mark.parametrize("N", [2, 3])
def test_identity_eigenvectors(N):
    """Phi = Psi = I: h^i_p = A^i_p / (N! (sum_m lam_{p_m} - lam_i)) and Psi_N[i,k] = -h^i_{k..k}."""
    n = 5
    rng = np.random.default_rng(1)
    lam = -rng.uniform(0.1, 2, n) + 1j * rng.uniform(-5, 5, n)
    I = np.eye(n, dtype=complex)
    pk = S.random_packed_tensor_dense_fill(n, N, 3)
    A = dense_from_packed(pk, n, N)
    h = oracle.h_fact(pk, n, N, I, I, lam)
    for idx in itertools.product(range(n), repeat=N + 1):
        i, p = idx[0], idx[1:]
        D = sum(lam[q] for q in p) - lam[i]
        assert abs(h[idx] - A[idx] / (math.factorial(N) * D)) <= 1e-14 * abs(h).max()
    Psi = oracle.psiN(pk, n, N, I, I, lam)
    for i in range(n):
        for k in range(n):
            np.testing.assert_allclose(Psi[i, k], -h[(i,) + (k,) * N], rtol=1e-13)


def test_eps_clamp_is_strict_and_real():
    """Alg. 2 step 9: |D| < eps -> D = eps (a real value)."""
    n, N = 3, 2
    lam = np.array([-1 + 2j, -0.5 + 1j, -1.5 + 3j + 1e-10])   # D^2_{01} = -1e-10
    I = np.eye(n, dtype=complex)
    pk = np.zeros((n, S.packed_count(n, N)))
    r01 = list(itertools.combinations_with_replacement(range(n), N)).index((0, 1))
    pk[2, r01] = 3.0
    eps = 1e-8
    h = oracle.h_fact(pk, n, N, I, I, lam, eps=eps)
    np.testing.assert_allclose(h[2, 0, 1], 3.0 / (2 * eps), rtol=1e-14)
    np.testing.assert_allclose(h[2, 1, 0], 3.0 / (2 * eps), rtol=1e-14)
    # just above eps the clamp does not fire
    lam2 = lam.copy()
    lam2[2] = lam[0] + lam[1] - 2e-8
    h2 = oracle.h_fact(pk, n, N, I, I, lam2, eps=eps)
    D = lam2[0] + lam2[1] - lam2[2]
    np.testing.assert_allclose(h2[2, 0, 1], 3.0 / (2 * D), rtol=1e-6)
    # exactly at eps it does not fire either (strict <): D = (3 + 4i) 2^-28, |D| = 5 * 2^-28, with
    # every sum exact, so a clamp that fired would turn the complex D into the real eps
    Dx = (3 + 4j) * 2.0 ** -28
    lam3 = lam.copy()
    lam3[2] = complex(-1.5 - 3 * 2.0 ** -28, 3 - 4 * 2.0 ** -28)
    assert (-lam3[2] + lam3[0]) + lam3[1] == Dx
    eps3 = 5 * 2.0 ** -28
    if abs(Dx) != eps3:
        pytest.skip("this libm's hypot does not return 5 * 2^-28 exactly for (3, 4) * 2^-28")
    h3 = oracle.h_fact(pk, n, N, I, I, lam3, eps=eps3)
    np.testing.assert_allclose(h3[2, 0, 1], 3.0 / (2 * Dx), rtol=1e-14)


@pytest.mark.parametrize("n,N", [(4, 2), (6, 2), (4, 3), (6, 3), (4, 4), (6, 4)])
def test_brute_equals_factorised(n, N):
    sysm = S.modal_system(n, 10 * n + N)
    pk = S.random_packed_tensor(n, N, n * N)
    hb = oracle.h_brute(oracle.unpack(pk, n, N), sysm.U, sysm.V, sysm.lam)
    hf = oracle.h_fact(pk, n, N, sysm.U, sysm.V, sysm.lam)
    np.testing.assert_allclose(hf, hb, rtol=0, atol=1e-13 * np.abs(hb).max())
    pb = oracle.psiN_brute(hb, sysm.V)
    pf = oracle.psiN(pk, n, N, sysm.U, sysm.V, sysm.lam, p1_block=2)
    np.testing.assert_allclose(pf, pb, rtol=0, atol=1e-13 * np.abs(pb).max())
    # the slab routine agrees with the full tensor
    pre = [(q * 5 + 1) % n for q in range(N - 1)]
    sl = oracle.h_slab(pk, n, N, sysm.U, sysm.V, sysm.lam, pre)
    np.testing.assert_allclose(sl, hb[(slice(None),) + tuple(pre)], rtol=0,
                               atol=1e-13 * np.abs(hb).max())


def test_psiN_khatri_rao_orientation():
    """Psi_N[i,k] = -sum_p h^i_p prod_m Psi[p_m, k]: rows of Psi are modes (p), columns states (k).
    Evaluated here as -h^i(zeta_k) with zeta_k = Psi[:, k] by plain polynomial evaluation."""
    n, N = 4, 3
    sysm = S.modal_system(n, 21)
    pk = S.random_packed_tensor_dense_fill(n, N, 2)
    h = oracle.h_brute(oracle.unpack(pk, n, N), sysm.U, sysm.V, sysm.lam)
    got = oracle.psiN(pk, n, N, sysm.U, sysm.V, sysm.lam)
    for k in range(n):
        zeta = sysm.V[:, k]
        np.testing.assert_allclose(got[:, k], -poly_eval(h, zeta, N), rtol=1e-12)


def test_npf_orders_cumulative():
    sysm = S.config_small(0, orders=(2, 3))
    P3 = oracle.npf_orders(sysm, 3, p1_block=5)
    S2 = oracle.psiN(sysm.tensors[2], 10, 2, sysm.U, sysm.V, sysm.lam)
    S3 = oracle.psiN(sysm.tensors[3], 10, 3, sysm.U, sysm.V, sysm.lam)
    np.testing.assert_allclose(P3, sysm.U * (sysm.V + S2 + S3).T, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("n,seed", [(4, 0), (10, 1), (20, 2)])
def test_order1_chain_gives_eigenvalues(n, seed):
    """The chain of Algorithm 2 (lower index with Phi, upper index with Psi, 1/1!) applied to the
    Jacobian A1 as an order-1 tensor, with the divide off, gives Psi A1 Phi = diag(lambda): the
    generator builds A1 = P B P^-1 with U = P W, so this is fixed by the eigen-decomposition, not
    by the oracle. A transposed Phi or Psi, or a wrong pairing of the upper index, breaks it."""
    sysm = S.modal_system(n, seed) if n % 4 else S.config_blocks(n, seed, orders=())
    A1 = np.ascontiguousarray(sysm.A1)           # packed order 1: coeffs[j, a] = A1[j, a]
    h = oracle.h_fact(A1, n, 1, sysm.U, sysm.V, sysm.lam, divide=False)
    assert h.shape == (n, n)
    scale = np.abs(sysm.lam).max()
    np.testing.assert_allclose(h, np.diag(sysm.lam), rtol=0, atol=1e-12 * scale)
    if n <= 10:
        hb = oracle.h_brute(A1, sysm.U, sysm.V, sysm.lam, divide=False)
        np.testing.assert_allclose(hb, np.diag(sysm.lam), rtol=0, atol=1e-12 * scale)
    # with the divide on, D = lambda_p - lambda_i: zero on the diagonal, clamped to eps (step 9)
    hd = oracle.h_fact(A1, n, 1, sysm.U, sysm.V, sysm.lam)
    np.testing.assert_allclose(np.diag(hd), sysm.lam / oracle.DEFAULT_EPS, rtol=1e-6)
