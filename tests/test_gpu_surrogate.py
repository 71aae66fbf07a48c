"""The learned surrogate end to end on the operating-point family (n = 40, order 3): labels from
the plain GPU method (checked against the CPU oracle), an ensemble of five BF16 MLPs
4 -> 256 -> 256 -> 256 -> 64 trained by the library's kernels on 4096 points, and 512 held-out
points evaluated by the plain method, with fallback to it where the members disagree by more than 5%.
The test states what the network gains over the method without it (throughput at bounded error).
"""
import time

import numpy as np
import pytest

import npf_synth as S
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_2509_08968_gb300 import build
    build.build()
    from paper_2509_08968_gb300 import surrogate as SG
    fam = S.surrogate_family(40, 0)
    lam_ref = np.linalg.eigvals(fam.A(fam.p0))
    solver = SG.PlainSolver(fam, 3, lam_ref, slots=256)
    idx = SG.top_indices(solver.npf(fam.p0[None])[0], 64)
    solver.indices = idx
    yield SG, fam, lam_ref, solver, idx
    solver.close()


def test_labels_match_oracle(setup):
    SG, fam, lam_ref, solver, idx = setup
    P = S.operating_points(fam, 3, 99)
    F = solver.npf(P)
    for j, p in enumerate(P):
        lam, U, V = SG.modal_data(fam.A(p), lam_ref)
        sysm = S.ModalSystem(n=40, A1=fam.A(p), lam=lam, U=U, V=V, P=np.eye(40),
                             tensors=dict(fam.tensors))
        ref = oracle.npf_orders(sysm, 3, p1_block=40)
        assert np.linalg.norm(F[j] - ref) / np.linalg.norm(ref) < 1e-10


def test_top_indices_tie_rule(setup):
    SG = setup[0]
    a = np.array([[1.0, 3.0, 3.0], [2.0, 3.0, 0.5]])
    assert SG.top_indices(a, 4).tolist() == [1, 2, 4, 3]


def test_surrogate_gain_over_plain_method(setup):
    SG, fam, lam_ref, solver, idx = setup
    Ptr = S.operating_points(fam, 4096, 0)
    Pte = S.operating_points(fam, 512, 1)
    Ytr = solver.values(Ptr)
    t0 = time.perf_counter()
    Yte = solver.values(Pte)
    t_plain = time.perf_counter() - t0
    sur = SG.Surrogate(fam, idx, [4, 256, 256, 256, 64], ensemble=5, seed=0)
    try:
        hist = sur.fit(Ptr, Ytr, epochs=300, batch=256, lr=1e-3, seed=0)
        assert hist[-1] < 0.05 * hist[0]
        sur.predict(Pte[:8])                      # warm-up
        t0 = time.perf_counter()
        mean, spread, fb = sur.predict(Pte, 0.05)
        t_sur = time.perf_counter() - t0
        t0 = time.perf_counter()
        out, spread_g, fb_g = sur.gated(Pte, solver, 0.05)
        t_gated = time.perf_counter() - t0
    finally:
        sur.close()
    np.testing.assert_array_equal(fb, fb_g)
    rel = np.abs(out - Yte) / Yte
    rowmax = (np.abs(mean - Yte) / Yte).max(axis=1)
    # error bars of the gated pipeline (fallback rows are exact to the plain method)
    assert fb.mean() <= 0.10
    assert np.median(rel) < 5e-3
    assert np.percentile(rel, 95) < 2e-2
    assert np.percentile(rowmax[~fb], 95) < 5e-2
    assert np.all(rel[fb] < 1e-9)
    # the gate tracks the error: rows it rejects are worse than rows it accepts
    assert np.median(rowmax[fb]) > np.median(rowmax[~fb])
    # gate misses: accepted rows whose worst output is off by more than the 5% gate. The spread
    # of five members estimates the error, so a few misses are expected; they stay rare and
    # bounded (one accepted row of 512 at 13% was measured)
    miss = rowmax[~fb] > 0.05
    assert miss.mean() <= 0.02, miss.mean()
    assert rowmax[~fb].max() < 0.25, rowmax[~fb].max()
    # the gain: queries per second against the plain method on the same points
    assert 512 / t_sur > 100 * (512 / t_plain)
    assert 512 / t_gated > 3 * (512 / t_plain)
