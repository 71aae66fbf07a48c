"""Write stored oracle results used by the GPU parity tests.

Calls only the CPU oracle (oracle/) on the seeded synthetic inputs of npf_synth:
  n120_seed0_order3.npz : Psi_3[i, k] for the n = 120 block-structured system (seed 0),
                          the full order-3 correction term of Eq. 7.
Run from the repository root:  python tests/golden/make_golden.py [order4 | radix128 | n120order4]
  order4:
    n60_seed2_order4.npz  : Psi_4 of the n = 60 system (seed 2).
    n120_seed0_order4_slabs.npz : three order-4 modal slabs of the n = 120 system (seed 0).
  radix128 (systems with 64 < n <= 128, whose digits use the row radix 128):
    n68_seed0_order4.npz  : Psi_4 of the n = 68 system (seed 0), ~10 min on 8 cores.
    n80_seed1_order4.npz  : Psi_4 of the n = 80 system (seed 1), ~25 min on 8 cores.
  n120order4:
    n120_seed0_order4.npz : Psi_4 of the n = 120 system (seed 0), the full order-4 term of the
                            benchmarked system, ~6 h on 8 cores.
  npf34 (after the two n = 120 terms exist):
    n120_seed0_npf34.npz  : NPF of the n = 120 system with its order-3 and order-4 terms
                            (Algorithm 2 step 20), the output of the benchmarked call.
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import npf_synth as S  # noqa: E402
import oracle  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    sysm = S.config_n120(0, orders=(3,))
    t = time.time()
    psi3 = oracle.psiN(sysm.tensors[3], 120, 3, sysm.U, sysm.V, sysm.lam, p1_block=4)
    np.savez_compressed(os.path.join(HERE, "n120_seed0_order3.npz"), psi3=psi3)
    print(f"n120 order 3: {time.time() - t:.1f} s, |Psi_3|_F = {np.linalg.norm(psi3):.6e}")


if __name__ == "__main__" and len(sys.argv) == 1:
    main()


def order4():
    """n = 60 full Psi_4 (seed 2) and three order-4 modal slabs of the n = 120 system (seed 0,
    first output index p_1 = 7): h^i_{7, p_2, p_3, q} for (p_2, p_3) in SLABS_120."""
    s60 = S.config_n60(2, orders=(4,))
    t = time.time()
    psi4 = oracle.psiN(s60.tensors[4], 60, 4, s60.U, s60.V, s60.lam, p1_block=1)
    np.savez_compressed(os.path.join(HERE, "n60_seed2_order4.npz"), psi4=psi4)
    print(f"n60 order 4: {time.time() - t:.1f} s")
    s120 = S.config_n120(0, orders=(4,))
    t = time.time()
    hb = oracle.h_fact(s120.tensors[4], 120, 4, s120.U, s120.V, s120.lam, p1_lo=7, p1_hi=8)
    slabs = np.stack([hb[:, 0, p2, p3, :] for (p2, p3) in SLABS_120])
    np.savez_compressed(os.path.join(HERE, "n120_seed0_order4_slabs.npz"), slabs=slabs,
                        prefixes=np.array([(7, p2, p3) for (p2, p3) in SLABS_120]))
    print(f"n120 order 4 slabs: {time.time() - t:.1f} s")


SLABS_120 = [(0, 0), (33, 91), (119, 64)]

if __name__ == "__main__" and "order4" in sys.argv:
    order4()


def radix128():
    """Full Psi_4 of two systems above 64 states (n = 68 seed 0, n = 80 seed 1)."""
    for n, seed in ((68, 0), (80, 1)):
        sysm = S.config_blocks(n, seed, orders=(4,))
        t = time.time()
        psi4 = oracle.psiN(sysm.tensors[4], n, 4, sysm.U, sysm.V, sysm.lam, p1_block=1)
        np.savez_compressed(os.path.join(HERE, f"n{n}_seed{seed}_order4.npz"), psi4=psi4)
        print(f"n{n} order 4: {time.time() - t:.1f} s, |Psi_4|_F = {np.linalg.norm(psi4):.6e}",
              flush=True)


def n120_order4():
    """Full Psi_4 of the n = 120 system (seed 0)."""
    sysm = S.config_n120(0, orders=(4,))
    t = time.time()
    psi4 = oracle.psiN(sysm.tensors[4], 120, 4, sysm.U, sysm.V, sysm.lam, p1_block=1)
    np.savez_compressed(os.path.join(HERE, "n120_seed0_order4.npz"), psi4=psi4)
    print(f"n120 order 4: {time.time() - t:.1f} s, |Psi_4|_F = {np.linalg.norm(psi4):.6e}",
          flush=True)


if __name__ == "__main__" and "radix128" in sys.argv:
    radix128()

if __name__ == "__main__" and "n120order4" in sys.argv:
    n120_order4()


def npf34():
    """NPF (Alg. 2 step 20) of the n = 120 system from the stored Psi_3 and Psi_4."""
    sysm = S.config_n120(0, orders=())
    psi3 = np.load(os.path.join(HERE, "n120_seed0_order3.npz"))["psi3"]
    psi4 = np.load(os.path.join(HERE, "n120_seed0_order4.npz"))["psi4"]
    npf = oracle.npf(sysm.U, sysm.V, psi3 + psi4)
    np.savez_compressed(os.path.join(HERE, "n120_seed0_npf34.npz"), npf=npf)
    print(f"n120 NPF of orders 3+4: |NPF|_F = {np.linalg.norm(npf):.6e}", flush=True)


if __name__ == "__main__" and "npf34" in sys.argv:
    npf34()
