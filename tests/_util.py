import numpy as np


def rel_fro(got, ref):
    """Relative Frobenius error ||got - ref||_F / ||ref||_F."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    return float(np.linalg.norm((got - ref).ravel()) / np.linalg.norm(ref.ravel()))


def make_plan(npf, sysm, N_max, precision, **kw):
    p = npf.Plan(sysm.lam, sysm.U, sysm.V, N_max, precision=precision, **kw)
    for N, t in sysm.tensors.items():
        if N <= N_max:
            p.set_tensor(N, t)
    return p
