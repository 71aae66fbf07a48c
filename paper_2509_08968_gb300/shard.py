"""Row-sharded and resumable order-N terms.

Psi_N[i, k] of Eq. 7 sums over the lower indices only, so its rows (the upper index i) are
independent: disjoint row ranges computed separately (npf_get_term_rows) add up to the whole term.
This module splits the rows over ranks of a process group (one GPU each; the only exchange is one
sum of the n x n partial terms, FP64 complex) and over resumable chunks whose partial sums are
checkpointed to a file after each chunk; sharded_npf is the whole row-sharded NPF computation
that the multi-GPU benchmark times.
"""
from __future__ import annotations

import os

import numpy as np


def row_ranges(n, parts):
    """`parts` contiguous row ranges [lo, hi) covering [0, n), sizes differing by at most one."""
    if parts < 1:
        raise ValueError("parts must be >= 1")
    base, extra = divmod(n, parts)
    out, lo = [], 0
    for r in range(parts):
        hi = lo + base + (1 if r < extra else 0)
        out.append((lo, hi))
        lo = hi
    return out


def allreduce_sum(x, dist, group=None):
    """Sum of a complex128 array over the ranks of a torch.distributed group (real and imaginary
    parts as float64; on the GPU with NCCL, on the host with gloo)."""
    import torch
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.from_numpy(np.ascontiguousarray(np.asarray(x, dtype=np.complex128)).view(np.float64))
    t = t.to(dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy().view(np.complex128).reshape(np.shape(x))


def term_sharded(plan, order, dist, group=None):
    """Psi_N of `plan` with its rows split over the ranks of the group: each rank forms its own
    rows, then one sum gives every rank the whole term."""
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    lo, hi = row_ranges(plan.n, world)[rank]
    part = plan.term_rows(order, lo, hi) if hi > lo else np.zeros((plan.n, plan.n), np.complex128)
    return allreduce_sum(part, dist, group)


def sharded_npf(plan, orders, dist=None, group=None, out=None):
    """NPF of the given orders with the upper-index rows of every term split over the ranks of
    the group: each rank forms its rows of each Psi_N (npf_get_term_rows) into one stacked
    [orders, n, n] array, one sum over the ranks (FP64 complex: on the GPU with NCCL, on the host
    with gloo) gives every rank the whole terms, and the library finishes the NPF from them
    (npf_finish_terms, Algorithm 2 step 20). Without a group the rank forms every row."""
    import torch
    rank, world = (dist.get_rank(group), dist.get_world_size(group)) if dist else (0, 1)
    lo, hi = row_ranges(plan.n, world)[rank]
    dev = "cuda" if dist is None or dist.get_backend(group) == "nccl" else "cpu"
    stack = torch.zeros((len(orders), plan.n, plan.n), dtype=torch.complex128, device=dev)
    for t, N in enumerate(orders):
        if hi > lo:
            plan.term_rows(N, lo, hi, out=stack[t])
    if dist is not None and world > 1:
        dist.all_reduce(torch.view_as_real(stack), op=dist.ReduceOp.SUM, group=group)
    return plan.finish_terms(stack, out)


class Interrupted(RuntimeError):
    """Raised by checkpointed_term when asked to stop after a number of chunks (tests)."""


def checkpointed_term(plan, order, path, chunk_rows, stop_after=None):
    """Psi_N computed in row chunks of `chunk_rows`; after each chunk the running sum and the list
    of finished chunks are written to `path` (a .npz, replaced atomically), and a call that finds
    the file resumes after the last finished chunk. stop_after: raise Interrupted after that many
    chunks of this call (to test resumption)."""
    n = plan.n
    chunks = [(lo, min(n, lo + chunk_rows)) for lo in range(0, n, chunk_rows)]
    acc = np.zeros((n, n), np.complex128)
    done = np.zeros(len(chunks), bool)
    if os.path.exists(path):
        with np.load(path) as f:
            if (int(f["n"]), int(f["order"]), int(f["chunk_rows"])) != (n, order, chunk_rows):
                raise ValueError(f"{path} belongs to another computation")
            acc = f["acc"].copy()
            done = f["done"].copy()
    ran = 0
    for c, (lo, hi) in enumerate(chunks):
        if done[c]:
            continue
        if stop_after is not None and ran == stop_after:
            raise Interrupted(f"stopped after {ran} chunks")
        acc += plan.term_rows(order, lo, hi)
        done[c] = True
        ran += 1
        tmp = path + ".tmp.npz"
        np.savez(tmp, n=n, order=order, chunk_rows=chunk_rows, acc=acc, done=done)
        os.replace(tmp, path)
    return acc
