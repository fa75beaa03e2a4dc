"""CPU emulation of the row-sharded design of the randomized SVD (one rank per
GPU, each owning a block of rows of A), on gloo ranks in FP64.

Every box of this build has one GPU, so the library runs replicas and this
mode exists as a design only.  The design follows from the structure of
Algorithm rqb with subspace iterations: Omega is regenerated on every rank
from its counter-based generator (no exchange), Y = A Omega and Y = A Q_n are
row-local, and only three exchanges are needed, each a sum over the ranks:

  (i)   the l x l Gram Y^T Y of each CholeskyQR step (the m-side QR),
  (ii)  the n x l products A^T Q of the power iterations,
  (iii) the l x n factor B = Q^T A.

The n-side QR, the SVD of B and the truncation are then computed redundantly
on every rank, and U = Q Ut stays row-local.  These tests run that exchange
pattern with torch.distributed all-reduces on gloo ranks and require the
gathered result to equal the unsharded oracle (any orthonormal basis of the
same span gives the same U, Sigma, V in exact arithmetic), on uneven row
splits; a rank that leaves before an exchange must make the others fail
with an error instead of hanging.
"""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rows(m, world, rank):
    return m * rank // world, m * (rank + 1) // world


def _sharded_rsvd(A_i, n, k, p, q, seed, allreduce, fail_before=None):
    """The rank-local part of the sharded method (FP64 numpy); allreduce sums
    a numpy array over the ranks.  Returns (d, U_i, V)."""
    import oracle

    l = min(k + p, n)
    Om = oracle.omega(n, l, seed).astype(np.float64)  # replicated, regenerated per rank
    calls = [0]

    def exchange(x):
        calls[0] += 1
        if fail_before is not None and calls[0] == fail_before:
            os._exit(3)  # an injected failure: the rank leaves before this exchange
        return allreduce(x)

    def cholqr(Y_i):  # CholeskyQR2 of the row-distributed Y, exchange (i) twice
        Q_i = Y_i
        for _ in range(2):
            G = exchange(Q_i.T @ Q_i)
            R = np.linalg.cholesky(G).T
            Q_i = np.linalg.solve(R.T, Q_i.T).T
        return Q_i

    Y_i = A_i @ Om
    for _ in range(q):
        Q_i = cholqr(Y_i)
        Z = exchange(A_i.T @ Q_i)  # exchange (ii)
        Qn, _ = np.linalg.qr(Z)    # n-side QR, redundant on every rank
        Y_i = A_i @ Qn
    Q_i = cholqr(Y_i)
    B = exchange(Q_i.T @ A_i)      # exchange (iii)
    Ut, d, Vt = np.linalg.svd(B, full_matrices=False)
    return d[:k], Q_i @ Ut[:, :k], Vt[:k].T


def _worker(rank, world, port, m, n, k, p, q, seed, out, fail_before):
    import datetime

    import torch
    import torch.distributed as dist

    from paper_1608_02148_gb300 import inputs
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=20))
    try:
        A = inputs.planted(m, n, inputs.exp_spectrum(n, 0.08), seed=seed, dtype=np.float64)
        r0, r1 = _rows(m, world, rank)

        def allreduce(x):
            t = torch.from_numpy(np.ascontiguousarray(x))
            dist.all_reduce(t)
            return t.numpy()

        fb = fail_before if rank == world - 1 else None
        d, U_i, V = _sharded_rsvd(A[r0:r1], n, k, p, q, 7, allreduce, fb)
        out.put((rank, "ok", d, U_i, V))
    except Exception as exc:
        out.put((rank, "error: " + type(exc).__name__, None, None, None))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def _run(world, m, n, k, p, q, seed, fail_before=None, expect=None):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, m, n, k, p, q, seed, out, fail_before))
             for r in range(world)]
    for pr in procs:
        pr.start()
    got = {}
    try:
        for _ in range(expect if expect is not None else world):
            rank, status, d, U_i, V = out.get(timeout=180)
            got[rank] = (status, d, U_i, V)
    finally:
        for pr in procs:
            pr.join(60)
            if pr.is_alive():
                pr.kill()
                pr.join(10)
    return got, procs


@pytest.mark.parametrize("world,m,n,k,p,q", [(2, 301, 80, 10, 6, 2), (3, 250, 120, 15, 5, 1)])
def test_row_sharded_rsvd_equals_the_unsharded_oracle(world, m, n, k, p, q):
    import oracle
    from paper_1608_02148_gb300 import inputs
    from tests.helpers import sin_theta

    seed = 40 + world
    got, procs = _run(world, m, n, k, p, q, seed)
    assert all(pr.exitcode == 0 for pr in procs)
    assert sorted(got) == list(range(world)) and all(g[0] == "ok" for g in got.values())
    A = inputs.planted(m, n, inputs.exp_spectrum(n, 0.08), seed=seed, dtype=np.float64)
    d_o, U_o, V_o = oracle.rsvd(A, k, p=p, q=q, seed=7)
    U = np.vstack([got[r][2] for r in range(world)])
    for r in range(world):  # the replicated parts agree across ranks
        np.testing.assert_allclose(got[r][1], got[0][1], rtol=1e-13)
    np.testing.assert_allclose(got[0][1], d_o, rtol=1e-10)
    assert U.shape == (m, k)
    assert sin_theta(U, U_o) < 1e-8
    assert sin_theta(got[0][3], V_o) < 1e-8
    np.testing.assert_allclose(U.T @ U, np.eye(k), atol=1e-12)


def test_a_rank_that_leaves_before_an_exchange_fails_the_others():
    """The last rank exits before the third exchange (the second Gram of the
    first CholeskyQR2 counts as the second); the remaining rank's all-reduce
    ends with an error within the process group's timeout."""
    got, procs = _run(2, 200, 60, 8, 4, 1, 5, fail_before=3, expect=1)
    assert procs[1].exitcode == 3
    assert got[0][0].startswith("error"), got[0][0]
