"""Row sharding of one fit across ranks (Algorithm 4's F = sum_s U_s^T X_s),
host logic on CPU: two gloo ranks, each computing its partial with the oracle.

* the row blocks tile [0, m) exactly;
* the gathered, rank-ordered FP64 sum equals the unsharded F and G to
  rounding, and is bit-identical on both ranks;
* the k x k step on the reduced F gives the unsharded fit's subspace;
* the timing reduction is the maximum over ranks.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1709_07175_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


@pytest.mark.parametrize("m,world", [(10, 1), (10, 3), (7, 7), (2000, 2), (5, 8)])
def test_row_range_tiles_rows(m, world):
    covered = []
    sizes = []
    for r in range(world):
        lo, hi = shard.row_range(m, world, r)
        covered += list(range(lo, hi))
        sizes.append(hi - lo)
    assert covered == list(range(m))
    assert max(sizes) - min(sizes) <= 1


def test_ordered_sum_is_fixed_order():
    a = torch.tensor([1e16], dtype=torch.float64)
    b = torch.tensor([1.0], dtype=torch.float64)
    c = torch.tensor([-1e16], dtype=torch.float64)
    # (a + b) + c = 0 in FP64 while a + (b + c) = 0 as well, but (a + c) + b = 1:
    assert shard.ordered_sum([a, b, c]).item() == 0.0
    assert shard.ordered_sum([a, c, b]).item() == 1.0


def _worker(rank, world, port, outdir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import lspca as O
        from oracle import philox as P
        from paper_1709_07175_gb300 import synthetic as S

        w = S.WORKLOADS["fp64_small"]
        X = S.generate(w).numpy()
        Om = P.omega_gaussian(w.omega_seed, w.n, w.k)
        lo, hi = shard.row_range(w.m, world, rank)
        U = O.sketch(X[lo:hi], Om)
        Fg = torch.from_numpy(O.chain(U, X[lo:hi]))
        Gg = torch.from_numpy(O.gram(U))
        F, G = shard.reduce_partials(Fg, Gg)
        t = shard.max_over_ranks(float(rank + 1))
        np.save(os.path.join(outdir, f"F{rank}.npy"), F.numpy())
        np.save(os.path.join(outdir, f"G{rank}.npy"), G.numpy())
        np.save(os.path.join(outdir, f"t{rank}.npy"), np.array([t]))
    finally:
        dist.destroy_process_group()


def test_two_rank_reduction_matches_unsharded(tmp_path):
    from oracle import lspca as O
    from oracle import metrics as M
    from oracle import philox as P
    from paper_1709_07175_gb300 import synthetic as S

    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    F0, F1 = (np.load(tmp_path / f"F{r}.npy") for r in range(world))
    G0, G1 = (np.load(tmp_path / f"G{r}.npy") for r in range(world))
    assert np.array_equal(F0, F1) and np.array_equal(G0, G1)  # bit-identical on every rank
    assert all(np.load(tmp_path / f"t{r}.npy")[0] == world for r in range(world))

    w = S.WORKLOADS["fp64_small"]
    X = S.generate(w).numpy()
    Om = P.omega_gaussian(w.omega_seed, w.n, w.k)
    U = O.sketch(X, Om)
    F = O.chain(U, X)
    G = O.gram(U)
    assert np.linalg.norm(F0 - F) <= 1e-13 * np.linalg.norm(F)
    assert np.linalg.norm(G0 - G) <= 1e-13 * np.linalg.norm(G)
    # the replicated k x k step on the reduced F: the unsharded fit's subspace
    Vs, sig_s, _ = O.decompose_eig(F0, w.m, w.n)
    ref = O.lspca_fit(X, Om, route="eig")
    assert M.max_sine(ref["V"], Vs) < 1e-10
    assert np.max(np.abs(sig_s - ref["sigma"]) / ref["sigma"]) < 1e-12


def test_reduce_partials_without_group_is_identity():
    F = torch.randn(3, 5, dtype=torch.float64)
    G = torch.randn(3, 3, dtype=torch.float64)
    F2, G2 = shard.reduce_partials(F, G)
    assert F2 is F and G2 is G
    assert shard.max_over_ranks(2.5) == 2.5
