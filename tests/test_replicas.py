"""Host logic for several GPUs on CPU ranks (gloo, world size 2): the slice partition, the
maximum over ranks used for timings, and the wavelength-split gradient of Eq. 4 (one
all-reduce), checked against the full-wavelength FP64 oracle gradient."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2505_22313_b300.replicas import grad_split_wavelengths, max_over_ranks, shard


def test_shard_partitions_exactly():
    for n in range(0, 9):
        for world in range(1, 5):
            parts = [list(shard(n, r, world)) for r in range(world)]
            assert sum(parts, []) == list(range(n))
            sizes = [len(p) for p in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard(4, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import oracle
    from paper_2505_22313_b300 import inputs

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), OMP_NUM_THREADS="1")
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m = max_over_ranks(10.0 + rank)
        N, dx, z = 16, 1e-6, 2e-3
        P = 2 * N
        lams = [450e-9, 550e-9, 650e-9]
        h = inputs.heights(N, 31)
        T = np.random.default_rng(32).random((3, P, P)).astype(np.float32)

        def grad_fn(sub):
            idx = [lams.index(l) for l in sub]
            g, loss = oracle.grad(h, dx, z, sub, T[idx])
            return torch.from_numpy(g), torch.tensor(loss)

        g, loss = grad_split_wavelengths(lams, grad_fn, (N, N))
        np.save(os.path.join(out_dir, f"g{rank}.npy"), g.numpy())
        np.save(os.path.join(out_dir, f"m{rank}.npy"), np.array([m, loss.item()]))
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks_gradient_and_max(tmp_path):
    import oracle
    from paper_2505_22313_b300 import inputs

    oracle.build()  # compile once, before the ranks start
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    N, dx, z = 16, 1e-6, 2e-3
    P = 2 * N
    lams = [450e-9, 550e-9, 650e-9]
    h = inputs.heights(N, 31)
    T = np.random.default_rng(32).random((3, P, P)).astype(np.float32)
    full, loss = oracle.grad(h, dx, z, lams, T)
    for r in range(world):
        g = np.load(tmp_path / f"g{r}.npy")
        m, lr = np.load(tmp_path / f"m{r}.npy")
        assert m == 11.0  # max over ranks of 10 + rank
        assert np.abs(g - full).max() <= 1e-12 * np.abs(full).max()
        # the loss is an FP64 sum whose order depends on the OpenMP thread count (one per rank here)
        assert abs(lr - loss) <= 1e-8 * abs(loss)
