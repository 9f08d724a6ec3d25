"""Shot sharding across ranks, on CPU with the gloo backend (world size 2):
the static partition is balanced and complete, and the sharded misfit and
gradient (here computed per shard by the oracle) equal the single-process
result on every rank."""
import os
import socket

import numpy as np
import pytest

from paper_2502_12350_gb300 import sharding, synth

torch = pytest.importorskip("torch")


def test_partition_balanced_and_complete():
    rng = np.random.default_rng(0)
    costs = rng.uniform(1, 10, 37)
    for world in (1, 2, 3, 8):
        parts = sharding.partition(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(37))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= costs.max() + 1e-9
    assert sharding.partition([5, 5], 4) == [[0], [1], [], []]


def test_subset_rebases_receivers():
    src = np.arange(9, dtype=np.float32).reshape(3, 3)
    off = np.array([0, 2, 5, 6])
    rec = np.arange(18, dtype=np.float32).reshape(6, 3)
    s, o, r, ap, rows = sharding.subset([0, 2], src, off, rec)
    np.testing.assert_array_equal(s, src[[0, 2]])
    np.testing.assert_array_equal(o, [0, 2, 3])
    np.testing.assert_array_equal(rows, [0, 1, 5])
    np.testing.assert_array_equal(r, rec[[0, 1, 5]])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    return synth.small_case(seed=71, nx=10, ny=9, nz=8, border=4, nt=30, density=True, n_src=5,
                            n_rec=4, fpeak=35.0)


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    from oracle import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = _case()
    og = oracle.make_grid(w.nx, w.ny, w.nz, w.border, w.h, w.dt, w.nt)
    dobs = np.zeros((int(w.rec_offset[-1]), w.nt))

    def compute(idx):
        if not idx:
            return 0.0, torch.zeros(w.vel.shape, dtype=torch.float64)
        src, off, rec, ap, rows = sharding.subset(idx, w.src_xyz, w.rec_offset, w.rec_xyz)
        J, g = oracle.gradient(og, w.vel, src, w.wavelet, off, rec, dobs[rows], rho=w.rho)
        return J, torch.from_numpy(g)

    costs = sharding.shot_costs(w.nx, w.ny, w.nz, w.border, w.n_src)
    J, g = sharding.sharded_gradient(compute, costs)
    np.save(os.path.join(out_dir, f"g{rank}.npy"), g.numpy())
    np.save(os.path.join(out_dir, f"J{rank}.npy"), np.array([J]))
    dist.destroy_process_group()


def test_sharded_gradient_equals_single_process(oracle, tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    w = _case()
    og = oracle.make_grid(w.nx, w.ny, w.nz, w.border, w.h, w.dt, w.nt)
    Jr, gr = oracle.gradient(og, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz,
                             np.zeros((int(w.rec_offset[-1]), w.nt)), rho=w.rho)
    g0, g1 = np.load(tmp_path / "g0.npy"), np.load(tmp_path / "g1.npy")
    np.testing.assert_array_equal(g0, g1)  # identical on every rank
    np.testing.assert_allclose(g0, gr, rtol=1e-12, atol=1e-12 * np.abs(gr).max())
    J0 = float(np.load(tmp_path / "J0.npy")[0])
    assert J0 == float(np.load(tmp_path / "J1.npy")[0])
    assert abs(J0 - Jr) <= 1e-12 * Jr
