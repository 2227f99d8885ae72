"""The multi-process path on CPU: two gloo ranks shard probes and frozen-phonon
configurations and gather the result, which must equal one process doing it all.

The per-rank computation here is the FP64 oracle (CPU); on GPUs the same
helpers drive libstem with NCCL.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1706_08563_b300.parallel import config_shards, shard_range


def test_shard_range_partitions():
    for n in (0, 1, 7, 64, 65):
        for world in (1, 2, 3, 8):
            blocks = [shard_range(n, r, world) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == n
            assert all(b[1] == c[0] for b, c in zip(blocks, blocks[1:]))
            sizes = [b - a for a, b in blocks]
            assert max(sizes) - min(sizes) <= 1
    assert config_shards(8, 1, 3) == [1, 4, 7]
    with pytest.raises(ValueError):
        shard_range(4, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    import workloads as W
    from oracle import stem as O
    w = W.Workload("g", (10.0, 10.0, 4.0), 12, 32, 2, 2.0, 200.0, 25.0, 3, 4.0, 20, fp_configs=3, fp_sigma=0.08)
    p = O.params_from(w)
    xyz, gauss = W.atoms(w, seed=3)
    xy = W.random_positions(w, 7, seed=4)
    return w, p, xyz, gauss, xy


def _worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import workloads as W
        from oracle import stem as O
        from paper_1706_08563_b300.parallel import sharded_configs, sharded_probes
        w, p, xyz, gauss, xy = _case()
        t = O.transmission(p, O.projected_potential(p, xyz, gauss))
        probes = sharded_probes(len(xy), lambda a, b: torch.from_numpy(O.multislice_rings(p, t, xy[a:b])))

        def one_config(c):
            xc = W.displaced(w, xyz, c)
            tc = O.transmission(p, O.projected_potential(p, xc, gauss))
            return torch.from_numpy(O.multislice_rings(p, tc, xy))
        configs = sharded_configs(w.fp_configs, one_config, like=torch.zeros((len(xy), w.n_rings), dtype=torch.float64))
        if rank == 0:
            np.savez(out_path, probes=probes.numpy(), configs=configs.numpy())
    finally:
        dist.destroy_process_group()


def _prism_case():
    import workloads as W
    from oracle import stem as O
    w = W.Workload("gp", (10.0, 12.0, 4.0), 14, 32, 2, 2.0, 200.0, 30.0, 3, 4.0, 20, f=(2,))
    p = O.params_from(w)
    xyz, gauss = W.atoms(w, seed=8)
    xy = W.random_positions(w, 7, seed=9)
    return w, p, xyz, gauss, xy


def _prism_worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import stem as O
        from paper_1706_08563_b300.parallel import sharded_prism
        w, p, xyz, gauss, xy = _prism_case()
        t = O.transmission(p, O.projected_potential(p, xyz, gauss))
        beams = O.prism_beams(p, 2)
        smat = torch.zeros((len(beams), p.n, p.n, 2), dtype=torch.float64)
        built = []

        def build(b0, b1):
            built.append((b0, b1))
            s = O.prism_smatrix(p, t, beams[b0:b1])
            smat[b0:b1] = torch.from_numpy(np.stack([s.real, s.imag], axis=-1))

        def output(a, b):
            s = smat[..., 0].numpy() + 1j * smat[..., 1].numpy()
            return torch.from_numpy(O.prism_rings(p, s, beams, 2, xy[a:b]))
        rings = sharded_prism(len(beams), len(xy), build, [smat], output)
        assert built[0][1] - built[0][0] < len(beams)          # each rank built only part of the beams
        if rank == 0:
            np.savez(out_path, rings=rings.numpy(), smat=smat.numpy())
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_prism_split_match_one_process(repo_tmp):
    """PRISM split over two ranks: beams sharded for the S-matrix and summed
    into every rank's copy, then probes sharded for the output step; the rings
    and the assembled S-matrix equal one process doing it all."""
    from oracle import stem as O
    out = os.path.join(repo_tmp, "p.npz")
    mp.spawn(_prism_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    got = np.load(out)
    w, p, xyz, gauss, xy = _prism_case()
    t = O.transmission(p, O.projected_potential(p, xyz, gauss))
    beams = O.prism_beams(p, 2)
    s = O.prism_smatrix(p, t, beams)
    assert np.array_equal(got["smat"][..., 0] + 1j * got["smat"][..., 1], s)
    assert np.allclose(got["rings"], O.prism_rings(p, s, beams, 2, xy), rtol=0, atol=1e-15)


def test_two_gloo_ranks_match_one_process(repo_tmp):
    import workloads as W
    from oracle import stem as O
    out = os.path.join(repo_tmp, "r.npz")
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    got = np.load(out)
    w, p, xyz, gauss, xy = _case()
    t = O.transmission(p, O.projected_potential(p, xyz, gauss))
    assert np.allclose(got["probes"], O.multislice_rings(p, t, xy), rtol=0, atol=1e-14)
    ref = O.frozen_phonon_rings(p, [W.displaced(w, xyz, c) for c in range(w.fp_configs)], gauss, xy)
    assert np.allclose(got["configs"], ref, rtol=1e-12, atol=1e-15)
