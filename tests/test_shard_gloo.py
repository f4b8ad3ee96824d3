"""Sharded PPP over two processes (gloo, CPU): each rank simulates its own
replicas of every window (disjoint uids from shard_uid_base) with the 1D
oracle, computes per-replica partials, and the ranks all-gather them with
gather_partials.  The merged estimates must equal the estimates of one
process holding every shard's samples."""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp

from oracle import _clib
from oracle import estimators as est
from paper_1105_4840_gb300 import inputs, shard

WORLD = 2
R_LOCAL = 3


def _workload():
    w = inputs.od1d_workload()
    run = w["run"]
    run.n_steps, run.n_equil, run.stride, run.replicas = 3000, 300, 10, R_LOCAL
    lam = np.linspace(-1.5, 1.5, 7)
    return w, run, lam


def _shard_samples(rank):
    w, run, lam = _workload()
    base = shard.shard_uid_base(rank, lam.size, R_LOCAL)
    out = []
    for wi, l in enumerate(lam):
        rows = [_clib.od1d_run(w["a"], l, run.k, run.kT, run.gamma, run.dt, run.n_steps, run.n_equil, run.stride,
                               run.seed, base + wi * R_LOCAL + r, w["x0"])[0] for r in range(R_LOCAL)]
        out.append(np.array(rows))
    return out


def _rank_main(rank, port, outdir):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        _, run, lam = _workload()
        local = est.window_partials(_shard_samples(rank), lam, run.k, run.kT)
        merged = shard.gather_partials(local)
        res = est.free_energy_from_partials(merged, lam, run.k, run.kT)
        np.savez(os.path.join(outdir, f"rank{rank}.npz"), merged=merged,
                 **{k: v for k, v in res.items()})
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_merge(tmp_path):
    import socket

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_rank_main, args=(port, str(tmp_path)), nprocs=WORLD, join=True, start_method="spawn")
    _, run, lam = _workload()
    every = [np.concatenate(parts, axis=0) for parts in zip(*[_shard_samples(r) for r in range(WORLD)])]
    want = est.free_energy_profile(every, lam, run.k, run.kT)
    got = [np.load(tmp_path / f"rank{r}.npz") for r in range(WORLD)]
    assert np.array_equal(got[0]["merged"], got[1]["merged"])  # every rank holds the same merge
    assert got[0]["merged"].shape == (lam.size, WORLD * R_LOCAL, 5)
    for key in ("dF_JE", "dF_fluct", "dF_G", "se_JE", "se_fluct", "mean_x", "var_x"):
        np.testing.assert_allclose(got[0][key], want[key], rtol=1e-10, atol=1e-12, err_msg=key)


def test_uid_blocks_are_disjoint():
    seen = set()
    for rank in range(4):
        b = shard.shard_uid_base(rank, 21, 32)
        block = set(range(b, b + 21 * 32))
        assert not (block & seen)
        seen |= block
    with pytest.raises(ValueError):
        shard.shard_uid_base(1, 2 ** 20, 2 ** 12)
