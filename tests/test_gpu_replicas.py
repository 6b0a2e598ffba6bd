"""Replicas through libsr in two processes (-m gpu): two gloo ranks, each with its
own session on the one GPU of this machine (ranks never wait on each other's
kernels), align their cell-balanced shards of one batch; rank 0 gathers and
concatenates the shards, and the result equals the whole batch aligned in one
call, byte for byte."""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

KEYS = ["bases", "read_off", "cand_off", "c_ref", "c_strand", "c_start", "c_len"]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _align(sr, w):
    s = sr.Session.open([bytes(r) for r in w["refs"]])
    g = s.align(*[w[k] for k in KEYS], sr.score_params(), sr.align_opts())
    out = {k: np.array(g[k]) for k in ["best", "best_per_ref", "item_score", "item_end", "cigar"]}
    s.close()
    return out


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    from paper_1805_00106_gb300 import replicas, sr, synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    w = synth.workload("c2", scale=0.003, seed=17, rc_frac=0.5)
    b = replicas.shard_bounds(w["read_off"], w["cand_off"], w["c_len"], world)
    part = _align(sr, replicas.take_shard(w, int(b[rank]), int(b[rank + 1])))
    parts = [None] * world
    dist.all_gather_object(parts, part)
    if rank == 0:
        q.put((replicas.concat_results(parts), _align(sr, w), b.tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_processes_replicas_equal_one_call():
    import torch.multiprocessing as mp
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    merged, full, bounds = q.get(timeout=600)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert bounds[0] == 0 < bounds[1] < bounds[2] == len(full["best"])
    for k in ["item_score", "item_end", "cigar"]:
        assert np.array_equal(merged[k], full[k]), k
    for f in full["best"].dtype.names:
        assert np.array_equal(merged["best"][f], full["best"][f]), f
        assert np.array_equal(merged["best_per_ref"][f], full["best_per_ref"][f]), f
