"""Multi-rank (replicas) host logic on CPU: two gloo ranks each align a
cell-balanced shard of one batch (with the oracle, no GPU), the shards'
results are gathered and concatenated, and the result equals the unsharded
batch.  Also checks the max-over-ranks timing reduction the benchmark uses."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1805_00106_gb300 import replicas, synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _oracle(w):
    from oracle import oracle as O
    o = O.run_batch([O.encode(bytes(r)) for r in w["refs"]], w["bases"], w["read_off"], w["cand_off"],
                    w["c_ref"], w["c_strand"], w["c_start"], w["c_len"])
    # adapt the oracle's CIGAR rows to the flat CIGAR layout of the library
    flat, off = [], 0
    best = o["best"]
    cig_off = np.zeros(len(best), np.int64)
    for r in range(len(best)):
        n = int(best["cigar_len"][r])
        flat.append(o["cigar"][r][:n])
        cig_off[r] = off
        off += n
    import numpy.lib.recfunctions as rf
    best = rf.append_fields(best, "cigar_off", cig_off, usemask=False)
    return dict(best=best, best_per_ref=o["best_per_ref"], item_score=o["item_score"],
                item_end=o["item_end_j"], cigar=np.concatenate(flat) if flat else np.zeros(0, np.uint32))


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = synth.workload("c2", scale=0.0002, seed=5)
    b = replicas.shard_bounds(w["read_off"], w["cand_off"], w["c_len"], world)
    part = _oracle(replicas.take_shard(w, int(b[rank]), int(b[rank + 1])))
    parts = [None] * world
    dist.all_gather_object(parts, part)
    import torch
    t = torch.tensor([0.5 + rank], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        q.put((replicas.concat_results(parts), _oracle(w), float(t.item()), b.tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_concat():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    merged, full, tmax, bounds = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert tmax == 1.5
    assert bounds[0] == 0 and bounds[-1] == len(full["best"]) and bounds[0] < bounds[1] < bounds[2]
    for k in ["item_score", "item_end", "cigar"]:
        assert np.array_equal(merged[k], full[k]), k
    for f in ["score", "second", "n_ties", "item", "cigar_off", "cigar_len", "ref_end"]:
        assert np.array_equal(merged["best"][f], full["best"][f]), f
    assert np.array_equal(merged["best_per_ref"]["item"], full["best_per_ref"]["item"])


def test_shard_bounds_balance_cells():
    w = synth.workload("c2", scale=0.001, seed=9)
    b = replicas.shard_bounds(w["read_off"], w["cand_off"], w["c_len"], 4)
    m = np.diff(w["read_off"])
    cells = []
    for k in range(4):
        s = replicas.take_shard(w, int(b[k]), int(b[k + 1]))
        cells.append(int((np.repeat(np.diff(s["read_off"]), np.diff(s["cand_off"])) * s["c_len"]).sum()))
    assert max(cells) - min(cells) < 0.02 * sum(cells)
    assert sum(cells) == int((np.repeat(m, np.diff(w["cand_off"])) * w["c_len"]).sum())
