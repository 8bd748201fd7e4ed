"""The multi-GPU path of bench.py, run as world_size-2 gloo ranks on CPU.

The filter partitions by reads with no exchange step: every rank gets the
same reference and its own read batch (weak scaling), and the job's time is
the slowest rank's.  This checks those host-side rules without a GPU."""
import hashlib
import os
import socket
import types

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import oracle
        args = types.SimpleNamespace(ref_bp=2_000_000, reads=400)
        w = bench.make_workload("gather", args, rank)
        o = oracle.Oracle()
        ob = o.build_bank(w.ref2bit, w.ref_len, w.q, w.bin_len, w.overlap)
        p, _ = o.filter(ob, w.q, w.bases, w.read_offsets, w.cand_bins, w.cand_offsets, w.E)
        slowest = bench.max_over_ranks(float(rank + 1) * 1.5, world)
        out.put((rank, hashlib.sha1(w.ref2bit.tobytes()).hexdigest(), hashlib.sha1(w.bases.tobytes()).hexdigest(),
                 w.n_checks, int(p.sum()), slowest))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_reads_not_reference():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = sorted(q.get(timeout=300) for _ in range(world))
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    (r0, ref0, reads0, n0, p0, t0), (r1, ref1, reads1, n1, p1, t1) = res
    assert ref0 == ref1                  # one reference on every rank
    assert reads0 != reads1              # each rank its own read batch
    assert n0 > 0 and n1 > 0 and p0 > 0 and p1 > 0
    assert t0 == t1 == 3.0               # job time = the slowest rank's
