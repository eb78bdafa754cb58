"""The multi-rank path on CPU: two gloo ranks survey their pivot ranges and sum
their tables with one all_reduce; the sum equals the single-process survey.
(The per-rank survey here is the oracle's pivot-range survey; on GPUs it is
tripoll_survey_range.)"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth
from paper_2107_12330_b300.shard import sharded_survey

KEYS = ("count", "hist", "vtri", "etri")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _graph():
    return synth.rmat_graph(11, 16, 6, ts_bits=18, num_vlabels=3, num_elabels=3)


def _worker(rank, world, port, bounds, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = _graph()

    def survey_range(lo, hi, out):
        r = oracle.survey_graph(g, pivot_range=(lo, hi), extras=())
        vec = np.concatenate([r[k] for k in KEYS]).astype(np.int64)
        out.copy_(torch.from_numpy(vec))

    words = 1 + 33 + 27 + 27
    out = torch.zeros(words, dtype=torch.int64)
    sharded_survey(survey_range, bounds, rank, out, dist.all_reduce)
    if rank == 0:
        q.put(out.numpy().copy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_sum_to_the_full_survey():
    g = _graph()
    full = oracle.survey_graph(g, extras=())
    want = np.concatenate([full[k] for k in KEYS]).astype(np.int64)
    bounds = [0, 1300, g.n]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, bounds, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert np.array_equal(got, want)
    assert want[0] > 0
