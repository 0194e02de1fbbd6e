"""Replica runs on CPU: shard plan, host map merge, and a world-size-2 gloo run.

Each gloo rank runs the oracle on its contiguous shard of the c1 records
(the GPU path needs a GPU; the exchange under test is host code), exports
its map with shard-local record indices, and rank 0 merges the gathered maps
through the library's as_map_merge. The result must equal the oracle's map
of one run over all records: global record indices, summed counts.
"""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp

import synth
import paper_2606_15650_b300.api as api
from paper_2606_15650_b300 import replicas
from oracle import pipeline as P
from oracle.encoder import Encoder
from oracle.tokenizer import build_vocab_index
from oracle.pseudonym import merge_maps

DIMS = synth.C1.dims
N_REC = 24


def _tuples(entries):
    return [(e.type, e.original, e.full_hash, e.slug, e.first_seen, e.last_seen, e.count) for e in entries]


def _oracle_run(recs, base=0):
    w = synth.make_weights(DIMS, seed=31, random_affine=True)
    vocab = build_vocab_index(synth.make_vocab())
    sch = P.Schema(synth.TYPE_NAMES_4)
    return P.anonymize(recs, sch, synth.make_key(), Encoder(DIMS, w), vocab, record_base=base, keep_traces=False)


def _records():
    rs = synth.make_records(synth.scaled(synth.C1, N_REC).records, synth.make_vocab(), seed=synth.SEED_RECORDS)
    return rs.records()


def test_shard_ranges_cover_and_balance():
    rng = np.random.default_rng(7)
    sizes = rng.integers(1, 5000, 1000)
    for world in (1, 2, 3, 8):
        rr = replicas.shard_ranges(sizes, world)
        assert rr[0][0] == 0 and rr[-1][1] == len(sizes)
        assert all(a[1] == b[0] for a, b in zip(rr, rr[1:]))
        loads = [int(sizes[a:b].sum()) for a, b in rr]
        assert max(loads) - min(loads) <= 2 * int(sizes.max())
    assert replicas.shard_ranges(np.array([5, 5]), 4)[-1] == (2, 2)


def test_map_merge_matches_oracle_merge():
    recs = _records()
    cut = 10
    a, b = _oracle_run(recs[:cut]), _oracle_run(recs[cut:])
    got = api.map_merge([[api.Entity(*_tuples([e])[0]) for e in a.map], [api.Entity(*_tuples([e])[0]) for e in b.map]],
                        [0, cut])
    whole = _oracle_run(recs)
    assert _tuples(got) == _tuples(whole.map)
    shifted = [P.MapEntry(e.type, e.original, e.full_hash, e.slug, e.first_seen + cut, e.last_seen + cut, e.count)
               for e in b.map]
    assert _tuples(got) == _tuples(merge_maps([a.map, shifted]))


def test_map_merge_rejects_key_mismatch_and_empty():
    e1 = api.Entity(0, b"10.0.0.1", "a" * 64, "a" * 10, 0, 0, 1)
    e2 = api.Entity(0, b"10.0.0.1", "b" * 64, "b" * 10, 3, 3, 1)
    with pytest.raises(api.AnonShieldError):
        api.map_merge([[e1], [e2]])
    assert api.map_merge([[], []]) == []
    assert api.map_merge([]) == []


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        recs = _records()
        a, b = replicas.shard_ranges(np.array([len(r) for r in recs]), world)[rank]
        res = _oracle_run(recs[a:b])
        merged = replicas.gather_merge([api.Entity(*t) for t in _tuples(res.map)], a)
        if rank == 0:
            q.put(_tuples(merged))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks_merge_equals_single_run():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 2000
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=300)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    assert got == _tuples(_oracle_run(_records()).map)
