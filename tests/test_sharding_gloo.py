"""Output-channel sharding of the batch-packed CNN (paper_2102_00319_gb300.
sharding): the partition logic, and two gloo ranks on the CPU that each run
their channels' share of the network, exchange the partial FC ciphertexts'
words through the module's all-gather and sum them modulo each prime; the
result equals the single-process network word for word.

The CPU ranks compute with the oracle (no GPU here); the product module
supplies only the index maps and the exchange, which is what this checks.
The same maps drive the GPU path (tests/test_gpu_sharding.py)."""
import os

import numpy as np
import pytest

from paper_2102_00319_gb300 import sharding as S


def test_shard_channels_partition():
    for cout in range(1, 9):
        for world in range(1, cout + 1):
            sh = S.shard_channels(cout, world)
            assert len(sh) == world
            assert sum(sh, []) == list(range(cout))  # contiguous, in order, each once
            sizes = [len(s) for s in sh]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
    with pytest.raises(ValueError):
        S.shard_channels(3, 4)
    with pytest.raises(ValueError):
        S.shard_channels(0, 1)


def test_plan_index_maps_partition_the_network():
    plan = S.ShardPlan(H=28, W=28, cin=1, cout=5, kh=5, kw=5, stride=2, n_out=10, world=2)
    assert (plan.Ho, plan.Wo, plan.Hp, plan.Wp, plan.n_in) == (12, 12, 6, 6, 180)
    ks = [plan.fc_inputs(r) for r in range(2)]
    assert sorted(ks[0] + ks[1]) == list(range(180))
    ws = [plan.conv_weight_indices(r) for r in range(2)]
    assert sorted(ws[0] + ws[1]) == list(range(5 * 25))
    fws = [plan.fc_weight_indices(r) for r in range(2)]
    assert sorted(fws[0] + fws[1]) == list(range(10 * 180))
    # channel-last flatten: input k of rank 1 belongs to one of its channels
    assert all(k % 5 in plan.channels(1) for k in ks[1])
    # class-major weight order: class r's weights of rank 0 are a contiguous run
    n0 = len(ks[0])
    assert fws[0][3 * n0:4 * n0] == [3 * 180 + k for k in ks[0]]


# --------------------------------------------------------------- two ranks
SHAPE = dict(H=6, W=6, cin=1, cout=3, kh=3, kw=3, stride=1, n_out=3)
PARAMS = (8, [60, 40, 40, 40, 40], [60], 40)
SEED = 91


def _inputs(ckks, op, pk):
    from paper_2102_00319_gb300 import workloads as W

    c = SHAPE
    n_in = ((c["H"] - c["kh"]) // c["stride"] + 1) // 2
    n_in = n_in * n_in * c["cout"]

    def enc(mseed, nonce):
        m = W.int_plaintext(mseed, op.N, 2 ** 30)
        return ckks.encrypt(op, pk, ckks.plaintext_from_ints(op, m, op.L, op.scale), SEED + 1, nonce)

    xs = [enc(100 + i, i) for i in range(c["H"] * c["W"])]
    ws = [enc(300 + i, 1000 + i) for i in range(c["cout"] * c["kh"] * c["kw"])]
    fws = [enc(500 + i, 2000 + i) for i in range(c["n_out"] * n_in)]
    return xs, ws, fws


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist

    from oracle import ckks, cnn

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        op = ckks.Params(*PARAMS)
        sk, pk, evk = ckks.keygen(op, SEED)
        xs, ws, fws = _inputs(ckks, op, pk)
        c = SHAPE
        plan = S.ShardPlan(world=world, **c)
        ch = plan.channels(rank)
        # this rank's share, with the oracle standing in for the library
        y = cnn.enc_conv2d_batch(op, evk, xs, c["H"], c["W"], 1, [ws[i] for i in plan.conv_weight_indices(rank)],
                                 len(ch), c["kh"], c["kw"], c["stride"])
        a = [cnn.enc_square(op, evk, t) for t in y]
        p = cnn.enc_pool_batch(op, a, len(ch), plan.Ho, plan.Wo)
        mine_w = [fws[i] for i in plan.fc_weight_indices(rank)]
        n_mine = len(p)
        partials = [ckks.tensor_sum(op, p, [ckks.drop_to_level(op, w, p[0].level)
                                            for w in mine_w[r * n_mine:(r + 1) * n_mine]])
                    for r in range(c["n_out"])]
        gathered = S.allgather_words([t.c for t in partials])
        assert len(gathered) == world
        assert all(np.array_equal(g, t.c) for g, t in zip(gathered[rank], partials))
        lv, sc = partials[0].level, partials[0].scale
        parts = [[ckks.Ciphertext(w, lv, sc) for w in words] for words in gathered]
        total = S.sum_partials(parts, lambda u, v: ckks.add(op, u, v))
        logits = [ckks.rescale(op, ckks.relin(op, evk, t)) for t in total]
        if rank == 0:
            np.save(out_path, np.stack([t.c for t in logits]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_match_the_single_process_network(tmp_path):
    import multiprocessing as mp
    import socket

    from oracle import ckks, cnn

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = str(tmp_path / "logits.npy")
    ctxm = mp.get_context("spawn")
    procs = [ctxm.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = np.load(out)
    # the whole network in one process
    op = ckks.Params(*PARAMS)
    sk, pk, evk = ckks.keygen(op, SEED)
    xs, ws, fws = _inputs(ckks, op, pk)
    c = SHAPE
    y = cnn.enc_conv2d_batch(op, evk, xs, c["H"], c["W"], 1, ws, c["cout"], c["kh"], c["kw"], c["stride"])
    a = [cnn.enc_square(op, evk, t) for t in y]
    Ho = (c["H"] - c["kh"]) // c["stride"] + 1
    p = cnn.enc_pool_batch(op, a, c["cout"], Ho, Ho)
    want = cnn.enc_fc(op, evk, p, fws, c["n_out"])
    assert got.shape == np.stack([t.c for t in want]).shape
    assert np.array_equal(got, np.stack([t.c for t in want]))
