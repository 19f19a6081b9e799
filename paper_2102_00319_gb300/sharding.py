"""Output-channel sharding of the batch-packed CNN, one GPU per rank.

The batch-packed network's channels are independent until the fully
connected layer: the response of each filter, its activation and its
pooling need no other filter (Sec. "Parallelization using
multi-threading", which runs filters on separate threads).  Each rank
holds every input ciphertext and the weights of its own channels, runs
conv -> activation -> pool for those channels and the FC layer's sums of
tensor products over its channels' activations (degree 2, before
relinearisation: hc_enc_fc_partial).

The one exchange is an all-gather of those partial ciphertexts' residue
words.  A collective sum would add words modulo 2^64, not modulo each
prime, so the collective only carries the words and the modular addition
runs in the library's own kernel (hc_add); every rank then relinearises and
rescales each class once.  Since the partial sums are exact residues, the
result has the words of hc_enc_fc over all inputs.

This module holds the partition logic and the exchange; all homomorphic
arithmetic goes through the library (`hecnn`).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def shard_channels(cout: int, world: int) -> list:
    """Contiguous blocks of output channels, sizes differing by at most one
    (the first cout % world ranks take one more).  Every rank needs a
    channel: world > cout is rejected."""
    if cout < 1 or world < 1 or world > cout:
        raise ValueError("need 1 <= world <= cout (cout=%d, world=%d)" % (cout, world))
    base, extra = divmod(cout, world)
    out, c0 = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append(list(range(c0, c0 + n)))
        c0 += n
    return out


@dataclass
class ShardPlan:
    """Index maps of one rank's share of a batch-packed CNN.

    Shapes follow the layer calls: inputs x[(h W + w) Cin + ci], conv
    weights w[((co kh + p) kw + q) Cin + ci], conv outputs and activations
    channel-last [(m Wo + n) C + c], pooled activations [(i Wp + j) C + c]
    (the FC's flattened input k), FC weights fc_w[r n_in + k]."""
    H: int
    W: int
    cin: int
    cout: int
    kh: int
    kw: int
    stride: int
    n_out: int
    world: int

    @property
    def Ho(self) -> int:
        return (self.H - self.kh) // self.stride + 1

    @property
    def Wo(self) -> int:
        return (self.W - self.kw) // self.stride + 1

    @property
    def Hp(self) -> int:
        return self.Ho // 2

    @property
    def Wp(self) -> int:
        return self.Wo // 2

    @property
    def n_in(self) -> int:
        return self.Hp * self.Wp * self.cout

    def channels(self, rank: int) -> list:
        return shard_channels(self.cout, self.world)[rank]

    def conv_weight_indices(self, rank: int) -> list:
        """Indices into the full conv weight list for this rank's channels, in
        the order a conv call over just those channels expects."""
        per = self.kh * self.kw * self.cin
        return [co * per + t for co in self.channels(rank) for t in range(per)]

    def fc_inputs(self, rank: int) -> list:
        """Flattened FC input indices k of this rank's pooled activations, in
        the order a pool call over just its channels returns them."""
        ch = self.channels(rank)
        return [(i * self.Wp + j) * self.cout + c for i in range(self.Hp) for j in range(self.Wp) for c in ch]

    def fc_weight_indices(self, rank: int) -> list:
        """FC weights of this rank's inputs, class-major: [r * len(k) + t]."""
        ks = self.fc_inputs(rank)
        return [r * self.n_in + k for r in range(self.n_out) for k in ks]


def allgather_words(arrays, group=None, device=None) -> list:
    """All-gather of equally shaped uint64 arrays (one list per rank, the same
    shapes on every rank) through torch.distributed; returns, per rank, its
    list of arrays.  The words travel as int64 bit patterns: no arithmetic
    happens in the collective.  `device`: where the collective's tensors
    live (a CUDA device for NCCL, None for gloo on the host)."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    flat = np.concatenate([np.ascontiguousarray(a, dtype=np.uint64).reshape(-1) for a in arrays])
    mine = torch.from_numpy(flat.view(np.int64).copy())
    if device is not None:
        mine = mine.to(device)
    bufs = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(bufs, mine, group=group)
    out = []
    for b in bufs:
        words = b.cpu().numpy().view(np.uint64)
        parts, o = [], 0
        for a in arrays:
            parts.append(words[o:o + a.size].reshape(a.shape).copy())
            o += a.size
        out.append(parts)
    return out


def sum_partials(parts_by_rank, add):
    """Per class, the partial ciphertexts of all ranks folded with `add`
    (the library's modular addition), ranks in order."""
    n_out = len(parts_by_rank[0])
    out = []
    for r in range(n_out):
        acc = parts_by_rank[0][r]
        for parts in parts_by_rank[1:]:
            acc = add(acc, parts[r])
        out.append(acc)
    return out


def rank_partials(H, ctx, evk, plan: ShardPlan, rank: int, xs, conv_w, fc_w, act):
    """This rank's conv -> activation -> pool for its channels and the FC's
    degree-2 partial sums over them (all through the library).  Returns the
    n_out partial ciphertexts."""
    ch = plan.channels(rank)
    w_mine = [conv_w[i] for i in plan.conv_weight_indices(rank)]
    y = H.hc_enc_conv2d(ctx, evk, H.HC_PACK_BATCH, xs, plan.H, plan.W, plan.cin, w_mine, len(ch), plan.kh, plan.kw,
                        plan.stride)
    a = H.hc_enc_poly_act(ctx, evk, y, act)
    del y
    p = H.hc_enc_pool(ctx, evk, H.HC_PACK_BATCH, a, len(ch), plan.Ho, plan.Wo)
    del a
    fw_mine = [fc_w[i] for i in plan.fc_weight_indices(rank)]
    return H.hc_enc_fc_partial(ctx, H.HC_PACK_BATCH, p, fw_mine, plan.n_out)


def exchange_partials(H, ctx, mine, group=None, device=None) -> list:
    """All ranks' partial ciphertexts, per rank in rank order: this rank's
    own handles and the others' imported from the gathered words.  All
    partials share level, degree and scale (the same circuit on every
    rank)."""
    import torch.distributed as dist

    exported = [H.hc_ct_export(ctx, c) for c in mine]
    gathered = allgather_words([e[0] for e in exported], group=group, device=device)
    meta = exported[0][1]
    me = dist.get_rank(group)
    return [mine if r == me else [H.hc_ct_import(ctx, w, meta.level, meta.degree, meta.scale) for w in words]
            for r, words in enumerate(gathered)]


def combine(H, ctx, evk, parts_by_rank):
    """The modular sum of every rank's partials (hc_add, ranks in order),
    then one batched relinearisation + rescale of the classes (the tail of
    hc_enc_fc)."""
    total = sum_partials(parts_by_rank, lambda a, b: H.hc_add(ctx, a, b))
    return H.hc_relin_rescale_batch(ctx, evk, total)


def sharded_cnn(H, ctx, evk, plan: ShardPlan, rank: int, xs, conv_w, fc_w, act, group=None, device=None):
    """The sharded forward pass on one rank: its partials, the exchange, the
    modular sum and the per-class relinearisation and rescale.  Every rank
    returns the n_out logits ciphertexts."""
    mine = rank_partials(H, ctx, evk, plan, rank, xs, conv_w, fc_w, act)
    parts = [mine] if plan.world == 1 else exchange_partials(H, ctx, mine, group=group, device=device)
    return combine(H, ctx, evk, parts)
