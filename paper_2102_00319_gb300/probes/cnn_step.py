"""One batched forward pass of the batch-packed CNN at N = 2^14 (8192
synthetic 28x28 images: conv 5x5 stride 2 x5 -> x^2 -> 2x2 mean pool -> FC
180 -> 10) between cudaProfilerStart and cudaProfilerStop (for ncu
--profile-from-start off).  Usage: python paper_2102_00319_gb300/probes/cnn_step.py"""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
import numpy as np  # noqa: E402
import torch  # noqa: E402

from paper_2102_00319_gb300 import build as B  # noqa: E402
from paper_2102_00319_gb300 import hecnn as H  # noqa: E402
from paper_2102_00319_gb300 import workloads as W  # noqa: E402

B.build()
torch.cuda.set_device(0)
ps, c = W.BATCH_N14, W.CNN_BATCH
params = H.hc_params_create(ps.log_n, list(ps.q_bits), list(ps.p_bits), ps.log2_scale)
ctx = H.hc_ctx_create(params, 0, torch.cuda.current_stream().cuda_stream)
K, seed, scale = ctx.n // 2, W.MASTER_SEED + 2, 2.0 ** ps.log2_scale
sk, pk, evk = H.hc_keygen(ctx, seed)
imgs = W.images(seed + 20, K, c["H"], c["W"])
cw = W.conv_weights(seed + 21, c["cout"], c["k"], c["k"])
Ho = (c["H"] - c["k"]) // c["stride"] + 1
n_in = (Ho // 2) ** 2 * c["cout"]
fw = W.fc_weights(seed + 22, c["n_out"], n_in)


def const_ct(v, nonce):
    m = np.zeros(ctx.n, dtype=np.int64)
    m[0] = int(np.round(v * scale))
    return H.hc_encrypt(ctx, pk, H.hc_pt_from_coeffs(ctx, m, ctx.L, scale), seed + 5, nonce)


xs = [H.hc_encrypt(ctx, pk, H.hc_encode(ctx, imgs[:, h, w], scale, ctx.L), seed + 5, h * c["W"] + w)
      for h in range(c["H"]) for w in range(c["W"])]
ws = [const_ct(cw[co, a, b, 0], 1000 + (co * c["k"] + a) * c["k"] + b)
      for co in range(c["cout"]) for a in range(c["k"]) for b in range(c["k"])]
fws = [const_ct(fw[r, i], 2000 + r * n_in + i) for r in range(c["n_out"]) for i in range(n_in)]


def forward():
    y = H.hc_enc_conv2d(ctx, evk, H.HC_PACK_BATCH, xs, c["H"], c["W"], 1, ws, c["cout"], c["k"], c["k"], c["stride"])
    a = H.hc_enc_poly_act(ctx, evk, y, c["act"])
    p = H.hc_enc_pool(ctx, evk, H.HC_PACK_BATCH, a, c["cout"], Ho, Ho)
    return H.hc_enc_fc(ctx, evk, H.HC_PACK_BATCH, p, fws, c["n_out"])


forward()
H.hc_sync(ctx)
torch.cuda.profiler.start()
out = forward()
H.hc_sync(ctx)
torch.cuda.profiler.stop()
print("ok", len(out))
