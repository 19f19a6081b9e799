"""One batched HMult + relin + rescale step at N = 2^16, L = 20 between
cudaProfilerStart and cudaProfilerStop (for ncu --profile-from-start off).
Usage: python paper_2102_00319_gb300/probes/one_step.py [batch]"""
import os, sys
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
import numpy as np, torch
from paper_2102_00319_gb300 import hecnn as H, workloads as W, build as B
B.build(); torch.cuda.set_device(0)
Bn = int(sys.argv[1]) if len(sys.argv) > 1 else 16
ps = W.DEEP_N16
params = H.hc_params_create(ps.log_n, list(ps.q_bits), list(ps.p_bits), ps.log2_scale)
ctx = H.hc_ctx_create(params, 0, torch.cuda.current_stream().cuda_stream)
n, L = ctx.n, ctx.L
sk, pk, evk = H.hc_keygen(ctx, 7)
A = [H.hc_encrypt(ctx, pk, H.hc_encode(ctx, W.slot_values(2 * i, n // 2), 2.0 ** ps.log2_scale, L), 17, 2 * i) for i in range(Bn)]
Bc = [H.hc_encrypt(ctx, pk, H.hc_encode(ctx, W.slot_values(2 * i + 1, n // 2), 2.0 ** ps.log2_scale, L), 17, 2 * i + 1) for i in range(Bn)]
for _ in range(2):
    out = H.hc_mul_relin_rescale_batch(ctx, evk, A, Bc)
H.hc_sync(ctx)
torch.cuda.profiler.start()
out = H.hc_mul_relin_rescale_batch(ctx, evk, A, Bc)
H.hc_sync(ctx)
torch.cuda.profiler.stop()
print("ok", len(out))
