#!/usr/bin/env python
"""Benchmark of the CKKS ciphertext-by-ciphertext hot path on GB300.

Metric: HMult + relin + rescale per second at N = 2^16, L = 20 (q_0 60 bits,
twenty 50-bit primes, seven 60-bit special primes, dnum = 3).  One step is
one batch of B independent (tensor product, hybrid key switch, rescale)
operations -- every kernel of the multiplication path -- over ciphertext
pairs already resident in HBM (B pairs occupy far more than the 129 MB L2,
so no flush is needed between steps).

The JSON line also carries:
  e2e           the same metric through the C ABI from pinned HOST buffers
                (coefficient-form import, NTT, compute, INTT, export),
  roofline      the dominant kernel's algorithmic bytes / its device time
                (CUDA events around every launch on the context stream),
  cpu_baseline  the CPU oracle on this host (bounded sample, rank 0, N=1),
  clocks        nvidia-smi samples taken during the timed region.

--impl reference times the CPU oracle itself (the paper publishes no code
for this path; the plain oracle is the reference arm).
Multi-GPU: replicas only (independent batches per rank, no collective on
the data path); value = all ranks' operations / max rank time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "HMult+relin+rescale/s at N=2^16,L=20"
UNIT = "ops/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--batch", type=int, default=32, help="ciphertext pairs per step")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-ops", type=int, default=1, help="oracle operations in the CPU sample")
    ap.add_argument("--summarize-ncu", metavar="CSV",
                    help="summarise an ncu launch list (gpu__time_duration.sum) of the timed step and exit")
    ap.add_argument("--step-occurrence", type=int, default=2,
                    help="which occurrence of the step's first kernel starts the timed step (warm-up = 1)")
    return ap.parse_args()


def summarize_ncu(path, occurrence):
    """Per-kernel launches, total time and share over one timed step of an ncu
    launch list: the step starts at the given occurrence of k_tensor_acc and
    ends before the next step's first kernel or the end of the step's kernels."""
    import csv
    import re

    rows = [r for r in csv.DictReader(l for l in open(path) if l.startswith('"'))
            if r.get("Metric Name") == "gpu__time_duration.sum"]
    names = [re.sub(r"^.*?::", "", r["Kernel Name"]).split("(")[0].split("<")[0] for r in rows]
    starts = [i for i, n in enumerate(names) if n == "k_tensor_acc"]
    a = starts[occurrence - 1]
    b = starts[occurrence] if occurrence < len(starts) else len(rows)
    # the step ends at its last rescale combine
    ends = [i for i in range(a, b) if names[i] == "k_rescale_combine"]
    b = ends[-1] + 1
    per = {}
    for i in range(a, b):
        t = float(rows[i]["Metric Value"]) * (1e-3 if rows[i]["Metric Unit"] == "ns" else 1.0)
        c, tot = per.get(names[i], (0, 0.0))
        per[names[i]] = (c + 1, tot + t)
    total = sum(v[1] for v in per.values())
    print("| kernel | launches | total us | share |")
    print("|---|---|---|---|")
    for k, (c, t) in sorted(per.items(), key=lambda kv: -kv[1][1]):
        print("| %s | %d | %.1f | %.3f |" % (k, c, t, t / total))
    print("| (step) | %d | %.1f | 1.000 |" % (b - a, total))


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi sampling (SM clock, throttle reasons) during the timed region."""

    def __init__(self, index):
        self.proc = None
        self.index = index
        self.path = os.path.join(ROOT, "gpurun_out", "bench_clocks_%d.csv" % os.getpid())

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.remove(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle: one HMult + relin + rescale at the same parameters
# ---------------------------------------------------------------------------
class OracleBench:
    """The CPU oracle at the benchmark's parameters: keys and two ciphertexts
    are made once (untimed); run(k) times k HMult+relin+rescale."""

    def __init__(self, seed=0x2102_0031_9004):
        import numpy as np

        from oracle import ckks
        from paper_2102_00319_gb300 import workloads as W

        self.ckks = ckks
        ps = W.DEEP_N16
        self.op = op = ckks.Params(ps.log_n, list(ps.q_bits), list(ps.p_bits), ps.log2_scale)
        self.sk, self.pk, self.evk = ckks.keygen(op, seed)
        # slot-constant plaintexts (constant polynomials) keep the untimed setup cheap
        self.cts = []
        for i in range(2):
            m = np.zeros(op.N, dtype=np.int64)
            m[0] = ckks.llround(float(W.slot_values(seed + i, 1)[0]) * op.scale)
            self.cts.append(ckks.encrypt(op, self.pk, ckks.plaintext_from_ints(op, m, op.L, op.scale), seed + 7, i))
        self.threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))

    def run(self, n_ops):
        c, op = self.ckks, self.op
        t0 = time.perf_counter()
        for _ in range(n_ops):
            c.rescale(op, c.relin(op, self.evk, c.mul(op, self.cts[0], self.cts[1])))
        return time.perf_counter() - t0

    def sample(self, n_ops):
        return ("%d oracle HMult+relin+rescale (tensor, hybrid key switch dnum=3, rescale) at N=2^16, L=20, "
                "textbook-NTT product mode, OpenMP over limbs" % n_ops)


def run_reference(args, rank, world):
    if rank != 0:
        return
    ob = OracleBench()
    ob.run(args.warmup)
    total = ob.run(args.steps)
    value = args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "deep_n16_l20", "N": 65536, "L": 20, "dnum": 3, "batch": 1},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": ob.threads, "kind": "oracle",
                         "sample": "each step: " + ob.sample(1)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
# Algorithmic HBM bytes per work unit (one N-word limb of the launch's output
# domain), per kernel; dnum = 3 at the top level of this workload.
def bytes_per_unit(name, n, dnum):
    limb = 8 * n
    if name.startswith("ntt_"):
        return 2 * limb                       # read + write the limb
    if name == "k_key_product":
        return (3 * dnum + 2) * limb          # dnum raised limbs + 2 dnum key limbs in, 2 out
    if name == "k_tensor_acc":
        return 7 * limb                       # 4 operand limbs in, 3 out (one term per output here)
    if name in ("k_moddown_combine",):
        return 4 * limb                       # acc, converted limb, base in; out
    if name in ("k_rescale_combine",):
        return 3 * limb
    return 2 * limb


def run_gpu(args, rank, world, local):
    import numpy as np
    import torch

    from paper_2102_00319_gb300 import build as B
    from paper_2102_00319_gb300 import hecnn as H
    from paper_2102_00319_gb300 import workloads as W

    B.build()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()
    ps = W.DEEP_N16
    params = H.hc_params_create(ps.log_n, list(ps.q_bits), list(ps.p_bits), ps.log2_scale)
    ctx = H.hc_ctx_create(params, local, stream.cuda_stream)
    n, L, alpha, dnum = ctx.n, ctx.L, ctx.alpha, ctx.dnum
    seed = W.MASTER_SEED + 4 + 1000 * rank
    sk, pk, evk = H.hc_keygen(ctx, seed)
    Bn = args.batch
    A, Bc = [], []
    for i in range(Bn):
        for lst, off in ((A, 0), (Bc, 1)):
            pt = H.hc_encode(ctx, W.slot_values(seed + 2 * i + off, n // 2), 2.0 ** ps.log2_scale, L)
            lst.append(H.hc_encrypt(ctx, pk, pt, seed + 17, 2 * i + off))
    H.hc_sync(ctx)

    def step():
        return H.hc_mul_relin_rescale_batch(ctx, evk, A, Bc)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    outs = None
    for _ in range(args.warmup):
        outs = step()
    # correctness guard on the timed configuration: decrypt one product
    got = H.hc_decode(ctx, H.hc_decrypt(ctx, sk, outs[0]))
    za, zb = W.slot_values(seed, n // 2), W.slot_values(seed + 1, n // 2)
    err = float(np.max(np.abs(got - za * zb)))
    assert err < 2.0 ** -15, "batched result decrypts wrong (max error %g)" % err
    outs = None
    barrier()
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    H.hc_profile_enable(ctx, True)
    launches0 = H.hc_kernel_launches(ctx)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        outs = step()
        outs = None
    e1.record(stream)
    barrier()
    launches = H.hc_kernel_launches(ctx) - launches0
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    kernels = {}
    for name in H.hc_profile_names(ctx):
        cnt, tot, units = H.hc_profile_kernel(ctx, name)
        kernels[name] = (cnt, tot, units)
    H.hc_profile_enable(ctx, False)
    t_local = ms / 1000.0
    if world > 1:
        t = torch.tensor([t_local], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_max = float(t.item())
    else:
        t_max = t_local
    value = Bn * args.steps * world / t_max

    # ---------------- e2e through the C ABI from pinned host memory
    host_in = []
    for c in A + Bc:
        data, meta = H.hc_ct_export(ctx, c)
        pin = torch.empty(data.size, dtype=torch.int64, pin_memory=True)
        arr = pin.numpy().view(np.uint64).reshape(data.shape)
        arr[...] = data
        host_in.append((pin, arr, meta))
    out_words = 2 * L * n
    host_out = [torch.empty(out_words, dtype=torch.int64, pin_memory=True) for _ in range(Bn)]
    h2d = sum(a.nbytes for _, a, _ in host_in)
    d2h = Bn * out_words * 8

    def e2e_step():
        ins = [H.hc_ct_import(ctx, a, m.level, m.degree, m.scale) for _, a, m in host_in]
        res = H.hc_mul_relin_rescale_batch(ctx, evk, ins[:Bn], ins[Bn:])
        for r, buf in zip(res, host_out):
            arr = buf.numpy().view(np.uint64).reshape(2, L, n)
            H.load().hc_ct_export(ctx.ptr, r.ptr, arr.ctypes.data_as(H.ctypes.POINTER(H.ctypes.c_uint64)),
                                  arr.size, None)
        return res

    e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        e2e_step()
    barrier()
    t_e2e = max(time.perf_counter() - t0, 1e-9)
    if world > 1:
        t = torch.tensor([t_e2e], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_e2e = float(t.item())
    e2e_value = Bn * args.e2e_steps * world / t_e2e if args.e2e_steps > 0 else None

    if rank != 0:
        return
    # ---------------- roofline of the dominant kernel
    dom = max(kernels, key=lambda k: kernels[k][1])
    cnt, tot, units = kernels[dom]
    alg_bytes = units * bytes_per_unit(dom, n, dnum)
    achieved = alg_bytes / (tot / 1000.0) / 1e9
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = peaks.get("hbm_gbs", 6800.0)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None,
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                "bytes_per_launch": alg_bytes / max(cnt, 1), "avg_launch_us": 1000.0 * tot / max(cnt, 1),
                "share_of_step": tot / ms}
    kern_summary = {k: {"launches": v[0], "ms": round(v[1], 3), "share": round(v[1] / ms, 4)}
                    for k, v in sorted(kernels.items(), key=lambda kv: -kv[1][1])}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "deep_n16_l20", "N": n, "L": L, "alpha": alpha, "dnum": dnum, "batch": Bn,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (%.2f GB of resident ciphertexts)" % (2 * Bn * 2 * (L + 1) * n * 8 / 1e9)},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches, "roofline": roofline, "clocks": clk, "kernels": kern_summary,
        "check": {"max_slot_error": err},
    }
    if world == 1 and not args.no_cpu_baseline:
        ob = OracleBench()
        dt = ob.run(args.cpu_ops)
        line["cpu_baseline"] = {"value": args.cpu_ops / dt, "unit": UNIT, "cores": ob.threads, "kind": "oracle",
                                "sample": ob.sample(args.cpu_ops)}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.summarize_ncu:
        summarize_ncu(args.summarize_ncu, args.step_occurrence)
        return
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_gpu(args, rank, world, local)


if __name__ == "__main__":
    main()
