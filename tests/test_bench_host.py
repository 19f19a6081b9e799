"""Host-side logic of bench.py (no GPU): the roofline unit counts, the
replica seeds and timing reduction, and the launch-list summary."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_butterfly_and_mulmod_counts(bench):
    n = 1 << 16
    # column pass: stages 0..7, row pass: stages 8..15, N/2 butterflies each
    assert bench.butterflies_per_unit("ntt_fwd_cols", n) == 8 * n // 2
    assert bench.butterflies_per_unit("ntt_inv_rows", n) == 8 * n // 2
    assert bench.butterflies_per_unit("ntt_fwd_cols", 1 << 15) == 7 * (1 << 14)
    assert bench.butterflies_per_unit("ntt_fwd_rows", 1 << 15) == 8 * (1 << 14)
    assert bench.mulmods_per_unit("ntt_fwd_rows", n) == 4 * n
    assert bench.mulmods_per_unit("ntt_fwd_rows_ksr", n) == 4 * n + n
    assert bench.mulmods_per_unit("ntt_fwd_cols_ksr", n) == 4 * n


def test_multiplier_peak_from_measured_rates(bench):
    # 1 / (2/15.2 + 1/7.0) Shoup products and 1 / (1/15.2 + 1/7.0) 128-bit
    # multiply-adds per SM per clock
    assert abs(bench.MULMODS_PER_SM_CLK - 1.0 / (2 / 15.2 + 1 / 7.0)) < 1e-12
    assert abs(bench.MULMODS_PER_SM_CLK - 3.6438) < 1e-3
    assert abs(bench.MULMODS_PER_SM_CLK * 152 * 2070e6 / 1e9 - 1146.50) < 0.1
    assert abs(bench.MAC128_PER_SM_CLK - 4.7928) < 1e-3
    # the measured unit-of-work rates sit below the derived ones
    assert bench.BUTTERFLY_PER_SM_CLK < bench.MULMODS_PER_SM_CLK
    assert bench.MAC128_CHAIN_PER_SM_CLK < bench.MAC128_PER_SM_CLK


def test_bytes_per_unit(bench):
    n, limb = 1 << 16, 8 << 16
    assert bench.bytes_per_unit("ntt_fwd_rows", n, 3) == 2 * limb
    assert bench.bytes_per_unit("ntt_fwd_rows_ksr", n, 3) == 4 * limb
    assert bench.bytes_per_unit("k_tensor_pair", n, 3) == 7 * limb
    assert bench.bytes_per_unit("k_key_product", n, 3) == 11 * limb


def test_summarize_launch_list(bench, tmp_path, capsys):
    """Two steps in a synthetic ncu CSV: the summary covers exactly the
    second one (from its tensor kernel to the fused-tail NTT after k_ksr_cl)."""
    step = ["k_tensor_pair", "k_rows", "k_cols", "k_modup_bconv_h", "k_key_product_t", "k_ksr_last",
            "k_ksr_cl", "k_cols", "k_rows"]
    lines = ['"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"']
    i = 0
    for rep in range(2):
        for k in step:
            us = 10.0 * (rep + 1)
            lines.append('"%d","void <unnamed>::%s<1>(int)","gpu__time_duration.sum","us","%.1f"' % (i, k, us))
            i += 1
    p = tmp_path / "launches.csv"
    p.write_text("\n".join(lines) + "\n")
    bench.summarize_ncu(str(p), 2)
    out = capsys.readouterr().out
    assert "| (step) | 9 | 180.0 | 1.000 |" in out
    assert "| k_rows | 2 | 40.0 |" in out
    # occurrence 0: every launch of the list (a capture of one profiled region)
    bench.summarize_ncu(str(p), 0)
    out = capsys.readouterr().out
    assert "| (step) | 18 | 270.0 | 1.000 |" in out
    assert "| k_rows | 4 | 60.0 |" in out


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the oracle timed on the host's cores)
    prints one JSON line with the contract's keys for its metric and config."""
    import json
    import subprocess
    import sys

    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == "HMult+relin+rescale/s at N=2^16,L=20"
    assert d["value"] > 0 and d["unit"] == "ops/s" and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["config"] == bench_config_of_default()


def test_plain_guards_equal_the_oracle_networks(bench):
    """The benchmark's FP64 decryption guards compute the same networks as the
    oracle's plaintext CNNs (batch-packed and single-image deep)."""
    import numpy as np

    from oracle import cnn

    rng = np.random.default_rng(5)
    for (hh, k, stride, cout, act) in ((28, 5, 2, 5, (0.0, 0.0, 1.0)), (12, 3, 1, 3, (0.47, 0.50, 0.09)),
                                       (9, 3, 1, 2, (0.1, 0.2, 0.3))):
        x = rng.random((4, hh, hh))
        cw = rng.normal(0, 0.3, (cout, k, k, 1))
        ho = (hh - k) // stride + 1
        fw = rng.normal(0, 0.3, (10, (ho // 2) ** 2 * cout))
        got = bench.plain_batch_network(np, x, cw, stride, act, fw)
        want = cnn.network(x[..., None], cw, stride, act, fw)
        assert np.allclose(got, want, rtol=1e-12, atol=1e-12)
    img = rng.random((28, 28))
    cw = rng.normal(0, 0.3, (4, 3, 3))
    act = list(rng.normal(0, 1, 8))
    fw = rng.normal(0, 0.3, (10, 13 * 13 * 4))
    assert np.allclose(bench.plain_deep_network(np, img, cw, act, fw), cnn.deep_network(img, cw, act, fw),
                       rtol=1e-11, atol=1e-11)


def test_both_arms_report_one_config(bench):
    c = bench.bench_config(64, 1)
    assert (c["workload"], c["N"], c["L"], c["alpha"], c["dnum"], c["batch"]) == ("deep_n16_l20", 65536, 20, 7, 3, 64)
    assert c["parallelism"] == "single" and bench.bench_config(64, 2)["parallelism"] == "replicas"


def bench_config_of_default():
    spec = importlib.util.spec_from_file_location("bench_cfg", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.bench_config(64, 1)


def test_oracle_cnn_slice_extrapolates_the_batch(bench):
    """The labelled CPU-oracle slice of the N = 2^14 CNN times each piece and
    extrapolates to 720 conv outputs, 720 activations, 180 pools, 10 classes."""
    r = bench.OracleCnnSlice().run()
    t = r["seconds"]
    assert set(t) == {"conv_output", "activation", "pool_output", "fc_class"}
    want = 720 * t["conv_output"] + 720 * t["activation"] + 180 * t["pool_output"] + 10 * t["fc_class"]
    assert abs(r["extrapolated_batch_s"] - want) < 0.01 * want + 0.01
    assert r["unit"] == "images/s" and r["kind"] == "oracle" and abs(r["value"] - 8192 / r["extrapolated_batch_s"]) < 1e-6


def test_schoolbook_slice_counts_the_operation_products(bench):
    """The schoolbook-mode slice extrapolates to the tensor's 4 x 21 and the
    key product's 2 x 3 x 28 limb products and restores the oracle's mode."""
    from oracle import _lib
    assert bench.OracleSchoolbookSlice.PRODUCTS_PER_OP == 252
    mode = _lib.lib().or_get_mode()
    r = bench.OracleSchoolbookSlice().run(log_n=10)
    assert _lib.lib().or_get_mode() == mode
    assert r["kind"] == "oracle" and r["value"] > 0 and "N = 2^10" in r["sample"] and "252" in r["sample"]
