"""The benchmark's bookkeeping on the CPU: the algorithmic byte and product counts behind the
roofline figures, the derived integer-multiply peak, and the aggregate rate of replicas."""
import argparse

import pytest

import bench

N, L, K, DNUM = 1 << 15, 12, 3, 4          # the bench ring: 12 + 3 primes, digits of 3 primes


def test_layer_algorithmic_bytes():
    # 24 Galois keys of [4 digits][2][15 limbs][N] words, 64 inputs and 64 x 5 outputs of
    # [2][12][N] words, 8 bytes a word
    keys = 24 * 4 * 2 * 15 * N * 8
    ct = 2 * 12 * N * 8
    assert keys == 754_974_720 and ct == 6_291_456
    assert bench.layer_algorithmic_bytes(64, 5, 24) == keys + 64 * ct + 64 * 5 * ct == 3_170_893_824


def test_tap_kernel_products_and_roofline():
    # per image, limb of Q u P and coefficient: 2 dnum = 8 products for each of the 24 rotated
    # taps and 2 r = 4 for each of the 25 taps: 292
    args = argparse.Namespace(pack="dp_shift_ext")
    roof = bench.taps_roofline({"taps": (8.6513, 1)}, args, 64, 24)
    assert roof["products_per_launch"] == 64 * N * 15 * 292 == 9_185_525_760
    assert roof["launch_us"] == pytest.approx(8651.3)
    assert roof["achieved"] == pytest.approx(9_185_525_760 / 8.6513e-3 / 1e12)
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    assert "k_ks_mac_ext_bulk" in roof["kernel"]
    # the DRAM capture belongs to the carry-chain kernel at batch 64 only
    assert roof["traffic"] == pytest.approx(4.534172160e9)
    assert bench.taps_roofline({"taps": (1.0, 1)}, args, 64, 24, arith="columns")["traffic"] is None
    assert bench.taps_roofline({"taps": (1.0, 1)}, argparse.Namespace(pack="dp_shift"), 64, 24) is None


def test_integer_peak():
    # 152 SMs x 64 multiply-add slots per clock / 4 mad.wide.u32 per 64 x 64 -> 128-bit
    # product x 2070 MHz; the SM count follows the device
    assert bench.mul64_peak_per_s(2070.0) == pytest.approx(5.03424e12)
    assert bench.mul64_peak_per_s(2070.0, sms=76) == pytest.approx(5.03424e12 / 2)


def test_whole_job_rate_is_the_sum_over_replicas():
    # every rank does the same units; the time is the slowest rank's
    assert bench.whole_job_rate(64 * 24 * 100, 4, 1588.4) == pytest.approx(4 * 64 * 24 * 100 / 1.5884)


def test_workload_name_names_the_packing():
    assert "dp_shift_ext" in bench.workload_name(argparse.Namespace(pack="dp_shift_ext"))
    assert "N=2^15" in bench.workload_name(argparse.Namespace(pack="dp_dot"))


def test_sweep_point_bytes_and_bound():
    # B input and B output ciphertexts of [2][L][N] words, the reused outputs of one batched
    # hoisted call (P ciphertexts x h), min(max(B, h), 64) keys of [dnum][2][L + K][N] words,
    # the rotation scratch
    n, L, K, B, h = 1 << 16, 24, 6, 1024, 24
    ct = 2 * L * n * 8
    key = 16 * 4 * (L + K) * n
    scratch = 64 * (L + 4 * (L + K) + 2 * (L + K) + 2 * L) * n * 8
    P = (16 << 30) // (h * ct)                     # 28 ciphertexts' outputs fit 16 GiB
    assert P == 28 and bench.sweep_hoist_batch(16, L, h) == P
    assert bench.sweep_point_bytes(16, L, K, B, h) == 2 * B * ct + P * h * ct + 64 * key + scratch
    # the batch stays within 8 .. 64 ciphertexts and below B
    assert bench.sweep_hoist_batch(13, 3, 8) == 64
    assert bench.sweep_point_bytes(13, 3, 1, 1, 8) == (2 * 2 * 3 * 8192 * 8 + 8 * 2 * 3 * 8192 * 8
                                                       + 8 * 16 * 3 * 4 * 8192
                                                       + (3 + 3 * 4 + 2 * 4 + 6) * 8192 * 8)
    # every point of the grid fits the 150 GB bound (none is skipped)
    for log_n in bench.SWEEP_LOG_N:
        for L, K in bench.SWEEP_L.items():
            for B in bench.SWEEP_B:
                assert bench.sweep_point_bytes(log_n, L, K, B, max(bench.SWEEP_H)) <= bench.SWEEP_MEM_LIMIT


def test_reference_step_runs_the_oracle_layer(monkeypatch):
    """One reference step is one image's DP_SHIFT_EXT layer by the oracle (a small ring here)."""
    monkeypatch.setattr(bench, "LOG_N", 11)          # 28 x 28 = 784 slots fit a row of N/2
    monkeypatch.setattr(bench, "N_Q", 3)
    monkeypatch.setattr(bench, "N_P", 1)
    monkeypatch.setattr(bench, "ALPHA", 1)
    monkeypatch.setattr(bench, "_ORACLE", {})
    dt, n_rot = bench.oracle_layer_step(3)
    assert dt > 0 and n_rot == 24
    assert bench._ORACLE["lay"].pack == "dp_shift_ext"


def test_bench_line_contract_is_checked():
    """The main line carries clocks as an object (sm_mhz, sm_max_mhz, reasons) and e2e as one;
    a line whose clocks became a bare number is refused before it is printed."""
    line = {"metric": "m", "value": 1.0, "unit": "u", "n_gpus": 1, "steps": 2, "warmup": 3,
            "ms_per_step": 1.0, "higher_is_better": True, "dtype": "u64", "config": {},
            "e2e": {"value": 1.0}, "gpu_launches": 4,
            "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}}
    assert bench.check_line(line) is line
    with pytest.raises(ValueError):
        bench.check_line(dict(line, clocks=2.07e9))
    with pytest.raises(ValueError):
        bench.check_line({k: v for k, v in line.items() if k != "e2e"})
