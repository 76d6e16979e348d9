"""The work model bench.py reports fractions with, against hand counts at
logN=16, 30 limbs, K=10, alpha=10 (HMult+relin reads 120 ciphertext limbs and
240 key limbs and writes 60; its key switch is 200 transforms of 2^19
butterflies, 1500 N conversion multiply-adds and 470 N other products), and
the kernel launch model against the launch sequence of one single-op step."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

N = 1 << 16


def test_op_work_matches_the_published_figures():
    w = bench.op_work(30, 10, 10, N)
    # HMult+relin: (120 ciphertext + 240 key + 60 output) limbs = 220.2 MB;
    # 104.9 M butterflies + 98.3 M conversion MACs + 30.8 M other = 234 M
    assert w["hmult"][0] == 420 * 8 * N
    assert w["hmult"][1] == 200 * 32768 * 16 + 1500 * N + 470 * N
    # HRotate: 360 limbs = 188.7 MB, about 226 M
    assert w["rotate"][0] == 360 * 8 * N
    assert w["rotate"][1] == 200 * 32768 * 16 + 1500 * N + 350 * N
    # Rescale 30 -> 29: 118 limbs = 61.9 MB; 60 transforms + 58 products
    assert w["rescale"][0] == 118 * 8 * N
    assert w["rescale"][1] == 60 * 32768 * 16 + 58 * N
    assert round(w["hmult"][0] / 1e6, 1) == 220.2 and round(w["hmult"][1] / 1e6) == 234
    assert round(w["rotate"][0] / 1e6, 1) == 188.7 and round(w["rotate"][1] / 1e6) == 226
    assert round(w["rescale"][0] / 1e6, 1) == 61.9


def test_op_work_at_a_ragged_level():
    # 17 limbs: digits of 10 and 7, beta = 2, 27 extended limbs
    w = bench.op_work(17, 10, 10, N)
    assert w["hmult"][0] == (4 * 17 + 2 * 2 * 27 + 2 * 17) * 8 * N
    conv = 10 * (27 - 10) + 7 * (27 - 7) + 2 * 10 * 17
    other = 17 + 2 * 2 * 27 + 2 * 10 + 2 * 17
    assert w["rotate"][1] == 4 * 27 * 32768 * 16 + conv * N + other * N


@pytest.mark.parametrize("nl", [30, 21, 5])
def test_launch_model_counts_one_step(nl):
    model = bench.launch_model(nl, 10, 10, N)
    count = {}
    for name, _, _ in model:
        count[name] = count.get(name, 0) + 1
    # HMult 12, Rescale 4, HRotate 11 launches
    assert sum(count.values()) == 27
    assert count["k_tensor"] == 1 and count["k_inner"] == 2 and count["k_bconv_tc"] == 4
    for k in ("k_ntt_fwd_cols", "k_ntt_fwd_rows", "k_ntt_inv_rows", "k_ntt_inv_cols"):
        assert count[k] == 5


def test_bconv_tc_flops():
    # per key switch: 3 ModUp jobs (10 sources, 30 targets) + 2 ModDown jobs
    # (10 sources, 30 targets), each 2 N (8 targets) (8 * 12) flops
    per_job = 2 * N * 8 * 30 * 8 * 12
    assert bench.bconv_tc_flops(30, 10, 10, N) == 2 * 5 * per_job
