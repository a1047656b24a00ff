"""Host-side logic of bench.py, on the CPU: the term counts it divides by, the stratified FP64
sample of the serving mix, the per-request serving policy, and the host CPU record.

The term counts are checked against brute-force enumeration of the Lemma's index sets (Sec. 2.3):
C2 = #{(k, l) in I_N^2 x I_N^2 : k + l = n in I_N} summed over n, and C3 the same for triples; the
closed forms (3N^2/4)^d and (2(N^3 - N)/3)^d are what the bench's throughput and roofline use.
"""
from __future__ import annotations

import itertools
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402
from paper_2110_13735_gb300 import inputs as I  # noqa: E402


def _brute_counts(d, N):
    h = N // 2
    idx = range(-h, h)
    # the index conditions act per dimension, so the counts are the 1-D counts to the power d
    one2 = sum(1 for k, l in itertools.product(idx, idx) if -h <= k + l < h)
    one3 = sum(1 for k, l, m in itertools.product(idx, idx, idx) if -h <= k + l + m < h)
    return one2 ** d, one3 ** d


@pytest.mark.parametrize("d,N", [(2, 4), (2, 8), (2, 16), (3, 4), (3, 6)])
def test_lemma_term_counts(d, N):
    c2, c3 = _brute_counts(d, N)
    assert bench.lemma_terms(d, N, False) == pytest.approx(c2)
    assert bench.lemma_terms(d, N, True) == pytest.approx(c2 + c3)


def test_lemma_terms_of_an_output_box():
    """The central box of outputs: enumerate the pairs and triples whose sum lands in it (2-D)."""
    N, lo, cnt = 8, -2, 3
    h = N // 2
    idx = range(-h, h)
    box = set(range(lo, lo + cnt))
    one2 = sum(1 for k, l in itertools.product(idx, idx) if k + l in box)
    one3 = sum(1 for k, l, m in itertools.product(idx, idx, idx) if k + l + m in box)
    assert bench.lemma_terms_box(N, lo, cnt, False) == pytest.approx(one2 ** 2)
    assert bench.lemma_terms_box(N, lo, cnt, True) == pytest.approx(one2 ** 2 + one3 ** 2)


def test_stratified_fp64_sample():
    reqs = I.serving_requests(n=512, rate=200.0, Ns=(16, 32, 64), kernels=(0, 1))
    per_n = {16: 6, 32: 5, 64: 2}
    sample = bench.serving_fp64_sample(reqs, per_n)
    assert len(sample) == len(set(sample)) == 13
    for N, k in per_n.items():
        mine = [reqs[i] for i in sample if reqs[i]["N"] == N]
        assert len(mine) == k
        quantum = sorted((r for r in reqs if r["N"] == N and r["eps"] != 0.0),
                         key=lambda r: (abs(r["eps"]) * r["fmax"], r["id"]))
        q = [r for r in mine if r["eps"] != 0.0]
        # the least and the most saturated quantum request of that N are always in the sample
        assert quantum[0]["id"] in [r["id"] for r in q] and quantum[-1]["id"] in [r["id"] for r in q]
        # one classical request when the sample has room for it
        assert sum(r["eps"] == 0.0 for r in mine) == (1 if k >= 3 else 0)


def test_request_options_policy():
    pol = {"beta_split_N": [16], "escalate_at_by_N": {32: 0.5}}
    base = dict(N=16, eps=1.0)
    assert bench.request_options(base, pol) == {"beta_split": 1}
    assert bench.request_options(dict(base, N=32), pol) == {"escalate_at": 0.5}
    assert bench.request_options(dict(base, N=64), pol) == {}
    assert bench.request_options(dict(base, N=64), {}) == {}


def test_whole_job_rate_and_single_rank_max():
    assert bench.whole_job_rate(10.0, 2.0, 4) == pytest.approx(20.0)
    assert bench.reduce_max_over_ranks(3.5, 1) == 3.5


def test_host_cpu_record():
    info = bench.host_cpu()
    assert set(info) >= {"model", "architecture", "cpus"}
    assert info["cpus"] is None or int(info["cpus"]) >= 1
    assert np.isfinite(bench.lemma_terms(2, 32, True))
