"""Host-side plan of the mixed 2-D operator kernel (include/bn.h: bn_plan_mixed2d), on the CPU.

The plan is what every solver with the mixed N <= 32 kernel uploads: per work item b of the
factorised Lemma sum (Sec. 3.3 step 2(c)) its boxes, the warp split of its sweep and its place in
the CTA order.  Checked here against what the factorisation fixes: the items are exactly the b with
non-empty boxes, their terms add up to the closed-form count C3 = (2(N^3 - N)/3)^2, every (task,
s_u row) of every item is covered exactly once by the split, and the CTA layout balances the work
better than dealing the items round-robin."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2110_13735_gb300 import bn

COL = {c: i for i, c in enumerate(bn.PLAN_COLUMNS)}


def boxes(N, b):
    """(L, S) of one dimension: outputs n with n, n - b in I_N; inner s with s, b - s in I_N."""
    h = N // 2
    nlo, nhi = max(-h, b - h), min(h - 1, b + h - 1)
    slo, shi = max(-h, b - h + 1), min(h - 1, b + h)
    return nhi - nlo + 1, shi - slo + 1


def expected_items(N):
    E = 2 * N
    out = {}
    for b1 in range(-N, N):
        for b2 in range(-N, N):
            (L1, S1), (L2, S2) = boxes(N, b1), boxes(N, b2)
            if min(L1, S1, L2, S2) > 0:
                out[(b1 + N) * E + (b2 + N)] = (L1, L2, S1, S2)
    return out


@pytest.fixture(scope="module")
def lib():
    try:
        return bn.load()
    except RuntimeError as e:
        pytest.skip(str(e))


@pytest.mark.parametrize("N", [2, 4, 8, 16, 24, 32])
@pytest.mark.parametrize("rw", [8, 16])
@pytest.mark.parametrize("oriented", [False, True])
def test_items_boxes_and_term_count(lib, N, rw, oriented):
    plan = bn.plan_mixed2d(N, rw, oriented, 456)
    exp = expected_items(N)
    ib = plan[:, COL["ib"]]
    assert sorted(ib.tolist()) == sorted(exp)          # every b with non-empty boxes, once
    terms = 0
    for row in plan:
        L1, L2, S1, S2 = exp[int(row[COL["ib"]])]
        o = int(row[COL["orient"]])
        assert o in (0, 1) and (oriented or o == 0)
        Lu, Lw, Su, Sw = (L1, L2, S1, S2) if o == 0 else (L2, L1, S2, S1)
        assert (row[COL["Lu"]], row[COL["Lw"]], row[COL["Su"]], row[COL["Sw"]]) == (Lu, Lw, Su, Sw)
        assert row[COL["base"]] == Lu * (-(-Lw // rw))
        terms += Lu * Lw * Su * Sw
    assert terms == round((2 * (N ** 3 - N) / 3) ** 2)   # C3 of the Lemma's triple sum


@pytest.mark.parametrize("N", [4, 16, 32])
@pytest.mark.parametrize("rw", [8, 16])
def test_split_covers_every_task_and_row_once(lib, N, rw):
    warps = 8
    for row in bn.plan_mixed2d(N, rw, True, 456):
        J, chunk, units = int(row[COL["J"]]), int(row[COL["chunk"]]), int(row[COL["units"]])
        J2, chunk2, units2, tail0 = (int(row[COL[c]]) for c in ("J2", "chunk2", "units2", "tail0"))
        base, Su = int(row[COL["base"]]), int(row[COL["Su"]])
        assert J in (1, 2, 4, 8) and chunk == -(-Su // J)
        cover = np.zeros((base, Su), dtype=np.int32)
        tpw = 32 // J
        for u in range(units):                        # full rounds (or all units without a tail split)
            for t in range(tpw):
                tau = u * tpw + t
                if tau >= (tail0 if units2 else base):
                    continue
                for j in range(J):
                    cover[tau, j * chunk:min(Su, (j + 1) * chunk)] += 1
        if units2:
            assert units % warps == 0 and tail0 == units * tpw
            assert J2 in (2, 4, 8, 16, 32) and J2 > J and chunk2 == -(-Su // J2)
            tpw2 = 32 // J2
            assert (units2 - 1) * tpw2 < base - tail0 <= units2 * tpw2
            for u in range(units2):
                for t in range(tpw2):
                    tau = tail0 + u * tpw2 + t
                    if tau >= base:
                        continue
                    for j in range(J2):
                        cover[tau, j * chunk2:min(Su, (j + 1) * chunk2)] += 1
        else:
            assert (units - 1) * tpw < base <= units * tpw
        assert (cover == 1).all()


def test_cta_layout_balances_better_than_plain_deal(lib):
    N, nblk = 32, 456
    plan = bn.plan_mixed2d(N, 8, True, nblk)
    w = (plan[:, COL["Lu"]] * plan[:, COL["Lw"]] * plan[:, COL["Su"]] * plan[:, COL["Sw"]]).astype(np.float64)
    fixed = 2.0e4   # a per-item share for the staging and setup, in terms
    load = np.zeros(nblk)
    np.add.at(load, np.arange(len(w)) % nblk, w + fixed)        # CTA j takes rows k nblk + j
    rr = np.zeros(nblk)
    order = np.argsort(-w, kind="stable")
    np.add.at(rr, np.arange(len(w)) % nblk, w[order] + fixed)   # heaviest first, dealt round-robin
    counts = np.bincount(np.arange(len(w)) % nblk, minlength=nblk)
    assert counts.max() - counts.min() <= 1
    # the plan balances an issue-cost estimate (padding and per-unit work included), not raw terms,
    # so only the comparison with the plain deal is asserted in terms
    print(f"max/mean terms per CTA: plan {load.max() / load.mean():.3f}, round-robin {rr.max() / rr.mean():.3f}")
    assert load.max() / load.mean() < rr.max() / rr.mean()


@pytest.mark.parametrize("args", [(31, 8, 1, 456), (34, 8, 1, 456), (0, 8, 1, 456), (32, 12, 1, 456), (32, 8, 1, 0)])
def test_rejects_bad_arguments(lib, args):
    with pytest.raises(bn.BNError):
        bn.plan_mixed2d(*args)
