"""The ensemble's CTA plan (lb_batch_plan), host logic only: no GPU.

With no more lattices than CTAs and no bins every lattice is a group of its
own, and the largest per-CTA share ceil(items / CTAs) must be the smallest
any split of the CTAs allows (checked by brute force on small cases); with
more lattices than CTAs, or with k bins, the groups are filled with whole
lattices by the longest-processing-time rule and the CTAs split over the
groups' work the same way."""
import itertools
import math
import random

import pytest

from paper_1405_6162_gb300 import LBError
from paper_1405_6162_gb300.batch import plan


def _shares(items, groups):
    return [math.ceil(it / m) for it, (_, m) in zip(items, groups)]


def _check_layout(items, ctas, group, groups):
    assert len(group) == len(items)
    c = 0
    for cta0, m in groups:          # consecutive CTAs from 0, at least one each
        assert cta0 == c and m >= 1
        c += m
    assert c <= ctas
    assert sorted(set(group)) == list(range(len(groups)))


def _best_max_share(items, ctas):
    best = None
    for ms in itertools.product(range(1, ctas + 1), repeat=len(items)):
        if sum(ms) <= ctas:
            v = max(math.ceil(i / m) for i, m in zip(items, ms))
            best = v if best is None else min(best, v)
    return best


@pytest.mark.parametrize("seed", range(12))
def test_one_group_per_lattice_is_min_max(seed):
    rng = random.Random(seed)
    n = rng.randint(1, 4)
    items = [rng.randint(1, 40) for _ in range(n)]
    ctas = rng.randint(n, 9)
    group, groups = plan(items, ctas)
    _check_layout(items, ctas, group, groups)
    assert group == list(range(n))
    assert max(_shares(items, groups)) == _best_max_share(items, ctas)


def test_leftover_ctas_stay_idle():
    group, groups = plan([1, 2], 10)
    assert group == [0, 1] and groups == [(0, 1), (1, 2)]


def test_ensemble_workload_balance():
    # 64 lattices of sides 16..64 in 128-site items over 912 CTAs: no CTA
    # carries more than the integer optimum allows
    import lb_inputs as L
    specs = L.ensemble(3, 64, lo=16, hi=64)
    items = [(d["nx"] * d["ny"] * d["nz"] + 127) // 128 for d in specs]
    group, groups = plan(items, 912)
    _check_layout(items, 912, group, groups)
    t = max(_shares(items, groups))
    # t is optimal: one share less would need more CTAs than there are
    assert sum(math.ceil(i / t) for i in items) <= 912 < sum(math.ceil(i / (t - 1)) for i in items)


def test_more_lattices_than_ctas_longest_first():
    group, groups = plan([5, 3, 9, 1, 7], 2)
    # 9 -> g0, 7 -> g1, 5 -> g1 (12), 3 -> g0 (12), 1 -> g0 (tie, lower group)
    assert group == [1, 0, 0, 0, 1] and groups == [(0, 1), (1, 1)]
    rng = random.Random(7)
    items = [rng.randint(1, 100) for _ in range(50)]
    group, groups = plan(items, 8)
    _check_layout(items, 8, group, groups)
    loads = [0] * 8
    for k, g in enumerate(group):
        loads[g] += items[k]
    # the LPT bound: no group exceeds the mean by more than the largest item
    assert max(loads) <= sum(items) / 8 + max(items)


@pytest.mark.parametrize("items,ctas,bins", [([], 4, 0), ([3, 0], 4, 0), ([3, -1], 4, 0), ([3], 0, 0), ([3], 4, -1)])
def test_invalid(items, ctas, bins):
    with pytest.raises(LBError):
        plan(items, ctas, bins)


@pytest.mark.parametrize("seed", range(6))
def test_bins_balance_whole_lattices(seed):
    # k groups of whole lattices: the LPT bound on each group's work, and the
    # CTA split over the groups' work is the integer min-max (brute force)
    rng = random.Random(100 + seed)
    n = rng.randint(3, 9)
    items = [rng.randint(1, 30) for _ in range(n)]
    bins = rng.randint(2, 3)
    ctas = rng.randint(bins, 7)
    group, groups = plan(items, ctas, bins)
    _check_layout(items, ctas, group, groups)
    assert len(groups) == min(bins, n, ctas)
    loads = [0] * len(groups)
    for k, g in enumerate(group):
        loads[g] += items[k]
    assert max(loads) <= sum(items) / len(groups) + max(items)
    assert max(_shares(loads, groups)) == _best_max_share(loads, ctas)


def test_one_bin_is_the_whole_grid():
    items = [5, 9, 2, 7]
    group, groups = plan(items, 12, 1)
    assert group == [0, 0, 0, 0] and groups == [(0, 12)]
    # fewer items than CTAs: one CTA per item, the rest idle
    group, groups = plan([2, 1], 10, 1)
    assert groups == [(0, 3)]


def test_bins_capped_by_lattices_and_ctas():
    assert len(plan([3, 4], 10, 5)[1]) == 2
    assert len(plan([3, 4, 5, 6], 3, 8)[1]) == 3
