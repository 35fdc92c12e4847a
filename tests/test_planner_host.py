"""Host-side planning through the C ABI, without a GPU: the transform planner
(rift2_fft_plan) and the launch-group planner (rift2_plan_groups).

The transform plans are checked for what makes them correct whatever the cost model picks:
the radices multiply to the pass length, a 13-smooth side is transformed directly, any
other side (up to 4096) through a Bluestein convolution of 13-smooth length between 2n - 1
and 2.5 n, the row kernels' plans have no radix 16, and no plan has more than 12 passes.
The group planner is checked for the ordering and grouping rift2_extract documents."""
import random

import pytest

import paper_2303_00319_gb300 as pkg

SMOOTH = (2, 3, 5, 7, 11, 13)
RADICES = {2, 3, 4, 5, 7, 8, 9, 11, 13, 16}


def smooth(n):
    for f in SMOOTH:
        while n % f == 0:
            n //= f
    return n == 1


def prod(xs):
    p = 1
    for x in xs:
        p *= x
    return p


@pytest.mark.parametrize("rows", [False, True])
def test_smooth_sides_are_direct(rows):
    for n in range(16, 8193):
        if not smooth(n):
            continue
        m, rad = pkg.fft_plan(n, rows)
        assert m == n and prod(rad) == n, (n, m, rad)
        assert set(rad) <= RADICES and len(rad) <= 12
        assert not (rows and 16 in rad)


@pytest.mark.parametrize("rows", [False, True])
def test_other_sides_take_bluestein(rows):
    for n in range(16, 4097):
        if smooth(n):
            continue
        m, rad = pkg.fft_plan(n, rows)
        assert 2 * n - 1 <= m <= 5 * n // 2 + 1 and smooth(m), (n, m)
        assert prod(rad) == m and set(rad) <= RADICES and len(rad) <= 12
        assert not (rows and 16 in rad)
        # the row and column plans of one side share the pass length (one plan per side)
        assert pkg.fft_plan(n, not rows)[0] == m


def test_plan_refusals_and_examples():
    for n, code in ((4099, pkg.E_UNIMPL), (8193, pkg.E_UNIMPL), (16384, pkg.E_UNIMPL), (1, pkg.E_INVAL)):
        with pytest.raises(pkg.Rift2Error) as e:
            pkg.fft_plan(n)
        assert e.value.code == code, n
    # the length whose two-halves row pass keeps two CTAs per SM (113.7 KB for 2816 would not)
    assert pkg.fft_plan(1289)[0] == 2704
    assert pkg.fft_plan(1024, rows=True)[1] == [8, 8, 4, 4]


def test_groups_order_by_size_and_cap_at_32():
    rng = random.Random(5)
    sizes = [(rng.randrange(384, 2049, 128), rng.randrange(384, 2049, 128)) for _ in range(100)]
    order, groups = pkg.plan_groups(sizes, hbm_budget=200 << 30)   # room for full groups
    assert sorted(order) == list(range(100))
    keys = [sizes[i] for i in order]
    assert keys == sorted(keys)                         # by height, then width
    for a, b in zip(order, order[1:]):                  # equal sizes keep their call order
        if sizes[a] == sizes[b]:
            assert a < b
    assert sum(groups) == 100 and all(1 <= g <= 32 for g in groups)
    assert groups == [32, 32, 32, 4]
    # the default 16 GiB budget halves the groups of the larger images
    _, g16 = pkg.plan_groups(sizes)
    assert sum(g16) == 100 and g16[:2] == [32, 32] and g16[2] < 32


def test_group_flags_and_budget():
    sizes = [(512, 512), (640, 384), (512, 512), (384, 640), (512, 512)]
    order, groups = pkg.plan_groups(sizes, pkg.default_params(flags=pkg.FLAG_NO_GROUPING))
    assert order == list(range(5)) and groups == [1] * 5
    order, groups = pkg.plan_groups(sizes, pkg.default_params(flags=pkg.FLAG_SIZE_GROUPS))
    assert order == list(range(5)) and groups == [1, 1, 1, 1, 1]   # no two neighbours match
    same = [(1024, 1024)] * 64
    order, groups = pkg.plan_groups(same)
    assert order == list(range(64)) and groups == [32, 32]
    # ~0.3 GB per 1024^2 image: a 2 GB budget halves the groups until they fit
    order, groups = pkg.plan_groups(same, hbm_budget=2 << 30)
    assert sum(groups) == 64 and max(groups) <= 8 and len(groups) > 2
    with pytest.raises(pkg.Rift2Error) as e:
        pkg.plan_groups(same, pkg.default_params(n_orient=8))
    assert e.value.code == pkg.E_UNIMPL
