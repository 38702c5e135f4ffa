"""The batch autotuner's host logic, without a GPU: the compiled variant list,
the selection rule applied to one class's timings, and the process-wide cache
keyed by a system's class (sides rounded up to multiples of 64, exact
half-bandwidths)."""
import math

import pytest

import paper_2408_05444_gb300 as g
from paper_2408_05444_gb300 import build as gbuild


@pytest.fixture(scope="module", autouse=True)
def built():
    gbuild.build()
    g.grbk_tune_clear()
    yield
    g.grbk_tune_clear()


def test_variants_are_listed():
    vs = g.grbk_tune_variants()
    assert len(vs) >= 4
    assert (512, 2) in vs                       # the default variant
    assert all(t in (256, 512) and r in (1, 2, 4) for t, r in vs)
    assert len(set(vs)) == len(vs)


def test_choose_fastest_and_prefer_fewer_threads_within_two_percent():
    vs = g.grbk_tune_variants()
    n = len(vs)
    big = [i for i, (t, _) in enumerate(vs) if t == 512]
    small = [i for i, (t, _) in enumerate(vs) if t == 256]
    ms = [10.0] * n
    ms[big[0]] = 5.0
    assert g.grbk_tune_choose(ms) == big[0]
    ms[small[0]] = 5.08                         # within 2 %: the 256-thread variant wins
    assert g.grbk_tune_choose(ms) == small[0]
    ms[small[0]] = 5.2                          # 4 % slower: the fastest stays
    assert g.grbk_tune_choose(ms) == big[0]
    # failed or missing trials are ignored; none at all gives the default (512, 2)
    ms = [0.0] * n
    ms[small[-1]] = 3.0
    ms[big[0]] = math.nan
    assert g.grbk_tune_choose(ms) == small[-1]
    assert vs[g.grbk_tune_choose([0.0] * n)] == (512, 2)
    assert g.grbk_tune_choose([1.0] * (n + 1)) == -1


def test_cache_keys_by_class():
    g.grbk_tune_clear()
    assert g.grbk_tune_lookup(464, 464, 464, 464, 3, 3) == -1
    g.grbk_tune_store(464, 464, 464, 464, 3, 3, 1)
    # same class: sides within the same multiple of 64, same bands
    assert g.grbk_tune_lookup(449, 512, 450, 460, 3, 3) == 1
    assert g.grbk_tune_lookup(513, 464, 464, 464, 3, 3) == -1      # other side class
    assert g.grbk_tune_lookup(464, 464, 464, 464, 4, 3) == -1      # other band
    assert g.grbk_tune_lookup(464, 464, 464, 464, -1, -1) == -1    # dense path
    g.grbk_tune_store(464, 464, 464, 464, 3, 3, 0)                 # a later choice replaces it
    assert g.grbk_tune_lookup(464, 464, 464, 464, 3, 3) == 0
    with pytest.raises(g.GrbkError):
        g.grbk_tune_store(64, 64, 64, 64, -1, -1, len(g.grbk_tune_variants()))
    g.grbk_tune_clear()
    assert g.grbk_tune_lookup(464, 464, 464, 464, 3, 3) == -1
