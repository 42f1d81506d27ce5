"""Host-only wave planner of the batch scheduler (adc_batch_plan): no GPU."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def lib():
    from conftest import build_library
    build_library()
    import paper_2511_21640_gb300 as m
    return m


def _uneven(n, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        o = int(rng.integers(10, 41))
        v = int(rng.integers(50, 251))
        out.append(dict(kind="IP" if i % 2 == 0 else "EA", nocc=o, nvir=v, naux=6 * v, order=3, x=0.5))
    return out


def test_plan_orders_by_cost_and_respects_budget(lib):
    probs = _uneven(64)
    budget = 40 * 10**9
    nw, order, wave, mem, cost = lib.batch_plan(probs, 6, budget)
    assert sorted(order.tolist()) == list(range(64))
    assert np.all(np.diff(cost[order]) <= 0)          # longest first
    for w in range(nw):
        members = np.nonzero(wave == w)[0]
        assert members.size > 0
        assert mem[members].sum() <= budget or members.size == 1
    # first fit: no problem would have fitted into an earlier wave at its turn
    used = np.zeros(nw, np.int64)
    for i in order:
        for w in range(wave[i]):
            assert used[w] + mem[i] > budget
        used[wave[i]] += mem[i]


def test_plan_single_wave_when_everything_fits(lib):
    probs = _uneven(8, seed=3)
    nw, order, wave, mem, cost = lib.batch_plan(probs, 6, 10**15)
    assert nw == 1 and np.all(wave == 0)


def test_plan_oversized_problem_gets_its_own_wave(lib):
    probs = [dict(kind="EA", nocc=40, nvir=250, naux=1500, order=3, x=0.5),
             dict(kind="IP", nocc=10, nvir=50, naux=300, order=3, x=0.5),
             dict(kind="IP", nocc=12, nvir=60, naux=360, order=2, x=0.0)]
    nw, order, wave, mem, cost = lib.batch_plan(probs, 6, 10**9)
    assert order[0] == 0
    assert mem[0] > 10**9 and wave[0] == 0
    assert wave[1] == wave[2] == 1 and nw == 2


def test_plan_memory_estimate_grows_with_size(lib):
    small = dict(kind="EA", nocc=10, nvir=50, naux=300, order=3, x=0.5)
    big = dict(kind="EA", nocc=40, nvir=250, naux=1500, order=3, x=0.5)
    _, _, _, mem, cost = lib.batch_plan([small, big], 6, 10**12)
    assert mem[1] > 100 * mem[0] and cost[1] > 100 * cost[0]
    adc2 = dict(big, order=2, x=0.0)
    _, _, _, mem2, _ = lib.batch_plan([adc2, big], 6, 10**12)
    assert mem2[0] < mem2[1]  # no ladder integrals at second order


def test_plan_rejects_bad_sizes(lib):
    with pytest.raises(lib.AdcError):
        lib.batch_plan([dict(kind="EA", nocc=0, nvir=5, naux=3)], 6, 10**9)
    with pytest.raises(lib.AdcError):
        lib.batch_plan([dict(kind="IP", nocc=4, nvir=5, naux=3)], 6, 0)
