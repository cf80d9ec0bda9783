"""Host logic of the serving loop: the slot arena and its take/give stacks."""
import numpy as np

from paper_2201_10473_gb300 import gf2x, serve


def test_slot_pool_carves_disjoint_aligned_slots_within_budget():
    sizes = {12323: 1, 17669: 2, 57637: 1}
    budget = 3 << 20
    pool = serve.SlotPool(sizes, budget, device="cpu")
    base = pool.arena.data_ptr()
    spans = []
    for n in sizes:
        L = pool.slot_limbs[n]
        assert L >= gf2x.limbs(n) and L % 2 == 0
        for ad in pool.free[n][: pool.top[n]]:
            assert (int(ad) - base) % 16 == 0
            spans.append((int(ad), int(ad) + 8 * L))
    spans.sort()
    assert all(a[1] <= b[0] for a, b in zip(spans, spans[1:]))     # no two slots overlap
    assert spans[0][0] >= base and spans[-1][1] <= base + budget    # all inside the arena
    # byte shares follow the weights
    bytes_of = {n: pool.capacity[n] * 8 * pool.slot_limbs[n] for n in sizes}
    assert abs(bytes_of[17669] / budget - 0.5) < 0.01


def test_slot_pool_take_and_give_many_conserve_slots():
    pool = serve.SlotPool({17669: 1}, 1 << 20, device="cpu")
    n = 17669
    cap = pool.capacity[n]
    all_slots = set(int(x) for x in pool.free[n][:cap])
    a = pool.take_many(n, 10)
    b = pool.take_many(n, cap - 10)
    assert pool.available(n) == 0 and pool.take(n) is None
    assert set(a.tolist()) | set(b.tolist()) == all_slots and len(set(a.tolist()) & set(b.tolist())) == 0
    try:
        pool.take_many(n, 1)
        raise AssertionError("took a slot that was not free")
    except ValueError:
        pass
    pool.give_many(n, b[::-1].copy())
    pool.give(n, int(a[0]))
    assert pool.available(n) == cap - 9
    c = pool.take_many(n, cap - 9)
    assert set(c.tolist()) == set(b.tolist()) | {int(a[0])}


def test_slot_pool_rejects_a_budget_without_a_slot_for_some_size():
    import pytest
    with pytest.raises(ValueError):
        serve.SlotPool({12323: 1, 57637: 1}, 8000, device="cpu")   # 4000 bytes each: no 57637 slot


def test_request_slots_hold_both_operands_and_the_result():
    """A request slot holds a, b and r (each part 16-byte aligned), so the
    budget admits a third of the requests a results-only pool would."""
    sizes = {17669: 1, 57637: 1}
    budget = 6 << 20
    full = serve.SlotPool(sizes, budget, device="cpu")
    res_only = serve.SlotPool(sizes, budget, device="cpu", operands=False)
    for n in sizes:
        P = full.part_limbs[n]
        assert P >= gf2x.limbs(n) and P % 2 == 0 and full.slot_limbs[n] == 3 * P
        assert abs(full.capacity[n] * 3 - res_only.capacity[n]) <= 3
        ad = int(full.free[n][0])
        a, b = full.operand_addrs(n, ad)
        assert (a, b, full.result_addr(n, ad)) == (ad, ad + 8 * P, ad + 16 * P)
        assert res_only.result_addr(n, ad) == ad


def test_server_budget_must_cover_its_lists():
    import pytest
    # the item and copy lists of 3 streams x 2048 items take 480 KiB of the budget
    assert serve.default_budget([17669], 0, max_batch=2048, streams=3) == 3 * 2048 * 80
