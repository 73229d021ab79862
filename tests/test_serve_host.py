"""Host-side logic of the serving path (no GPU): admission by memory budget,
slot reuse and eviction, and the arrival trace."""
import numpy as np
import pytest

from paper_2005_02704_gb300 import serve


def make_pool(budget):
    made = []
    freed = []

    def alloc(key):
        made.append(key)
        return ("slot", key, len(made))

    return serve.SlotPool(budget, alloc, size_of=lambda k: k[0] * k[1], free_fn=freed.append), made, freed


def test_admission_waits_for_memory_and_reuses_slots():
    pool, made, _ = make_pool(100)
    a = pool.acquire((4, 10, 1))          # 40
    b = pool.acquire((4, 10, 1))          # 80
    assert a is not None and b is not None and pool.used == 80
    assert pool.acquire((4, 10, 1)) is None  # would exceed: waits
    pool.release((4, 10, 1), a)
    c = pool.acquire((4, 10, 1))          # reuses the released slot, no new allocation
    assert c is a and len(made) == 2 and pool.used == 80


def test_idle_slots_of_other_shapes_are_evicted_for_a_new_shape():
    pool, made, freed = make_pool(100)
    a = pool.acquire((2, 20, 1))          # 40
    b = pool.acquire((2, 20, 1))          # 80
    pool.release((2, 20, 1), a)
    c = pool.acquire((3, 20, 1))          # 60: needs the idle slot's memory
    assert c is not None and freed == [a] and pool.used == 100
    assert pool.acquire((3, 20, 1)) is None  # b is live and cannot be evicted
    pool.release((2, 20, 1), b)
    assert pool.acquire((3, 20, 1)) is None  # 60 + 60 > 100 even after evicting b (40)
    assert pool.peak <= 100


def test_oversized_scan_is_refused():
    pool, _, _ = make_pool(100)
    with pytest.raises(ValueError):
        pool.acquire((11, 10, 1))


def test_slot_bytes_counts_the_slot_tensors_in_allocator_blocks():
    # a slot holds x,y,z,r, elevations, mesh bytes, normals, labels and the
    # segment count, each rounded up to 512-byte allocator blocks; the pass's
    # workspace belongs to the lanes' contexts, not to slots
    H, W = 128, 4096
    assert serve.slot_bytes((H, W, 1)) == H * W * 16 + 512 + H * W + H * W * 12 + H * W * 4 + 512
    assert serve.slot_bytes((3, 5, 1)) == 6 * 512
    assert serve.slot_bytes((64, 2048, 2)) < serve.slot_bytes((64, 2048, 1))


def test_arrival_trace_rates_and_burst():
    rates = [10.0, 20.0]
    tr = serve.arrival_trace(rates, duration_s=60.0, burst=(30.0, 40.0, 4.0), seed=3)
    t = np.array([x[0] for x in tr])
    assert np.all(np.diff(t) >= 0) and t.min() >= 0 and t.max() < 60.0
    for k, r in enumerate(rates):
        tk = t[[x[1] == k for x in tr]]
        base = ((tk < 30) | (tk >= 40)).sum() / 50.0
        burst = ((tk >= 30) & (tk < 40)).sum() / 10.0
        assert abs(base - r) < 0.25 * r
        assert abs(burst - 4 * r) < 0.3 * 4 * r
