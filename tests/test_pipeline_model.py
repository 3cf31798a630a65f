"""CPU model of the fused kernel's row pipeline (no GPU).

The fused update streams lattice rows through RING shared-memory slots: a producer warp loads
rows ahead and stores final rows; compute threads do the even update of row r and the odd
update of row r-1 at loop step r and hand row r-2 back at step r (row n+1 after the loop).
The producer processes hand-backs in row order: store the row (rows 2..n+1 of the slab), wait
for the store to finish reading the slot, load the row RING further down into it.  This model
replays that protocol step by step and checks, for every slab of several lattice sizes and ring
depths, that a row is always loaded before it is read, that no slot is overwritten while a row
in it is still in use or being stored, that every slab row is stored exactly once, and that
neither side can wait on the other in a cycle (the producer never needs a hand-back the
compute side has not yet produced)."""
import pytest


def model(L, nslabs, ring):
    stored = [0] * L
    for b in range(nslabs):
        y0, y1 = b * L // nslabs, (b + 1) * L // nslabs
        n = y1 - y0
        total = n + 4                          # rows y0-2 .. y1+1
        slot_row = {}
        loaded = set()
        last_use = {}
        released = set()

        def load(r, when):
            s = r % ring
            if s in slot_row:
                old = slot_row[s]
                assert old in released, "slot refilled before its row was handed back"
                assert last_use.get(old, -1) < when
            slot_row[s] = r
            loaded.add(r)

        def use(r, when):
            assert r in loaded and slot_row[r % ring] == r, (L, nslabs, ring, b, r, when)
            last_use[r] = max(last_use.get(r, -1), when)

        producer_next = 0                      # next hand-back the producer will take

        def producer_progress(when):
            nonlocal producer_next
            while producer_next in released:
                k = producer_next
                if k >= 2:
                    stored[(y0 - 2 + k) % L] += 1
                if k + ring < total:
                    load(k + ring, when)
                producer_next += 1

        for r in range(min(ring, total)):
            load(r, -1)
        use(0, 0)
        use(1, 0)
        for r in range(1, n + 3):
            # the compute side waits for row r+1; it must already be loaded (no cycle)
            use(r + 1, r)
            if r - 2 >= 1:
                use(r - 2, r)                  # odd carry of row r-2
            use(r, r)
            use(r + 1, r)                      # even update of row r
            if r >= 2:
                released.add(r - 2)
            producer_progress(r + 0.25)
            use(r, r + 0.5)                    # even carry of row r
            if r >= 2:
                use(r - 1, r + 0.5)
                use(r, r + 0.5)                # odd update of row r-1
        use(n + 1, n + 3)
        released.add(n + 1)
        producer_progress(n + 3.5)
        assert producer_next == n + 2
        assert len(loaded) == total
    assert all(c == 1 for c in stored), "a lattice row was not stored exactly once"


@pytest.mark.parametrize("ring", [6, 8, 12])
@pytest.mark.parametrize("L", [2048, 8192, 65536])
def test_fused_pipeline_protocol(L, ring):
    for nslabs in (L // 8, 304, 152, 7, 1):
        if nslabs <= L // 8:
            model(L, nslabs, ring)


def test_model_detects_a_short_ring():
    """With 3 slots the compute side would wait for a row the producer can only load after a
    hand-back that comes later in the same step (a cycle): the model must flag it.  (4 slots
    would already be correct but leave no room to prefetch; the kernel uses 6, 8 or 12.)"""
    with pytest.raises(AssertionError):
        model(2048, 16, 3)
    model(2048, 16, 4)
