"""Bank behaviour of the shared-memory layout of the merge stage
(merge_runs_block_kernel): element i of a key array sits at slot
i + i/16 (8-byte keys) or i + i/32 (4-byte keys), element i of a 16-bit
index array at i + 2 (i/64); thread t of 512 owns outputs [8t, 8t + 8).

Shared memory has 32 banks of 4 bytes.  A warp's 8-byte accesses are served
in two halves of 16 lanes (16 eight-byte bank pairs); its 4-byte and 2-byte
accesses in one pass (two lanes on the same 4-byte word do not conflict).
The test enumerates every warp's addresses for the 8-strided accesses of the
merge rounds and for the linear loads and stores of a chunk, and checks
that no two lanes touch different words of one bank: the gaps remove the
conflicts a power-of-two stride would otherwise cause (checked too)."""
import pytest

R, IPT, NT = 4096, 8, 512


def key_slot(i, key_bytes):
    return i + (i >> (4 if key_bytes == 8 else 5))


def idx_slot(i):
    return i + ((i >> 6) << 1)


def worst_way(addrs_bytes, width):
    """Largest number of distinct bank words one bank serves for these lane
    byte addresses (accesses of `width` bytes)."""
    if width == 8:
        groups = [addrs_bytes[:16], addrs_bytes[16:]]
        way = 0
        for g in groups:
            banks = {}
            for a in g:
                banks.setdefault((a // 8) % 16, set()).add(a // 8)
            way = max(way, max(len(v) for v in banks.values()))
        return way
    banks = {}
    for a in addrs_bytes:
        banks.setdefault((a // 4) % 32, set()).add(a // 4)
    return max(len(v) for v in banks.values())


@pytest.mark.parametrize("key_bytes", [4, 8])
def test_strided_and_linear_key_accesses_are_conflict_free(key_bytes):
    for warp in range(NT // 32):
        for q in range(IPT):
            lanes = [key_slot((warp * 32 + l) * IPT + q, key_bytes) * key_bytes
                     for l in range(32)]
            assert worst_way(lanes, key_bytes) == 1, (warp, q)
    for c in range(R // 32):
        lanes = [key_slot(32 * c + l, key_bytes) * key_bytes for l in range(32)]
        assert worst_way(lanes, key_bytes) == 1, c


def test_strided_and_linear_index_accesses_are_conflict_free():
    for warp in range(NT // 32):
        for q in range(IPT):
            lanes = [idx_slot((warp * 32 + l) * IPT + q) * 2 for l in range(32)]
            assert worst_way(lanes, 2) == 1, (warp, q)
    for c in range(R // 32):
        lanes = [idx_slot(32 * c + l) * 2 for l in range(32)]
        assert worst_way(lanes, 2) == 1, c


def test_unpadded_layout_would_conflict():
    """Without the gaps the 8-strided writes are 8-way (8-byte keys) and
    4-way (16-bit indices) conflicted: the gaps are what removes it."""
    lanes = [(l * IPT) * 8 for l in range(32)]
    assert worst_way(lanes, 8) == 8
    lanes = [(l * IPT) * 2 for l in range(32)]
    assert worst_way(lanes, 2) == 4


def test_slots_fit_the_layout():
    """The largest slot used (element R, read one past a pair) is inside the
    arrays the kernel allocates: R + R/16 + 1 (8-byte keys), R + R/32 + 1
    (4-byte keys), R + 2 R/64 + 1 (indices)."""
    assert key_slot(R, 8) == R + R // 16
    assert key_slot(R, 4) == R + R // 32
    assert idx_slot(R - 1) < R + 2 * (R // 64) + 1
    for i in range(R):
        assert key_slot(i + 1, 8) > key_slot(i, 8) and idx_slot(i + 1) > idx_slot(i)
