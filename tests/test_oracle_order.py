"""Pins of the oracle's key-order map (order_key / merge_in_order) to what
the IEEE 754 standard and plain integer arithmetic fix, independently of the
map itself:

* the totalOrder ladder of IEEE 754-2008 Section 5.10 written out as explicit
  bit patterns (NaN signs, quiet/signaling, payloads, signed zeros,
  subnormals, infinities);
* numeric order of random finite floats and integers (numpy's stable sort of
  the values);
* descending = the reverse stable order (Python's stable sort on negated
  integers);
* merges in every order against Python's stable sort of the concatenation.
"""
import numpy as np
import pytest

import oracle


def _f32(bits):
    return np.array(bits, dtype=np.uint32).view(np.float32)


def _f64(bits):
    return np.array(bits, dtype=np.uint64).view(np.float64)


# totalOrder, ascending (Section 5.10): negative NaNs below -inf, quiet below
# signaling and greater payload below lesser for negative NaNs, the reverse
# for positive NaNs; -0 below +0.
LADDER32 = [
    0xFFFFFFFF,  # -qNaN, largest payload
    0xFFC00001,  # -qNaN, payload 1
    0xFFC00000,  # -qNaN, payload 0
    0xFFBFFFFF,  # -sNaN, largest payload
    0xFF800001,  # -sNaN, payload 1
    0xFF800000,  # -inf
    0xFF7FFFFF,  # -largest finite
    0xBF800000,  # -1.0
    0x80800000,  # -smallest normal
    0x807FFFFF,  # -largest subnormal
    0x80000001,  # -smallest subnormal
    0x80000000,  # -0
    0x00000000,  # +0
    0x00000001,  # +smallest subnormal
    0x007FFFFF,  # +largest subnormal
    0x00800000,  # +smallest normal
    0x3F800000,  # +1.0
    0x7F7FFFFF,  # +largest finite
    0x7F800000,  # +inf
    0x7F800001,  # +sNaN, payload 1
    0x7FBFFFFF,  # +sNaN, largest payload
    0x7FC00000,  # +qNaN, payload 0
    0x7FC00001,  # +qNaN, payload 1
    0x7FFFFFFF,  # +qNaN, largest payload
]
LADDER64 = [
    0xFFFFFFFFFFFFFFFF, 0xFFF8000000000001, 0xFFF8000000000000, 0xFFF7FFFFFFFFFFFF,
    0xFFF0000000000001, 0xFFF0000000000000, 0xFFEFFFFFFFFFFFFF, 0xBFF0000000000000,
    0x8010000000000000, 0x800FFFFFFFFFFFFF, 0x8000000000000001, 0x8000000000000000,
    0x0000000000000000, 0x0000000000000001, 0x000FFFFFFFFFFFFF, 0x0010000000000000,
    0x3FF0000000000000, 0x7FEFFFFFFFFFFFFF, 0x7FF0000000000000, 0x7FF0000000000001,
    0x7FF7FFFFFFFFFFFF, 0x7FF8000000000000, 0x7FF8000000000001, 0x7FFFFFFFFFFFFFFF,
]


@pytest.mark.parametrize("kt,ladder,mk", [("f32", LADDER32, _f32), ("f64", LADDER64, _f64)])
def test_float_total_order_ladder(kt, ladder, mk):
    vals = mk(ladder)
    keys = oracle.order_key(vals, kt).astype(object)
    assert all(int(a) < int(b) for a, b in zip(keys, keys[1:]))
    # shuffled, the stable order of the keys restores the ladder
    rng = np.random.default_rng(0)
    perm = rng.permutation(len(ladder))
    got = vals[perm][np.argsort(oracle.order_key(vals[perm], kt), kind="stable")]
    assert got.tobytes() == vals.tobytes()
    # descending: exactly the reverse
    desc = oracle.order_key(vals, kt + ":desc").astype(object)
    assert all(int(a) > int(b) for a, b in zip(desc, desc[1:]))


@pytest.mark.parametrize("kt,dt", [("f32", np.float32), ("f64", np.float64)])
def test_float_order_is_numeric_on_finite_values(kt, dt):
    rng = np.random.default_rng(1)
    x = (rng.standard_normal(5000) * 10.0 ** rng.integers(-30, 30, 5000)).astype(dt)
    x = x[x != 0]
    o_key = np.argsort(oracle.order_key(x, kt), kind="stable")
    o_num = np.argsort(x, kind="stable")
    assert np.array_equal(x[o_key], x[o_num])


@pytest.mark.parametrize("kt,dt", [("i32", np.int32), ("u32", np.uint32), ("i64", np.int64),
                                   ("u64", np.uint64)])
def test_integer_orders_and_descending(kt, dt):
    rng = np.random.default_rng(2)
    info = np.iinfo(dt)
    x = rng.integers(info.min, info.max, 3000, dtype=dt, endpoint=True)
    x[:40] = x[40:80]                              # ties
    x[80], x[81] = info.min, info.max
    asc = np.argsort(oracle.order_key(x, kt), kind="stable")
    assert np.array_equal(asc, np.argsort(x, kind="stable"))
    desc = np.argsort(oracle.order_key(x, kt + ":desc"), kind="stable")
    ref = sorted(range(len(x)), key=lambda i: -int(x[i]))   # stable: ties keep input order
    assert np.array_equal(desc, ref)


@pytest.mark.parametrize("kt", ["i32", "u32:desc", "i64:desc", "f32", "f64:desc", "f32:desc"])
def test_merge_in_order_brute_force(kt):
    """merge_in_order against Python's stable sort of A||B by order position:
    every output element, and stability (A before B on ties)."""
    rng = np.random.default_rng(3)
    base = kt.split(":")[0]
    dt = {"i32": np.int32, "u32": np.uint32, "i64": np.int64, "f32": np.float32,
          "f64": np.float64}[base]
    for _ in range(300):
        m, n = rng.integers(0, 12, 2)
        if base[0] != "f":
            pool = rng.integers(-4, 5, 8).astype(dt)
        elif base == "f32":
            pool = _f32(LADDER32)[rng.integers(0, len(LADDER32), 8)]
        else:
            pool = _f64(LADDER64)[rng.integers(0, len(LADDER64), 8)]
        A = pool[rng.integers(0, len(pool), m)]
        B = pool[rng.integers(0, len(pool), n)]
        A = A[np.argsort(oracle.order_key(A, kt), kind="stable")]
        B = B[np.argsort(oracle.order_key(B, kt), kind="stable")]
        C, src = oracle.merge_in_order(A, B, kt)
        # rank of each distinct bit pattern in the order, computed by sorting
        # the pool with the already pinned map
        ka = oracle.order_key(np.concatenate([A, B]), kt).astype(object)
        ref = sorted(range(m + n), key=lambda i: int(ka[i]))
        assert list(src) == ref
        assert C.tobytes() == np.concatenate([A, B])[ref].tobytes()


@pytest.mark.parametrize("kt", ["pair_u32", "pair_i32", "pair_i32:desc", "pair_u32:desc"])
def test_pair_orders_are_lexicographic(kt):
    """(major, minor) pairs in one 64-bit word, major in the high half:
    order_key order equals Python's stable sort of the (major, minor) tuples
    with the halves read as uint32 or int32 (reversed for ':desc')."""
    rng = np.random.default_rng(4)
    n = 4000
    major = rng.integers(0, 2**32, n, dtype=np.uint64)
    major[: n // 2] = major[n // 2:]                       # repeated majors
    minor = rng.integers(0, 2**32, n, dtype=np.uint64)
    minor[:50] = minor[50:100]
    major[:50] = major[50:100]                             # full ties
    words = (major << np.uint64(32)) | minor
    signed = kt.startswith("pair_i32")

    def half(v):
        v = int(v)
        return v - (1 << 32) if signed and v >= (1 << 31) else v
    tup = [(half(a), half(b)) for a, b in zip(major, minor)]
    if kt.endswith(":desc"):
        ref = sorted(range(n), key=lambda i: (-tup[i][0], -tup[i][1]))
    else:
        ref = sorted(range(n), key=lambda i: tup[i])
    got = np.argsort(oracle.order_key(words, kt), kind="stable")
    assert np.array_equal(got, ref)
