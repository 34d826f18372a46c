"""GPU parity of the recorded merge pass and its key-free backward
(cr_merge_pass_record / cr_merge_pass_backward_recorded) against the CPU
oracle: output keys and payloads bit for bit, every recorded source bit, and
the routed gradient; then the whole merge-sort chain in both backward forms."""
import numpy as np
import pytest
import torch

import oracle
import paper_1303_4312_gb300 as cr
from gpu_util import dev, host, key_type, same_bits

pytestmark = pytest.mark.gpu

KEY_DTYPES = [np.int32, np.uint32, np.int64, np.uint64]
VAL_DTYPES = {4: np.float32, 8: np.float64}


def run_sorted_keys(rng, N, w, dt, spread):
    """N keys of dtype dt whose runs of w are each sorted (ties frequent)."""
    info = np.iinfo(dt)
    if spread is None:
        X = rng.integers(info.min, info.max, size=N, dtype=dt, endpoint=True)
    else:
        X = (rng.integers(0, spread, size=N).astype(dt) * dt(info.max // spread)).astype(dt)
        if info.min < 0:
            X = (X - dt(info.max // 2)).astype(dt)
    for a0 in range(0, N, w):
        X[a0:a0 + w].sort(kind="stable")
    return X


def expected_flags(src, N, w, tile):
    """The per-tile source bits of one pass, from the oracle's source indices:
    tile t of pair q owns TILE/32 words; bit x is set when output x of the
    tile came from the pair's second run."""
    w = min(w, N)
    words = []
    for a0 in range(0, N, 2 * w):
        m = min(w, N - a0)
        n = min(w, N - a0 - m)
        from_b = src[a0:a0 + m + n] >= a0 + m
        for r0 in range(0, m + n, tile):
            bits = np.zeros(tile, dtype=bool)
            part = from_b[r0:r0 + tile]
            bits[:len(part)] = part
            words.append(np.packbits(bits, bitorder="little").view("<u4"))
    return np.concatenate(words) if words else np.zeros(0, "<u4")


CASES = [(50000, 1000), (1 << 16, 1024), (12345, 7), (9000, 6000), (100, 1000), (1, 1),
         (33, 16), (200003, 4096)]


@pytest.mark.parametrize("dt", KEY_DTYPES)
@pytest.mark.parametrize("vb", [4, 8])
def test_recorded_pass_forward_flags_backward(dt, vb):
    rng = np.random.default_rng(300 + vb)
    vdt = VAL_DTYPES[vb]
    kt = key_type(np.empty(0, dt))
    tile = cr.tile_size(kt, vb, cls="pass")     # merge passes use the pass class
    for N, w in CASES:
        for spread in (None, 5):
            X = run_sorted_keys(rng, N, w, dt, spread)
            Xv = rng.standard_normal(N).astype(vdt)
            Y, Yv, rec = cr.merge_pass_record(dev(X), dev(Xv), w, key_type=kt)
            gY = rng.standard_normal(N).astype(vdt)
            gX = cr.merge_pass_backward_recorded(rec, dev(gY))
            torch.cuda.synchronize()
            cr.workspace_status(rec.ws)
            wy, wyv, src = oracle.merge_pass(X, Xv, w)
            assert same_bits(host(Y, dt), wy), (N, w, spread)
            assert same_bits(host(Yv, vdt), wyv), (N, w, spread)
            want_f = expected_flags(src, N, w, tile)
            got_f = host(rec.flags, np.uint32)[:len(want_f)]
            assert np.array_equal(got_f, want_f), (N, w, spread)
            want = np.empty_like(gY)
            want[src] = gY
            assert same_bits(host(gX, vdt), want), (N, w, spread)


@pytest.mark.parametrize("shape", range(6))
def test_recorded_pass_every_tile_shape(shape):
    """Each tile shape (its own TILE and flag-word count) records and routes
    correctly; the previous shape is restored afterwards."""
    from paper_1303_4312_gb300 import _lib
    lib = _lib.load()
    code = _lib.KEY_TYPES["u64"]
    before = lib.cr_get_tile_shape_for(code, 4, 4)
    if lib.cr_set_tile_shape_for(code, 4, 4, shape) != 0:
        pytest.skip("shape does not fit recorded passes of uint64 keys with 4-byte payloads")
    try:
        rng = np.random.default_rng(310 + shape)
        tile = cr.tile_size("u64", 4, cls="pass")
        for N, w in ((5 * tile + 77, 2 * tile - 3), (40000, 512), (3 * tile, tile)):
            X = run_sorted_keys(rng, N, w, np.uint64, 9)
            Xv = rng.standard_normal(N).astype(np.float32)
            Y, Yv, rec = cr.merge_pass_record(dev(X), dev(Xv), w, key_type="u64")
            gY = rng.standard_normal(N).astype(np.float32)
            gX = cr.merge_pass_backward_recorded(rec, dev(gY))
            torch.cuda.synchronize()
            cr.workspace_status(rec.ws)
            wy, wyv, src = oracle.merge_pass(X, Xv, w)
            assert same_bits(host(Y, np.uint64), wy)
            assert same_bits(host(Yv, np.float32), wyv)
            want_f = expected_flags(src, N, w, tile)
            assert np.array_equal(host(rec.flags, np.uint32)[:len(want_f)], want_f)
            want = np.empty_like(gY)
            want[src] = gY
            assert same_bits(host(gX, np.float32), want)
    finally:
        lib.cr_set_tile_shape_for(code, 4, 4, before)


def test_recorded_backward_refuses_other_table():
    """A record made for another width (another tile count) is refused on
    the device and nothing is written."""
    rng = np.random.default_rng(320)
    N = 100000
    X = run_sorted_keys(rng, N, 1000, np.int32, None)
    Xv = rng.standard_normal(N).astype(np.float32)
    _, _, rec = cr.merge_pass_record(dev(X), dev(Xv), 1000, key_type="i32")
    torch.cuda.synchronize()
    rec.width = N     # one pair: fewer tiles than the table holds
    gX = torch.full((N,), 7.0, device="cuda")
    cr.merge_pass_backward_recorded(rec, dev(rng.standard_normal(N).astype(np.float32)), out=gX)
    with pytest.raises(cr.CorankError) as e:
        cr.workspace_status(rec.ws)
    assert e.value.name == "CR_EINTERNAL"
    assert bool((gX == 7.0).all())


@pytest.mark.parametrize("record", [True, False])
@pytest.mark.parametrize("run", [None, 64, 1000])
def test_merge_sort_both_backward_forms(record, run):
    """The merge-sort chain with recorded or recomputed backward, with and
    without run formation, against numpy's stable argsort."""
    rng = np.random.default_rng(330)
    for N in (1, 999, 70001, 1 << 18):
        vals = rng.integers(0, 2**64, 3000, dtype=np.uint64)
        X = vals[rng.integers(0, len(vals), N)]
        if run is not None:
            for a0 in range(0, N, run):
                X[a0:a0 + run].sort(kind="stable")
        Xv = rng.standard_normal(N).astype(np.float32)
        Xt = dev(X)
        Xvt = dev(Xv).requires_grad_(True)
        Y, Yv = cr.merge_sort(Xt, Xvt, run=run, key_type="u64", record=record)
        gY = rng.standard_normal(N).astype(np.float32)
        Yv.backward(dev(gY))
        torch.cuda.synchronize()
        o = np.argsort(X, kind="stable")
        assert same_bits(host(Y, np.uint64), X[o]), N
        assert same_bits(host(Yv.detach(), np.float32), Xv[o]), N
        g = np.empty_like(gY)
        g[o] = gY
        assert same_bits(host(Xvt.grad, np.float32), g), N


@pytest.mark.parametrize("dt", KEY_DTYPES)
@pytest.mark.parametrize("vb", [4, 8])
def test_recorded_run_formation(dt, vb):
    """sort_runs_record: every run of sort_run_length() elements stably
    sorted with its payloads, the written permutation equal to numpy's stable
    argsort of the run, and the recorded backward routing gY through it; the
    plain and replayed forms give the same results."""
    rng = np.random.default_rng(340 + vb)
    vdt = VAL_DTYPES[vb]
    kt = key_type(np.empty(0, dt))
    R = cr.sort_run_length()
    info = np.iinfo(dt)
    for N in (1, R - 1, R, R + 1, 7 * R + 123, 100003):
        for spread in (None, 4):
            if spread is None:
                X = rng.integers(info.min, info.max, N, dtype=dt, endpoint=True)
            else:
                X = rng.integers(0, spread, N).astype(dt)
            Xv = rng.standard_normal(N).astype(vdt)
            gY = rng.standard_normal(N).astype(vdt)
            Y, Yv, perm = cr.sort_runs_record(dev(X), dev(Xv), key_type=kt)
            gX = cr.sort_runs_backward_recorded(perm, dev(gY))
            Y2, Yv2 = cr.sort_runs(dev(X), dev(Xv), key_type=kt)
            gX2 = cr.sort_runs_backward(dev(X), dev(gY), key_type=kt)
            torch.cuda.synchronize()
            p = host(perm, np.uint16).astype(np.int64)
            wy, wyv, wg = np.empty_like(X), np.empty_like(Xv), np.empty_like(gY)
            for b0 in range(0, N, R):
                o = np.argsort(X[b0:b0 + R], kind="stable")
                assert np.array_equal(p[b0:b0 + len(o)], o), (N, b0)
                wy[b0:b0 + len(o)] = X[b0:b0 + R][o]
                wyv[b0:b0 + len(o)] = Xv[b0:b0 + R][o]
                g = np.empty(len(o), dtype=vdt)
                g[o] = gY[b0:b0 + len(o)]
                wg[b0:b0 + len(o)] = g
            assert same_bits(host(Y, dt), wy) and same_bits(host(Yv, vdt), wyv), N
            assert same_bits(host(gX, vdt), wg), N
            assert same_bits(host(Y2, dt), wy) and same_bits(host(Yv2, vdt), wyv), N
            assert same_bits(host(gX2, vdt), wg), N


@pytest.mark.parametrize("dt", KEY_DTYPES)
@pytest.mark.parametrize("vb", [0, 4, 8])
def test_merge_runs_block(dt, vb):
    """The shared-memory stage equals the chain of merge passes it replaces
    (oracle merge_pass, width by width up to the chunk length), keys and
    payloads bit for bit; its recorded permutation routes gradients like the
    passes' composed permutation.  Widths 1, 2 and 4 (run formation: groups
    of 8 sorted in registers first) equal the passes from that width."""
    rng = np.random.default_rng(350 + vb)
    R = cr.merge_runs_block_length()
    kt = key_type(np.empty(0, dt))
    for N, w in [(R, 1024), (5 * R + 333, 8), (100003, 1024), (1, 64), (3 * R, 2048),
                 (R - 1, 512), (5 * R + 333, 1), (R, 2), (3 * R + 5, 4), (1, 1), (13, 1),
                 (100003, 1)]:
        X = run_sorted_keys(rng, N, w, dt, 7 if vb else None)
        Xv = rng.standard_normal(N).astype(VAL_DTYPES.get(vb, np.float32))
        want, wv, src = X.copy(), Xv.copy(), np.arange(N)
        ww = w
        while ww < R and ww < N:
            # chunks of R are independent: merge pass by pass inside each
            want, wv, s = oracle.merge_pass(want, wv, ww)
            src = src[s]
            ww *= 2
        # merge_pass runs over the whole array; restricted to widths < R its
        # pairs never cross a chunk boundary, so it equals the chunked stage
        Y, Yv, perm = cr.merge_runs_block(dev(X), dev(Xv) if vb else None, w, key_type=kt,
                                          record=vb != 0)
        torch.cuda.synchronize()
        assert same_bits(host(Y, dt), want), (N, w)
        if vb:
            assert same_bits(host(Yv, Xv.dtype), wv), (N, w)
            base = (np.arange(N) // R) * R
            assert np.array_equal(host(perm, np.uint16).astype(np.int64) + base, src), (N, w)
            gY = rng.standard_normal(N).astype(Xv.dtype)
            gX = cr.merge_runs_block_backward_recorded(perm, dev(gY))
            torch.cuda.synchronize()
            g = np.empty_like(gY)
            g[src] = gY
            assert same_bits(host(gX, Xv.dtype), g), (N, w)
