"""The tile-shape autotuner: its table is applied class by class (CPU, no
kernel runs), refused when made for another list of shapes, and on a GPU
tune() times every class and produces a table that apply() installs."""
import json

import pytest

from paper_1303_4312_gb300 import _lib, autotune, build


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


CLASS_NAMES = [c for c, _ in autotune.CLASSES]


def _snapshot(lib):
    return {(kt, vb, c): lib.cr_get_tile_shape_for(_lib.KEY_TYPES[kt], vb, c)
            for kt, vb in autotune.COMBOS for c in range(len(CLASS_NAMES))}


def _restore(lib, snap):
    for (kt, vb, c), s in snap.items():
        lib.cr_set_tile_shape_for(_lib.KEY_TYPES[kt], vb, c, s)


def test_apply_round_trip_changes_shapes(lib, tmp_path):
    """A table that picks shapes other than the current ones, class by class
    (batched and pass included), is installed by apply(); one made for
    another list of shapes is ignored."""
    snap = _snapshot(lib)
    try:
        table = {"gpu": "test", "cc": "10.3", "shape_list": autotune.shape_list(lib),
                 "shapes": {}}
        want = {}
        for kt, vb in autotune.COMBOS:
            code = _lib.KEY_TYPES[kt]
            entry = {}
            for cls, idx in autotune.CLASSES:
                cur = lib.cr_get_tile_shape_for(code, vb, idx)
                pick = None
                for s in range(lib.cr_tile_shape_count()):
                    if s != cur and lib.cr_set_tile_shape_for(code, vb, idx, s) == 0:
                        pick = s
                        break
                lib.cr_set_tile_shape_for(code, vb, idx, cur)
                if pick is not None:
                    entry[cls] = {"shape": pick}
                    want[(code, vb, idx)] = pick
            table["shapes"][f"{kt}:{vb}"] = entry
        assert any(idx == 3 for _, _, idx in want) and any(idx == 4 for _, _, idx in want)
        path = tmp_path / "t.json"
        path.write_text(json.dumps(table))
        assert autotune.apply(lib, path=str(path)) is not None
        for (code, vb, idx), s in want.items():
            assert lib.cr_get_tile_shape_for(code, vb, idx) == s
        _restore(lib, snap)
        # another list of shapes: ignored, nothing changes
        table["shape_list"] = table["shape_list"][:-1]
        path.write_text(json.dumps(table))
        assert autotune.apply(lib, path=str(path)) is None
        assert _snapshot(lib) == snap
    finally:
        _restore(lib, snap)


def test_committed_table_matches_the_library(lib):
    """The committed GB300 table names shapes of this library's list, every
    class of every combination, and each choice is accepted."""
    path = autotune.table_path("NVIDIA GB300")
    table = json.load(open(path))
    assert table["shape_list"] == autotune.shape_list(lib)
    snap = _snapshot(lib)
    try:
        for kt, vb in autotune.COMBOS:
            entry = table["shapes"][f"{kt}:{vb}"]
            for cls, idx in autotune.CLASSES:
                assert cls in entry, (kt, vb, cls)
                assert lib.cr_set_tile_shape_for(_lib.KEY_TYPES[kt], vb, idx,
                                                 entry[cls]["shape"]) == 0, (kt, vb, cls)
    finally:
        _restore(lib, snap)


@pytest.mark.gpu
def test_tune_small_times_every_class(lib, tmp_path):
    """tune() at a small size: every combination and class gets timings for
    the shapes that fit and a fastest one; apply() installs that table."""
    snap = _snapshot(lib)
    try:
        out = tmp_path / "tuned.json"
        table = autotune.tune(log2_size=20, reps=2, write=True, out=str(out))
        assert table["shape_list"] == autotune.shape_list(lib)
        for kt, vb in autotune.COMBOS:
            entry = table["shapes"][f"{kt}:{vb}"]
            for cls, idx in autotune.CLASSES:
                e = entry[cls]
                assert e["ms"], (kt, vb, cls)
                # the table keeps times rounded to 0.1 us: the choice is within
                # that rounding of the fastest listed time
                tot = {int(s): sum(v.values()) for s, v in e["ms"].items()}
                assert tot[e["shape"]] <= min(tot.values()) + 1e-4 * len(e["ms"][str(e["shape"])])
                if cls == "pass" and vb:
                    assert all(autotune.shape_list(lib)[int(s)][0] *
                               autotune.shape_list(lib)[int(s)][1] *
                               autotune.shape_list(lib)[int(s)][2] <= 4096 for s in e["ms"])
        # tune() leaves the shapes as they were
        assert _snapshot(lib) == snap
        assert autotune.apply(lib, path=str(out)) is not None
        for kt, vb in autotune.COMBOS:
            for cls, idx in autotune.CLASSES:
                assert lib.cr_get_tile_shape_for(_lib.KEY_TYPES[kt], vb, idx) == \
                    table["shapes"][f"{kt}:{vb}"][cls]["shape"]
    finally:
        _restore(lib, snap)
