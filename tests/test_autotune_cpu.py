"""The autotuner's host side (CPU only): the tuning knobs of the C ABI reject
values out of range before any device work, choices turn into call flags,
and the cache is plain JSON that survives a reload."""
import json

import pytest

from paper_1803_01237_gb300 import hss


def test_set_tuning_validates_and_round_trips():
    hss.reset_tuning()
    assert hss.get_tuning() == {"chip_max_keys": 4096, "child_interp": 0, "child_bucket_keys": 384, "pack_keys": 1024,
                                "first_split": 0, "split_scatter": 0}
    hss.set_tuning(14336, 1, 768, 2048, 1, 1)
    assert hss.get_tuning() == {"chip_max_keys": 14336, "child_interp": 1, "child_bucket_keys": 768, "pack_keys": 2048,
                                "first_split": 1, "split_scatter": 1}
    for bad in ((5000, 0, 0), (4096, 2, 0), (4096, 1, 64), (4096, 1, 5000), (4096, 0, 0, 5000), (4096, 0, 0, 0, 2),
                (4096, 0, 0, 0, 0, 2)):
        with pytest.raises(hss.HSSError):
            hss.set_tuning(*bad)
    assert hss.get_tuning()["chip_max_keys"] == 14336  # a refused call changes nothing
    hss.reset_tuning()
    assert hss.get_tuning()["chip_max_keys"] == 4096


def test_choice_flags_and_cache_file(tmp_path):
    from paper_1803_01237_gb300 import autotune
    c = autotune.Choice(oversample=8.0, hist_flags=hss.FLAG_HIST_STAGED, host_rounds=1)
    assert c.flags() == hss.FLAG_HIST_STAGED | hss.FLAG_HOST_ROUNDS
    s, flags = c.apply()
    assert s == 8.0 and flags == c.flags()
    hss.reset_tuning()
    path = tmp_path / "tuning.json"
    t = autotune.Tuner(str(path))
    t.cache["GPU|u64|n20|p6|uniform"] = {"choice": {"oversample": 3.0, "hist_flags": 0, "host_rounds": 0,
                                                     "chip_max_keys": 4096, "child_interp": 1,
                                                     "child_bucket_keys": 384}, "ms": 1.0}
    t.save()
    t2 = autotune.Tuner(str(path))
    assert t2.cache == json.load(open(path))
    assert autotune.Choice(**t2.cache["GPU|u64|n20|p6|uniform"]["choice"]).child_interp == 1


def test_default_space_tilings_map_to_choices():
    """Every tiling of the search space becomes a Choice whose knobs the C ABI
    accepts (3-tuples leave packing and the first split at their defaults)."""
    from paper_1803_01237_gb300 import autotune
    over, tiles = autotune.default_space(1024)
    assert 5.0 in over
    for t in tiles:
        c = autotune.Choice(oversample=5.0, **autotune._tiling_fields(t))
        assert (c.chip_max_keys, c.child_interp, c.child_bucket_keys) == tuple(t[:3])
        if len(t) > 3:
            assert (c.pack_keys, c.first_split) == tuple(t[3:5])
        s, flags = c.apply()
        assert hss.get_tuning()["first_split"] == c.first_split
        hss.reset_tuning()
    assert any(len(t) > 4 and t[4] == 1 for t in tiles)  # the sampled-splitter first split is searched
