"""Host-side logic of the autotuner (CPU): the z-block candidates it times and its JSON cache."""
import json

from paper_1901_09593_gb300 import autotune


def test_zblock_candidates():
    for sx in (1, 2, 4):
        limit = ((256 - 32 * sx - 32) // 32) * 32          # the staged right span fits 256 columns
        for dk in (1, 31, 32, 33, 40, 100, 1000):
            opts = autotune._zblock_options(sx, dk)
            assert opts and all(z % 32 == 0 and 32 <= z <= max(32, limit) for z in opts)
            # no block wider than needed: the largest option covers at most dk + 31 candidates
            assert max(opts) < dk + 32 or opts == [32]
            assert opts == sorted(set(opts))
    assert autotune._zblock_options(1, 40) == [32, 64]
    assert autotune._zblock_options(1, 1000) == [32, 64, 96, 128, 160, 192]
    assert autotune._zblock_options(4, 1000) == [32, 64, 96]


def test_cache_roundtrip_and_damaged_files(tmp_path):
    path = str(tmp_path / "sub" / "cache.json")
    assert autotune._load_cache(path) == {}                 # missing
    autotune._save_cache(path, {"k": {"sx": 2, "zblock": 64}})
    assert autotune._load_cache(path) == {"k": {"sx": 2, "zblock": 64}}
    assert json.load(open(path)) == {"k": {"sx": 2, "zblock": 64}}
    with open(path, "w") as f:
        f.write("{not json")
    assert autotune._load_cache(path) == {}                 # damaged: start afresh
