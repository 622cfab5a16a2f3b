"""Host-side logic of the autotuner (no GPU): cache keys, selection, caching."""
from paper_2609_21204_b300 import autotune as at
from synth import assoc_ab


def test_cache_key_buckets():
    k1 = at.cache_key("B300", "mixed", 1_000_000, 1.59, 1)
    k2 = at.cache_key("B300", "mixed", 1_040_000, 1.61, 1)
    assert k1 == k2
    assert at.cache_key("B300", "fp64", 1_000_000, 1.59, 1) != k1
    assert at.cache_key("B300", "mixed", 1_000_000, 1.59, 256) != k1


def test_choose_fastest_and_skips_failures():
    trials = [({"block_size": 64, "skin": 0.3}, 0.5), ({"block_size": 128, "skin": 0.3}, None),
              ({"block_size": 256, "skin": 0.4}, 0.4), ({"block_size": 128, "skin": 0.4}, 0.4)]
    best = at.choose(trials)
    assert best["block_size"] == 256 and best["skin"] == 0.4 and best["ms_per_step"] == 0.4


def test_autotune_with_fake_timer_caches(tmp_path):
    s = assoc_ab(seed=1, n_a=50, n_b=50)
    calls = []

    def timer(cfg):
        calls.append(cfg)
        return 1.0 + abs(cfg["skin"] - 0.3) + cfg["block_size"] / 1000.0

    path = tmp_path / "tune.json"
    r = at.autotune(s, timer=timer, cache_path=path)
    assert r["block_size"] == 64 and r["skin"] == 0.3 and not r["cached"]
    n_trials = len(at.BLOCKS) * len(at.SKINS) + len(at.LIST_BLOCKS) - 1 + len(at.LIST_SUBCELLS) - 1
    assert len(calls) == n_trials
    r2 = at.autotune(s, timer=timer, cache_path=path)
    assert r2["cached"] and r2["block_size"] == 64
    assert len(calls) == n_trials


def test_autotune_searches_list_block_at_the_best_shape(tmp_path):
    """The list build's block size is searched after (block, skin), at the
    best of those; a faster list block wins, a slower one does not."""
    s = assoc_ab(seed=2, n_a=50, n_b=50)
    calls = []

    def timer(cfg):
        calls.append(cfg)
        return 1.0 + abs(cfg["skin"] - 0.4) + cfg["block_size"] / 1000.0 + {128: 0.01, 256: 0.0, 64: 0.02}[cfg["list_block"]]

    r = at.autotune(s, timer=timer, cache_path=tmp_path / "t.json")
    assert (r["block_size"], r["skin"], r["list_block"]) == (64, 0.4, 256)
    stage2 = calls[len(at.BLOCKS) * len(at.SKINS):][:len(at.LIST_BLOCKS) - 1]
    assert [c["list_block"] for c in stage2] == list(at.LIST_BLOCKS[1:])
    assert all((c["block_size"], c["skin"]) == (64, 0.4) for c in stage2)


def test_autotune_searches_list_subcells_after_the_list_block(tmp_path):
    """The sub-cells per cell are searched last, at the best (block, skin,
    list block); a faster choice wins."""
    s = assoc_ab(seed=3, n_a=50, n_b=50)
    calls = []

    def timer(cfg):
        calls.append(cfg)
        return (1.0 + abs(cfg["skin"] - 0.3) + cfg["block_size"] / 1000.0
                + {128: 0.0, 256: 0.01, 64: 0.02}[cfg["list_block"]] + {0: 0.01, 8: 0.0, 2: 0.02}[cfg["list_subcells"]])

    r = at.autotune(s, timer=timer, cache_path=tmp_path / "t.json")
    assert (r["block_size"], r["skin"], r["list_block"], r["list_subcells"]) == (64, 0.3, 128, 8)
    stage3 = calls[-(len(at.LIST_SUBCELLS) - 1):]
    assert [c["list_subcells"] for c in stage3] == list(at.LIST_SUBCELLS[1:])
    assert all((c["block_size"], c["skin"], c["list_block"]) == (64, 0.3, 128) for c in stage3)
