"""Host-side logic of the autotuner: cache keys separate problem shapes,
shot counts, density, kernel kinds and apertures, and the JSON cache
round-trips atomically (no GPU needed)."""
import json
import os
import subprocess
import sys

import numpy as np

from paper_2502_12350_gb300 import autotune, mamute


def test_keys_separate_problems():
    g = mamute.make_grid(64, 48, 32, 8, 10.0, 1e-3, 100)
    k = autotune.key(g, 1, False, "fwd")
    assert k == "fwd:80x64x48:s1:d0:full"
    assert autotune.key(g, 2, False, "fwd") != k
    assert autotune.key(g, 1, True, "fwd") != k
    assert autotune.key(g, 1, False, "adj-1") != k
    ap1 = np.array([[0, 32, 0, 16]], np.int32)
    ap2 = np.array([[4, 36, 0, 16]], np.int32)
    assert autotune.key(g, 1, False, "fwd", ap1) != autotune.key(g, 1, False, "fwd", ap2)
    assert autotune.key(g, 1, False, "fwd", ap1) == autotune.key(g, 1, False, "fwd", ap1.copy())


def test_cache_round_trip(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "tiles.json"
    monkeypatch.setenv("MAMUTE_AUTOTUNE_CACHE", str(path))
    assert autotune._load() == {}
    autotune._store({"fwd:1": {"tiles": [64, 16, 2, 0, 0, 0], "ms_per_step": 0.3}})
    assert json.load(open(path))["fwd:1"]["tiles"] == [64, 16, 2, 0, 0, 0]
    assert autotune._load()["fwd:1"]["ms_per_step"] == 0.3
    path.write_text("{not json")
    assert autotune._load() == {}  # a damaged cache is ignored, not fatal


def test_aperture_key_stable_across_processes():
    """The key of an aperture workload is the same in processes with
    different hash salts (PYTHONHASHSEED), so the cache is reused."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import numpy as np; from paper_2502_12350_gb300 import autotune, mamute; "
            "g = mamute.make_grid(64, 48, 32, 8, 10.0, 1e-3, 100); "
            "print(autotune.key(g, 2, False, 'adj-1', np.array([[0, 32, 0, 16], [4, 36, 8, 40]], np.int32)))")
    keys = set()
    for seed in ("1", "2", "12345"):
        env = dict(os.environ, PYTHONHASHSEED=seed, PYTHONPATH=root)
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                             check=True, cwd=root).stdout.strip()
        keys.add(out)
    assert len(keys) == 1, keys
    g = mamute.make_grid(64, 48, 32, 8, 10.0, 1e-3, 100)
    here = autotune.key(g, 2, False, "adj-1", np.array([[0, 32, 0, 16], [4, 36, 8, 40]], np.int32))
    assert keys == {here}
