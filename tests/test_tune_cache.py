"""The autotuner's cache as the library reads it (no GPU): the mesh key and
hqn_tune_lookup, on cache lines written by autotune.cache_line."""
import os
import shutil

import numpy as np
import pytest

from paper_1604_07378_gb300 import workloads as W

pytestmark = pytest.mark.skipif(
    shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
    reason="needs the CUDA toolkit to build the library")

DEV = "NVIDIA GB300"


@pytest.fixture(scope="module")
def at():
    from paper_1604_07378_gb300 import autotune, build
    build.build_library()
    return autotune


def _choice(leaf, t, kb, n, pf, top=0, lkb=0, lt=0, dp=0):
    return {"leaf_size": leaf, "solve_dense_top": top, "solve_threads": t, "solve_item_kb": kb, "solve_items": n,
            "solve_prefetch": pf, "solve_leaf_kb": lkb, "solve_leaf_threads": lt, "solve_dense_prefetch": dp}


def test_mesh_key_identifies_the_mesh(at):
    w = W.lattice_workload((3, 2, 4), W.Material(W.NEOHOOKEAN, 1e5, 0.4))
    k = at.mesh_key(w.rest_pos, w.tets, w.clamped)
    assert k != 0 and k == at.mesh_key(w.rest_pos.copy(), w.tets.copy(), w.clamped.copy())
    cl = w.clamped.copy()
    cl[-1] ^= 1
    X = w.rest_pos.copy()
    X[5, 1] += 1e-9
    T = w.tets.copy()
    T[0, [2, 3]] = T[0, [3, 2]]
    assert len({k, at.mesh_key(w.rest_pos, w.tets, cl), at.mesh_key(X, w.tets, w.clamped),
                at.mesh_key(w.rest_pos, T, w.clamped), at.mesh_key(w.rest_pos, w.tets, None)}) == 5


def test_lookup_hits_misses_and_overrides(at, tmp_path):
    path = str(tmp_path / "cache.txt")
    assert at.lookup(path, DEV, 123, 1) is None  # no file yet
    lines = ["# tuned on a GB300",
             at.cache_line(DEV, 1, 123, _choice(128, 512, 96, 152, 3, 3, 24, 128, 1), step_ms=2.0, workload="cube40"),
             at.cache_line(DEV, 0, 123, _choice(64, 256, 64, 400, 2)),
             at.cache_line("Other GPU", 1, 123, _choice(256, 256, 32, 800, -1)),
             at.cache_line(DEV, 1, 999, _choice(256, 256, 32, 800, 1))]
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")
    assert at.lookup(path, DEV, 123, 1) == {**_choice(128, 512, 96, 152, 3, 3, 24, 128, 1), "ls_batch": 8}
    assert at.lookup(path, DEV, 123, 0) == {**_choice(64, 256, 64, 400, 2), "ls_batch": 8}
    assert at.lookup(path, "Other GPU", 123, 1)["solve_prefetch"] == -1
    assert at.lookup(path, DEV, 124, 1) is None
    # a later line for the same key wins
    with open(path, "a") as f:
        f.write(at.cache_line(DEV, 1, 123, _choice(64, 256, 48, 304, 1)) + "\n")
    assert at.lookup(path, DEV, 123, 1)["solve_item_kb"] == 48


@pytest.mark.parametrize("bad", ["hqn-tune 2 device=X precision=1 key=%016x leaf_size=64 solve_threads=256 "
                                 "solve_item_kb=64 solve_items=400 solve_prefetch=2",
                                 "hqn-tune 1 device=X precision=1 key=%016x leaf_size=64 solve_threads=256",
                                 "hqn-tune 1 device=X precision=1 key=%016x leaf_size=64 solve_threads=256 "
                                 "solve_item_kb=64 solve_items=400 solve_prefetch=99",
                                 "tuned: leaf 64"])
def test_malformed_cache_is_an_error(at, tmp_path, bad):
    from paper_1604_07378_gb300 import hqn
    path = str(tmp_path / "cache.txt")
    with open(path, "w") as f:
        f.write((bad % 7 if "%" in bad else bad) + "\n")
    with pytest.raises(hqn.HQNError) as e:
        at.lookup(path, "X", 7, 1)
    assert e.value.code == hqn.HQN_ERR_ARG


def test_committed_cache_parses(at):
    """The cache shipped with the package is well formed."""
    if os.path.exists(at.DEFAULT_CACHE):
        at.lookup(at.DEFAULT_CACHE, DEV, 0, 1)


def test_entry_with_library_defaults_and_a_tuned_ls_batch(at, tmp_path):
    """An entry that keeps the library's size-dependent defaults (zeros) and
    tunes only the line search's trials per pass."""
    path = str(tmp_path / "cache.txt")
    choice = {**_choice(0, 0, 0, 0, 0), "ls_batch": 4}
    with open(path, "w") as f:
        f.write(at.cache_line(DEV, 1, 77, choice, step_ms=1.0) + "\n")
    assert at.lookup(path, DEV, 77, 1) == {**_choice(0, 0, 0, 0, 0), "ls_batch": 4}
