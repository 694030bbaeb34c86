"""Host-side set-up through the C ABI without a GPU (hqn_analyse): mesh
counts, the fitted stiffness against the oracle, the factor's size against
A0's own nonzeros, the default leaf-size rule, supernode amalgamation and
the rejection of bad input."""
import os
import shutil

import numpy as np
import pytest

from oracle import hqn_oracle as O
from paper_1604_07378_gb300 import workloads as W

pytestmark = pytest.mark.skipif(
    shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
    reason="needs the CUDA toolkit to build the library")

FP64, FP32 = 0, 1


@pytest.fixture(scope="module")
def hqn():
    from paper_1604_07378_gb300 import build, hqn as H
    build.build_library()
    return H


@pytest.fixture(scope="module")
def lat12():
    return W.lattice_workload((12, 12, 12), W.Material(W.NEOHOOKEAN, 5e5, 0.4), name="lat12")


def test_counts_stiffness_and_factor_size(hqn, lat12):
    w = lat12
    P = O.problem_from_workload(w)
    for prec in (FP64, FP32):
        a = hqn.analyse_workload(w, precision=prec)
        assert a["n_verts"] == w.n_verts and a["n_tets"] == w.n_tets
        assert a["n_free"] == int((~w.clamped.astype(bool)).sum())
        assert a["precision"] == prec and a["n_sims"] == 1 and a["device_bytes"] == 0
        # Eq. stiffness: the same least-squares slope as the oracle's fit
        assert abs(a["stiffness_k"] - P.k) <= 1e-9 * P.k
        # L holds at least the lower triangle of A0 on the free vertices
        A = O.assemble_A(P)
        assert a["factor_nnz"] >= (A.nnz + A.shape[0]) // 2
        # every free vertex is a column of exactly one supernode
        assert 1 <= a["n_levels"] <= a["n_supernodes"] <= a["n_free"]


def test_default_leaf_size_rule(hqn, lat12):
    """0 = 128-vertex leaves in FP32 up to 150,000 free vertices, else 64."""
    def key(a):
        return a["n_supernodes"], a["n_levels"], a["factor_nnz"]
    w = lat12
    assert key(hqn.analyse_workload(w, precision=FP32)) == key(hqn.analyse_workload(w, precision=FP32, leaf_size=128))
    assert key(hqn.analyse_workload(w, precision=FP64)) == key(hqn.analyse_workload(w, precision=FP64, leaf_size=64))
    assert key(hqn.analyse_workload(w, precision=FP32, leaf_size=64)) != key(hqn.analyse_workload(w, precision=FP32))
    # a long bar of 160,752 vertices (160,480 free): 64 in both forms
    big = W.lattice_workload((590, 16, 15), W.Material(W.NEOHOOKEAN, 5e5, 0.4), name="bar590")
    a = hqn.analyse_workload(big, precision=FP32)
    assert a["n_free"] > 150000
    assert key(a) == key(hqn.analyse_workload(big, precision=FP32, leaf_size=64))


def test_merge_depths_shorten_the_chain(hqn, lat12):
    w = lat12
    for prec in (FP64, FP32):
        a0, a1, a5 = (hqn.analyse_workload(w, precision=prec, merge_depths=m) for m in (0, 1, 5))
        assert a1["n_levels"] == a0["n_levels"] - 1 and a5["n_levels"] == a0["n_levels"] - 2
        assert a1["n_supernodes"] == a0["n_supernodes"] - 2
        assert a0["factor_nnz"] < a1["factor_nnz"] < a5["factor_nnz"]
    with pytest.raises(hqn.HQNError) as e:
        hqn.analyse_workload(w, merge_depths=6)
    assert e.value.code == hqn.HQN_ERR_ARG


def test_rejects_degenerate_and_bad_input(hqn, lat12):
    w = lat12
    X = w.rest_pos.copy()
    t0 = w.tets[0]
    X[t0[3]] = X[t0[0]]  # collapse one rest tetrahedron
    with pytest.raises(hqn.HQNError) as e:
        hqn.analyse(X, w.tets, w.clamped, kind=W.NEOHOOKEAN, E=5e5, nu=0.4)
    assert e.value.code == hqn.HQN_ERR_DEGENERATE_TET
    with pytest.raises(hqn.HQNError) as e:
        hqn.analyse_workload(w, precision=7)
    assert e.value.code == hqn.HQN_ERR_ARG
    assert hqn.MAX_HISTORY == 128  # the paper's convergence study runs m = 100
    hqn.analyse_workload(w, history_m=hqn.MAX_HISTORY)
    for kw in (dict(ls_batch=3), dict(history_m=hqn.MAX_HISTORY + 1), dict(history_m=-1), dict(h=0.0),
               dict(gamma=1.0)):
        with pytest.raises(hqn.HQNError) as e:
            hqn.analyse_workload(w, **kw)
        assert e.value.code == hqn.HQN_ERR_ARG, kw
    for E, nu in ((-1.0, 0.4), (5e5, 0.5), (5e5, -1.0)):
        with pytest.raises(hqn.HQNError) as e:
            hqn.analyse(w.rest_pos, w.tets, w.clamped, kind=W.NEOHOOKEAN, E=E, nu=nu)
        assert e.value.code == hqn.HQN_ERR_ARG, (E, nu)
    for X0, T0 in ((np.zeros((0, 3)), np.zeros((0, 4), np.int32)), (w.rest_pos, np.zeros((0, 4), np.int32))):
        with pytest.raises(hqn.HQNError) as e:  # no vertices, or no tets
            hqn.analyse(X0, T0, kind=W.NEOHOOKEAN, E=5e5, nu=0.4)
        assert e.value.code == hqn.HQN_ERR_ARG
    X = w.rest_pos.copy()
    X[5, 1] = np.nan
    with pytest.raises(hqn.HQNError) as e:
        hqn.analyse(X, w.tets, w.clamped, kind=W.NEOHOOKEAN, E=5e5, nu=0.4)
    assert e.value.code == hqn.HQN_ERR_NONFINITE
    tets = w.tets.copy()
    tets[0, 0] = w.n_verts  # vertex index out of range
    with pytest.raises(hqn.HQNError) as e:
        hqn.analyse(w.rest_pos, tets, w.clamped, kind=W.NEOHOOKEAN, E=5e5, nu=0.4)
    assert e.value.code == hqn.HQN_ERR_ARG
    with pytest.raises(hqn.HQNError) as e:
        hqn.analyse(w.rest_pos, w.tets, np.ones(w.n_verts, np.uint8), kind=W.NEOHOOKEAN, E=5e5, nu=0.4)
    assert e.value.code == hqn.HQN_ERR_ARG


def test_collider_parameters_are_checked(hqn):
    """The parameter checks sim_create shares with the analysis: a torus
    needs 0 < tube radius < ring radius and a nonzero axis; a sphere a
    positive radius; a plane a nonzero normal."""
    w = W.collision_drop(2, torus=True)
    assert hqn.analyse_workload(w)["n_free"] == w.n_verts  # the drop is unclamped
    bad = [W.Collider("torus", (0.0, 0.0, 0.0), (0.0, 0.0, 1.0), radius=0.2, major=0.1),
           W.Collider("torus", (0.0, 0.0, 0.0), (0.0, 0.0, 0.0), radius=0.1, major=0.2),
           W.Collider("sphere", (0.0, 0.0, 0.0), radius=0.0),
           W.Collider("plane", (0.0, 0.0, 0.0), (0.0, 0.0, 0.0))]
    for c in bad:
        with pytest.raises(hqn.HQNError) as e:
            hqn.analyse_workload(w, colliders=(c,))
        assert e.value.code == hqn.HQN_ERR_ARG, c


def test_non_spd_and_material_table_errors(hqn, lat12):
    """A negative density makes A0 = M/h^2 + L indefinite: HQN_ERR_NOT_SPD
    from the host set-up.  A per-tet material index outside the mesh's
    material table, or too many materials, is HQN_ERR_ARG."""
    w = lat12
    with pytest.raises(hqn.HQNError) as e:
        hqn.analyse(w.rest_pos, w.tets, w.clamped, kind=W.NEOHOOKEAN, E=5e5, nu=0.4, density=-1000.0)
    assert e.value.code == hqn.HQN_ERR_NOT_SPD
    b = W.Material(W.STVK, 6e5, 0.35)
    tm = np.zeros(w.n_tets, np.int32)
    tm[3] = 2  # two materials: indices 0 and 1 only
    with pytest.raises(hqn.HQNError) as e:
        hqn.analyse(w.rest_pos, w.tets, w.clamped, kind=W.NEOHOOKEAN, E=5e5, nu=0.4, extra_materials=(b,),
                    tet_material=tm)
    assert e.value.code == hqn.HQN_ERR_ARG
    with pytest.raises(hqn.HQNError) as e:
        hqn.analyse(w.rest_pos, w.tets, w.clamped, kind=W.NEOHOOKEAN, E=5e5, nu=0.4,
                    extra_materials=(b,) * hqn.MAX_MATERIALS, tet_material=np.zeros(w.n_tets, np.int32))
    assert e.value.code == hqn.HQN_ERR_ARG
    tm[3] = 1
    a = hqn.analyse(w.rest_pos, w.tets, w.clamped, kind=W.NEOHOOKEAN, E=5e5, nu=0.4, extra_materials=(b,),
                    tet_material=tm)
    assert a["n_tets"] == w.n_tets
