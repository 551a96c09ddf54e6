"""Pins of the oracle's box cluster tree (Section 3.2, Alg. 1) and of its nearfield and
interaction lists (Section 3.3, Eq. 03:ILtemp, 03:Iarea, def_st_nearfield,
def_st_interaction_list)."""
import json
import os

import pytest

import oracle as O
from paper_2106_15911_gb300.inputs import cube_mesh

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_paper_example_temporal_lists():
    g = json.load(open(os.path.join(GOLD, "temporal_lists.json")))
    assert O.nearfield_list(g["interval"]) == g["nearfield"]
    assert O.interaction_list(g["interval"]) == g["interaction"]


def test_temporal_lists_small_cases():
    assert O.nearfield_list(0) == [0]
    assert O.interaction_list(0) == [] and O.interaction_list(1) == []
    assert O.interaction_list(2) == [0] and O.interaction_list(3) == [0, 1]
    for k in range(2, 64):
        js = O.interaction_list(k)
        # separated from k (dist(I, J) > 0) and the parents are temporal neighbours
        assert all(k - j >= 2 for j in js)
        assert all(k // 2 - j // 2 in (0, 1) for j in js)


@pytest.mark.parametrize("case", json.load(open(os.path.join(GOLD, "tree_shapes.json")))["cases"],
                         ids=lambda c: c["name"])
def test_tree_shape_matches_algorithm_1(case):
    V, T = cube_mesh(case["n_a"])
    P = O.make_problem(V, T, 1.0, case["Et"], c_st=case["c_st"])
    info = O.tree_info(P)
    assert info["p"] == case["p"]
    assert info["lx"] == case["lx"]
    assert info["nbox"] == case["nbox"]
    assert max(info["pad"]) == 0.0  # cube grids align with box faces: no padding needed
    if "m2l_pairs" in case:
        n = 0
        for l in range(2, info["p"] + 1):
            for k in range(1 << l):
                n += len(O.interaction_list(k)) * info["nbox"][l] ** 2
        assert n == case["m2l_pairs"]


@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_every_causal_step_pair_is_covered_exactly_once(p):
    """Nearfield at the leaves plus M2L on the ancestor chain cover each pair (k_t >= j_t) once
    and no acausal pair (Alg. 2 with the lists of Eq. 03:ILtemp)."""
    ls = 2
    Et = ls << p
    for kt in range(Et):
        for jt in range(Et):
            ip, jp = kt // ls, jt // ls
            cover = 0
            if jp in O.nearfield_list(ip):
                cover += 1
            far = 0
            for l in range(2, p + 1):
                il, jl = ip >> (p - l), jp >> (p - l)
                if jl in O.interaction_list(il):
                    far += 1
            if jt <= kt:
                assert cover + far == 1, (kt, jt)
            else:
                assert far == 0


def test_padding_grows_with_coarser_levels_on_a_sphere():
    from paper_2106_15911_gb300.inputs import cube_sphere_mesh

    V, T = cube_sphere_mesh(8)
    P = O.make_problem(V, T, 1.0, 64, c_st=0.25)
    info = O.tree_info(P)
    pad = info["pad"]
    assert all(pad[l] >= pad[l + 1] for l in range(len(pad) - 1))
    assert pad[-1] > 0.0
