"""The C-ABI library loads, exports every symbol include/gpm.h declares, and
its host-side planner (no GPU needed) derives the right pattern facts."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2011_03135_b300 import build
    build.build()
    from paper_2011_03135_b300 import gpm
    return gpm


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"^\s*(?:int|uint64_t|const char \*|const char\*)\s*(gpm_\w+)\s*\(", txt, flags=re.M))
    return names


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 15
    so = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in sorted(names) if not hasattr(so, n)]
    assert not missing, missing


def test_version_and_errors_without_gpu(lib):
    assert "sm_103a" in lib.version()
    with pytest.raises(lib.GpmError) as e:
        lib.Pattern.spec(np.array([[0, 1, 0], [1, 0, 0], [0, 0, 0]]))
    assert e.value.name == "DISCONNECTED_PATTERN"
    with pytest.raises(lib.GpmError) as e:
        lib.Pattern.spec(np.array([[0, 1], [0, 0]]))
    assert e.value.name == "INVALID_ARG"
    with pytest.raises(lib.GpmError) as e:
        lib.Pattern.clique(9)
    assert e.value.name == "K_TOO_LARGE"


def test_count_cliques_validates_before_any_device_work(lib):
    # a null graph handle and a null output are rejected on the host
    so = ctypes.CDLL(lib.LIB_PATH)
    so.gpm_count_cliques.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                     ctypes.c_void_p, ctypes.c_void_p]
    out = ctypes.c_uint64(0)
    invalid = so.gpm_count_cliques(None, 7, 0, 0, ctypes.byref(out), None)
    assert invalid != 0
    assert so.gpm_count_cliques(None, 7, 0, 0, None, None) == invalid


def test_orientation_and_existence_validate_on_the_host(lib):
    # null handles and outputs are rejected before any device work
    so = ctypes.CDLL(lib.LIB_PATH)
    so.gpm_graph_set_orientation.argtypes = [ctypes.c_void_p, ctypes.c_uint32]
    so.gpm_graph_core_numbers.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    so.gpm_exists.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert so.gpm_graph_set_orientation(None, 1) != 0
    assert so.gpm_graph_core_numbers(None, None, None) != 0
    found = ctypes.c_int(7)
    assert so.gpm_exists(None, None, ctypes.byref(found), None, None) != 0
    assert found.value == 7  # untouched on error


@pytest.mark.parametrize("idx", range(6))
def test_planner_motif4(lib, idx):
    pats = lib.Pattern.motifs(4)
    info = pats[idx].info()
    adj = O.MOTIF4_PATTERNS[idx]
    assert info["motif_index"] == idx
    assert info["automorphisms"] == O.automorphisms(adj)
    # the constraints leave exactly one vertex order per distinct subgraph
    assert O.orders_satisfying(4, info["sb_pairs"]) * info["automorphisms"] == math.factorial(4)
    assert info["min_degree"] == [int(x) for x in adj.sum(axis=1)]
    assert sorted(info["matching_order"]) == [0, 1, 2, 3]


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7, 8])
def test_planner_cliques(lib, k):
    info = lib.Pattern.clique(k).info()
    assert info["automorphisms"] == math.factorial(k)
    assert info["is_clique"] == 1
    assert O.orders_satisfying(k, info["sb_pairs"]) == 1
    if k >= 3:
        assert info["strategy"] == lib.STRATEGY_CLIQUE_DAG


def test_planner_diamond_matching_order_is_triangle_first(lib):
    # appendix "Pattern-Guided Search": the diamond is matched triangle first,
    # starting with the two degree-3 vertices that carry a partial order
    info = lib.Pattern.spec(O.DIAMOND, induced=False).info()
    mo = info["matching_order"]
    assert set(mo[:2]) == {0, 1}
    assert (0, 1) in info["sb_pairs"] and (2, 3) in info["sb_pairs"]
    assert info["strategy"] == lib.STRATEGY_LOCAL_COUNT


def test_planner_other_numberings(lib):
    # diamond with the shared edge on vertices 2,3; 4-cycle 0-1-2-3-0
    d = O.pattern(4, [(2, 3), (2, 0), (2, 1), (3, 0), (3, 1)])
    c = O.pattern(4, [(0, 1), (1, 2), (2, 3), (3, 0)])
    for a in (d, c):
        info = lib.Pattern.spec(a, induced=False).info()
        assert O.orders_satisfying(4, info["sb_pairs"]) * info["automorphisms"] == 24


def test_planner_five_vertex_pattern(lib):
    # a 5-vertex house: counted by the pattern-oblivious enumeration
    house = O.pattern(5, [(0, 1), (1, 2), (2, 3), (3, 0), (0, 4), (1, 4)])
    info = lib.Pattern.spec(house).info()
    assert info["automorphisms"] == O.automorphisms(house)
    assert O.orders_satisfying(5, info["sb_pairs"]) * info["automorphisms"] == 120
    assert info["strategy"] == lib.STRATEGY_ENUMERATE and info["motif_index"] < 21


def _connected_patterns(kmin, kmax):
    import networkx as nx
    for G in nx.graph_atlas_g():
        k = G.number_of_nodes()
        if kmin <= k <= kmax and nx.is_connected(G):
            yield k, G.number_of_edges(), nx.to_numpy_array(G, dtype=np.uint8)


def test_planner_every_connected_pattern_up_to_7_vertices(lib):
    # appendix "Symmetry Breaking (Partial Order)" and "Pattern-Guided Search
    # (Matching Order)", Section 4.3: over all 994 connected patterns of 3..7
    # vertices (the networkx graph atlas), |Aut| equals the brute-force count,
    # the partial order leaves exactly one of the |Aut| equivalent vertex
    # orders, every vertex of the matching order after the first has a matched
    # neighbour before it, and the degree filter is the pattern degree
    seen = 0
    for k, m, a in _connected_patterns(3, 7):
        aut = O.automorphisms(a)
        for induced in (True, False):
            info = lib.Pattern.spec(a, induced=induced).info()
            assert info["automorphisms"] == aut
            assert O.orders_satisfying(k, info["sb_pairs"]) * aut == math.factorial(k)
            mo = info["matching_order"]
            assert sorted(mo) == list(range(k))
            assert all(any(a[mo[j], mo[i]] for i in range(j)) for j in range(1, k))
            assert info["min_degree"] == [int(x) for x in a.sum(axis=1)]
            clique = m == k * (k - 1) // 2
            want = (lib.STRATEGY_CLIQUE_DAG if clique else lib.STRATEGY_LOCAL_COUNT if k <= 4
                    else lib.STRATEGY_ENUMERATE if k == 5 else lib.STRATEGY_GUIDED)
            assert info["strategy"] == want
        seen += 1
    assert seen == 2 + 6 + 21 + 112 + 853


def test_planner_random_eight_vertex_patterns(lib):
    import networkx as nx
    rng = np.random.default_rng(8)
    seen = 0
    while seen < 60:
        G = nx.gnp_random_graph(8, float(rng.uniform(0.25, 0.8)), seed=int(rng.integers(1 << 30)))
        if not nx.is_connected(G):
            continue
        a = nx.to_numpy_array(G, dtype=np.uint8)
        info = lib.Pattern.spec(a, induced=False).info()
        aut = O.automorphisms(a)
        assert info["automorphisms"] == aut
        assert O.orders_satisfying(8, info["sb_pairs"]) * aut == 40320
        mo = info["matching_order"]
        assert sorted(mo) == list(range(8))
        assert all(any(a[mo[j], mo[i]] for i in range(j)) for j in range(1, 8))
        seen += 1


def test_options_roundtrip(lib):
    old = lib.get_options()
    lib.set_options(warp_max_degree=64, cta_max_degree=512)
    assert lib.get_options()["warp_max_degree"] == 64
    with pytest.raises(lib.GpmError):
        lib.set_options(warp_max_degree=8)
    assert old["c4_hub_bound"] == 1048576
    lib.set_options(c4_hub_bound=4000)
    assert lib.get_options()["c4_hub_bound"] == 4000
    for bad in (512, 1048577):
        with pytest.raises(lib.GpmError):
            lib.set_options(c4_hub_bound=bad)
    assert old["batch_direct_us"] == 1000
    lib.set_options(batch_direct_us=5)
    assert lib.get_options()["batch_direct_us"] == 5
    assert old["c4_range_bound"] == 1048576 and old["c4_range_width"] == 98304
    lib.set_options(c4_range_bound=0xffffffff, c4_range_width=512)
    assert lib.get_options()["c4_range_bound"] == 0xffffffff
    assert lib.get_options()["c4_range_width"] == 512
    assert old["c4_pull_bound"] == 262144
    lib.set_options(c4_pull_bound=600)
    assert lib.get_options()["c4_pull_bound"] == 600
    for bad in (dict(c4_range_bound=100), dict(c4_range_width=63), dict(c4_range_width=98306),
                dict(c4_range_width=1001), dict(c4_pull_bound=511)):
        with pytest.raises(lib.GpmError):
            lib.set_options(**bad)
    # a call with one invalid field applies none of its fields
    before = lib.get_options()
    with pytest.raises(lib.GpmError):
        lib.set_options(warp_max_degree=96, c4_hub_bound=2000, c4_pull_bound=511)
    assert lib.get_options() == before
    lib.set_options(**{k: v for k, v in old.items() if v})


def test_binding_structs_match_the_header(lib, tmp_path):
    # every struct the binding passes through the ABI has the header's size
    # and field offsets (compiled here with the host C compiler)
    import subprocess
    pairs = {"gpm_graph_info_t": lib.GraphInfo, "gpm_pattern_info_t": lib.PatternInfo, "gpm_query_t": lib.Query,
             "gpm_server_opts_t": lib.ServerOpts, "gpm_completion_t": lib.Completion, "gpm_options_t": lib.Options}
    lines = ['#include <stdio.h>', '#include "gpm.h"', "int main(void) {"]
    for cname, py in pairs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'  printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        cname, field, value = line.split()
        got[(cname, field)] = int(value)
    for cname, py in pairs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for field, _ in py._fields_:
            assert got[(cname, field)] == getattr(py, field).offset, (cname, field)


def test_binding_declares_every_call_with_the_header_arity(lib):
    # each call of include/gpm.h is declared in the binding with as many
    # arguments as its prototype has
    txt = ""
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt += open(os.path.join(ROOT, "include", h)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    protos = re.findall(r"^\s*(?:int|uint64_t|const char\s*\*)\s*(gpm_\w+)\s*\(([^;]*?)\)\s*;", txt,
                        flags=re.M | re.S)
    assert len(protos) == len(_declared())
    for name, args in protos:
        args = args.strip()
        arity = 0 if args in ("", "void") else args.count(",") + 1
        declared = getattr(lib._lib, name).argtypes
        assert declared is not None, name
        assert len(declared) == arity, (name, arity, len(declared))


def test_binding_constants_match_the_header(lib):
    txt = open(os.path.join(ROOT, "include", "gpm.h")).read()
    codes = {name: int(v) for name, v in re.findall(r"#define GPM_E_(\w+) \((-\d+)\)", txt)}
    assert codes == {name: code for code, name in lib.ERRORS.items()}
    defs = {name: int(v) for name, v in re.findall(r"#define GPM_(\w+) (\d+)u?\b", txt)}
    for name in ("GRAPH_VALIDATE", "GRAPH_DEVICE_INPUT", "STRATEGY_CLIQUE_DAG", "STRATEGY_LOCAL_COUNT",
                 "STRATEGY_EDGE", "STRATEGY_ENUMERATE", "STRATEGY_GUIDED", "QUERY_MOTIF3", "QUERY_MOTIF4",
                 "QUERY_TC", "QUERY_CLIQUE4", "QUERY_CLIQUE5"):
        assert getattr(lib, name) == defs[name], name
