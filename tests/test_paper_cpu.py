"""The paper's own CPU method in float / double (oracle/paper_cpu.c) against exact arithmetic.

Not a parity test of this library: it records what the inexact method decides
differently, on the same snapped inputs, and checks the facts the comparison rests
on (inputs whose determinants are exactly representable give no differences;
tie-heavy inputs give many in float, and some in double when the products exceed
53 bits).
"""
import numpy as np
import pytest

import oracle
from paper_2106_01326_gb300 import meshgen as mg


def test_exactly_representable_inputs_agree(oracle_lib):
    """The unjittered 16^3 lattice at 64^3: every coordinate difference is a small multiple
    of s, so every product is exact in float and double and nothing may differ."""
    ijk, tets = mg.kuhn_lattice_int(16)
    xyz = (ijk * ((1 << 20) // 16)).astype(np.int32)
    d = oracle.paper_cpu_disagreements(xyz, tets, 64)
    assert d["tests"] > 1_000_000
    assert d["float_closed"] == d["float_strict"] == d["double_closed"] == d["double_strict"] == 0
    for mode in (0, 1):
        ex = oracle.voxelize_fixed(xyz, tets, 64, mode=mode)
        for prec in ("float", "double"):
            assert oracle.mismatches(oracle.paper_cpu(xyz, tets, 64, prec, mode), ex) == (0, 0)


def test_ties_break_float_and_double(oracle_lib):
    xyz, tets = mg.coplanar_face_soup(400, 64, seed=1, spread=60)
    d = oracle.paper_cpu_disagreements(xyz, tets, 64)
    assert d["float_closed"] > 0 and d["float_strict"] > 0
    assert d["double_closed"] > 0 and d["double_strict"] > 0
    assert d["float_closed"] > d["double_closed"]
    # at the grid level the float path loses closed samples on faces and keeps on-face samples
    # that the paper's own strict statement excludes
    closed = oracle.voxelize_fixed(xyz, tets, 64, mode=0)
    strict = oracle.voxelize_fixed(xyz, tets, 64, mode=1)
    assert oracle.mismatches(oracle.paper_cpu(xyz, tets, 64, "float", 0), closed)[1] > 0
    assert oracle.mismatches(oracle.paper_cpu(xyz, tets, 64, "float", 1), strict)[0] > 0


def test_counts_cover_every_box_sample(oracle_lib):
    """The disagreement counter visits exactly the samples of each tet's box (the oracle's
    count of samples tested) and rejects a bad slab."""
    ijk, tets = mg.kuhn_lattice_int(2)
    xyz = (ijk * (1 << 19)).astype(np.int32)
    g, st = oracle.voxelize_fixed(xyz, tets, 8, with_stats=True)
    d = oracle.paper_cpu_disagreements(xyz, tets, 8)
    assert d["tests"] == st["tested"]
    with pytest.raises(oracle.OracleError):
        oracle.paper_cpu_disagreements(xyz, tets, 8, z0=3, z1=2)
