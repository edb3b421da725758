"""The C-ABI library: it builds, loads, exports every symbol include/gpm.h
declares, and its host-only logic (pattern dictionary, argument checks)
behaves -- no GPU needed."""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest

from oracle import oracle as O
from paper_2212_04551_gb300 import gpm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gpm.h")
GOLDEN = os.path.join(ROOT, "tests", "golden", "graph_classes.txt")


def declared_symbols() -> list[str]:
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:gpm_status|void|const\s+char\s*\*)\s*(gpm_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    return gpm.load()


def test_every_declared_symbol_is_exported(lib):
    syms = declared_symbols()
    assert len(syms) >= 12
    for name in syms:
        assert hasattr(lib, name), f"{name} declared in gpm.h but not exported"
        assert name in gpm.SIGNATURES, f"{name} has no Python binding"
    # and nothing the binding wraps is missing from the header
    assert set(gpm.SIGNATURES) <= set(syms)


def _golden_connected():
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        k, c, _ = (int(x) for x in line.split())
        out[k] = c
    return out


def test_pattern_counts_match_oeis(lib):
    golden = _golden_connected()
    for k in range(1, gpm.GPM_MOTIF_MAX_K + 1):
        assert gpm.gpm_motif_num_patterns(k) == golden[k]


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7, 8])
def test_pattern_codes_are_canonical_and_ordered(lib, k):
    """Each id's code is the smallest code of its class (checked with the
    oracle's relabelling-minimum), connected, distinct, and the ids are
    ordered by (edge count, code)."""
    npat = gpm.gpm_motif_num_patterns(k)
    codes = [gpm.gpm_motif_pattern(k, p) for p in range(npat)]
    assert len(set(codes)) == npat
    keys = [(bin(c).count("1"), c) for c in codes]
    assert keys == sorted(keys)
    if k <= 6:
        assert codes == sorted(O.classes(k, True), key=lambda c: (bin(c).count("1"), c))
    canon = O.canon_many(k, codes)
    assert [int(x) for x in canon] == codes
    for c in codes:
        assert O.code_connected(k, c)


def test_argument_errors_without_gpu(lib):
    with pytest.raises(gpm.GpmError) as e:
        gpm.gpm_motif_num_patterns(0)
    assert e.value.status == gpm.GPM_EINVAL
    with pytest.raises(gpm.GpmError) as e:
        gpm.gpm_motif_pattern(4, 6)
    assert e.value.status == gpm.GPM_EINVAL
    assert "out of range" in gpm.gpm_last_error()
    # NULL graph handle
    assert lib.gpm_graph_info(None, None, None, None) == gpm.GPM_EINVAL
    out = ctypes.c_uint64()
    assert lib.gpm_clique_count(None, 3, ctypes.byref(out)) == gpm.GPM_EINVAL
    # host-side CSR checks happen before any device work
    with pytest.raises(gpm.GpmError) as e:
        gpm.gpm_graph_create(np.array([1, 2], dtype=np.int32), np.array([0, 0], dtype=np.int32), 1)
    assert e.value.status == gpm.GPM_EINVAL
    with pytest.raises(gpm.GpmError) as e:
        gpm.gpm_graph_create(np.array([0, 1], dtype=np.int32), np.array([0], dtype=np.int32), 1)
    assert e.value.status == gpm.GPM_EINVAL   # odd number of adjacency entries
    with pytest.raises(gpm.GpmError) as e:
        gpm.gpm_graph_create(np.array([0], dtype=np.int32), np.array([], dtype=np.int32), -1)
    assert e.value.status == gpm.GPM_EINVAL
    gpm.gpm_graph_destroy(gpm.Graph(0))      # NULL-safe


def test_no_oracle_in_library():
    """The CUDA sources and the binding never include or import the oracle."""
    pkg = os.path.join(ROOT, "paper_2212_04551_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                for pat in ("import oracle", "from oracle", "gpm_oracle", "orc_"):
                    assert pat not in txt, (f, pat)
