"""Python face of the CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this module.  The CUDA library never imports or links it, and
it imports nothing from the CUDA package (the two share no code; only the
seeded graph generators serve both).

``gpm_oracle.c`` is compiled with gcc on first use (or by ``build()``) into
``oracle/_build/``.  Every function here is marshalling only: the counting is
the C code, which restates the paper's Eq. 1 and Algorithm 4.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gpm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libgpm_oracle.so")
_lock = threading.Lock()
_lib = None

ORDER_ID = 0
ORDER_DEGREE = 1

_i32p = ctypes.POINTER(ctypes.c_int32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, -O2, portable: no -march flags)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    # -mpopcnt on x86-64 only speeds up the bitset route (hardware population
    # count); the results are the same on every machine
    extra = ["-mpopcnt"] if platform.machine() in ("x86_64", "AMD64") else []
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared"] + extra + ["-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_clique_count.argtypes = [ctypes.c_int32, _i32p, _i32p, ctypes.c_int, ctypes.c_int,
                                             _i32p, ctypes.c_int64, _u64p, _u64p]
            lib.orc_clique_count.restype = ctypes.c_int
            lib.orc_motif_count.argtypes = [ctypes.c_int32, _i32p, _i32p, ctypes.c_int, _i32p,
                                            ctypes.c_int64, ctypes.c_int64, _u64p, _u64p, _u64p,
                                            _i64p, _u64p, _u64p]
            lib.orc_motif_count.restype = ctypes.c_int
            lib.orc_motif_count_esu.argtypes = lib.orc_motif_count.argtypes
            lib.orc_motif_count_esu.restype = ctypes.c_int
            lib.orc_brute_force.argtypes = [ctypes.c_int32, _i32p, _i32p, ctypes.c_int, ctypes.c_int64,
                                            _u64p, _u64p, _u64p, _u8p, _i64p]
            lib.orc_brute_force.restype = ctypes.c_int
            lib.orc_canon.argtypes = [ctypes.c_int, ctypes.c_uint64]
            lib.orc_canon.restype = ctypes.c_uint64
            lib.orc_canon_many.argtypes = [ctypes.c_int, _u64p, ctypes.c_int64, _u64p]
            lib.orc_canon_many.restype = ctypes.c_int
            lib.orc_code_connected.argtypes = [ctypes.c_int, ctypes.c_uint64]
            lib.orc_code_connected.restype = ctypes.c_int
            lib.orc_classes.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, _u64p, _i64p]
            lib.orc_classes.restype = ctypes.c_int
            lib.orc_clique_instrument.argtypes = [ctypes.c_int32, _i32p, _i32p, ctypes.c_int, _i32p,
                                                  ctypes.c_int64, _u64p, _u64p]
            lib.orc_clique_instrument.restype = ctypes.c_int
            lib.orc_clique_count_bits.argtypes = [ctypes.c_int32, _i32p, _i32p, ctypes.c_int, _i32p,
                                                  ctypes.c_int64, _u64p, _u64p]
            lib.orc_clique_count_bits.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _csr(g):
    ip = np.ascontiguousarray(g.indptr, dtype=np.int32)
    ix = np.ascontiguousarray(g.indices, dtype=np.int32)
    if ix.size == 0:
        ix = np.zeros(1, dtype=np.int32)
    return ip, ix


def _roots(roots):
    if roots is None:
        return None, 0, None
    r = np.ascontiguousarray(roots, dtype=np.int32)
    if r.size == 0:
        r = np.zeros(1, dtype=np.int32)
        return r, 0, _ptr(r, _i32p)
    return r, int(r.shape[0]), _ptr(r, _i32p)


def clique_count(g, k: int, order: int = ORDER_ID, roots=None, per_root: bool = False):
    """Exact number of k-cliques (a Python int, may exceed 2^64).

    With ``roots`` given, only cliques whose first vertex under ``order`` is
    one of them; with ``per_root`` also returns each root's count (uint64)."""
    lib = _load()
    ip, ix = _csr(g)
    r, nr, rp = _roots(roots)
    tot = np.zeros(2, dtype=np.uint64)
    pr = None
    if per_root:
        pr = np.zeros(max(nr if roots is not None else g.n, 1), dtype=np.uint64)
    rc = lib.orc_clique_count(g.n, _ptr(ip, _i32p), _ptr(ix, _i32p), k, order, rp, nr,
                              _ptr(tot, _u64p), _ptr(pr, _u64p) if pr is not None else None)
    if rc != 0:
        raise ValueError(f"orc_clique_count failed ({rc})")
    total = int(tot[0]) | (int(tot[1]) << 64)
    if per_root:
        return total, pr[: (nr if roots is not None else g.n)]
    return total


def clique_instrument(g, k: int, roots=None) -> dict:
    """Search tree of the degree-oriented clique enumeration to depth k:
    ``nodes[s]`` = s-cliques reached (s = 1 .. k; index 0 unused) and
    ``b_alg`` = bytes a sorted-list merge moves over every expansion of a
    node of size <= k-2 (4 (|C(S)| + d+(v)) per child v).  With ``roots``,
    only cliques whose first vertex in the orientation is listed."""
    lib = _load()
    ip, ix = _csr(g)
    r, nr, rp = _roots(roots)
    nodes = np.zeros(2 * (k + 1), dtype=np.uint64)
    b = np.zeros(2, dtype=np.uint64)
    rc = lib.orc_clique_instrument(g.n, _ptr(ip, _i32p), _ptr(ix, _i32p), k, rp, nr,
                                   _ptr(nodes, _u64p), _ptr(b, _u64p))
    if rc != 0:
        raise ValueError(f"orc_clique_instrument failed ({rc})")
    return {"nodes": [int(nodes[2 * s]) | (int(nodes[2 * s + 1]) << 64) for s in range(k + 1)],
            "b_alg": int(b[0]) | (int(b[1]) << 64)}


def clique_count_bits(g, k: int, roots=None, per_root: bool = False):
    """Clique counts of every size s = 1 .. k in one degree-oriented search
    whose candidate sets are bitsets over the root's out-neighbourhood:
    returns ``counts`` (list, index s; index 0 unused), plus with
    ``per_root`` a uint64 array [roots, k + 1] of each root's s-cliques.
    With ``roots``, only cliques whose first vertex in the orientation is
    listed (all vertices when None)."""
    lib = _load()
    ip, ix = _csr(g)
    r, nr, rp = _roots(roots)
    tot = np.zeros(2 * (k + 1), dtype=np.uint64)
    pr = None
    if per_root:
        pr = np.zeros((max(nr if roots is not None else g.n, 1), k + 1), dtype=np.uint64)
    rc = lib.orc_clique_count_bits(g.n, _ptr(ip, _i32p), _ptr(ix, _i32p), k, rp, nr, _ptr(tot, _u64p),
                                   _ptr(pr, _u64p) if pr is not None else None)
    if rc != 0:
        raise ValueError(f"orc_clique_count_bits failed ({rc})")
    counts = [int(tot[2 * s]) | (int(tot[2 * s + 1]) << 64) for s in range(k + 1)]
    if per_root:
        return counts, pr[: (nr if roots is not None else g.n)]
    return counts


def motif_count(g, k: int, roots=None, per_root: bool = False, method: str = "arabesque"):
    """Connected induced k-vertex subgraphs aggregated by canonical code:
    returns ``{canonical_code: count}`` (Python ints), plus per-root totals
    when ``per_root``.  With ``roots``, only sets whose smallest vertex is a
    listed root.  ``method``: "arabesque" (Algorithm 4 with the Arabesque
    canonical filter) or "esu" (ESU exclusive extension; same results,
    faster, for full-size checks)."""
    lib = _load()
    fn = {"arabesque": lib.orc_motif_count, "esu": lib.orc_motif_count_esu}[method]
    ip, ix = _csr(g)
    r, nr, rp = _roots(roots)
    cap = 1 << 14
    codes = np.zeros(cap, dtype=np.uint64)
    lo = np.zeros(cap, dtype=np.uint64)
    hi = np.zeros(cap, dtype=np.uint64)
    nout = np.zeros(1, dtype=np.int64)
    tot = np.zeros(2, dtype=np.uint64)
    pr = None
    if per_root:
        pr = np.zeros(max(nr if roots is not None else g.n, 1), dtype=np.uint64)
    rc = fn(g.n, _ptr(ip, _i32p), _ptr(ix, _i32p), k, rp, nr, cap,
                             _ptr(codes, _u64p), _ptr(lo, _u64p), _ptr(hi, _u64p),
                             _ptr(nout, _i64p), _ptr(tot, _u64p),
                             _ptr(pr, _u64p) if pr is not None else None)
    if rc != 0:
        raise ValueError(f"orc_motif_count failed ({rc})")
    m = int(nout[0])
    if m > cap:
        raise ValueError("too many distinct patterns")
    out = {int(codes[i]): int(lo[i]) | (int(hi[i]) << 64) for i in range(m)}
    if per_root:
        return out, pr[: (nr if roots is not None else g.n)]
    return out


def brute_force(g, k: int):
    """Every k-subset classified: ``{canonical_code: (count, connected)}``."""
    lib = _load()
    ip, ix = _csr(g)
    cap = 1 << 14
    codes = np.zeros(cap, dtype=np.uint64)
    lo = np.zeros(cap, dtype=np.uint64)
    hi = np.zeros(cap, dtype=np.uint64)
    conn = np.zeros(cap, dtype=np.uint8)
    nout = np.zeros(1, dtype=np.int64)
    rc = lib.orc_brute_force(g.n, _ptr(ip, _i32p), _ptr(ix, _i32p), k, cap, _ptr(codes, _u64p),
                             _ptr(lo, _u64p), _ptr(hi, _u64p), _ptr(conn, _u8p), _ptr(nout, _i64p))
    if rc != 0:
        raise ValueError(f"orc_brute_force failed ({rc})")
    m = int(nout[0])
    return {int(codes[i]): (int(lo[i]) | (int(hi[i]) << 64), bool(conn[i])) for i in range(m)}


def canon(k: int, code: int) -> int:
    """Smallest full code over all relabelings of a k-vertex graph."""
    return int(_load().orc_canon(k, code))


def canon_many(k: int, codes) -> np.ndarray:
    lib = _load()
    a = np.ascontiguousarray(codes, dtype=np.uint64)
    out = np.zeros_like(a)
    if a.size:
        rc = lib.orc_canon_many(k, _ptr(a, _u64p), a.shape[0], _ptr(out, _u64p))
        if rc != 0:
            raise ValueError("orc_canon_many failed")
    return out


def code_connected(k: int, code: int) -> bool:
    return bool(_load().orc_code_connected(k, code))


def classes(k: int, connected_only: bool) -> list[int]:
    """All canonical codes of k-vertex graphs (k <= 6), ascending."""
    lib = _load()
    cap = 1 << 12
    out = np.zeros(cap, dtype=np.uint64)
    nout = np.zeros(1, dtype=np.int64)
    rc = lib.orc_classes(k, int(connected_only), cap, _ptr(out, _u64p), _ptr(nout, _i64p))
    if rc != 0:
        raise ValueError("orc_classes failed")
    return [int(x) for x in out[: int(nout[0])]]


def full_code(adj_pairs, k: int) -> int:
    """Full code of a k-vertex graph from its edge list: bit i(i-1)/2 + j for j < i."""
    code = 0
    for a, b in adj_pairs:
        j, i = min(a, b), max(a, b)
        code |= 1 << (i * (i - 1) // 2 + j)
    return code
