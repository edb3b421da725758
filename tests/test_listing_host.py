"""Host-side bookkeeping of gpm_list in the binding (CPU, with a stand-in
for the library's gpm_list that calls the consumer as the real one does).

While a listing kernel runs, the consumer is called on the calling thread
and the kernel waits for it; nothing on that thread may wait for the device
meanwhile.  The binding therefore turns Python's cyclic garbage collector
off for the call (a collected graph would free device memory, which waits
for the device) and defers the destruction of graphs released during it.
Checked here: the collector is off inside the consumer and restored after,
also when the consumer raises and when listings nest; a graph released
inside the consumer is destroyed only after the call returns.
"""
from __future__ import annotations

import ctypes
import gc

import numpy as np
import pytest

from paper_2212_04551_gb300 import gpm


class FakeLib:
    """gpm_list delivers `batches` batches of 3 records of k + 1 words."""

    def __init__(self, batches=2, k=3):
        self.batches = batches
        self.k = k
        self.destroyed = []
        self.during = []
        self.graphs = []

    def gpm_list(self, g, app, k, pattern, ring, cb, user, out):
        words = self.k + 1
        recs = np.arange(3 * words, dtype=np.int32)
        n = 0
        for _ in range(self.batches):
            self.during.append(gc.isenabled())
            if cb(recs.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), 3, words, None):
                break
            n += 3
        out._obj.value = n
        return 0

    def gpm_graph_destroy(self, handle):
        self.destroyed.append(handle.value)

    def graph(self, handle):
        """A binding Graph over a stand-in handle, forgotten (never passed to
        the real library) when the test ends."""
        g = gpm.Graph(handle)
        self.graphs.append(g)
        return g

    def gpm_last_error(self):
        return b""


@pytest.fixture
def fake(monkeypatch):
    lib = FakeLib()
    monkeypatch.setattr(gpm, "load", lambda build_if_missing=True: lib)
    yield lib
    assert gpm._LISTING[0] == 0
    for g in lib.graphs:          # stand-in handles must never reach the real library
        g.handle = None


def test_collector_off_inside_and_restored(fake):
    assert gc.isenabled()
    seen = []
    n = gpm.gpm_list(fake.graph(1), gpm.GPM_APP_CLIQUE, 3, lambda r: seen.append(r.shape) and False)
    assert n == 6 and seen == [(3, 4), (3, 4)]
    assert fake.during == [False, False]
    assert gc.isenabled()


def test_collector_restored_when_the_consumer_raises(fake):
    def boom(recs):
        raise KeyError("consumer failed")
    with pytest.raises(KeyError):
        gpm.gpm_list(fake.graph(2), gpm.GPM_APP_CLIQUE, 3, boom)
    assert gc.isenabled()


def test_collector_left_off_if_it_was_off(fake):
    gc.disable()
    try:
        gpm.gpm_list(fake.graph(3), gpm.GPM_APP_CLIQUE, 3, lambda r: False)
        assert not gc.isenabled()
    finally:
        gc.enable()


def test_graph_released_in_the_consumer_is_destroyed_after(fake):
    held = {"g": gpm.Graph(77)}      # its only reference: released inside the consumer

    def consumer(recs):
        held.pop("g", None)          # the last reference goes away here
        assert fake.destroyed == []  # ... but nothing is freed while listing
        return False

    gpm.gpm_list(fake.graph(4), gpm.GPM_APP_CLIQUE, 3, consumer)
    assert 77 in fake.destroyed
    assert gpm._DEFERRED == []


def test_nested_listing_keeps_the_collector_off(fake):
    inner = []

    def consumer(recs):
        if not inner:
            inner.append(gpm.gpm_list(fake.graph(5), gpm.GPM_APP_CLIQUE, 3, lambda r: False))
            assert not gc.isenabled()  # the outer listing still runs
        return False

    gpm.gpm_list(fake.graph(6), gpm.GPM_APP_CLIQUE, 3, consumer)
    assert inner == [6] and gc.isenabled()
