"""Argument marshalling of the Python binding on the CPU: what
Context.forces_at hands to rbsog_forces_at, what it refuses before any
library call, and how a library error code becomes an exception (a stand-in
for the loaded library; no GPU)."""
import ctypes

import numpy as np
import pytest

from paper_2512_24970_gb300 import rbsog


class FakeLib:
    def __init__(self, rc=0):
        self.rc = rc
        self.calls = []

    def rbsog_forces_at(self, h, pos, step, forces, kind):
        self.calls.append((h, pos.value, step, forces.value, kind))
        if self.rc == 0:                         # the library writes the forces
            ctypes.memmove(forces.value, np.full(self.n3, 1.5).ctypes.data, 8 * self.n3)
        return self.rc

    def rbsog_last_error(self, h):
        return b"kept lists: an atom moved by more than skin/2"


def context(n, rc=0):
    ctx = rbsog.Context.__new__(rbsog.Context)   # no device: the library is a stand-in
    ctx.h = ctypes.c_void_p(1234)
    ctx.n = n
    ctx._L = FakeLib(rc)
    ctx._L.n3 = 3 * n
    return ctx


def test_forces_at_host_arrays():
    ctx = context(5)
    pos = np.arange(15, dtype=np.float64).reshape(5, 3)
    F = ctx.forces_at(pos, 42)
    assert F.shape == (5, 3) and np.all(F == 1.5)
    (h, pp, step, fp, kind), = ctx._L.calls
    assert step == 42 and kind == rbsog.PTR_HOST
    assert pp == pos.ctypes.data and fp == F.ctypes.data
    out = np.zeros((5, 3))
    assert ctx.forces_at(pos, 43, out) is out and np.all(out == 1.5)


def test_forces_at_converts_positions_only():
    ctx = context(2)
    pos = [[0, 0, 0], [1, 2, 3]]                 # a list: converted to a contiguous FP64 array
    F = ctx.forces_at(np.asarray(pos, dtype=np.int64), 1)
    assert np.all(F == 1.5)
    with pytest.raises(ValueError):              # the output is written in place: never converted
        ctx.forces_at(np.zeros((2, 3)), 1, np.zeros((2, 3), dtype=np.float32))
    with pytest.raises(ValueError):
        ctx.forces_at(np.zeros((2, 3)), 1, np.zeros((3, 3)))
    with pytest.raises(ValueError):
        ctx.forces_at(np.zeros((3, 3)), 1)
    with pytest.raises(ValueError):
        ctx.forces_at(np.zeros((2, 3)), 1, np.zeros((3, 2)).T)   # not C-contiguous
    assert len(ctx._L.calls) == 1                # the refused calls never reached the library


def test_forces_at_cpu_tensor_is_host_memory():
    # a CPU torch tensor is host memory: written in place like a numpy array
    # (host and CUDA buffers mixed are refused; tests/test_gpu_kept.py checks that)
    torch = pytest.importorskip("torch")
    ctx = context(2)
    out = torch.zeros((2, 3), dtype=torch.float64)
    assert ctx.forces_at(np.zeros((2, 3)), 1, out) is out
    assert ctx._L.calls[0][4] == rbsog.PTR_HOST and bool((out == 1.5).all())
    with pytest.raises(ValueError):
        ctx.forces_at(np.zeros((2, 3)), 1, torch.zeros((2, 3), dtype=torch.float32))


def test_library_error_becomes_exception():
    ctx = context(2, rc=-9)
    with pytest.raises(rbsog.RbsogError) as e:
        ctx.forces_at(np.zeros((2, 3)), 1)
    assert e.value.code == -9 and "RBSOG_E_SKIN" in str(e.value) and "skin/2" in str(e.value)
