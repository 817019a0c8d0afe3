"""Host-side argument checks of the binding (CPU only): a workspace smaller
than the plan of a call's arguments is refused before the library is
called (the C signature of the batched call carries no workspace size), and
the answer is cached per arguments and buffer."""
import os

import pytest

from paper_1901_06101_gb300 import binding as B


class _DeviceBuffer:
    """Stands in for a device tensor: only what the check reads."""
    is_cuda = True

    def __init__(self, nbytes, ptr=0x7f0000000000):
        self.nbytes, self.ptr = nbytes, ptr

    def data_ptr(self):
        return self.ptr

    def numel(self):
        return self.nbytes

    def element_size(self):
        return 1


class _HostBuffer(_DeviceBuffer):
    is_cuda = False


def test_small_workspace_is_refused():
    B._WS_CHECKED.clear()
    with pytest.raises(B.HbacaError):
        B._check_workspace(_DeviceBuffer(4095), lambda: 4096, ("args",))
    B._check_workspace(_DeviceBuffer(4096), lambda: 4096, ("args",))


def test_host_workspace_is_refused():
    B._WS_CHECKED.clear()
    with pytest.raises(B.HbacaError):
        B._check_workspace(_HostBuffer(1 << 20), lambda: 4096, ("args",))


def test_answer_cached_per_arguments_and_buffer():
    B._WS_CHECKED.clear()
    calls = []

    def need():
        calls.append(1)
        return 4096
    buf = _DeviceBuffer(8192)
    B._check_workspace(buf, need, ("a",))
    B._check_workspace(buf, need, ("a",))
    assert len(calls) == 1
    B._check_workspace(buf, need, ("b",))           # other arguments: planned again
    B._check_workspace(_DeviceBuffer(8192, ptr=0x7f0000100000), need, ("a",))  # other buffer
    assert len(calls) == 3


def test_workspace_need_comes_from_the_planner():
    """The size the check compares with is hbaca_workspace_size of the same
    arguments (host planning, no device needed)."""
    if not os.path.exists(B.LIB_PATH):
        pytest.skip("libhbaca.so not built")
    g = B.Gen(kind=B.GEN_GAUSSIAN, dtype=B.F64, m=2000, n=1800, x=4096, y=8192, dim=3, h=0.7)
    opts = B.make_opts(1e-6, 8, 2, seed=0, rank_cap=128, leaf_rank_cap=256)
    need = B.workspace_size(g, opts)
    B._WS_CHECKED.clear()
    with pytest.raises(B.HbacaError):
        B._check_workspace(_DeviceBuffer(need - 256), lambda: B.workspace_size(g, opts), ("g",))
    B._check_workspace(_DeviceBuffer(need), lambda: B.workspace_size(g, opts), ("g",))
