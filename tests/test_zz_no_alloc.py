"""The allocation-free root-cell entry point (afd_root_cell_static), for
callers that cannot allocate device memory: its result must equal the root
cell the context path (afd_tree_build) computes, call after call, with its
scratch in a static device array shared by every call. Kept in a file that
pytest collects last."""
import ctypes

import numpy as np
import pytest

import ics

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1907_02290_gb300 as afd

    return torch, afd


def _dev(torch, arrays):
    return [torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda:0")
            for a in arrays]


def _context_root(afd, torch, x, y, z, m):
    g = afd.Gravity(afd.Config(n_grp=64), 0, torch.cuda.current_stream())
    afd.afd_tree_build(g.ctx, x, y, z, m)
    root = g.export("root")
    g.close()
    return root


def test_static_root_matches_context_path_on_consecutive_calls(env):
    torch, afd = env
    stream = torch.cuda.current_stream()
    # two calls in a row on different particle sets: the second must not see
    # the first call's partials, counter or flag
    for k, p in enumerate((ics.plummer(300000 + 17, 61), ics.galaxy(50000, 62))):
        x, y, z, m = _dev(torch, (p.x, p.y, p.z, p.m))
        root = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda:0")
        flag = torch.full((1,), -1, dtype=torch.int32, device="cuda:0")
        afd.afd_root_cell_static(x, y, z, m, root, flag, stream)
        torch.cuda.synchronize()
        ref = _context_root(afd, torch, x, y, z, m)
        assert np.array_equal(root.cpu().numpy(), ref), k
        assert int(flag.item()) == 0


def test_static_root_flags_nonfinite_and_handles_empty(env):
    torch, afd = env
    stream = torch.cuda.current_stream()
    p = ics.plummer(5000, 63)
    x, y, z, m = _dev(torch, (p.x, p.y, p.z, p.m))
    m[123] = float("inf")
    root = torch.zeros(4, dtype=torch.float64, device="cuda:0")
    flag = torch.zeros(1, dtype=torch.int32, device="cuda:0")
    afd.afd_root_cell_static(x, y, z, m, root, flag, stream)
    torch.cuda.synchronize()
    assert int(flag.item()) == 1
    e = torch.zeros(0, dtype=torch.float64, device="cuda:0")
    afd.afd_root_cell_static(e, e, e, e, root, flag, stream)
    torch.cuda.synchronize()
    assert root.cpu().tolist() == [0.0, 0.0, 0.0, 1.0] and int(flag.item()) == 0


def test_static_root_rejects_sizes_above_the_limit(env):
    torch, afd = env
    L = afd.lib()
    root = torch.zeros(4, dtype=torch.float64, device="cuda:0")
    flag = torch.zeros(1, dtype=torch.int32, device="cuda:0")
    dummy = ctypes.c_void_p(root.data_ptr())
    rc = L.afd_root_cell_static(dummy, dummy, dummy, dummy, (1 << 31), ctypes.c_void_p(root.data_ptr()),
                                ctypes.c_void_p(flag.data_ptr()), None)
    assert rc == -11
    assert "limit" in afd.afd_error_string(rc)
