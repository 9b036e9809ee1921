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


def test_static_root_matches_context_path_bit_for_bit_on_signed_zeros(env):
    """Coordinates of -0.0 and +0.0 (and a box whose lower and upper bounds are
    zeros of opposite sign): both paths reduce the box on the same
    order-preserving integer keys of the doubles, so the centre's sign of zero
    agrees bit for bit, not only as equal values."""
    torch, afd = env
    stream = torch.cuda.current_stream()
    gen = np.random.default_rng(64)
    n = 40000
    for case in range(3):
        pos = gen.normal(size=(n, 3))
        if case == 0:  # every coordinate a zero of either sign on the x axis
            pos[:, 0] = np.where(gen.random(n) < 0.5, -0.0, 0.0)
        elif case == 1:  # only -0.0 on y, only +0.0 on z
            pos[:, 1] = -0.0
            pos[:, 2] = 0.0
        else:  # zeros of both signs sprinkled through, the rest symmetric
            sel = gen.random((n, 3)) < 0.2
            pos[sel] = np.where(gen.random(sel.sum()) < 0.5, -0.0, 0.0)
        m = np.full(n, 1.0 / n)
        x, y, z, md = _dev(torch, (pos[:, 0], pos[:, 1], pos[:, 2], m))
        root = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda:0")
        flag = torch.full((1,), -1, dtype=torch.int32, device="cuda:0")
        afd.afd_root_cell_static(x, y, z, md, root, flag, stream)
        torch.cuda.synchronize()
        ref = _context_root(afd, torch, x, y, z, md)
        got = root.cpu().numpy()
        assert np.array_equal(got.view(np.uint64), np.asarray(ref, np.float64).view(np.uint64)), case
        assert int(flag.item()) == 0


def test_static_root_flags_sets_without_a_root_cell(env):
    """An infinite coordinate, or finite coordinates whose extent has no
    power-of-two side in doubles, set the flag (the side is read off the bits
    of the extent, so the call ends); the next call on a good set is clean."""
    torch, afd = env
    stream = torch.cuda.current_stream()
    p = ics.plummer(7000, 65)
    root = torch.zeros(4, dtype=torch.float64, device="cuda:0")
    flag = torch.zeros(1, dtype=torch.int32, device="cuda:0")
    for v0, v1 in ((float("inf"), None), (float("-inf"), None), (-1e308, 1e308),
                   (0.0, 2.0 ** 1023)):
        x, y, z, m = _dev(torch, (p.x, p.y, p.z, p.m))
        z[11] = v0
        if v1 is not None:
            z[4000] = v1
        flag.fill_(-1)
        afd.afd_root_cell_static(x, y, z, m, root, flag, stream)
        torch.cuda.synchronize()
        assert int(flag.item()) == 1, (v0, v1)
    x, y, z, m = _dev(torch, (p.x, p.y, p.z, p.m))
    afd.afd_root_cell_static(x, y, z, m, root, flag, stream)
    torch.cuda.synchronize()
    assert int(flag.item()) == 0
    assert np.array_equal(root.cpu().numpy(), _context_root(afd, torch, x, y, z, m))
