"""Pins for the FP64 CPU oracle: each test checks the oracle against something
other than itself -- brute force on tiny inputs, closed forms, invariants, or
special cases that reduce to a textbook computation. No GPU needed."""
import math

import numpy as np
import pytest

import ics

LEVELS = 21


def _decode(key):
    """Bit-by-bit de-interleave of a 63-bit key into (qx, qy, qz)."""
    q = [0, 0, 0]
    for k in range(LEVELS):
        q[0] |= ((key >> (3 * k + 2)) & 1) << k
        q[1] |= ((key >> (3 * k + 1)) & 1) << k
        q[2] |= ((key >> (3 * k)) & 1) << k
    return q


# ---------------------------------------------------------------- root cell


def test_root_cell_hand_cases(orc):
    # two points at 0 and 1: extent 1 -> 1.000001 -> next power of two is 2
    r = orc.root_cell([0.0, 1.0], [0.0, 1.0], [0.0, 1.0])
    assert list(r) == [0.5, 0.5, 0.5, 2.0]
    # extent 0.9 -> L = 1
    r = orc.root_cell([0.0, 0.9], [0.0, 0.0], [0.0, 0.0])
    assert list(r) == [0.45, 0.0, 0.0, 1.0]
    # one particle: extent 0 -> L = 1, centred on it
    r = orc.root_cell([3.0], [-2.0], [7.5])
    assert list(r) == [3.0, -2.0, 7.5, 1.0]
    # tiny extent -> negative power of two
    r = orc.root_cell([0.0, 0.001], [0.0, 0.0], [0.0, 0.0])
    assert r[3] == 2.0 ** -9
    with pytest.raises(ValueError):
        orc.root_cell([0.0, np.nan], [0.0, 0.0], [0.0, 0.0])


def test_root_cell_rejects_sets_no_double_cube_holds(orc):
    """An infinite coordinate, or finite coordinates whose extent overflows a
    double or needs a side above 2^1023, have no root cell in doubles: the
    oracle reports them as non-finite input (and ends)."""
    for xs in ([0.0, np.inf], [-np.inf, 0.0], [-1e308, 1e308], [0.0, 2.0 ** 1023],
               [0.0, 1.7976931348623157e308]):
        with pytest.raises(ValueError):
            orc.root_cell(xs, [0.0, 0.0], [0.0, 0.0])
    # the largest side that still exists: an extent of 2^1022 needs 2^1023
    r = orc.root_cell([0.0, 2.0 ** 1022], [0.0, 0.0], [0.0, 0.0])
    assert r[3] == 2.0 ** 1023
    # subnormal extents reach the smallest powers of two exactly
    r = orc.root_cell([0.0, 5e-324], [0.0, 0.0], [0.0, 0.0])
    assert r[3] == 5e-324  # 1.000001 x 2^-1074 rounds back to 2^-1074
    r = orc.root_cell([0.0, 3 * 5e-324], [0.0, 0.0], [0.0, 0.0])
    assert r[3] == 4 * 5e-324


def test_root_cell_contains_and_is_minimal(orc):
    p = ics.plummer(5000, 11)
    c = orc.root_cell(p.x, p.y, p.z)
    L = c[3]
    assert math.frexp(L)[0] == 0.5  # power of two
    for d, arr in enumerate(p.pos()):
        assert np.all(arr >= c[d] - L / 2) and np.all(arr < c[d] + L / 2)
    ext = max(a.max() - a.min() for a in p.pos())
    assert L >= ext and L / 2 < ext * 1.000001


# ---------------------------------------------------------------- keys


def test_morton_keys_hand_worked(orc):
    root = np.array([0.0, 0.0, 0.0, 2.0])  # cube [-1, 1)^3, cell of level 21 = 2^-20
    h = 2.0 ** -20
    pts = np.array([
        [-1.0, -1.0, -1.0],                    # min corner -> q = 0
        [1.0 - h / 2, 1.0 - h / 2, 1.0 - h / 2],  # max corner -> all ones
        [0.5, -0.5, -0.5],                     # +x half only -> top digit 4
        [-0.5, 0.5, -0.5],                     # +y -> 2
        [-0.5, -0.5, 0.5],                     # +z -> 1
        [5.0, -5.0, 0.0],                      # outside: clamped
    ])
    keys = orc.morton_keys(pts[:, 0], pts[:, 1], pts[:, 2], root)
    assert int(keys[0]) == 0
    assert int(keys[1]) == (1 << 63) - 1
    assert int(keys[2]) >> 60 == 4
    assert int(keys[3]) >> 60 == 2
    assert int(keys[4]) >> 60 == 1
    q = _decode(int(keys[5]))
    assert q == [2 ** 21 - 1, 0, 2 ** 20]
    # a point in the x-upper, y-lower, z-upper octant at levels 1 and 2
    k = int(orc.morton_keys([0.75 + h / 4], [-0.75 + h / 4], [0.25 + h / 4], root)[0])
    assert (k >> 60) & 7 == 0b101
    assert (k >> 57) & 7 == 0b100  # level 2: x in [0.5,1) upper, y in [-1,-0.5) lower, z in [0,0.5) lower
    qx, qy, qz = _decode(k)
    assert qx == int((0.75 + h / 4 + 1.0) / h)
    assert qy == int((-0.75 + h / 4 + 1.0) / h)
    assert qz == int((0.25 + h / 4 + 1.0) / h)


def test_morton_keys_containment(orc):
    """Decoded key coordinates place each particle inside its level-21 cell."""
    p = ics.plummer(3000, 12)
    root = orc.root_cell(p.x, p.y, p.z)
    keys = orc.morton_keys(p.x, p.y, p.z, root)
    L = root[3]
    h = L / 2 ** LEVELS
    for i in range(0, p.n, 7):
        q = _decode(int(keys[i]))
        for d, arr in enumerate(p.pos()):
            lo = root[d] - L / 2 + q[d] * h
            assert lo <= arr[i] < lo + h


# ---------------------------------------------------------------- sort


def test_radix_sort_is_stable_argsort(orc):
    g = np.random.Generator(np.random.Philox(7))
    keys = g.integers(0, 50, 20000).astype(np.uint64) << np.uint64(40)
    keys |= g.integers(0, 3, 20000).astype(np.uint64)
    ks, perm = orc.radix_sort(keys)
    ref = np.argsort(keys, kind="stable")
    assert np.array_equal(perm, ref)
    assert np.array_equal(ks, keys[ref])
    wide = g.integers(0, 2 ** 63, 5000, dtype=np.uint64)
    ks, perm = orc.radix_sort(wide)
    assert np.array_equal(perm, np.argsort(wide, kind="stable"))


# ---------------------------------------------------------------- tree


def _recursive_tree(keys, n_leaf):
    """The octree by its definition: split a cell while it holds more than
    n_leaf particles and is above level 21; emit (level, first, count) in
    depth-first pre-order, children in octant order."""
    out = []

    def rec(level, lo, hi):
        out.append((level, lo, hi - lo))
        if hi - lo <= n_leaf or level == LEVELS:
            return
        shift = 3 * (LEVELS - level - 1)
        digits = [(int(k) >> shift) & 7 for k in keys[lo:hi]]
        start = lo
        for o in range(8):
            cnt = sum(1 for d in digits if d == o)
            if cnt:
                rec(level + 1, start, start + cnt)
                start += cnt

    if len(keys):
        rec(0, 0, len(keys))
    return out


@pytest.mark.parametrize("model,n,n_leaf", [("plummer", 3000, 16), ("uniform_sphere", 1500, 4),
                                            ("plummer", 17, 16), ("plummer", 16, 16)])
def test_tree_matches_recursive_definition(orc, model, n, n_leaf):
    p = ics.make(model, n, 21)
    t = orc.Tree(p.x, p.y, p.z, p.m, n_leaf=n_leaf, n_grp=64)
    keys, perm = t.order()
    ref_keys, ref_perm = orc.radix_sort(orc.morton_keys(p.x, p.y, p.z, t.root()))
    assert np.array_equal(keys, ref_keys) and np.array_equal(perm, ref_perm)
    c = t.cells()
    got = list(zip(c.level.tolist(), c.first.tolist(), c.count.tolist()))
    assert got == _recursive_tree(keys, n_leaf)


def test_tree_invariants(orc):
    p = ics.plummer(20000, 5)
    t = orc.Tree(p.x, p.y, p.z, p.m, n_leaf=16, n_grp=64)
    c = t.cells()
    nc = len(c.level)
    leaf = c.n_child == 0
    assert np.all(c.count[leaf] <= 16) or np.all(c.level[leaf & (c.count > 16)] == LEVELS)
    assert np.all(c.count[~leaf] > 16)
    # leaves partition the particles
    cover = np.zeros(p.n, dtype=np.int64)
    for f, n in zip(c.first[leaf], c.count[leaf]):
        cover[f:f + n] += 1
    assert np.all(cover == 1)
    # children: counts add up, contiguous, Morton ordered, pre-order ids
    for ci in range(nc):
        kids = [k for k in c.child[ci] if k >= 0]
        assert len(kids) == c.n_child[ci]
        if kids:
            assert kids[0] == ci + 1
            assert sum(c.count[k] for k in kids) == c.count[ci]
            assert c.first[kids[0]] == c.first[ci]
            for a, b in zip(kids, kids[1:]):
                assert c.first[b] == c.first[a] + c.count[a] and c.skip[a] == b
            assert all(c.parent[k] == ci and c.level[k] == c.level[ci] + 1 for k in kids)
        assert c.skip[ci] > ci
    assert c.skip[0] == nc


def test_moments_match_direct_sums(orc):
    p = ics.plummer(6000, 8)
    t = orc.Tree(p.x, p.y, p.z, p.m, n_leaf=16, n_grp=64, quad=True)
    c = t.cells()
    M, com, Q = t.moments()
    _, perm = t.order()
    xs, ys, zs, ms = (a[perm] for a in (p.x, p.y, p.z, p.m))
    for ci in range(0, len(M), 3):
        sl = slice(c.first[ci], c.first[ci] + c.count[ci])
        m = ms[sl]
        assert M[ci] == pytest.approx(m.sum(), rel=1e-13)
        g = np.array([np.dot(m, xs[sl]), np.dot(m, ys[sl]), np.dot(m, zs[sl])]) / m.sum()
        assert np.allclose(com[ci], g, rtol=0, atol=1e-13 * (1 + np.abs(g).max()))
        d = np.stack([xs[sl] - g[0], ys[sl] - g[1], zs[sl] - g[2]])
        r2 = (d * d).sum(0)
        ref = [np.sum(m * (3 * d[0] * d[0] - r2)), np.sum(m * (3 * d[1] * d[1] - r2)),
               np.sum(m * (3 * d[2] * d[2] - r2)), np.sum(m * 3 * d[0] * d[1]),
               np.sum(m * 3 * d[0] * d[2]), np.sum(m * 3 * d[1] * d[2])]
        scale = np.sum(m * r2) + 1e-300
        assert np.allclose(Q[ci], ref, rtol=0, atol=1e-10 * scale)
        assert abs(Q[ci][0] + Q[ci][1] + Q[ci][2]) <= 1e-10 * scale  # traceless


def test_massless_cell_takes_geometric_centre(orc):
    p = ics.plummer(200, 9)
    m = np.zeros(p.n)
    m[:100] = 1.0 / 100
    t = orc.Tree(p.x, p.y, p.z, m, n_leaf=4, n_grp=8)
    c = t.cells()
    M, com, _ = t.moments()
    root = t.root()
    keys, _ = t.order()
    for ci in np.nonzero(M == 0)[0]:
        lvl = int(c.level[ci])
        q = _decode(int(keys[c.first[ci]]) >> (3 * (LEVELS - lvl)) << (3 * (LEVELS - lvl)))
        s = root[3] / 2 ** lvl
        for d in range(3):
            qd = q[d] >> (LEVELS - lvl)
            assert com[ci][d] == pytest.approx(root[d] - root[3] / 2 + (qd + 0.5) * s, abs=1e-15)


# ---------------------------------------------------------------- groups and lists


def test_groups_partition_and_are_maximal(orc):
    p = ics.plummer(20000, 6)
    t = orc.Tree(p.x, p.y, p.z, p.m, n_grp=64)
    g = t.groups()
    c = t.cells()
    assert g["first"][0] == 0
    assert np.all(g["first"][1:] == g["first"][:-1] + g["count"][:-1])
    assert g["first"][-1] + g["count"][-1] == p.n
    assert np.all(g["count"] <= 64)
    for cell in g["cell"]:
        par = c.parent[cell]
        assert c.count[cell] <= 64 or c.n_child[cell] == 0
        assert par < 0 or c.count[par] > 64


def test_coincident_particles_max_depth_chunks(orc):
    n = 300
    z = np.zeros(n)
    t = orc.Tree(z + 0.25, z, z, np.full(n, 1.0 / n), n_leaf=16, n_grp=64, eps=0.01)
    c = t.cells()
    assert c.level.max() == LEVELS
    leaf = c.n_child == 0
    assert leaf.sum() == 1 and c.count[leaf][0] == n
    g = t.groups()
    assert list(g["count"]) == [64, 64, 64, 64, 44]
    ax, ay, az, pot = t.force()
    assert np.all(ax == 0) and np.all(ay == 0) and np.all(az == 0)
    assert np.allclose(pot, -(n - 1) / n / 0.01, rtol=1e-14)


def _check_lists_geometry(t, theta):
    """Partition invariant plus the opening criterion checked in FP64 with a
    relative band: every accepted cell is well separated (s < theta d), every
    opened ancestor is not."""
    c = t.cells()
    M, com, _ = t.moments()
    g = t.groups()
    eo, e, so, s = t.lists()
    n = t.n
    L = t.root()[3]
    band = 1e-5

    def sep(ci, box):
        lo, hi = box[:3], box[3:]
        d = np.maximum(0.0, np.maximum(lo - com[ci], com[ci] - hi))
        return L / 2 ** c.level[ci], float(np.sqrt((d * d).sum()))

    for gi in range(len(g["first"])):
        box = g["box"][gi]
        cover = np.zeros(n, dtype=np.int64)
        ep = e[eo[gi]:eo[gi + 1]]
        np.add.at(cover, ep, 1)
        sp = s[so[gi]:so[gi + 1]]
        for ci in sp:
            cover[c.first[ci]:c.first[ci] + c.count[ci]] += 1
            size, d = sep(ci, box)
            assert size < theta * d * (1 + band)
            a = c.parent[ci]
            while a >= 0:
                size, d = sep(a, box)
                assert size >= theta * d * (1 - band)
                a = c.parent[a]
        assert np.all(cover == 1), gi
        assert np.all(np.diff(sp) > 0) and np.all(np.diff(ep) > 0)  # depth-first = ascending


def test_lists_partition_and_criterion(orc):
    p = ics.plummer(8000, 3)
    for theta in (0.3, 0.5, 0.8):
        t = orc.Tree(p.x, p.y, p.z, p.m, n_grp=32, theta=theta)
        _check_lists_geometry(t, theta)


def test_theta_zero_is_direct_sum(orc):
    p = ics.plummer(4000, 4)
    eps = 1.0 / 256
    t = orc.Tree(p.x, p.y, p.z, p.m, n_grp=64, theta=0.0, eps=eps)
    eo, e, so, s = t.lists()
    assert len(s) == 0 and len(e) == len(t.groups()["first"]) * p.n
    got = t.force()
    ref = orc.direct_sum(p.x, p.y, p.z, p.m, eps)
    for a, b in zip(got, ref):
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))
    amag = np.sqrt(ref[0] ** 2 + ref[1] ** 2 + ref[2] ** 2)
    err = np.sqrt((got[0] - ref[0]) ** 2 + (got[1] - ref[1]) ** 2 + (got[2] - ref[2]) ** 2)
    assert np.max(err / amag) < 1e-11


def _rms_rel(got, ref, idx=None):
    ax, ay, az = got[:3]
    rx, ry, rz = ref[:3]
    if idx is not None:
        ax, ay, az = ax[idx], ay[idx], az[idx]
    num = (ax - rx) ** 2 + (ay - ry) ** 2 + (az - rz) ** 2
    return float(np.sqrt(np.mean(num / (rx ** 2 + ry ** 2 + rz ** 2))))


def test_error_falls_with_theta_and_quadrupole_helps(orc):
    p = ics.plummer(16384, 1)
    eps = 1.0 / 256
    idx = np.arange(0, p.n, 13)
    ref = orc.direct_sum(p.x, p.y, p.z, p.m, eps, idx)
    errs = {}
    for quad in (False, True):
        for theta in (0.8, 0.5, 0.3):
            t = orc.Tree(p.x, p.y, p.z, p.m, n_grp=64, theta=theta, eps=eps, quad=quad)
            errs[quad, theta] = _rms_rel(t.force(), ref, idx)
    for quad in (False, True):
        assert errs[quad, 0.8] > errs[quad, 0.5] > errs[quad, 0.3]
    for theta in (0.8, 0.5, 0.3):
        assert errs[True, theta] < 0.5 * errs[False, theta]
    assert errs[False, 0.5] < 5e-3


def test_quadrupole_two_masses_closed_form(orc):
    """Two equal masses at COM +/- d z and a far test particle on the z axis:
    the exact field is -m/(r-d)^2 - m/(r+d)^2; the monopole misses the
    -6 m d^2 / r^4 term and the quadrupole supplies it. Two massless anchors
    at (0,0,0) and (1.5,1.5,1.5) fix the root cube to [-0.25, 1.75)^3, so the
    pair at z = 0.3 +/- 0.01 shares a level-2 cell of side 0.5."""
    m, d, r = 0.5, 0.01, 1.0
    x = np.array([0.3, 0.3, 0.3, 0.0, 1.5])
    y = np.array([0.3, 0.3, 0.3, 0.0, 1.5])
    z = np.array([0.3 + d, 0.3 - d, 0.3 + r, 0.0, 1.5])
    mass = np.array([m, m, 1e-30, 1e-30, 1e-30])
    exact = -m / (r - d) ** 2 - m / (r + d) ** 2
    res = {}
    for quad in (False, True):
        t = orc.Tree(x, y, z, mass, n_leaf=2, n_grp=1, theta=0.9, eps=0.0, quad=quad)
        ax, ay, az, pot = t.force()
        res[quad] = (az[2], pot[2])
        assert abs(ax[2]) < 1e-20 and abs(ay[2]) < 1e-20
        # the pair reached the test particle as one superparticle
        _, perm = t.order()
        k = int(np.nonzero(perm == 2)[0][0])
        g = t.groups()
        gi = int(np.nonzero(g["first"] == k)[0][0])
        eo, e, so, s = t.lists()
        c = t.cells()
        pair = [ci for ci in s[so[gi]:so[gi + 1]] if c.count[ci] == 2]
        assert len(pair) == 1
    mono, quadr = res[False][0], res[True][0]
    assert mono == pytest.approx(-2 * m / r ** 2, rel=1e-12)
    assert quadr == pytest.approx(-2 * m / r ** 2 - 6 * m * d * d / r ** 4, rel=1e-12)
    assert abs(quadr - exact) < 1e-3 * abs(mono - exact)
    exact_pot = -m / (r - d) - m / (r + d)
    assert res[True][1] == pytest.approx(-2 * m / r - 2 * m * d * d / r ** 3, rel=1e-12)
    assert abs(res[True][1] - exact_pot) < 1e-3 * abs(res[False][1] - exact_pot)


def test_momentum_direct_and_tree(orc):
    p = ics.plummer(4096, 14)
    eps = 1.0 / 256
    ref = orc.direct_sum(p.x, p.y, p.z, p.m, eps)
    scale = np.sum(p.m * np.sqrt(ref[0] ** 2 + ref[1] ** 2 + ref[2] ** 2))
    for a in ref[:3]:
        assert abs(np.sum(p.m * a)) < 1e-13 * scale
    t = orc.Tree(p.x, p.y, p.z, p.m, n_grp=64, theta=0.5, eps=eps)
    got = t.force()
    for a in got[:3]:
        assert abs(np.sum(p.m * a)) < 1e-3 * scale


def test_plummer_closed_form_potential_and_field(orc):
    """Binned mean potential and radial field of a 16k Plummer sphere against
    phi = -1/sqrt(r^2+1) and a_r = -r/(r^2+1)^(3/2) (G = M = a = 1)."""
    p = ics.plummer(16384, 1)
    t = orc.Tree(p.x, p.y, p.z, p.m, n_grp=64, theta=0.4, eps=1.0 / 256)
    ax, ay, az, pot = t.force()
    r = np.sqrt(p.x ** 2 + p.y ** 2 + p.z ** 2)
    ar = (ax * p.x + ay * p.y + az * p.z) / r
    edges = np.array([0.1, 0.3, 0.5, 0.8, 1.2, 2.0, 3.5])
    for lo, hi in zip(edges[:-1], edges[1:]):
        sel = (r >= lo) & (r < hi)
        assert sel.sum() > 300
        rr = r[sel]
        phi_ref = np.mean(-1.0 / np.sqrt(rr ** 2 + 1.0))
        ar_ref = np.mean(-rr / (rr ** 2 + 1.0) ** 1.5)
        assert np.mean(pot[sel]) == pytest.approx(phi_ref, rel=0.02)
        assert np.mean(ar[sel]) == pytest.approx(ar_ref, rel=0.05)


def test_reuse_step_keeps_lists_and_matches_rebuild_at_same_positions(orc):
    p = ics.plummer(4000, 15)
    kw = dict(n_grp=64, theta=0.5, eps=1.0 / 256)
    t = orc.Tree(p.x, p.y, p.z, p.m, **kw)
    lists0 = t.lists()
    # the update with unchanged positions reproduces the construction step
    f0 = t.force()
    t.update(p.x, p.y, p.z, p.m)
    f1 = t.force()
    for a, b in zip(f0, f1):
        assert np.array_equal(a, b)
    # after a small drift the lists are unchanged and the moments follow
    dx = 1e-3 * p.vx
    t.update(p.x + dx, p.y, p.z, p.m)
    for a, b in zip(lists0, t.lists()):
        assert np.array_equal(a, b)
    M, com, _ = t.moments()
    assert com[0][0] == pytest.approx(np.sum(p.m * (p.x + dx)) / np.sum(p.m), abs=1e-14)
    with pytest.raises(ValueError):
        t.update(p.x * np.nan, p.y, p.z, p.m)


def test_leapfrog_energy_and_momentum(orc):
    p = ics.plummer(2048, 16)
    eps = 1.0 / 64
    out = orc.leapfrog(p.x, p.y, p.z, p.vx, p.vy, p.vz, p.m, dt=1.0 / 256, n_steps=32, n_reuse=4,
                       n_grp=64, theta=0.4, eps=eps)
    x, y, z, vx, vy, vz = out[:6]

    def energy(x, y, z, vx, vy, vz):
        _, _, _, pot = orc.direct_sum(x, y, z, p.m, eps)
        return 0.5 * np.sum(p.m * (vx ** 2 + vy ** 2 + vz ** 2)) + 0.5 * np.sum(p.m * pot)

    e0 = energy(p.x, p.y, p.z, p.vx, p.vy, p.vz)
    e1 = energy(x, y, z, vx, vy, vz)
    assert abs(e1 - e0) < 2e-4 * abs(e0)
    mom0 = np.array([np.sum(p.m * v) for v in p.vel()])
    mom1 = np.array([np.sum(p.m * v) for v in (vx, vy, vz)])
    assert np.max(np.abs(mom1 - mom0)) < 1e-4
    # without reuse (rebuild every step) the trajectory stays close
    out1 = orc.leapfrog(p.x, p.y, p.z, p.vx, p.vy, p.vz, p.m, dt=1.0 / 256, n_steps=32, n_reuse=1,
                        n_grp=64, theta=0.4, eps=eps)
    assert np.max(np.abs(out1[0] - x)) < 1e-4


def test_empty_and_single_particle(orc):
    e = np.zeros(0)
    t = orc.Tree(e, e, e, e)
    assert t.sizes() == {"n": 0, "n_cells": 0, "n_groups": 0, "n_epj": 0, "n_spj": 0}
    assert all(len(a) == 0 for a in t.force())
    t = orc.Tree([1.0], [2.0], [3.0], [1.0], eps=0.1)
    assert t.sizes()["n_cells"] == 1 and t.sizes()["n_groups"] == 1
    assert [float(a[0]) for a in t.force()] == [0.0, 0.0, 0.0, 0.0]
    with pytest.raises(ValueError):
        orc.Tree([1.0, np.inf], [0.0, 0.0], [0.0, 0.0], [1.0, 1.0])


def test_list_length_near_paper_estimate(orc):
    """Eq. n_list (Section 6.2) estimates the mean list length for a uniform
    sphere; the walk's lists should land within a factor of two of it (a
    loose sanity check: the equation models FDPS's own criterion)."""
    n = 1 << 16
    p = ics.uniform_sphere(n, 5)
    theta = 0.5
    for n_grp in (64, 256):
        t = orc.Tree(p.x, p.y, p.z, p.m, n_grp=n_grp, theta=theta)
        g = t.groups()
        eo, _, so, _ = t.lists()
        ni = float(np.mean(g["count"]))
        nlist = float(np.sum(g["count"] * ((eo[1:] - eo[:-1]) + (so[1:] - so[:-1])))) / n
        est = (ni + 14 * ni ** (2 / 3) / theta + 21 * math.pi * ni ** (1 / 3) / theta ** 2
               + 28 * math.pi / (3 * theta ** 3) * math.log2(theta / 2.8 * (n ** (1 / 3) - ni ** (1 / 3))))
        assert 0.5 * est < nlist < 2.0 * est, (ni, nlist, est)
