"""Pins for the oracle's short-range neighbour walk and density (readings
R17 and R18 of the oracle: the tree walk with a search-radius criterion of
Section 2, kept over steps as Section 4.2 allows). Checked against what the
mathematics fixes -- the kernel integrates to one over space, is continuous
with a continuous slope at q = 1/2 and vanishes at the support radius; a
lattice of spacing a has density m / a^3 -- against brute force (the lists
equal the particles of every leaf whose tight box meets the group's search
box, computed here in numpy without the walk; the density over the lists
equals the sum over all particles), and against reuse within the margin.
No GPU needed."""
import numpy as np
import pytest

import ics


def _two_body_w(orc, q, h=0.7):
    """W(q h, h) read off a two-particle system: a massless particle at the
    origin and a unit mass at distance q h."""
    q = np.asarray(q, dtype=np.float64)
    out = np.empty_like(q)
    for k, qk in enumerate(q):
        rho, _ = orc.density_direct([0.0, qk * h], [0.0, 0.0], [0.0, 0.0], [0.0, 1.0],
                                    [h, h], targets=[0])
        out[k] = rho[0]
    return out


def test_kernel_integrates_to_one_and_has_the_spline_shape(orc):
    h = 0.7
    n = 2000  # Simpson intervals on [0, h]; q = 1/2 is a node
    q = np.linspace(0.0, 1.0, n + 1)
    W = _two_body_w(orc, q, h)
    r = q * h
    f = 4.0 * np.pi * r * r * W
    simpson = (h / n) / 3.0 * (f[0] + f[-1] + 4.0 * f[1:-1:2].sum() + 2.0 * f[2:-1:2].sum())
    assert simpson == pytest.approx(1.0, abs=1e-12)  # piecewise cubic: Simpson is exact
    assert np.all(W >= 0.0)
    w0 = W[0]
    assert W[-1] == 0.0 and _two_body_w(orc, [1.3], h)[0] == 0.0
    assert W[n // 2] / w0 == pytest.approx(0.25, rel=1e-14)
    assert _two_body_w(orc, [0.75], h)[0] / w0 == pytest.approx(1.0 / 32.0, rel=1e-14)
    # the slope is continuous at q = 1/2 (one-sided differences agree)
    d = 1e-6
    wl, wm, wr = _two_body_w(orc, [0.5 - d, 0.5, 0.5 + d], h)
    assert (wm - wl) / d == pytest.approx((wr - wm) / d, rel=1e-4)


@pytest.mark.parametrize("h_over_a", [2.0, 4.0])
def test_lattice_density_and_neighbour_number(orc, h_over_a):
    k, a = 20, 0.05
    g = (np.arange(k) - k / 2 + 0.5) * a
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    x, y, z = X.ravel(), Y.ravel(), Z.ravel()
    m = np.full(x.size, 1.0 / x.size)
    h = np.full(x.size, h_over_a * a)
    t = orc.Tree(x, y, z, m, n_grp=64)
    t.neighbour_lists(h, 0.0)
    rho, nnb = t.density(h)
    edge = g.max() - h_over_a * a - 1e-9
    inner = (np.abs(x) < edge) & (np.abs(y) < edge) & (np.abs(z) < edge)
    assert inner.sum() >= 1000
    assert np.abs(rho[inner] / (m[0] / a ** 3) - 1.0).max() < 5e-4
    assert np.abs(nnb[inner] / (4.0 * np.pi / 3.0 * h_over_a ** 3) - 1.0).max() < 5e-4


def _down(v):
    f = v.astype(np.float32)
    over = f.astype(np.float64) > v
    f[over] = np.nextafter(f[over], np.float32(-np.inf))
    return f


def _up(v):
    f = v.astype(np.float32)
    under = f.astype(np.float64) < v
    f[under] = np.nextafter(f[under], np.float32(np.inf))
    return f


def _brute_lists(orc, t, p, h, skin):
    """The lists of R17 without the walk: every leaf whose tight box meets
    the group's search box, in ascending particle position."""
    keys, perm = t.order()
    P = np.stack([p.x[perm], p.y[perm], p.z[perm]], 1)
    cells = t.cells()
    leaf = cells.n_child == 0
    nc = len(cells.first)
    tb = np.zeros((nc, 6), np.float32)
    for c in range(nc):
        s = P[cells.first[c]:cells.first[c] + cells.count[c]]
        tb[c, :3] = _down(s.min(0))
        tb[c, 3:] = _up(s.max(0))
    gr = t.groups()
    r = h[perm] + skin
    ng = len(gr["first"])
    sb = np.zeros((ng, 6), np.float32)
    lists = []
    lf = np.nonzero(leaf)[0]
    for g in range(ng):
        f, n = gr["first"][g], gr["count"][g]
        sb[g, :3] = _down((P[f:f + n] - r[f:f + n, None]).min(0))
        sb[g, 3:] = _up((P[f:f + n] + r[f:f + n, None]).max(0))
        meet = np.all((tb[lf, :3] <= sb[g, 3:]) & (tb[lf, 3:] >= sb[g, :3]), axis=1)
        sel = lf[meet]
        sel = sel[np.argsort(cells.first[sel])]
        lists.append(np.concatenate([np.arange(cells.first[c], cells.first[c] + cells.count[c])
                                     for c in sel]) if len(sel) else np.zeros(0, np.int64))
    return tb, sb, lists


@pytest.mark.parametrize("n_grp,skin", [(16, 0.0), (64, 0.0), (64, 0.03), (256, 0.01)])
def test_lists_are_the_leaves_meeting_the_search_box(orc, n_grp, skin):
    p = ics.plummer(3000, 21)
    h = ics.plummer_search_radii(p, 32)
    t = orc.Tree(p.x, p.y, p.z, p.m, n_grp=n_grp)
    t.neighbour_lists(h, skin)
    off, idx, tb, sb = t.neighbour_data()
    want_tb, want_sb, want = _brute_lists(orc, t, p, h, skin)
    assert np.array_equal(tb, want_tb) and np.array_equal(sb, want_sb)
    gr = t.groups()
    for g in range(len(want)):
        got = idx[off[g]:off[g + 1]]
        assert np.array_equal(got, want[g])
        f, n = gr["first"][g], gr["count"][g]
        assert np.all(np.isin(np.arange(f, f + n), got))  # a group's own particles
    assert np.all(np.diff(idx[off[0]:off[1]]) > 0)


@pytest.mark.parametrize("n_grp", [8, 64, 256])
def test_density_over_lists_equals_the_sum_over_all_particles(orc, n_grp):
    p = ics.plummer(5000, 22)
    h = ics.plummer_search_radii(p, 40)
    t = orc.Tree(p.x, p.y, p.z, p.m, n_grp=n_grp)
    t.neighbour_lists(h, 0.0)
    rho, nnb = t.density(h)
    rd, nd = orc.density_direct(p.x, p.y, p.z, p.m, h)
    assert np.allclose(rho, rd, rtol=1e-12, atol=0.0)
    assert np.allclose(nnb, nd, rtol=1e-12, atol=0.0)
    assert 25.0 < np.median(nnb) < 60.0  # the radii hold about 40 neighbours


def test_reuse_within_the_skin_keeps_every_neighbour(orc):
    p = ics.plummer(5000, 23)
    h = ics.plummer_search_radii(p, 40)
    g = np.random.default_rng(5)
    d = g.normal(size=(3, p.n))
    d *= 0.0099 / np.linalg.norm(d, axis=0)  # every particle moves 0.0099
    x, y, z = p.x + d[0], p.y + d[1], p.z + d[2]
    rd, nd = orc.density_direct(x, y, z, p.m, h)
    t = orc.Tree(p.x, p.y, p.z, p.m, n_grp=64)
    t.neighbour_lists(h, 0.02)  # margin 2 x the displacement
    t.update(x, y, z, p.m)
    rho, nnb = t.density(h)
    assert np.allclose(rho, rd, rtol=1e-12, atol=0.0)
    assert np.allclose(nnb, nd, rtol=1e-12, atol=0.0)
    # moves of h / 2 without a margin: the kept lists miss neighbours
    d2 = d / 0.0099 * (0.5 * h)
    x2, y2, z2 = p.x + d2[0], p.y + d2[1], p.z + d2[2]
    r2, _ = orc.density_direct(x2, y2, z2, p.m, h)
    t0 = orc.Tree(p.x, p.y, p.z, p.m, n_grp=64)
    t0.neighbour_lists(h, 0.0)
    t0.update(x2, y2, z2, p.m)
    r0, _ = t0.density(h)
    assert np.abs(r0 / r2 - 1.0).max() > 1e-2


def test_coincident_particles_and_bad_radii(orc):
    n = 100  # one level-21 leaf cut into groups of 16
    z0 = np.zeros(n)
    m = np.full(n, 0.01)
    h = np.full(n, 0.5)
    t = orc.Tree(z0 + 0.25, z0, z0, m, n_grp=16)
    off, idx = t.neighbour_lists(h, 0.0)
    assert len(off) == 8 and np.all(np.diff(off) == n)
    rho, nnb = t.density(h)
    r1, n1 = orc.density_direct([0.25], [0.0], [0.0], [0.01], [0.5])
    assert np.allclose(rho, n * r1[0], rtol=1e-13) and np.allclose(nnb, n * 32.0 / 3.0, rtol=1e-13)
    for bad in (0.0, -1.0, np.nan, np.inf):
        hb = h.copy()
        hb[7] = bad
        with pytest.raises(ValueError):
            t.neighbour_lists(hb, 0.0)
    with pytest.raises(ValueError):
        t.neighbour_lists(h, -0.1)
    e = orc.Tree(np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0))
    off, idx = e.neighbour_lists(np.zeros(0), 0.0)
    assert list(off) == [0] and len(idx) == 0
