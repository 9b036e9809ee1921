"""GPU parity of the short-range neighbour walk and the gather density
(readings R17 and R18 of the oracle; Section 2, Section 4.2) through the C
ABI.

Bit-exact: the cells' tight boxes, the groups' search boxes and the
neighbour lists (every decision is a comparison of FP32 values both sides
round from FP64 the same way). Floating point: the FP32 density and smooth
neighbour number against the oracle's FP64 sums on the same lists, per
particle relative error <= RHO_TOL. The bound: each pair costs a few FP32
roundings in r^2 and q (relative 2e-7, and |dw/dq| <= 1.5), the sums run in
two levels (chunks of at most 32 terms, then one addition per chunk: at most
about (32 + list length / 32) unit roundoffs, 5e-6 for lists of 2000), the
mass and the normalisation add a few more roundings: 2e-5 leaves a factor
two over that worst case."""
import numpy as np
import pytest

import ics
from test_gpu_parity import env  # noqa: F401 (fixture)

pytestmark = pytest.mark.gpu

RHO_TOL = 2e-5


def _T(torch, a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda:0")


def _run(env, p, h, *, n_grp=64, skin=0.0):
    torch, afd, _ = env
    g = afd.Gravity(afd.Config(n_grp=n_grp), 0, torch.cuda.current_stream())
    X = [_T(torch, a) for a in (p.x, p.y, p.z, p.m)]
    afd.afd_tree_build(g.ctx, *X)
    H = _T(torch, h)
    g.neighbour_lists(H, skin)
    rho = torch.full((p.n,), float("nan"), dtype=torch.float32, device="cuda:0")
    nnb = torch.full_like(rho, float("nan"))
    g.density(H, rho, nnb)
    torch.cuda.synchronize()
    return g, X, H, rho.cpu().numpy().astype(np.float64), nnb.cpu().numpy().astype(np.float64)


def _check_lists(g, t):
    off, idx, tb, sb = t.neighbour_data()
    assert np.array_equal(g.export("nbr_off").astype(np.int64), off)
    assert np.array_equal(g.export("nbr_idx").astype(np.int64), idx)
    gtb = g.export("cell_tbox").reshape(-1, 8)
    assert np.array_equal(gtb[:, [0, 1, 2, 4, 5, 6]], tb)
    assert not gtb[:, [3, 7]].any()
    assert np.array_equal(g.export("group_sbox").reshape(-1, 6), sb)


def _rel(a, ref):
    return float(np.max(np.abs(a - ref) / np.abs(ref)))


def _clumps(n, seed):
    """Tight clumps with exact duplicates: deep trees and level-21 leaves."""
    gen = np.random.default_rng(seed)
    c = gen.uniform(-1.0, 1.0, (8, 3))
    k = gen.integers(0, 8, n)
    x = c[k] + gen.normal(0.0, 1e-3, (n, 3))
    x[: n // 10] = c[0]  # a tenth of the particles on one point
    m = np.full(n, 1.0 / n)
    return ics.Particles(x[:, 0], x[:, 1], x[:, 2], m * 0, m * 0, m * 0, m)


CASES = {  # particles, search radii, n_grp, skin
    "plummer_grp16": (lambda: ics.plummer(20003, 91),
                      lambda p: ics.plummer_search_radii(p, 40), 16, 0.0),
    "plummer_grp64": (lambda: ics.plummer(20003, 92),
                      lambda p: ics.plummer_search_radii(p, 40), 64, 0.0),
    "plummer_grp256_skin": (lambda: ics.plummer(20003, 93),
                            lambda p: ics.plummer_search_radii(p, 64), 256, 0.01),
    # one radius for all, about 40 neighbours in the unit sphere
    "uniform_const_h": (lambda: ics.uniform_sphere(30000, 94),
                        lambda p: np.full(p.n, (40.0 / p.n) ** (1.0 / 3.0)), 32, 0.005),
    "clumps": (lambda: _clumps(12000, 95), lambda p: np.full(p.n, 2e-3), 64, 0.0),
}


@pytest.mark.parametrize("case", list(CASES))
def test_lists_boxes_and_density_match_oracle(env, case):
    torch, afd, orc = env
    make, radii, n_grp, skin = CASES[case]
    p = make()
    h = radii(p)
    g, _, _, rho, nnb = _run(env, p, h, n_grp=n_grp, skin=skin)
    t = orc.Tree(p.x, p.y, p.z, p.m, n_grp=n_grp)
    t.neighbour_lists(h, skin)
    _check_lists(g, t)
    r_ref, n_ref = t.density(h)
    assert _rel(rho, r_ref) <= RHO_TOL
    assert _rel(nnb, n_ref) <= RHO_TOL
    st = afd.afd_neighbour_stats(g.ctx)
    off, _ = t.neighbour_data()[:2]
    cnt = t.groups()["count"]
    assert st["entries"] == off[-1] and st["pairs"] == int(np.sum(cnt * np.diff(off)))
    g.close()


def test_reuse_within_skin_and_new_radii(env):
    """Lists made with a margin, particles moved by less than half of it
    (afd_reuse_lists), then the density with the old and with smaller radii:
    the oracle's direct sums on the moved particles."""
    torch, afd, orc = env
    p = ics.plummer(20000, 96)
    h = ics.plummer_search_radii(p, 40)
    skin = 0.02
    g, X, H, _, _ = _run(env, p, h, n_grp=64, skin=skin)
    gen = np.random.default_rng(6)
    d = gen.normal(size=(3, p.n))
    d *= 0.0099 / np.linalg.norm(d, axis=0)
    q = [p.x + d[0], p.y + d[1], p.z + d[2]]
    afd.afd_reuse_lists(g.ctx, *(_T(torch, a) for a in q), X[3])
    for scale in (1.0, 0.9):
        hs = h * scale
        rho = torch.empty(p.n, dtype=torch.float32, device="cuda:0")
        g.density(_T(torch, hs), rho)
        torch.cuda.synchronize()
        r_ref, _ = orc.density_direct(*q, p.m, hs)
        assert _rel(rho.cpu().numpy().astype(np.float64), r_ref) <= RHO_TOL
    # the kept lists are the oracle's kept lists after its update
    t = orc.Tree(p.x, p.y, p.z, p.m, n_grp=64)
    t.neighbour_lists(h, skin)
    t.update(*q, p.m)
    assert np.array_equal(g.export("nbr_idx").astype(np.int64), t.neighbour_data()[1])
    g.close()


def test_neighbour_lists_of_independent_systems(env):
    torch, afd, orc = env
    sizes = [3000, 17, 1, 9000, 0, 700]
    n_grp = [64, 8, 64, 128, 16, 256]
    parts, hs = [], []
    for k, n in enumerate(sizes):
        p = ics.plummer(max(n, 1), 400 + k)
        if n == 0:
            p = ics.Particles(*(np.zeros(0) for _ in range(7)))
        parts.append((p.x + 3.0 * k, p.y, p.z - 3.0 * k, p.m))
        hs.append(ics.plummer_search_radii(p, 32) if n else np.zeros(0))
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    X = [np.concatenate([q[i] for q in parts]) for i in range(4)]
    h = np.concatenate(hs)
    g = afd.Gravity(afd.Config(n_grp=64), 0, torch.cuda.current_stream())
    afd.afd_set_systems(g.ctx, off, n_grp)
    afd.afd_tree_build(g.ctx, *(_T(torch, a) for a in X))
    H = _T(torch, h)
    g.neighbour_lists(H, 0.0)
    rho = torch.empty(off[-1], dtype=torch.float32, device="cuda:0")
    g.density(H, rho)
    torch.cuda.synchronize()
    rho = rho.cpu().numpy().astype(np.float64)
    no, ni = g.export("nbr_off"), g.export("nbr_idx")
    gbase = 0
    for k, n in enumerate(sizes):
        if n == 0:
            continue
        t = orc.Tree(*parts[k], n_grp=n_grp[k])
        t.neighbour_lists(hs[k], 0.0)
        toff, tidx, _, _ = t.neighbour_data()
        ng = len(toff) - 1
        assert np.array_equal(np.diff(no[gbase:gbase + ng + 1]).astype(np.int64), np.diff(toff))
        assert np.array_equal(ni[no[gbase]:no[gbase + ng]].astype(np.int64), tidx + off[k])
        r_ref, _ = t.density(hs[k])
        assert _rel(rho[off[k]:off[k + 1]], r_ref) <= RHO_TOL
        gbase += ng
    g.close()


def test_small_and_degenerate_inputs(env):
    torch, afd, orc = env
    for n in (1, 2, 31, 33, 100):
        if n == 100:  # coincident particles: one level-21 leaf cut into groups of 16
            p = ics.Particles(*(np.zeros(n) + v for v in (0.25, 0.0, 0.0, 0, 0, 0, 0.01)))
            n_grp = 16
        else:
            p = ics.plummer(n, 500 + n)
            n_grp = 64
        h = np.full(n, 0.7)
        g, _, _, rho, nnb = _run(env, p, h, n_grp=n_grp)
        t = orc.Tree(p.x, p.y, p.z, p.m, n_grp=n_grp)
        t.neighbour_lists(h, 0.0)
        _check_lists(g, t)
        r_ref, n_ref = orc.density_direct(p.x, p.y, p.z, p.m, h)
        assert _rel(rho, r_ref) <= RHO_TOL and _rel(nnb, n_ref) <= RHO_TOL
        g.close()
    # empty input
    g = afd.Gravity(afd.Config(), 0, torch.cuda.current_stream())
    e = torch.zeros(0, dtype=torch.float64, device="cuda:0")
    afd.afd_tree_build(g.ctx, e, e, e, e)
    g.neighbour_lists(e, 0.0)
    g.density(e, torch.zeros(0, dtype=torch.float32, device="cuda:0"))
    assert afd.afd_neighbour_stats(g.ctx) == {"entries": 0, "pairs": 0}
    g.close()


def test_errors_leave_the_context_usable(env):
    torch, afd, orc = env
    p = ics.plummer(2000, 97)
    X = [_T(torch, a) for a in (p.x, p.y, p.z, p.m)]
    h = np.full(p.n, 0.2)
    g = afd.Gravity(afd.Config(), 0, torch.cuda.current_stream())
    rho = torch.empty(p.n, dtype=torch.float32, device="cuda:0")
    with pytest.raises(afd.AfdError) as ei:  # before any tree
        afd.afd_make_neighbour_lists(g.ctx, _T(torch, h), 0.0)
    assert ei.value.status == -8
    afd.afd_tree_build(g.ctx, *X)
    with pytest.raises(afd.AfdError) as ei:  # no lists yet
        g.density(_T(torch, h), rho)
    assert ei.value.status == -4
    with pytest.raises(afd.AfdError) as ei:
        g.neighbour_lists(_T(torch, h), -1.0)
    assert ei.value.status == -1
    for bad in (0.0, -0.5, float("nan"), float("inf")):
        hb = h.copy()
        hb[123] = bad
        with pytest.raises(afd.AfdError) as ei:
            g.neighbour_lists(_T(torch, hb), 0.0)
        assert ei.value.status == -13
    g.neighbour_lists(_T(torch, h), 0.0)  # usable again
    hb = h.copy()
    hb[5] = -1.0
    g.density(_T(torch, hb), rho)  # stream-ordered: reported at the next sync
    with pytest.raises(afd.AfdError) as ei:
        afd.afd_sync(g.ctx)
    assert ei.value.status == -13
    out = rho.cpu().numpy()
    assert np.isnan(out[5]) and np.isfinite(np.delete(out, 5)).all()
    afd.afd_sync(g.ctx)  # the status word was cleared
    afd.afd_tree_build(g.ctx, *X)  # a new tree drops the lists
    with pytest.raises(afd.AfdError) as ei:
        g.density(_T(torch, h), rho)
    assert ei.value.status == -4
    g.close()


def test_full_size_density_on_sampled_particles(env):
    """The 2^20 Plummer sphere with radii for 64 neighbours, groups of 256
    (the measured configuration): density of 2000 sampled particles against
    the oracle's sum over all 2^20 particles; the lists hold each group's
    own particles in ascending order."""
    torch, afd, orc = env
    p = ics.plummer(1 << 20, 2020)
    h = ics.plummer_search_radii(p, 64)
    g, _, _, rho, nnb = _run(env, p, h, n_grp=256)
    sel = np.random.default_rng(9).choice(p.n, 2000, replace=False)
    r_ref, n_ref = orc.density_direct(p.x, p.y, p.z, p.m, h, targets=sel)
    assert _rel(rho[sel], r_ref) <= RHO_TOL and _rel(nnb[sel], n_ref) <= RHO_TOL
    assert 40.0 < np.median(nnb) < 90.0
    off, idx = g.export("nbr_off"), g.export("nbr_idx")
    gf, gc = g.export("group_first"), g.export("group_count")
    for k in np.random.default_rng(10).choice(len(gf), 50, replace=False):
        lst = idx[off[k]:off[k + 1]]
        assert np.all(np.diff(lst.astype(np.int64)) > 0)
        assert np.all(np.isin(np.arange(gf[k], gf[k] + gc[k]), lst))
    g.close()


def test_moments_follow_a_neighbour_only_reuse(env):
    """A reusing step that keeps only neighbour lists reorders the particles
    and leaves the moments for later: interaction lists made afterwards, and
    a local essential tree export, see the moved particles' moments -- the
    oracle's update, relist and export on the same data."""
    torch, afd, orc = env
    p = ics.plummer(12000, 98)
    h = ics.plummer_search_radii(p, 32)
    kw = dict(theta=0.5, eps=1.0 / 256, n_grp=64)
    g = afd.Gravity(afd.Config(**kw), 0, torch.cuda.current_stream())
    X = [_T(torch, a) for a in (p.x, p.y, p.z, p.m)]
    afd.afd_tree_build(g.ctx, *X)
    g.neighbour_lists(_T(torch, h), 0.02)
    gen = np.random.default_rng(8)
    q = [v + gen.normal(0.0, 1e-3, p.n) for v in (p.x, p.y, p.z)]
    afd.afd_reuse_lists(g.ctx, *(_T(torch, a) for a in q), X[3])
    t = orc.Tree(p.x, p.y, p.z, p.m, **kw)
    t.update(*q, p.m)
    # the LET export reads the refreshed moments
    box = [-0.3, -0.3, -0.3, 0.3, 0.3, 0.3]
    lx, _, _, lm, lk = afd.afd_let_export(g.ctx, box, 0.5)
    want = t.let_export(box, theta=0.5)
    assert np.array_equal(lx.cpu().numpy(), want[0]) and np.array_equal(lm.cpu().numpy(), want[3])
    # so do lists made now
    afd.afd_make_interaction_lists(g.ctx, afd.AFD_MAKE_LIST)
    acc = torch.empty(p.n, 4, dtype=torch.float32, device="cuda:0")
    afd.afd_calc_force(g.ctx, acc)
    torch.cuda.synchronize()
    t.relist()
    eo, e, so, sp = t.lists()
    assert np.array_equal(g.export("epj_idx").astype(np.int64), e)
    assert np.array_equal(g.export("spj_idx").astype(np.int64), sp)
    from test_gpu_parity import rms_rel_acc
    assert rms_rel_acc(acc.cpu().numpy().astype(np.float64), t.force()) <= 1e-6
    # the density still reads the moved particles through the kept lists
    rho = torch.empty(p.n, dtype=torch.float32, device="cuda:0")
    g.density(_T(torch, h), rho)
    r_ref, _ = orc.density_direct(*q, p.m, h)
    assert _rel(rho.cpu().numpy().astype(np.float64), r_ref) <= RHO_TOL
    g.close()


@pytest.mark.parametrize("h_value,n_grp", [(1000.0, 1024), (1000.0, 16), (1e-4, 64)])
def test_extreme_radii(env, h_value, n_grp):
    """A radius that puts every particle in every group's search box (each
    list is all N particles: whole-subtree records, the compaction's strided
    path, lists of several density segments) and one so small that lists
    hold little beyond the group's own leaves: lists bit for bit and the
    density within the bound, against the oracle."""
    torch, afd, orc = env
    p = ics.plummer(5000, 99)
    h = np.full(p.n, h_value)
    g, _, _, rho, nnb = _run(env, p, h, n_grp=n_grp)
    t = orc.Tree(p.x, p.y, p.z, p.m, n_grp=n_grp)
    t.neighbour_lists(h, 0.0)
    _check_lists(g, t)
    if h_value > 1.0:
        off = g.export("nbr_off")
        assert np.all(np.diff(off.astype(np.int64)) == p.n)
    r_ref, n_ref = t.density(h)
    assert _rel(rho, r_ref) <= RHO_TOL and _rel(nnb, n_ref) <= RHO_TOL
    g.close()
