"""GPU parity: the sm_103a library (through its C ABI) against the FP64 CPU
oracle on the same seeded inputs.

Bit-exact: root cell, Morton keys, permutation, tree topology, monopole
moments, groups, group boxes and the theta-criterion lists (both sides take
every decision in the same IEEE precision with the same operation order).
Floating point: the FP32 force kernel against the FP64 oracle force on the
same lists, rms relative acceleration error <= 1e-6 (the bound the method's
accuracy target states), potential likewise.
"""
import numpy as np
import pytest

import ics

pytestmark = pytest.mark.gpu

NONE = 0xFFFFFFFF
FORCE_RMS_TOL = 1e-6
POT_RMS_TOL = 1e-6


@pytest.fixture(scope="module")
def env(orc):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1907_02290_gb300 as afd

    return torch, afd, orc


def run_gpu(env, p, *, n_leaf=16, n_grp=64, theta=0.5, eps=1.0 / 256, quad=False,
            mode=None):
    torch, afd, _ = env
    cfg = afd.Config(eps=eps, theta=theta, n_leaf=n_leaf, n_grp=n_grp, multipole=int(quad))
    g = afd.Gravity(cfg, 0, torch.cuda.current_stream())
    dev = torch.device("cuda:0")
    x, y, z, m = (torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
                  for a in (p.x, p.y, p.z, p.m))
    acc = torch.full((p.n, 4), float("nan"), dtype=torch.float32, device=dev)
    g.force_all(x, y, z, m, acc, afd.AFD_MAKE_LIST_FOR_REUSE if mode is None else mode)
    torch.cuda.synchronize()
    return g, acc.cpu().numpy().astype(np.float64), (x, y, z, m, acc)


def rms_rel_acc(a, ref):
    ax, ay, az = ref[:3]
    num = (a[:, 0] - ax) ** 2 + (a[:, 1] - ay) ** 2 + (a[:, 2] - az) ** 2
    return float(np.sqrt(np.mean(num / (ax ** 2 + ay ** 2 + az ** 2))))


def rms_rel_pot(a, ref):
    return float(np.sqrt(np.mean((a[:, 3] - ref[3]) ** 2 / ref[3] ** 2)))


def u32(a):
    return np.where(a < 0, NONE, a).astype(np.uint32)


def check_structure(g, t, quad=False):
    """Everything the method decides, bit for bit."""
    assert np.array_equal(g.export("root"), t.root())
    keys, perm = t.order()
    assert np.array_equal(g.export("keys"), keys)
    assert np.array_equal(g.export("perm"), perm.astype(np.uint32))
    c = t.cells()
    assert np.array_equal(g.export("cell_level"), c.level.astype(np.uint32))
    assert np.array_equal(g.export("cell_first"), c.first.astype(np.uint32))
    assert np.array_equal(g.export("cell_count"), c.count.astype(np.uint32))
    assert np.array_equal(g.export("cell_skip"), c.skip.astype(np.uint32))
    assert np.array_equal(g.export("cell_parent"), u32(c.parent))
    assert np.array_equal(g.export("cell_child").reshape(-1, 8), u32(c.child))
    M, com, Q = t.moments()
    assert np.array_equal(g.export("cell_mass"), M)
    assert np.array_equal(g.export("cell_com").reshape(-1, 3), com)
    if quad:
        gq = g.export("cell_quad").reshape(-1, 6)
        scale = np.abs(Q).max(axis=1, keepdims=True) + 1e-300
        assert np.max(np.abs(gq - Q) / scale) < 1e-12
    gr = t.groups()
    assert np.array_equal(g.export("group_first"), gr["first"].astype(np.uint32))
    assert np.array_equal(g.export("group_count"), gr["count"].astype(np.uint32))
    assert np.array_equal(g.export("group_box").reshape(-1, 6), gr["box"])
    eo, e, so, s = t.lists()
    gself = g.export("group_self")
    assert np.array_equal(gself > 0, gr["self_in"] > 0)
    for gi in np.nonzero(gself)[0][::7]:  # the group's own particles, contiguous
        p0 = eo[gi] + int(gself[gi]) - 1
        assert np.array_equal(e[p0:p0 + gr["count"][gi]],
                              np.arange(gr["first"][gi], gr["first"][gi] + gr["count"][gi]))
    assert np.array_equal(g.export("epj_off"), eo.astype(np.uint64))
    assert np.array_equal(g.export("spj_off"), so.astype(np.uint64))
    assert np.array_equal(g.export("epj_idx"), e.astype(np.uint32))
    assert np.array_equal(g.export("spj_idx"), s.astype(np.uint32))
    st = g.stats()
    assert st["n_cells"] == len(c.level) and st["n_groups"] == len(gr["first"])
    assert st["interactions"] == t.interactions()


CASES = {
    # name: (particles, kwargs)
    "plummer_16k_ragged": (lambda: ics.plummer(16384 + 123, 1),
                           dict(n_grp=64, theta=0.5, eps=1.0 / 256)),
    "uniform_20k_grp256": (lambda: ics.uniform_sphere(20000, 5),
                           dict(n_grp=256, theta=0.7, eps=1.0 / 512)),
    "plummer_5k_leaf4_theta03": (lambda: ics.plummer(5000, 9),
                                 dict(n_leaf=4, n_grp=16, theta=0.3, eps=1.0 / 128)),
    "galaxy_40k_quad": (lambda: ics.galaxy(40000, 3),
                        dict(n_grp=512, theta=0.4, eps=1.0 / 2048, quad=True)),
    # leaves of up to 80 particles: long link windows (n_leaf + 1 keys) and
    # groups of up to 160
    "plummer_30k_leaf80": (lambda: ics.plummer(30000 + 11, 12),
                           dict(n_leaf=80, n_grp=160, theta=0.5, eps=1.0 / 512)),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_structure_and_force_parity(env, name):
    _, _, orc = env
    make, kw = CASES[name]
    p = make()
    g, a, _ = run_gpu(env, p, **kw)
    t = orc.Tree(p.x, p.y, p.z, p.m, **kw)
    check_structure(g, t, quad=kw.get("quad", False))
    ref = t.force()
    assert np.all(np.isfinite(a))
    assert rms_rel_acc(a, ref) <= FORCE_RMS_TOL
    assert rms_rel_pot(a, ref) <= POT_RMS_TOL
    g.close()


def test_clustered_and_coincident(env):
    """Clumps, exact duplicates and a max-depth leaf cut into chunks."""
    _, _, orc = env
    a = ics.plummer(3000, 4)
    b = ics.plummer(2000, 5)
    n_dup = 700
    x = np.concatenate([a.x, 0.01 * b.x + 3.0, np.full(n_dup, -2.0)])
    y = np.concatenate([a.y, 0.01 * b.y, np.full(n_dup, 1.0)])
    z = np.concatenate([a.z, 0.01 * b.z, np.full(n_dup, 0.5)])
    m = np.full(x.shape[0], 1.0 / x.shape[0])
    p = ics.Particles(x, y, z, x * 0, x * 0, x * 0, m)
    kw = dict(n_grp=64, theta=0.6, eps=1.0 / 512)
    g, acc, _ = run_gpu(env, p, **kw)
    t = orc.Tree(x, y, z, m, **kw)
    check_structure(g, t)
    assert g.stats()["max_level"] == 21
    ref = t.force()
    assert rms_rel_acc(acc[:5000], [r[:5000] for r in ref]) <= FORCE_RMS_TOL
    # duplicates: zero acceleration from each other, potential of the clump exact-ish
    g.close()


@pytest.mark.parametrize("quad", [False, True])
@pytest.mark.parametrize("sizes,n_grp", [
    ([33, 63, 64, 65, 95, 96, 97, 128], 128),
    ([129, 159, 160, 161, 191, 192, 193, 256], 256),
    ([48, 49, 80, 81, 112, 113, 176, 177], 256),
])
def test_group_sizes_around_the_unit_pairing(env, sizes, n_grp, quad):
    """One clump per octant of the root, so each clump is one group of the
    given size: groups of 48, 49, 63, 64, 65, 95, 96, 97, 128 ... particles
    cover every case of the force kernel's work items (a 32-particle unit
    alone, a full unit and the next one of more than 16 particles taken by
    one warp -- 49, 81, 113, 177 -- or of at most 16 left on its own -- 48,
    80, 112, 176 --, a partial last unit split into j-streams), with
    monopole and with quadrupole superparticles (both kernels take the same
    items). Structure bit-exact, forces against the oracle."""
    _, _, orc = env
    rng = np.random.default_rng(31)
    xs, ys, zs = [], [], []
    for o, k in enumerate(sizes):
        c = np.array([(o >> 2) & 1, (o >> 1) & 1, o & 1], dtype=np.float64) - 0.5
        d = rng.normal(scale=0.02, size=(k, 3))
        xs.append(c[0] + d[:, 0]); ys.append(c[1] + d[:, 1]); zs.append(c[2] + d[:, 2])
    x, y, z = (np.concatenate(a) for a in (xs, ys, zs))
    n = x.size
    p = ics.Particles(x, y, z, np.zeros(n), np.zeros(n), np.zeros(n), np.full(n, 1.0 / n))
    kw = dict(n_grp=n_grp, theta=0.5, eps=1.0 / 256, quad=quad)
    g, acc, _ = run_gpu(env, p, **kw)
    t = orc.Tree(p.x, p.y, p.z, p.m, **kw)
    check_structure(g, t, quad=quad)
    assert sorted(t.groups()["count"].tolist()) == sorted(sizes)
    ref = t.force()
    assert rms_rel_acc(acc, ref) <= FORCE_RMS_TOL
    assert rms_rel_pot(acc, ref) <= POT_RMS_TOL
    if quad:  # the far field holds quadrupole terms: other clumps' cells
        assert g.stats()["n_spj"] > 0
    g.close()


@pytest.mark.parametrize("n", [0, 1, 2, 16, 17, 33])
def test_tiny_sizes(env, n):
    _, _, orc = env
    p = ics.plummer(max(n, 1), 12)
    if n == 0:
        p = ics.Particles(*(np.zeros(0) for _ in range(7)))
    kw = dict(n_grp=8, theta=0.5, eps=0.05)
    g, acc, _ = run_gpu(env, p, **kw)
    t = orc.Tree(p.x, p.y, p.z, p.m, **kw)
    if n == 0:
        assert g.stats()["n_cells"] == 0
        g.close()
        return
    check_structure(g, t)
    ref = t.force()
    if n == 1:
        assert np.all(acc == 0)
    else:
        assert rms_rel_acc(acc, ref) <= FORCE_RMS_TOL
    g.close()


def test_signed_zero_coordinates(env):
    """Coordinates of exactly -0.0 and +0.0 on every axis (the root and group
    boxes take min / max on an order-preserving integer key of each double,
    which orders -0 below +0 while the oracle keeps the first of two equal
    values): the boxes compare equal, and everything the method decides is
    the oracle's."""
    _, _, orc = env
    gen = np.random.default_rng(14)
    q = ics.plummer(3000, 14)
    n = q.n
    pos = np.stack([q.x, q.y, q.z], 1)
    # 30% of the particles get one or two coordinates of -0.0 or +0.0 (none
    # sits at the centre, where the net force vanishes and its relative
    # error means nothing)
    sel = gen.random(n) < 0.3
    for i in np.nonzero(sel)[0]:
        axes = gen.choice(3, size=gen.integers(1, 3), replace=False)
        pos[i, axes] = np.where(gen.random(len(axes)) < 0.5, -0.0, 0.0)
    zeros = pos[pos == 0.0]
    assert np.signbit(zeros).any() and (~np.signbit(zeros)).any()
    m = q.m
    p = ics.Particles(pos[:, 0], pos[:, 1], pos[:, 2], m * 0, m * 0, m * 0, m)
    kw = dict(n_grp=32, theta=0.5, eps=1.0 / 64)
    g, acc, _ = run_gpu(env, p, **kw)
    t = orc.Tree(p.x, p.y, p.z, m, **kw)
    check_structure(g, t)
    assert rms_rel_acc(acc, t.force()) <= FORCE_RMS_TOL
    g.close()


@pytest.mark.parametrize("quad", [False, True])
def test_zero_softening(env, quad):
    """eps = 0 takes the guarded kernel: coincident pairs contribute nothing
    (monopole and quadrupole superparticles)."""
    _, _, orc = env
    p = ics.plummer(6000, 21)
    x = p.x.copy()
    x[:10] = x[10]  # ten coincident with particle 10
    y, z = p.y.copy(), p.z.copy()
    y[:10] = y[10]
    z[:10] = z[10]
    q = ics.Particles(x, y, z, p.vx, p.vy, p.vz, p.m)
    kw = dict(n_grp=64, theta=0.5, eps=0.0, quad=quad)
    g, acc, _ = run_gpu(env, q, **kw)
    t = orc.Tree(x, y, z, p.m, **kw)
    check_structure(g, t, quad=quad)
    ref = t.force()
    assert np.all(np.isfinite(acc))
    assert rms_rel_acc(acc[20:], [r[20:] for r in ref]) <= 2e-6
    g.close()


def test_reuse_step_parity(env):
    """MAKE_LIST_FOR_REUSE, drift, REUSE_LIST: same lists, new moments/forces."""
    torch, afd, orc = env
    p = ics.plummer(12000, 31)
    kw = dict(n_grp=64, theta=0.5, eps=1.0 / 256)
    g, _, (x, y, z, m, acc) = run_gpu(env, p, **kw)
    t = orc.Tree(p.x, p.y, p.z, p.m, **kw)
    lists0 = [g.export(k) for k in ("epj_off", "epj_idx", "spj_off", "spj_idx")]
    dt = 0.01
    x2, y2, z2 = p.x + dt * p.vx, p.y + dt * p.vy, p.z + dt * p.vz
    x.copy_(torch.tensor(x2, device=x.device))
    y.copy_(torch.tensor(y2, device=x.device))
    z.copy_(torch.tensor(z2, device=x.device))
    afd.afd_calc_force_all(g.ctx, x, y, z, m, acc, afd.AFD_REUSE_LIST)
    torch.cuda.synchronize()
    t.update(x2, y2, z2, p.m)
    for a, b in zip(lists0, [g.export(k) for k in ("epj_off", "epj_idx", "spj_off", "spj_idx")]):
        assert np.array_equal(a, b)
    M, com, _ = t.moments()
    assert np.array_equal(g.export("cell_mass"), M)
    assert np.array_equal(g.export("cell_com").reshape(-1, 3), com)
    ref = t.force()
    a = acc.cpu().numpy().astype(np.float64)
    assert rms_rel_acc(a, ref) <= FORCE_RMS_TOL
    # a list construction on the moved particles without a new tree
    afd.afd_make_interaction_lists(g.ctx, afd.AFD_MAKE_LIST_FOR_REUSE)
    t.relist()
    check_structure(g, t)
    g.close()


def test_host_entry_point_matches_device(env):
    torch, afd, _ = env
    p = ics.plummer(9000, 41)
    kw = dict(n_grp=64, theta=0.5, eps=1.0 / 256)
    g, a_dev, _ = run_gpu(env, p, **kw)
    out = np.zeros((p.n, 4), dtype=np.float32)
    afd.afd_calc_force_all_host(g.ctx, p.x, p.y, p.z, p.m, out, afd.AFD_MAKE_LIST_FOR_REUSE)
    assert np.array_equal(out.astype(np.float64), a_dev)
    # pinned arrays: the force kernel writes the pinned output directly
    # (construction and reusing steps), the same numbers
    hx, hy, hz, hm = (torch.tensor(a).pin_memory() for a in (p.x, p.y, p.z, p.m))
    pout = torch.full((p.n, 4), float("nan"), dtype=torch.float32).pin_memory()
    for mode in (afd.AFD_MAKE_LIST_FOR_REUSE, afd.AFD_REUSE_LIST):
        pout.fill_(float("nan"))
        afd.afd_calc_force_all_host(g.ctx, hx, hy, hz, hm, pout, mode)
        assert np.array_equal(pout.numpy().astype(np.float64), a_dev)
    g.close()


def test_leapfrog_against_oracle(env):
    torch, afd, orc = env
    p = ics.plummer(4096, 51)
    kw = dict(n_grp=64, theta=0.4, eps=1.0 / 64)
    dt, steps, reuse = 1.0 / 256, 8, 4
    g, _, (x, y, z, m, acc) = run_gpu(env, p, **kw)
    dev = x.device
    vx, vy, vz = (torch.tensor(v, device=dev) for v in p.vel())
    afd.afd_leapfrog(g.ctx, x, y, z, vx, vy, vz, m, acc, dt, steps, reuse)
    ref = orc.leapfrog(p.x, p.y, p.z, p.vx, p.vy, p.vz, p.m, dt=dt, n_steps=steps,
                       n_reuse=reuse, **kw)
    for got, want in zip((x, y, z, vx, vy, vz), ref[:6]):
        assert np.max(np.abs(got.cpu().numpy() - want)) < 1e-7
    K, W = afd.afd_energy(g.ctx, vx, vy, vz, m, acc)
    assert K == pytest.approx(0.5 * np.sum(p.m * (ref[3] ** 2 + ref[4] ** 2 + ref[5] ** 2)), rel=1e-6)
    assert W == pytest.approx(0.5 * np.sum(p.m * ref[9]), rel=1e-5)
    g.close()


def test_errors_are_reported(env):
    torch, afd, _ = env
    dev = torch.device("cuda:0")
    cfg = afd.Config(eps=0.01, theta=0.5, n_grp=32)
    g = afd.Gravity(cfg, 0, torch.cuda.current_stream())
    acc = torch.zeros(100, 4, dtype=torch.float32, device=dev)
    x = torch.rand(100, dtype=torch.float64, device=dev)
    m = torch.full((100,), 0.01, dtype=torch.float64, device=dev)
    with pytest.raises(afd.AfdError) as e:
        afd.afd_calc_force_all(g.ctx, x, x, x, m, acc, afd.AFD_REUSE_LIST)
    assert e.value.status == -4  # no saved lists
    with pytest.raises(afd.AfdError) as e:
        afd.afd_calc_force(g.ctx, acc)
    assert e.value.status == -8  # no tree
    bad = x.clone()
    bad[17] = float("nan")
    with pytest.raises(afd.AfdError) as e:
        afd.afd_calc_force_all(g.ctx, bad, x, x, m, acc, afd.AFD_MAKE_LIST)
    assert e.value.status == -3
    afd.afd_calc_force_all(g.ctx, x, x, x, m, acc, afd.AFD_MAKE_LIST)  # context still usable
    with pytest.raises(afd.AfdError) as e:
        afd.afd_calc_force_all(g.ctx, x, x, x, m, acc, afd.AFD_REUSE_LIST)
    assert e.value.status == -4  # MAKE_LIST does not keep lists
    afd.afd_calc_force_all(g.ctx, x, x, x, m, acc, afd.AFD_MAKE_LIST_FOR_REUSE)
    with pytest.raises(afd.AfdError) as e:
        afd.afd_calc_force_all(g.ctx, x[:50], x[:50], x[:50], m[:50], acc, afd.AFD_REUSE_LIST)
    assert e.value.status == -5
    with pytest.raises(afd.AfdError):
        afd.Gravity(afd.Config(n_grp=0), 0)
    g.close()


def test_sets_without_a_root_cell_are_nonfinite(env):
    """An infinite coordinate, or finite coordinates whose extent has no
    power-of-two side in doubles (+-1e308, or an extent just above 2^1023),
    end the tree build with AFD_ERR_NONFINITE -- the root side is read off the
    bits of the extent, with no loop -- for one system and for a forest, and
    the context stays usable."""
    torch, afd, _ = env
    dev = torch.device("cuda:0")
    n = 3000
    x = torch.rand(n, dtype=torch.float64, device=dev)
    m = torch.full((n,), 1.0 / n, dtype=torch.float64, device=dev)
    acc = torch.zeros(n, 4, dtype=torch.float32, device=dev)
    cases = []
    for v0, v1 in ((float("inf"), None), (float("-inf"), None), (-1e308, 1e308),
                   (0.0, 2.0 ** 1023), (0.0, 1.7976931348623157e308)):
        b = x.clone()
        b[5] = v0
        if v1 is not None:
            b[2000] = v1
        cases.append(b)
    for forest in (False, True):
        g = afd.Gravity(afd.Config(eps=0.01, theta=0.5, n_grp=32), 0, torch.cuda.current_stream())
        if forest:
            afd.afd_set_systems(g.ctx, [0, 1000, n])
        for b in cases:
            for axis in range(3):
                xyz = [x, x, x]
                xyz[axis] = b
                with pytest.raises(afd.AfdError) as e:
                    afd.afd_calc_force_all(g.ctx, *xyz, m, acc, afd.AFD_MAKE_LIST)
                assert e.value.status == -3
        afd.afd_calc_force_all(g.ctx, x, x, x, m, acc, afd.AFD_MAKE_LIST)  # still usable
        torch.cuda.synchronize()
        assert torch.isfinite(acc).all()
        g.close()


def test_full_size_plummer_1m(env):
    """The 2^20-particle Plummer workload in the bench's launch configuration:
    keys, topology, groups and lists bit-exact; forces of sampled groups."""
    _, _, orc = env
    wl = ics.WORKLOADS["plummer_1m"]
    p = ics.plummer(wl["n"], wl["seed"])
    kw = dict(n_grp=wl["n_grp"], theta=wl["theta"], eps=wl["eps"])
    g, a, _ = run_gpu(env, p, **kw)
    t = orc.Tree(p.x, p.y, p.z, p.m, **kw)
    check_structure(g, t)
    ng = t.sizes()["n_groups"]
    sel = np.arange(0, ng, 61)
    ref = t.force_groups(sel)
    mask = np.isfinite(ref[0])
    assert mask.sum() > 5000
    assert rms_rel_acc(a[mask], [r[mask] for r in ref]) <= FORCE_RMS_TOL
    assert rms_rel_pot(a[mask], [r[mask] for r in ref]) <= POT_RMS_TOL
    g.close()


def test_full_size_galaxy_8m(env):
    """The 2^23 galaxy workload (Hernquist halo and exponential disk,
    quadrupole superparticles, theta 0.4, n_grp 512) with the force launch
    shape autotuned on its lists, as the bench runs it: keys, topology,
    moments, groups and lists bit-exact (quadrupoles to 1e-12); forces of
    every 97th group against the oracle's FP64 sum on the same lists."""
    torch, afd, orc = env
    wl = ics.WORKLOADS["galaxy_8m"]
    p = ics.make(wl["model"], wl["n"], wl["seed"])
    kw = dict(n_grp=wl["n_grp"], theta=wl["theta"], eps=wl["eps"], quad=True)
    g, _, (_, _, _, _, acc) = run_gpu(env, p, **kw)
    afd.afd_autotune_launch(g.ctx, acc, reps=1)
    afd.afd_calc_force(g.ctx, acc)
    torch.cuda.synchronize()
    a = acc.cpu().numpy().astype(np.float64)
    t = orc.Tree(p.x, p.y, p.z, p.m, **kw)
    check_structure(g, t, quad=True)
    ng = t.sizes()["n_groups"]
    ref = t.force_groups(np.arange(0, ng, 97))
    mask = np.isfinite(ref[0])
    assert mask.sum() > 50000
    assert rms_rel_acc(a[mask], [r[mask] for r in ref]) <= FORCE_RMS_TOL
    assert rms_rel_pot(a[mask], [r[mask] for r in ref]) <= POT_RMS_TOL
    g.close()


def test_full_size_batch32(env):
    """The 32-system batched workload (N log-uniform in [2^12, 2^20], 7.1M
    particles in all) with n_grp autotuned per system and one launch per
    kernel over all systems, as the bench runs it: for four systems (the
    largest, the smallest and two others) root, keys, permutation, topology,
    groups and lists equal those of an oracle run on the system alone with
    the system's tuned n_grp (ids shifted by the system's offsets), and the
    system's forces match the oracle's."""
    torch, afd, orc = env
    wl = ics.WORKLOADS["batch32"]
    p, off, _ = ics.make_batch(wl["n_systems"], wl["seed"])
    dev = torch.device("cuda:0")
    x, y, z, m = (torch.tensor(a, dtype=torch.float64, device=dev) for a in (p.x, p.y, p.z, p.m))
    acc = torch.zeros(p.n, 4, dtype=torch.float32, device=dev)
    kw = dict(theta=wl["theta"], eps=wl["eps"])
    g = afd.Gravity(afd.Config(n_grp=wl["n_grp"], **kw), 0, torch.cuda.current_stream())
    afd.afd_set_systems(g.ctx, off)
    tuned = afd.afd_autotune_n_grp(g.ctx, x, y, z, m, acc, [32, 64, 128, 256, 512], 4,
                                   n_sys=wl["n_systems"])
    g.force_all(x, y, z, m, acc, afd.AFD_MAKE_LIST_FOR_REUSE)
    torch.cuda.synchronize()
    a = acc.cpu().numpy().astype(np.float64)
    roots = g.export("root").reshape(-1, 4)
    keys, perm = g.export("keys"), g.export("perm")
    lv, fi, ct = g.export("cell_level"), g.export("cell_first"), g.export("cell_count")
    pa, sk = g.export("cell_parent"), g.export("cell_skip")
    gf, gc = g.export("group_first"), g.export("group_count")
    eo, e, so, s = (g.export(k) for k in ("epj_off", "epj_idx", "spj_off", "spj_idx"))
    sizes = np.diff(off)
    # each system's cells and groups are contiguous, found by their first particle
    csys = np.searchsorted(off, fi.astype(np.int64), side="right") - 1
    gsys = np.searchsorted(off, gf.astype(np.int64), side="right") - 1
    picks = sorted({int(np.argmax(sizes)), int(np.argmin(sizes)), 7, 20})
    for k in picks:
        sl = slice(off[k], off[k + 1])
        q = [v[sl] for v in (p.x, p.y, p.z, p.m)]
        t = orc.Tree(*q, n_grp=int(tuned[k]), **kw)
        assert np.array_equal(roots[k], t.root())
        tk, tp = t.order()
        assert np.array_equal(keys[sl], tk)
        assert np.array_equal(perm[sl].astype(np.int64), tp + off[k])
        cidx = np.nonzero(csys == k)[0]
        c0, nc = int(cidx[0]), len(cidx)
        assert np.array_equal(cidx, np.arange(c0, c0 + nc))
        c = t.cells()
        cs = slice(c0, c0 + nc)
        assert nc == len(c.level)
        assert np.array_equal(lv[cs], c.level) and np.array_equal(ct[cs], c.count)
        assert np.array_equal(fi[cs].astype(np.int64), c.first + off[k])
        assert np.array_equal(sk[cs].astype(np.int64), c.skip + c0)
        assert np.array_equal(np.where(pa[cs] == NONE, -1, pa[cs].astype(np.int64) - c0), c.parent)
        gidx = np.nonzero(gsys == k)[0]
        g0, ng = int(gidx[0]), len(gidx)
        gr = t.groups()
        assert ng == len(gr["first"])
        assert np.array_equal(gf[g0:g0 + ng].astype(np.int64), gr["first"] + off[k])
        assert np.array_equal(gc[g0:g0 + ng], gr["count"].astype(np.uint32))
        teo, te, tso, ts = t.lists()
        assert np.array_equal(np.diff(eo[g0:g0 + ng + 1]).astype(np.int64), np.diff(teo))
        assert np.array_equal(np.diff(so[g0:g0 + ng + 1]).astype(np.int64), np.diff(tso))
        assert np.array_equal(e[eo[g0]:eo[g0 + ng]].astype(np.int64), te + off[k])
        assert np.array_equal(s[so[g0]:so[g0 + ng]].astype(np.int64), ts + c0)
        ref = t.force()
        assert rms_rel_acc(a[sl], ref) <= FORCE_RMS_TOL
        assert rms_rel_pot(a[sl], ref) <= POT_RMS_TOL
    g.close()


@pytest.mark.parametrize("learned", [False, True])
def test_batched_systems_match_per_system_oracle(env, learned):
    """Several independent systems in one context (one set of launches): each
    system's root, keys, tree, groups, lists and forces equal those of an
    oracle run on that system alone (ids shifted by the system's offsets) --
    with the theta criterion, and with the learned criterion (reference |a|
    per system from the oracle's direct sum, random FP16 network)."""
    torch, afd, orc = env
    sizes = [3000, 17, 1, 12000, 5000, 0, 700]
    n_grp = [64, 8, 64, 128, 32, 16, 256]
    parts = []
    for k, n in enumerate(sizes):
        p = ics.plummer(max(n, 1), 300 + k, virial=0.3 + 0.05 * k)
        if n == 0:
            p = ics.Particles(*(np.zeros(0) for _ in range(7)))
        shift = 5.0 * k  # systems apart in space (independent regardless)
        parts.append((p.x + shift, p.y - shift, p.z, p.m))
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    X = [np.concatenate([q[i] for q in parts]) for i in range(4)]
    kw = dict(theta=0.5, eps=1.0 / 256)
    dev = torch.device("cuda:0")
    g = afd.Gravity(afd.Config(n_grp=64, mac=int(learned), **kw), 0, torch.cuda.current_stream())
    afd.afd_set_systems(g.ctx, off, n_grp)
    x, y, z, m = (torch.tensor(a, device=dev) for a in X)
    mac, amags = None, []
    if learned:
        gen = np.random.default_rng(77)
        w = gen.normal(0.0, 0.3, orc.MAC_NP).astype(np.float32)
        w[:8] = gen.normal(0.0, 2.0, 8)
        w[8:16] = 0.25
        mac = dict(params=orc.fp16_round(w), theta_lo=0.25, theta_hi=1.0, tau=0.0)
        for q in parts:
            if len(q[0]) == 0:
                amags.append(np.zeros(0, np.float32))
                continue
            ax, ay, az, _ = orc.direct_sum(*q, kw["eps"])
            amags.append(np.sqrt(ax * ax + ay * ay + az * az).astype(np.float32))
        afd.afd_mac_set(g.ctx, w, 0.25, 1.0, 0.0)
        afd.afd_mac_set_reference(g.ctx, torch.tensor(np.concatenate(amags), device=dev))
    acc = torch.full((off[-1], 4), float("nan"), dtype=torch.float32, device=dev)
    g.force_all(x, y, z, m, acc, afd.AFD_MAKE_LIST_FOR_REUSE)
    torch.cuda.synchronize()
    a = acc.cpu().numpy().astype(np.float64)
    roots = g.export("root").reshape(-1, 4)
    keys, perm = g.export("keys"), g.export("perm")
    lv, fi, ct = g.export("cell_level"), g.export("cell_first"), g.export("cell_count")
    pa, sk = g.export("cell_parent"), g.export("cell_skip")
    gf, gc = g.export("group_first"), g.export("group_count")
    eo, e, so, s = (g.export(k) for k in ("epj_off", "epj_idx", "spj_off", "spj_idx"))
    cbase = gbase = 0
    gspj = {}
    for k, n in enumerate(sizes):
        sl = slice(off[k], off[k + 1])
        q = parts[k]
        t = orc.Tree(*q, n_grp=n_grp[k], mac=mac, amag=amags[k] if learned else None, **kw)
        if n == 0:
            assert t.sizes()["n_cells"] == 0
            continue
        assert np.array_equal(roots[k], t.root())
        tk, tp = t.order()
        assert np.array_equal(keys[sl], tk) and np.array_equal(perm[sl].astype(np.int64), tp + off[k])
        c = t.cells()
        nc = len(c.level)
        cs = slice(cbase, cbase + nc)
        assert np.array_equal(lv[cs], c.level) and np.array_equal(ct[cs], c.count)
        assert np.array_equal(fi[cs].astype(np.int64), c.first + off[k])
        assert np.array_equal(sk[cs].astype(np.int64), c.skip + cbase)
        assert np.array_equal(np.where(pa[cs] == NONE, -1, pa[cs].astype(np.int64) - cbase), c.parent)
        gr = t.groups()
        ng = len(gr["first"])
        gs = slice(gbase, gbase + ng)
        assert np.array_equal(gf[gs].astype(np.int64), gr["first"] + off[k])
        assert np.array_equal(gc[gs], gr["count"].astype(np.uint32))
        if learned:
            # pairs within the rounding bound of tau take the kernel's
            # decision (two FP32 summation orders of the network's output)
            gspj[k] = (so[gbase:gbase + ng + 1].astype(np.int64) - int(so[gbase]),
                       s[so[gbase]:so[gbase + ng]].astype(np.int64) - cbase)
            band, flips = t.relist_band(*gspj[k])
            assert flips <= band <= max(10, len(gspj[k][1]) // 20)
        teo, te, tso, ts = t.lists()
        assert np.array_equal(np.diff(eo[gbase:gbase + ng + 1]).astype(np.int64), np.diff(teo))
        assert np.array_equal(np.diff(so[gbase:gbase + ng + 1]).astype(np.int64), np.diff(tso))
        assert np.array_equal(e[eo[gbase]:eo[gbase + ng]].astype(np.int64), te + off[k])
        assert np.array_equal(s[so[gbase]:so[gbase + ng]].astype(np.int64), ts + cbase)
        ref = t.force()
        if n > 1:
            assert rms_rel_acc(a[sl], ref) <= FORCE_RMS_TOL
            assert rms_rel_pot(a[sl], ref) <= POT_RMS_TOL
        else:
            assert np.all(a[sl] == 0)
        cbase += nc
        gbase += ng
    assert cbase == len(lv) and gbase == len(gf)
    # a reusing step on the batch after a drift
    x += 1e-3
    afd.afd_calc_force_all(g.ctx, x, y, z, m, acc, afd.AFD_REUSE_LIST)
    torch.cuda.synchronize()
    a2 = acc.cpu().numpy().astype(np.float64)
    for k, n in enumerate(sizes):
        if n < 2:
            continue
        sl = slice(off[k], off[k + 1])
        t = orc.Tree(*parts[k], n_grp=n_grp[k], mac=mac, amag=amags[k] if learned else None,
                     **kw)
        if learned:
            t.relist_band(*gspj[k])
        t.update(parts[k][0] + 1e-3, parts[k][1], parts[k][2], parts[k][3])
        assert rms_rel_acc(a2[sl], t.force()) <= FORCE_RMS_TOL
    g.close()


def test_graph_replay_equals_direct_steps(env):
    """A captured reusing timestep replays exactly what the direct calls do."""
    torch, afd, _ = env
    p = ics.plummer(20000, 77)
    kw = dict(n_grp=64, theta=0.5, eps=1.0 / 256)
    dev = torch.device("cuda:0")
    stream = torch.cuda.Stream()
    dt = 1.0 / 256
    results = []
    for use_graph in (False, True):
        with torch.cuda.stream(stream):
            g = afd.Gravity(afd.Config(**kw), 0, stream)
            x, y, z, vx, vy, vz, m = (torch.tensor(a, device=dev) for a in
                                      (p.x, p.y, p.z, p.vx, p.vy, p.vz, p.m))
            acc = torch.zeros(p.n, 4, dtype=torch.float32, device=dev)
            afd.afd_calc_force_all(g.ctx, x, y, z, m, acc, afd.AFD_MAKE_LIST_FOR_REUSE)
            if use_graph:
                afd.afd_graph_capture_step(g.ctx, x, y, z, vx, vy, vz, m, acc, dt)
                for _ in range(3):
                    afd.afd_graph_launch(g.ctx)
            else:
                for _ in range(3):
                    afd.afd_kick_drift(g.ctx, x, y, z, vx, vy, vz, acc, 0.5 * dt, dt)
                    afd.afd_calc_force_all(g.ctx, x, y, z, m, acc, afd.AFD_REUSE_LIST)
                    afd.afd_kick(g.ctx, vx, vy, vz, acc, 0.5 * dt)
            stream.synchronize()
            results.append([t.cpu().numpy() for t in (x, y, z, vx, vy, vz, acc)])
            g.close()
    for a, b in zip(*results):
        assert np.array_equal(a, b)


def test_autotuner_installs_candidates_and_stays_exact(env):
    torch, afd, orc = env
    sizes = [4000, 9000, 600, 2500]
    parts = [ics.plummer(n, 500 + k) for k, n in enumerate(sizes)]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    X = [np.concatenate([getattr(q, a) for q in parts]) for a in "xyzm"]
    kw = dict(theta=0.5, eps=1.0 / 256)
    dev = torch.device("cuda:0")
    g = afd.Gravity(afd.Config(n_grp=64, **kw), 0, torch.cuda.current_stream())
    afd.afd_set_systems(g.ctx, off)
    x, y, z, m = (torch.tensor(a, device=dev) for a in X)
    acc = torch.zeros(off[-1], 4, dtype=torch.float32, device=dev)
    cand = [16, 64, 256]
    best = afd.afd_autotune_n_grp(g.ctx, x, y, z, m, acc, cand, 4, n_sys=len(sizes))
    assert all(b in cand for b in best)
    g.force_all(x, y, z, m, acc, afd.AFD_MAKE_LIST_FOR_REUSE)
    torch.cuda.synchronize()
    a = acc.cpu().numpy().astype(np.float64)
    inter, entries = afd.afd_system_stats(g.ctx, len(sizes))
    for k, q in enumerate(parts):
        t = orc.Tree(q.x, q.y, q.z, q.m, n_grp=int(best[k]), **kw)
        assert inter[k] == t.interactions()
        sl = slice(off[k], off[k + 1])
        assert rms_rel_acc(a[sl], t.force()) <= FORCE_RMS_TOL
    g.close()


@pytest.mark.parametrize("far,tol", [(1, 2e-3), (2, 2e-4)])
def test_half_precision_far_field(env, far, tol):
    """BF16 (far=1) / FP16 (far=2) far-field terms (formed in half precision
    with a per-group power-of-two scale, accumulated in FP32) on the same
    lists as the FP64 oracle: the difference stays within a few units of the
    half format's roundoff times the far field's share of the force."""
    torch, afd, orc = env
    p = ics.plummer(60000, 91)
    kw = dict(n_grp=256, theta=0.6, eps=1.0 / 1024)
    dev = torch.device("cuda:0")
    cfg = afd.Config(multipole=1, far_precision=far, **kw)
    g = afd.Gravity(cfg, 0, torch.cuda.current_stream())
    x, y, z, m = (torch.tensor(a, device=dev) for a in (p.x, p.y, p.z, p.m))
    acc = torch.zeros(p.n, 4, dtype=torch.float32, device=dev)
    g.force_all(x, y, z, m, acc, afd.AFD_MAKE_LIST_FOR_REUSE)
    torch.cuda.synchronize()
    t = orc.Tree(p.x, p.y, p.z, p.m, quad=True, **kw)
    check_structure(g, t, quad=True)
    ref = t.force()
    a = acc.cpu().numpy().astype(np.float64)
    assert rms_rel_acc(a, ref) <= tol
    assert rms_rel_pot(a, ref) <= tol
    g.close()


def test_half_far_field_scale_holds_any_mass_unit(env):
    """The per-group power-of-two scale of the half-precision far field: with
    every mass multiplied by 2^-60 or 2^+60 the terms M / rs^2 lie far
    outside FP16's range (2^-24 .. 2^16), yet the scaled terms do not: each
    group's scale moves by exactly 2^-+60, so the half-precision operands are
    the unit-mass run's bit for bit, and the forces scale exactly with the
    masses (every other quantity stays a normal FP32 / FP64 number)."""
    torch, afd, orc = env
    p = ics.plummer(30000, 93)
    kw = dict(n_grp=128, theta=0.6, eps=1.0 / 512)
    dev = torch.device("cuda:0")
    x, y, z = (torch.tensor(a, device=dev) for a in (p.x, p.y, p.z))
    out = {}
    for k in (0, -60, 60):
        m = torch.tensor(p.m * 2.0 ** k, device=dev)
        g = afd.Gravity(afd.Config(multipole=1, far_precision=2, **kw), 0,
                        torch.cuda.current_stream())
        acc = torch.zeros(p.n, 4, dtype=torch.float32, device=dev)
        g.force_all(x, y, z, m, acc, afd.AFD_MAKE_LIST)
        torch.cuda.synchronize()
        out[k] = acc.cpu().numpy().astype(np.float64)
        g.close()
    assert np.all(np.isfinite(out[0]))
    for k in (-60, 60):
        assert np.array_equal(out[k] * 2.0 ** -k, out[0]), k


def test_mixed_precision_workload_against_direct_sum(env, capsys):
    """The N = 2^22 Plummer workload with quadrupole superparticles at
    theta = 0.6: FP32, BF16 and FP16 far field, rms and max relative force
    error against the FP64 direct sum on 4096 seeded sample particles. The
    whole far-field term is formed in half precision: FP16 (11 significant
    bits) adds little to the multipole error; BF16 (8 bits, unit roundoff
    2^-9 per operation of the term) adds about as much again, so its bound
    is twice the FP32 error."""
    torch, afd, orc = env
    wl = ics.WORKLOADS["plummer_4m_mixed"]
    p = ics.plummer(wl["n"], wl["seed"])
    samples = np.random.Generator(np.random.Philox(4096)).choice(p.n, 4096, replace=False)
    ref = orc.direct_sum(p.x, p.y, p.z, p.m, wl["eps"], samples)
    dev = torch.device("cuda:0")
    x, y, z, m = (torch.tensor(a, device=dev) for a in (p.x, p.y, p.z, p.m))
    acc = torch.zeros(p.n, 4, dtype=torch.float32, device=dev)
    errs = {}
    for far in (0, 1, 2):
        cfg = afd.Config(eps=wl["eps"], theta=wl["theta"], n_grp=wl["n_grp"], multipole=1,
                         far_precision=far)
        g = afd.Gravity(cfg, 0, torch.cuda.current_stream())
        g.force_all(x, y, z, m, acc, afd.AFD_MAKE_LIST_FOR_REUSE)
        torch.cuda.synchronize()
        a = acc.cpu().numpy().astype(np.float64)[samples]
        num = np.sqrt((a[:, 0] - ref[0]) ** 2 + (a[:, 1] - ref[1]) ** 2 + (a[:, 2] - ref[2]) ** 2)
        rel = num / np.sqrt(ref[0] ** 2 + ref[1] ** 2 + ref[2] ** 2)
        errs[far] = (float(np.sqrt(np.mean(rel ** 2))), float(rel.max()))
        g.close()
    with capsys.disabled():
        for far, name in ((0, "fp32"), (1, "bf16"), (2, "fp16")):
            print(f"\nmixed-precision far field {name}: rms rel err {errs[far][0]:.4e} "
                  f"max {errs[far][1]:.4e}")
    # the far-field precision barely moves the tree's own error
    assert errs[0][0] < 5e-3
    assert errs[2][0] < 1.05 * errs[0][0] and errs[1][0] < 2.0 * errs[0][0]


def test_force_launch_shapes(env):
    """Every launch shape the autotuner can pick gives oracle-matching forces."""
    torch, afd, orc = env
    p = ics.plummer(20000 + 5, 61)
    kw = dict(n_grp=128, theta=0.5, eps=1.0 / 256)
    g, _, (x, y, z, m, acc) = run_gpu(env, p, **kw)
    t = orc.Tree(p.x, p.y, p.z, p.m, **kw)
    ref = t.force()
    for chunk in (32, 64):
        for warps in (2, 4, 8):
            afd.afd_set_launch(g.ctx, warps, chunk)
            acc.fill_(float("nan"))
            afd.afd_calc_force(g.ctx, acc)
            torch.cuda.synchronize()
            a = acc.cpu().numpy().astype(np.float64)
            assert np.all(np.isfinite(a)), (warps, chunk)
            assert rms_rel_acc(a, ref) <= FORCE_RMS_TOL, (warps, chunk)
    w, c, ms = afd.afd_autotune_launch(g.ctx, acc, reps=2)
    assert (w, c) in [(ww, cc) for cc in (32, 64) for ww in (2, 4, 8)]
    assert ms.shape == (2, 3) and np.all(ms > 0)
    assert afd.afd_get_launch(g.ctx) == (w, c)
    with pytest.raises(afd.AfdError):
        afd.afd_set_launch(g.ctx, 3, 32)
    g.close()


def test_materialized_lists_ablation_is_bit_identical(env):
    """The non-indirect ablation (j-data copied into list order, read without
    indices) computes the same forces as the indirect kernel, bit for bit,
    and both match the oracle's FP64 force on the oracle's own lists."""
    torch, afd, orc = env
    p = ics.plummer(20000 + 11, 71)
    kw = dict(n_grp=64, theta=0.5, eps=1.0 / 256)
    g, a_ind, (x, y, z, m, acc) = run_gpu(env, p, **kw)
    t = orc.Tree(p.x, p.y, p.z, p.m, **kw)
    check_structure(g, t)
    acc.fill_(float("nan"))
    t_copy, t_force = afd.afd_calc_force_materialized(g.ctx, acc)
    assert t_copy > 0 and t_force > 0
    a_mat = acc.cpu().numpy().astype(np.float64)
    assert np.array_equal(a_mat, a_ind)
    ref = t.force()
    assert rms_rel_acc(a_mat, ref) <= FORCE_RMS_TOL
    assert rms_rel_pot(a_mat, ref) <= POT_RMS_TOL
    g.close()
    gq, _, (_, _, _, _, accq) = run_gpu(env, p, quad=True, **kw)
    with pytest.raises(afd.AfdError):
        afd.afd_calc_force_materialized(gq.ctx, accq)
    gq.close()


@pytest.mark.parametrize("parts", [2, 3, 8])
def test_work_share_slices_sum_to_the_whole_force(env, parts):
    """A force step split by group slices (afd_set_work_share): every part
    writes only its groups' rows; the parts summed equal the unshared forces
    bit for bit, the slices tile the groups, and their interactions add up --
    also on a reusing step."""
    torch, afd, orc = env
    p = ics.plummer(20000, 41)
    kw = dict(n_grp=64, theta=0.5, eps=1.0 / 256)
    dev = torch.device("cuda:0")
    X = [torch.tensor(a, device=dev) for a in (p.x, p.y, p.z, p.m)]
    whole = afd.Gravity(afd.Config(**kw), 0, torch.cuda.current_stream())
    ref = torch.zeros(p.n, 4, dtype=torch.float32, device=dev)
    whole.force_all(*X, ref, afd.AFD_MAKE_LIST_FOR_REUSE)
    n_groups, inter = whole.stats()["n_groups"], whole.stats()["interactions"]
    moved = [X[0] + 1e-4, X[1], X[2], X[3]]
    ref2 = torch.zeros_like(ref)
    afd.afd_calc_force_all(whole.ctx, *moved, ref2, afd.AFD_REUSE_LIST)
    tot = torch.zeros_like(ref)
    tot2 = torch.zeros_like(ref)
    bounds, inters = [0], 0
    for part in range(parts):
        g = afd.Gravity(afd.Config(**kw), 0, torch.cuda.current_stream())
        afd.afd_set_work_share(g.ctx, part, parts)
        acc = torch.zeros_like(ref)
        g.force_all(*X, acc, afd.AFD_MAKE_LIST_FOR_REUSE)
        sh = afd.afd_get_work_share(g.ctx)
        assert sh["g0"] == bounds[-1]
        bounds.append(sh["g1"])
        inters += sh["interactions"]
        tot += acc
        acc2 = torch.zeros_like(ref)
        afd.afd_calc_force_all(g.ctx, *moved, acc2, afd.AFD_REUSE_LIST)
        tot2 += acc2
        g.close()
    torch.cuda.synchronize()
    assert bounds[-1] == n_groups and inters == inter
    assert torch.equal(tot, ref) and torch.equal(tot2, ref2)
    whole.close()


def test_bounded_walk_loops_stop_with_a_status(env):
    """The walks' bounded device loops, made to run out on a small tree by
    lowered limits: the iteration cap returns AFD_ERR_TIMEOUT (gravity and
    neighbour walks), the stack bound AFD_ERR_WALK_STACK, a record arena
    capped below what the lists need AFD_ERR_LIST_OVERFLOW; after each the
    context has no lists, and with the limits restored it makes the oracle's
    lists again."""
    torch, afd, orc = env
    p = ics.plummer(20000, 81)
    kw = dict(n_grp=64, theta=0.5, eps=1.0 / 256)
    dev = torch.device("cuda:0")
    X = [torch.tensor(a, device=dev) for a in (p.x, p.y, p.z, p.m)]
    g = afd.Gravity(afd.Config(**kw), 0, torch.cuda.current_stream())
    afd.afd_tree_build(g.ctx, *X)
    acc = torch.zeros(p.n, 4, dtype=torch.float32, device=dev)
    h = torch.full((p.n,), 0.05, dtype=torch.float64, device=dev)
    t = orc.Tree(p.x, p.y, p.z, p.m, **kw)
    for limits, status in (((3, 0, 0), -7), ((0, 12, 0), -10), ((0, 0, 8), -6)):
        afd.afd_set_walk_limits(g.ctx, *limits)
        with pytest.raises(afd.AfdError) as e:
            afd.afd_make_interaction_lists(g.ctx, afd.AFD_MAKE_LIST_FOR_REUSE)
        assert e.value.status == status, limits
        assert g.stats()["saved"] == 0
        with pytest.raises(afd.AfdError) as e:
            afd.afd_calc_force(g.ctx, acc)
        assert e.value.status == -4  # no lists
        if status == -7:
            with pytest.raises(afd.AfdError) as e:
                afd.afd_make_neighbour_lists(g.ctx, h, 0.0)
            assert e.value.status == -7
        afd.afd_set_walk_limits(g.ctx, 0, 0, 0)
        afd.afd_make_interaction_lists(g.ctx, afd.AFD_MAKE_LIST_FOR_REUSE)
        afd.afd_calc_force(g.ctx, acc)
        torch.cuda.synchronize()
        check_structure(g, t)
        assert rms_rel_acc(acc.cpu().numpy().astype(np.float64), t.force()) <= FORCE_RMS_TOL
    for bad in ((-1, 0, 0), (0, 449, 0), (0, -1, 0), (0, 0, (1 << 30) + 1)):
        with pytest.raises(afd.AfdError) as e:
            afd.afd_set_walk_limits(g.ctx, *bad)
        assert e.value.status == -1
    g.close()
