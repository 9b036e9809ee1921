"""Pins for the oracle's learned opening criterion (readings R12-R15 of the
oracle; the criterion is not in the paper, which opens cells by angle only,
Section 2). Each test checks the oracle against a closed form, a finite
difference, a special case that reduces to the theta criterion, or brute
force. No GPU needed."""
import math

import numpy as np
import pytest

import ics


# ---------------------------------------------------------------- lg2


def test_lg2_exact_at_powers_of_two(orc):
    e = np.arange(-126, 128)
    x = np.ldexp(np.float32(1.0), e).astype(np.float32)
    assert np.array_equal(orc.lg2(x), e.astype(np.float32))


def test_lg2_close_to_log2_and_special_values(orc):
    g = np.random.default_rng(3)
    x = np.exp2(g.uniform(-120, 120, 20000)).astype(np.float32)
    err = np.abs(orc.lg2(x).astype(np.float64) - np.log2(x.astype(np.float64)))
    # fit error 1.8e-5 plus the FP32 rounding of values up to 127
    assert err.max() < 2e-5 + 127 * 2.0 ** -23
    special = np.array([0.0, -1.0, np.float32(1e-40), np.nan, np.inf], dtype=np.float32)
    assert list(orc.lg2(special)) == [-127.0, -127.0, -127.0, -127.0, 128.0]


# ---------------------------------------------------------------- features


def _features_case(orc, **over):
    """Group box [0,1]^3, cell COM at (3, 0.5, 0.5) (d = 2, u = (-2.5, 0, 0)),
    s = 0.5, M = 0.25, Q = q diag(2, -1, -1), 8 particles, eps = 1/64,
    smallest reference |a| = 4."""
    q = 0.01
    args = dict(bmin=[0.0, 0.0, 0.0], bmax=[1.0, 1.0, 1.0], com=[3.0, 0.5, 0.5], s2=0.25,
                M=0.25, Q=[2 * q, -q, -q, 0.0, 0.0, 0.0], count=8, eps2=(1 / 64) ** 2, amin=4.0)
    args.update(over)
    return orc.mac_features(**args), args


def test_features_closed_form(orc):
    f, a = _features_case(orc)
    q = 0.01
    d, s, M, A = 2.0, 0.5, 0.25, 4.0
    qf = q * math.sqrt(6.0)  # Frobenius norm of q diag(2, -1, -1)
    expect = [math.log2(s / d), math.log2(M / (d * d * A)), math.log2(qf / (M * s * s)),
              math.log2(math.sqrt(3.0) / 2 / d), math.log2(8), math.log2((1 / 64) / d),
              2.0 / math.sqrt(6.0),  # u along x: u.Q.u / (|u|^2 |Q|) = 2q / (sqrt(6) q)
              math.log2(2.5 / d)]
    assert np.allclose(f, expect, rtol=0, atol=1e-4), (f, expect)


def test_features_each_input_moves_its_own_feature(orc):
    base, _ = _features_case(orc)
    cases = {  # input change -> the features it must move (and only those)
        "M": (dict(M=0.5), {1, 2}),
        "amin": (dict(amin=8.0), {1}),
        "count": (dict(count=64), {4}),
        "eps2": (dict(eps2=(1 / 32) ** 2), {5}),
        "s2": (dict(s2=1.0), {0, 2}),
        "Q": (dict(Q=[0.0, 0.02, -0.02, 0.0, 0.0, 0.0]), {2, 6}),
        "box": (dict(bmax=[1.0, 2.0, 1.0]), {3, 6, 7}),  # u turns as well
    }
    for name, (over, moved) in cases.items():
        f, _ = _features_case(orc, **over)
        changed = {k for k in range(8) if f[k] != base[k]}
        assert changed == moved, (name, changed)


def test_features_degenerate_inputs_clamp(orc):
    f, _ = _features_case(orc, Q=[0.0] * 6, count=1, bmin=[1.0, 1.0, 1.0], eps2=0.0, amin=0.0)
    assert f[2] == -32.0 and f[6] == 0.0  # no quadrupole
    assert f[3] == -32.0                  # point-like group
    assert f[4] == 0.0                    # one particle
    assert f[5] == -32.0                  # no softening
    assert f[1] == 32.0                   # zero reference acceleration


# ---------------------------------------------------------------- network


def _rand_params(orc, seed, scale=0.4):
    g = np.random.default_rng(seed)
    p = g.normal(0.0, scale, orc.MAC_NP).astype(np.float32)
    p[:8] = g.normal(0.0, 2.0, 8)       # mu
    p[8:16] = g.uniform(0.2, 1.0, 8)    # isd
    return orc.fp16_round(p)


def _np_forward(orc, p, f):
    mu, isd, W1, b1, W2, b2, w3, b3 = orc.mlp_unpack(np.asarray(p, np.float64))
    X = (np.asarray(f, np.float64) - mu) * isd
    H1 = np.maximum(X @ W1.T + b1, 0.0)
    H2 = np.maximum(H1 @ W2.T + b2, 0.0)
    return H2 @ w3 + b3[0]


def test_mlp_forward_hand_worked(orc):
    p = np.zeros(orc.MAC_NP, np.float32)
    mu, isd, W1, b1, W2, b2, w3, b3 = orc.mlp_unpack(p)  # views into p
    isd[:] = 1.0
    mu[:] = 1.0
    for k in range(8):
        W1[k, k] = 1.0
        W2[k, k] = 2.0
        w3[k] = k + 1
    b3[0] = 0.5
    f = np.array([3.0, 0.0, 2.0, 1.0, -4.0, 1.5, 1.0, 5.0], np.float32)
    # h1 = relu(f - 1) = [2, 0, 1, 0, 0, 0.5, 0, 4]; h2 = 2 h1; y = 0.5 + sum (k+1) h2_k
    expect = 0.5 + 2 * (1 * 2 + 3 * 1 + 6 * 0.5 + 8 * 4)
    assert orc.mlp_forward(p, f)[0] == np.float32(expect)


def test_mlp_output_unit_is_the_plain_sequential_sum(orc):
    """R13: the output unit is b3 followed by fused multiply-adds in index
    order. With b3 = 1 and 32 terms of 2^-25 each, every step rounds back to
    1 (a term is below half an ulp of 1), so the definition gives exactly 1;
    a pairwise order would first add the terms exactly (2^-20) and give
    1 + 2^-20. The returned bound covers that other order's result."""
    p = np.zeros(orc.MAC_NP, np.float32)
    mu, isd, W1, b1, W2, b2, w3, b3 = orc.mlp_unpack(p)
    b2[:] = 2.0 ** -13  # h2_j = 2^-13 (all inputs and hidden layers zero)
    w3[:] = 2.0 ** -12  # w3_j h2_j = 2^-25
    b3[0] = 1.0
    f = np.zeros((1, 8), np.float32)
    y, bound = orc.mlp_forward_bound(p, f)
    assert y[0] == np.float32(1.0)
    pairwise = 1.0 + 2.0 ** -20  # exact in FP32
    assert abs(pairwise - float(y[0])) <= bound[0] < 2.0 ** -15
    assert orc.mlp_forward(p, f)[0] == y[0]


def test_rn16_is_the_fp16_rounding(orc):
    """RN16 of R13 against numpy's FP16 conversion (round to nearest, ties
    to even) over normal, subnormal and tie values."""
    g = np.random.default_rng(12)
    v = np.concatenate([
        g.normal(0.0, 10.0, 4000), np.exp2(g.uniform(-30, 15.9, 4000)) * g.choice([-1, 1], 4000),
        (np.arange(-2000, 2000) + 0.5) * 2.0 ** -10,   # ties at the ulp of [1, 2)
        (np.arange(0, 1024) + 0.5) * 2.0 ** -24,       # subnormal ties
        [0.0, -0.0, 65504.0, -65504.0, 6.1e-5, 5.96e-8, 2.9e-8, 3.0e-8]]).astype(np.float32)
    got = np.array([orc.rn16(x) for x in v], np.float32)
    ref = v.astype(np.float16).astype(np.float32)
    assert np.array_equal(got, ref)
    assert np.array_equal(np.signbit(got), np.signbit(ref))


def test_mlp_inputs_and_first_layer_are_fp16(orc):
    """R13 rounds the normalised inputs and the first-layer activations to
    FP16 (ties to even) and saturates the activations at 65504: an input of
    1 + 2^-12 reaches the output as 1, an activation of 2049 as 2048 (FP16
    spacing 2 there), one of 70000 as 65504."""
    p = np.zeros(orc.MAC_NP, np.float32)
    mu, isd, W1, b1, W2, b2, w3, b3 = orc.mlp_unpack(p)
    isd[:] = 1.0
    W1[0, 0] = 1.0   # h1_0 = x_0
    b1[1] = 2049.0   # h1_1 = 2049 -> 2048
    b1[2] = 70000.0  # h1_2 = 70000 -> 65504 (not FP16, but a sum can reach it)
    W2[0, 0] = W2[1, 1] = W2[2, 2] = 1.0
    f = np.array([[1.0 + 2.0 ** -12, 0, 0, 0, 0, 0, 0, 0]], np.float32)
    for k, want in ((0, 1.0), (1, 2048.0), (2, 65504.0)):
        w3[:] = 0.0
        w3[k] = 1.0
        assert orc.mlp_forward(p, f)[0] == np.float32(want), k


def test_mlp_forward_matches_fp64_network(orc):
    """The FP64 evaluation of the same definition (FP16 roundings of inputs
    and first-layer activations, sums in FP64) lies within the returned
    bound, which is small next to the output."""
    p = _rand_params(orc, 5)
    f = np.random.default_rng(6).normal(0.0, 3.0, (500, 8)).astype(np.float32)
    y32, bound = orc.mlp_forward_bound(p, f)
    mu, isd, W1, b1, W2, b2, w3, b3 = orc.mlp_unpack(np.asarray(p, np.float64))
    X = ((f - mu.astype(np.float32)) * isd.astype(np.float32)).astype(np.float16).astype(np.float64)
    P1 = X @ W1.T + b1
    H1 = np.minimum(np.maximum(P1, 0.0), 65504.0).astype(np.float16).astype(np.float64)
    H2 = np.maximum(H1 @ W2.T + b2, 0.0)
    y64 = H2 @ w3 + b3[0]
    assert np.all(np.abs(y32.astype(np.float64) - y64) <= bound)
    assert np.median(bound) < 1e-3 * (1 + np.abs(y64).max())


def test_mlp_backward_matches_finite_differences(orc):
    p = _rand_params(orc, 7).astype(np.float64)
    g = np.random.default_rng(8)
    f = g.normal(0.0, 2.0, (64, 8))
    lab = g.normal(-10.0, 3.0, 64)
    loss, grad = orc.mlp_loss_grad(p, f, lab)
    assert loss == pytest.approx(orc.mlp_loss(p, f, lab), rel=1e-14)
    assert np.all(grad[:16] == 0.0)  # mu, isd are not trained
    h = 1e-6
    idx = np.r_[16:16 + 256:17, 272:304:3, 304:1328:37, 1328:1360:5, 1360:1393:4]
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (orc.mlp_loss(p + e, f, lab) - orc.mlp_loss(p - e, f, lab)) / (2 * h)
        assert fd == pytest.approx(grad[i], rel=1e-5, abs=1e-7), i


# ---------------------------------------------------------------- labels


def test_label_single_particle_cell_is_exact(orc):
    lab = orc.mac_label([[0.0, 0.0, 0.0]], [1.0], [[3.0, 1.0, 0.0]], [0.5], 0.5,
                        [3.0, 1.0, 0.0], np.zeros(6), 0.0, 0)
    assert lab == -40.0


def test_label_symmetric_pair_closed_forms(orc):
    # masses m at (D +- b, 0, 0), one group particle at the origin, eps = 0
    m, b, D, A = 0.125, 0.1, 2.0, 0.5
    xj = [[D - b, 0, 0], [D + b, 0, 0]]
    exact = m / (D - b) ** 2 + m / (D + b) ** 2      # a_x toward +x
    mono = 2 * m / D ** 2
    lab = orc.mac_label([[0, 0, 0]], [A], xj, [m, m], 2 * m, [D, 0, 0], np.zeros(6), 0.0, 0)
    assert lab == pytest.approx(math.log2(abs(mono - exact) / A), abs=1e-9)
    # quadrupole of the pair about its COM: Q_xx = 4 m b^2, Q_yy = Q_zz = -2 m b^2;
    # its term at r = -D x_hat adds 6 m b^2 / D^4 toward +x
    Q = np.array([4 * m * b * b, -2 * m * b * b, -2 * m * b * b, 0, 0, 0])
    quad = mono + 6 * m * b * b / D ** 4
    labq = orc.mac_label([[0, 0, 0]], [A], xj, [m, m], 2 * m, [D, 0, 0], Q, 0.0, 1)
    assert labq == pytest.approx(math.log2(abs(quad - exact) / A), abs=1e-6)
    assert labq < lab - 6  # the next order is (b/D)^2 smaller


def test_label_scales_with_reference_and_takes_the_worst_particle(orc):
    xj = [[2.0, 0.3, 0.0], [2.5, -0.2, 0.1], [2.2, 0.0, -0.3]]
    mj = [0.1, 0.2, 0.15]
    M = sum(mj)
    com = np.sum(np.array(xj) * np.array(mj)[:, None], axis=0) / M
    xi = [[0.0, 0.0, 0.0], [0.5, 0.1, 0.0]]
    l1 = orc.mac_label(xi[:1], [1.0], xj, mj, M, com, np.zeros(6), 0.01, 0)
    l2 = orc.mac_label(xi[1:], [1.0], xj, mj, M, com, np.zeros(6), 0.01, 0)
    both = orc.mac_label(xi, [1.0, 1.0], xj, mj, M, com, np.zeros(6), 0.01, 0)
    assert both == max(l1, l2)
    l8 = orc.mac_label(xi[:1], [8.0], xj, mj, M, com, np.zeros(6), 0.01, 0)
    assert l8 == pytest.approx(l1 - 3.0, abs=1e-12)


# ---------------------------------------------------------------- tree level


@pytest.fixture(scope="module")
def plummer_ref(orc):
    p = ics.plummer(3000, 21)
    ax, ay, az, _ = orc.direct_sum(p.x, p.y, p.z, p.m, 1.0 / 256)
    amag = np.sqrt(ax * ax + ay * ay + az * az).astype(np.float32)
    return p, amag


def _mac(params, lo, hi, tau):
    return dict(params=params, theta_lo=lo, theta_hi=hi, tau=tau)


def test_learned_walk_reduces_to_theta_walks(orc, plummer_ref):
    """A network that always answers 'accept' gives the theta_hi lists, one
    that always answers 'open' the theta_lo lists (theta_hi < 1/sqrt(3): the
    theta criterion never accepts a cell containing the group there)."""
    p, amag = plummer_ref
    kw = dict(n_grp=32, eps=1.0 / 256)
    for b3, th in ((-100.0, 0.55), (100.0, 0.3)):
        w = np.zeros(orc.MAC_NP, np.float32)
        w[8:16] = 1.0
        w[-1] = b3
        tl = orc.Tree(p.x, p.y, p.z, p.m, theta=0.9, mac=_mac(w, 0.3, 0.55, 0.0), amag=amag, **kw)
        tr = orc.Tree(p.x, p.y, p.z, p.m, theta=th, **kw)
        for a, b in zip(tl.lists(), tr.lists()):
            assert np.array_equal(a, b)


def test_learned_lists_partition_and_monotone_in_tau(orc, plummer_ref):
    p, amag = plummer_ref
    w = _rand_params(orc, 9, scale=0.3)
    w[:8] = 0.0
    w[8:16] = 0.25
    prev = None
    M_tot = p.m.sum()
    for tau in (-3.0, 0.0, 3.0):
        t = orc.Tree(p.x, p.y, p.z, p.m, n_grp=32, eps=1.0 / 256,
                     mac=_mac(w, 0.2, 1.2, tau), amag=amag)
        eo, e, so, s = t.lists()
        M, _, _ = t.moments()
        _, perm = t.order()
        ms = p.m[perm]
        c = t.cells()
        gr = t.groups()
        lens = (eo[1:] - eo[:-1]) + (so[1:] - so[:-1])
        for g in range(len(gr["first"])):
            spj = s[so[g]:so[g + 1]]
            tot = ms[e[eo[g]:eo[g + 1]]].sum() + M[spj].sum()
            assert tot == pytest.approx(M_tot, rel=1e-12)
            f0 = gr["first"][g]
            inside = (c.first[spj] <= f0) & (f0 < c.first[spj] + c.count[spj])
            assert not inside.any()  # never approximates a cell holding the group
        if prev is not None:
            assert np.all(lens <= prev)  # a larger tau accepts more, lists shrink
        prev = lens


def test_band_pairs_match_brute_force(orc, plummer_ref):
    """Band pairs of the walk = cells whose every ancestor is opened by the
    'accept below theta_lo' rule and that lie in [theta_lo, theta_hi)."""
    p, amag = plummer_ref
    lo, hi = 0.3, 0.8
    t = orc.Tree(p.x, p.y, p.z, p.m, n_grp=64, eps=1.0 / 256, amag=amag)
    pairs = t.band_pairs(lo, hi)
    c = t.cells()
    gr = t.groups()
    _, com, _ = t.moments()
    L = np.float32(t.root()[3])
    s = np.ldexp(L, -c.level).astype(np.float32)
    s2 = (s * s).astype(np.float32)
    comf = com.astype(np.float32)
    lo2, hi2 = np.float32(lo) * np.float32(lo), np.float32(hi) * np.float32(hi)
    want = set()
    for g in range(len(gr["first"])):
        box = gr["box"][g].astype(np.float32)
        d = np.maximum(np.maximum(box[:3] - comf, comf - box[3:]), np.float32(0))
        d2 = ((d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]).astype(np.float32)
        f0 = gr["first"][g]
        contains = (c.first <= f0) & (f0 < c.first + c.count)
        accept_lo = ~contains & (s2 < lo2 * d2)
        band = ~contains & ~accept_lo & (s2 < hi2 * d2)
        opens = ~accept_lo  # band cells are opened too
        reach = np.zeros(len(c.level), bool)
        reach[0] = True
        for k in range(1, len(c.level)):  # pre-order: parents come first
            reach[k] = reach[c.parent[k]] and opens[c.parent[k]]
        want |= {(g, k) for k in np.nonzero(reach & band)[0]}
    got = {(int(a), int(b)) for a, b in pairs}
    assert len(got) == len(pairs) and got == want


def test_pair_features_and_labels_gather_the_right_data(orc, plummer_ref):
    p, amag = plummer_ref
    t = orc.Tree(p.x, p.y, p.z, p.m, n_grp=32, eps=1.0 / 256, amag=amag)
    pairs = t.band_pairs(0.3, 0.9)[::97]
    f = t.pair_features(pairs)
    lab = t.pair_labels(pairs)
    c = t.cells()
    gr = t.groups()
    M, com, Q = t.moments()
    _, perm = t.order()
    xs = np.stack([p.x[perm], p.y[perm], p.z[perm]], 1)
    ms, am = p.m[perm], amag[perm]
    L = np.float32(t.root()[3])
    e = np.float32(1.0 / 256)
    for (g, k), fk, lk in zip(pairs, f, lab):
        s = np.float32(np.ldexp(L, -int(c.level[k])))
        gi = slice(gr["first"][g], gr["first"][g] + gr["count"][g])
        ref = orc.mac_features(gr["box"][g][:3], gr["box"][g][3:], com[k], s * s, M[k], Q[k],
                               c.count[k], e * e, am[gi].min())
        assert np.array_equal(fk, ref)
        cj = slice(c.first[k], c.first[k] + c.count[k])
        ref_l = orc.mac_label(xs[gi], am[gi], xs[cj], ms[cj], M[k], com[k], Q[k], 1.0 / 256, 0)
        assert lk == ref_l


def test_band_relist_takes_the_other_decision_only_within_the_bound(orc, plummer_ref):
    """The comparison the GPU tests make with the learned walk. A constant
    network b3 = tau puts every band pair exactly on tau (inside the
    rounding bound): the oracle then follows another implementation's
    decisions -- here one that accepts every band cell -- and counts every
    such pair as in the band and as flipped. With b3 = 1, tau = 2 the output
    lies further than the bound from tau: the other implementation's
    decisions (opening every band cell) are ignored, so a kernel that
    decides differently there would show as different lists."""
    p, amag = plummer_ref
    kw = dict(n_grp=32, eps=1.0 / 256)
    lo, hi = 0.3, 0.55

    def const_net(b3):
        w = np.zeros(orc.MAC_NP, np.float32)
        w[8:16] = 1.0
        w[-1] = b3
        return w

    acc = orc.Tree(p.x, p.y, p.z, p.m, mac=_mac(const_net(0.0), lo, hi, 1.0), amag=amag, **kw)
    opn = orc.Tree(p.x, p.y, p.z, p.m, mac=_mac(const_net(2.0), lo, hi, 1.0), amag=amag, **kw)
    a_eo, a_e, a_so, a_s = acc.lists()
    o_eo, o_e, o_so, o_s = opn.lists()
    assert len(a_s) != len(o_s)
    # output on tau: the other (accept-all) decisions are taken, every one a flip
    t = orc.Tree(p.x, p.y, p.z, p.m, mac=_mac(const_net(1.0), lo, hi, 1.0), amag=amag, **kw)
    own = t.lists()
    for a, b in zip(own, opn.lists()):
        assert np.array_equal(a, b)  # its own decision: 1 < 1 is false, open
    band, flips = t.relist_band(a_so, a_s)
    assert band > 0 and flips == band
    for a, b in zip(t.lists(), acc.lists()):
        assert np.array_equal(a, b)
    # every band pair the accept-all walk accepted was visited in the band
    bp = acc.band_pairs(lo, hi)
    band_set = set(zip(bp[:, 0].tolist(), bp[:, 1].tolist()))
    grp = np.repeat(np.arange(len(a_so) - 1), np.diff(a_so))
    accepted_in_band = sum(1 for g, c in zip(grp.tolist(), a_s.tolist()) if (g, c) in band_set)
    assert band >= accepted_in_band > 0
    # output away from tau: the override does not apply
    t2 = orc.Tree(p.x, p.y, p.z, p.m, mac=_mac(const_net(1.0), lo, hi, 2.0), amag=amag, **kw)
    band2, flips2 = t2.relist_band(o_so, o_s)
    assert band2 == 0 and flips2 == 0
    for a, b in zip(t2.lists(), acc.lists()):
        assert np.array_equal(a, b)
