"""GPU parity of the learned opening criterion (not in the paper; the walk
falls back to the paper's theta criterion, Section 2) against the oracle's
readings R12-R15, through the C ABI.

Bit-exact: quadrupole moments (the criterion reads them), the features of
every sampled pair and the set of pairs the band leaves to the network.
The network's output (R13: FP16 inputs and first-layer activations, FP32
sums): the oracle sums in index order, the kernel on the tensor cores in the
tensor core's order; the two must lie within the bound R13 states for two
FP32 summation orders. The interaction lists of the learned walk: equal to
the oracle's, except that for pairs whose oracle output lies within that
bound of tau (where two correct implementations may decide differently)
the oracle takes the kernel's decision; those pairs are counted and
reported. Within tolerance: the targets (GPU FP32 compensated
sums vs oracle FP64) and the network gradients of the GPU backward pass (vs
the oracle's FP64 chain rule, itself pinned by finite differences). Finally
the trained network is judged by brute force: its force error against the
direct sum, compared with the theta criterion at equal error.
"""
import numpy as np
import pytest

import ics
from test_gpu_parity import check_structure, env, rms_rel_acc  # noqa: F401 (fixture)

pytestmark = pytest.mark.gpu

EPS = 1.0 / 256


def dev(torch, a, dtype):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda:0")


def rand_params(orc, seed, scale=0.3):
    g = np.random.default_rng(seed)
    p = g.normal(0.0, scale, orc.MAC_NP).astype(np.float32)
    p[:8] = g.normal(0.0, 2.0, 8)
    p[8:16] = g.uniform(0.2, 1.0, 8)
    return p


@pytest.fixture(scope="module")
def plummer(env):
    """20k Plummer particles and FP32 reference |a| from the oracle's direct sum."""
    _, _, orc = env
    p = ics.plummer(20000 + 77, 41)
    ax, ay, az, _ = orc.direct_sum(p.x, p.y, p.z, p.m, EPS)
    amag = np.sqrt(ax * ax + ay * ay + az * az).astype(np.float32)
    return p, amag


def gpu_ctx(env, p, amag, *, n_grp=64, theta=0.5, quad=False):
    torch, afd, _ = env
    cfg = afd.Config(eps=EPS, theta=theta, n_grp=n_grp, multipole=int(quad), mac=1)
    g = afd.Gravity(cfg, 0, torch.cuda.current_stream())
    xs = [dev(torch, a, torch.float64) for a in (p.x, p.y, p.z, p.m)]
    afd.afd_tree_build(g.ctx, *xs)
    if amag is not None:
        afd.afd_mac_set_reference(g.ctx, dev(torch, amag, torch.float32))
    return g, xs


# ---------------------------------------------------------------- network


def test_forward_within_the_summation_bound_with_fp16_weights(env):
    """Same FP16-rounded parameters and FP16 inputs; the layers' sums in the
    tensor core's order: every output within the bound of R13 of the
    oracle's (many rows of 16, a ragged last one, clamped features)."""
    torch, afd, orc = env
    p = rand_params(orc, 3)
    f = np.random.default_rng(4).normal(0.0, 4.0, (20000, 8)).astype(np.float32)
    f[:100] = 32.0  # clamp edges
    f[100:200] = -32.0
    out = torch.empty(f.shape[0], dtype=torch.float32, device="cuda:0")
    afd.afd_mlp_forward(p, dev(torch, f, torch.float32), out)
    ref, bound = orc.mlp_forward_bound(orc.fp16_round(p), f)
    got = out.cpu().numpy()
    diff = np.abs(got.astype(np.float64) - ref.astype(np.float64))
    assert np.all(diff <= bound), float(np.max(diff / bound))
    equal = float(np.mean(got == ref))
    print(f"network output: {equal:.3f} of rows equal, largest difference "
          f"{float(np.max(diff / bound)):.3f} of the bound")
    # a ragged count: 16 rows per warp step, the last rows padded
    out2 = torch.empty(37, dtype=torch.float32, device="cuda:0")
    afd.afd_mlp_forward(p, dev(torch, f[:37], torch.float32), out2)
    assert np.array_equal(out2.cpu().numpy(), got[:37])


def test_gradient_matches_oracle_backward(env):
    torch, afd, orc = env
    p = rand_params(orc, 5)
    g = np.random.default_rng(6)
    for n in (1, 127, 5000):  # one sample, a ragged tile, many tiles
        f = g.normal(0.0, 2.0, (n, 8)).astype(np.float32)
        lab = g.normal(-10.0, 3.0, n).astype(np.float32)
        loss, grad = afd.afd_mlp_loss_grad(p, dev(torch, f, torch.float32),
                                           dev(torch, lab, torch.float32))
        ref_loss, ref_grad = orc.mlp_loss_grad(p, f, lab)
        assert loss == pytest.approx(ref_loss, rel=1e-4)
        assert np.all(grad[:16] == 0)
        err = np.linalg.norm(grad - ref_grad) / np.linalg.norm(ref_grad)
        assert err <= 1e-3, (n, err)
        big = np.abs(ref_grad) > 1e-3 * np.abs(ref_grad).max()
        assert np.max(np.abs(grad[big] - ref_grad[big]) / np.abs(ref_grad[big])) < 2e-2


def test_training_fits_a_known_function_deterministically(env):
    torch, afd, orc = env
    g = np.random.default_rng(7)
    n = 60000
    f = g.normal(0.0, 1.0, (n, 8)).astype(np.float32)
    lab = (2.0 * f[:, 0] + np.abs(f[:, 1]) - 0.5 * f[:, 2] * f[:, 3] - 12.0).astype(np.float32)
    fd, ld = dev(torch, f, torch.float32), dev(torch, lab, torch.float32)
    p1, h1 = afd.afd_mlp_train(fd, ld, epochs=8, batch=512, lr=3e-3, seed=11)
    p2, h2 = afd.afd_mlp_train(fd, ld, epochs=8, batch=512, lr=3e-3, seed=11)
    assert np.array_equal(p1, p2) and np.array_equal(h1, h2)
    assert h1[-1] < 0.05 * np.var(lab) and h1[-1] < h1[0]
    # the trained FP32 weights, rounded to FP16, still predict well
    pred = orc.mlp_forward(orc.fp16_round(p1), f[:5000])
    assert np.sqrt(np.mean((pred - lab[:5000]) ** 2)) < 0.35


# ---------------------------------------------------------------- samples


def test_samples_match_oracle(env, plummer):
    torch, afd, orc = env
    p, amag = plummer
    lo, hi = 0.3, 0.9
    g, _ = gpu_ctx(env, p, amag)
    t = orc.Tree(p.x, p.y, p.z, p.m, n_grp=64, eps=EPS, amag=amag)
    M, com, Q = t.moments()
    assert np.array_equal(g.export("cell_quad").reshape(-1, 6), Q)  # bit-exact quadrupoles
    want = t.band_pairs(lo, hi)
    cap = len(want) + 10
    feat = torch.empty((cap, 8), dtype=torch.float32, device="cuda:0")
    lab = torch.empty(cap, dtype=torch.float32, device="cuda:0")
    pair = torch.empty((cap, 2), dtype=torch.int32, device="cuda:0")
    n = afd.afd_mac_samples(g.ctx, lo, hi, 1.0, 0, feat, lab, pair)
    assert n == len(want)
    gp = pair[:n].cpu().numpy().astype(np.int64)
    order = np.lexsort((gp[:, 1], gp[:, 0]))
    gp = gp[order]
    ref_order = np.lexsort((want[:, 1], want[:, 0]))
    assert np.array_equal(gp, want[ref_order])
    gf = feat[:n].cpu().numpy()[order]
    assert np.array_equal(gf, t.pair_features(gp))
    # targets: both sides clamp at -40; the GPU sums in FP32 with compensation
    sel = np.arange(0, n, 7)
    gl = lab[:n].cpu().numpy()[order][sel].astype(np.float64)
    rl = t.pair_labels(gp[sel])
    deep = rl < -24  # below the FP32 noise floor of the exact sum
    assert np.all(gl[deep] < -20)
    d = np.abs(gl[~deep] - rl[~deep])
    assert np.percentile(d, 99) < 0.02 and d.max() < 0.2, (np.percentile(d, 99), d.max())
    # a subsample: the keep rule is a fixed hash, so two calls agree
    n2 = afd.afd_mac_samples(g.ctx, lo, hi, 0.25, 9, feat, lab, pair)
    keep = pair[:min(n2, cap)].cpu().numpy().copy()
    n3 = afd.afd_mac_samples(g.ctx, lo, hi, 0.25, 9, feat, lab, pair)
    assert n3 == n2 and 0.2 * n < n2 < 0.3 * n
    assert np.array_equal(keep, pair[:min(n3, cap)].cpu().numpy())
    g.close()


def test_samples_need_reference_and_tree(env, plummer):
    torch, afd, _ = env
    p, _ = plummer
    g, _ = gpu_ctx(env, p, None)
    feat = torch.empty((4, 8), dtype=torch.float32, device="cuda:0")
    lab = torch.empty(4, dtype=torch.float32, device="cuda:0")
    with pytest.raises(afd.AfdError) as e:
        afd.afd_mac_samples(g.ctx, 0.3, 0.9, 1.0, 0, feat, lab)
    assert e.value.status == -12
    g.close()
    g2 = afd.Gravity(afd.Config(eps=EPS, mac=0), 0, torch.cuda.current_stream())
    with pytest.raises(afd.AfdError):
        afd.afd_mac_set(g2.ctx, np.zeros(afd.AFD_MAC_PARAMS, np.float32), 0.3, 0.9, 0.0)
    g2.close()


# ---------------------------------------------------------------- learned walk


@pytest.mark.parametrize("case", ["random", "random_quad", "accept_all", "open_all"])
def test_learned_lists_bit_exact_and_forces(env, plummer, case):
    torch, afd, orc = env
    p, amag = plummer
    quad = case == "random_quad"
    params = rand_params(orc, 13)
    params[8:16] = 0.25
    lo, hi, tau = 0.25, 1.0, 0.0
    if case == "accept_all":
        params[16:] = 0.0
        params[-1] = -1000.0
    if case == "open_all":
        params[16:] = 0.0
        params[-1] = 1000.0
    g, xs = gpu_ctx(env, p, amag, quad=quad)
    afd.afd_mac_set(g.ctx, params, lo, hi, tau)
    afd.afd_make_interaction_lists(g.ctx, afd.AFD_MAKE_LIST_FOR_REUSE)
    acc = torch.empty((p.n, 4), dtype=torch.float32, device="cuda:0")
    afd.afd_calc_force(g.ctx, acc)
    info = afd.afd_mac_info(g.ctx)
    assert info["learned"] == 1 and info["evaluations"] > 0
    if case == "accept_all":
        assert info["accepted"] == info["evaluations"]
    if case == "open_all":
        assert info["accepted"] == 0
    mac = dict(params=orc.fp16_round(params), theta_lo=lo, theta_hi=hi, tau=tau)
    t = orc.Tree(p.x, p.y, p.z, p.m, n_grp=64, eps=EPS, quad=quad, mac=mac, amag=amag)
    band, flips = t.relist_band(g.export("spj_off"), g.export("spj_idx"))
    print(f"learned walk ({case}): {info['evaluations']} network evaluations, "
          f"{band} within the rounding bound of tau, {flips} decided otherwise than the oracle")
    assert flips <= band and band <= max(10, info["evaluations"] // 100)
    check_structure(g, t, quad=quad)
    ref = t.force()
    assert rms_rel_acc(acc.cpu().numpy().astype(np.float64), ref) <= 1e-6
    # the force evaluation stored |a| as the next reference
    info = afd.afd_mac_info(g.ctx)
    assert info["reference"] == 1
    g.close()


def test_learned_walk_falls_back_to_theta(env, plummer):
    torch, afd, orc = env
    p, amag = plummer
    t = orc.Tree(p.x, p.y, p.z, p.m, n_grp=64, eps=EPS, theta=0.5)
    # no weights
    g, _ = gpu_ctx(env, p, amag)
    afd.afd_make_interaction_lists(g.ctx, afd.AFD_MAKE_LIST)
    assert afd.afd_mac_info(g.ctx)["learned"] == 0
    assert np.array_equal(g.export("spj_idx"), t.lists()[3].astype(np.uint32))
    g.close()
    # weights but no reference magnitudes
    g, _ = gpu_ctx(env, p, None)
    afd.afd_mac_set(g.ctx, rand_params(orc, 1), 0.2, 0.9, 0.0)
    afd.afd_make_interaction_lists(g.ctx, afd.AFD_MAKE_LIST)
    assert afd.afd_mac_info(g.ctx)["learned"] == 0
    assert np.array_equal(g.export("epj_idx"), t.lists()[1].astype(np.uint32))
    # removing the weights again
    afd.afd_mac_set(g.ctx, None, 0, 0, 0)
    g.close()


def test_direct_sum_matches_oracle(env, plummer):
    torch, afd, orc = env
    p, _ = plummer
    tg = np.arange(0, p.n, 97).astype(np.int32)
    out = torch.empty((len(tg), 4), dtype=torch.float64, device="cuda:0")
    xs = [dev(torch, a, torch.float64) for a in (p.x, p.y, p.z, p.m)]
    afd.afd_direct_sum(*xs, dev(torch, tg, torch.int32), EPS, out)
    got = out.cpu().numpy()
    ref = orc.direct_sum(p.x, p.y, p.z, p.m, EPS, targets=tg)
    for k in range(4):
        assert np.allclose(got[:, k], ref[k], rtol=1e-11, atol=1e-12 * np.abs(ref[k]).max())


# ---------------------------------------------------------------- what it gains


def test_trained_criterion_beats_theta_at_equal_error(env):
    """Train on the targets of one Plummer sphere (GPU sampling, GPU training),
    then on another sphere compare interactions at equal rms force error
    (error against the FP64 direct sum of sampled particles)."""
    torch, afd, orc = env
    n = 1 << 16
    lo, hi = 0.25, 1.0

    def setup(seed):
        p = ics.plummer(n, seed)
        xs = [dev(torch, a, torch.float64) for a in (p.x, p.y, p.z, p.m)]
        return p, xs

    def run(xs, theta, mac=None):
        cfg = afd.Config(eps=EPS, theta=theta, n_grp=64, mac=1)
        g = afd.Gravity(cfg, 0, torch.cuda.current_stream())
        acc = torch.empty((n, 4), dtype=torch.float32, device="cuda:0")
        if mac is not None:  # reference |a| from a tight theta pass
            g0 = afd.Gravity(afd.Config(eps=EPS, theta=0.3, n_grp=64, mac=1), 0,
                             torch.cuda.current_stream())
            g0.force_all(*xs, acc, afd.AFD_MAKE_LIST)
            amag = torch.sqrt((acc[:, :3].double() ** 2).sum(1)).float().contiguous()
            g0.close()
            afd.afd_mac_set(g.ctx, mac, lo, hi, mac_tau[0])
            afd.afd_tree_build(g.ctx, *xs)
            afd.afd_mac_set_reference(g.ctx, amag)
            afd.afd_make_interaction_lists(g.ctx, afd.AFD_MAKE_LIST)
            afd.afd_calc_force(g.ctx, acc)
        else:
            g.force_all(*xs, acc, afd.AFD_MAKE_LIST)
        inter = g.stats()["interactions"]
        g.close()
        return acc, inter

    # training data
    _, xs_a = setup(101)
    cfg = afd.Config(eps=EPS, theta=0.3, n_grp=64, mac=1)
    g = afd.Gravity(cfg, 0, torch.cuda.current_stream())
    acc = torch.empty((n, 4), dtype=torch.float32, device="cuda:0")
    g.force_all(*xs_a, acc, afd.AFD_MAKE_LIST)
    cap = 400000
    feat = torch.empty((cap, 8), dtype=torch.float32, device="cuda:0")
    lab = torch.empty(cap, dtype=torch.float32, device="cuda:0")
    total = afd.afd_mac_samples(g.ctx, lo, hi, 1.0, 0, feat, lab)
    m = min(total, cap)
    if total > cap:
        m = afd.afd_mac_samples(g.ctx, lo, hi, cap / total * 0.95, 1, feat, lab)
    g.close()
    params, hist = afd.afd_mlp_train(feat[:m], lab[:m], epochs=12, batch=1024, lr=2e-3, seed=3)
    assert hist[-1] < hist[0]

    # evaluation sphere and its exact forces
    p, xs = setup(202)
    tg = np.arange(0, n, 16).astype(np.int32)
    ex = torch.empty((len(tg), 4), dtype=torch.float64, device="cuda:0")
    afd.afd_direct_sum(*xs, dev(torch, tg, torch.int32), EPS, ex)
    ex = ex.cpu().numpy()

    def err(acc):
        a = acc.cpu().numpy().astype(np.float64)[tg]
        return rms_rel_acc(a, [ex[:, k] for k in range(4)])

    th_pts = []
    for th in (0.3, 0.4, 0.5, 0.6, 0.7, 0.8):
        a, inter = run(xs, th)
        th_pts.append((err(a), inter))
    mac_tau = [0.0]
    le_pts = []
    for tau in (-14.0, -13.0, -12.0, -11.0):
        mac_tau[0] = tau
        a, inter = run(xs, 0.5, mac=params)
        le_pts.append((err(a), inter))
    th_e, th_i = np.log(np.array(th_pts)).T
    gains = []
    for e_l, i_l in le_pts:
        le = np.log(e_l)
        if th_e.min() <= le <= th_e.max():
            o = np.argsort(th_e)
            i_theta = np.exp(np.interp(le, th_e[o], th_i[o]))
            gains.append(i_theta / i_l)
    assert gains, (th_pts, le_pts)
    # fewer interactions than the theta criterion at the same error
    assert min(gains) > 1.2, (th_pts, le_pts, gains)
