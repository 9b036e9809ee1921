"""Pins for the oracle's local essential tree (reading R16: the superparticles
and particles a remote domain needs, Section 3 / Section 4.3). Checked
against the direct sum (theta = 0 exports every particle, so the split
computation must equal the whole-system direct sum), conservation of mass
and mass moment, and the whole-system tree. No GPU needed."""
import numpy as np
import pytest

import ics

EPS = 1.0 / 256


def _split(p):
    a = p.x < 0.0
    return a, ~a


def _box(p, sel):
    return [p.x[sel].min(), p.y[sel].min(), p.z[sel].min(),
            p.x[sel].max(), p.y[sel].max(), p.z[sel].max()]


def _rms_rel(a, ref):
    num = sum((a[k] - ref[k]) ** 2 for k in range(3))
    den = sum(ref[k] ** 2 for k in range(3))
    return float(np.sqrt(np.mean(num / den)))


def test_let_conserves_mass_and_moment(orc):
    p = ics.plummer(4000, 12)
    A, B = _split(p)
    tb = orc.Tree(p.x[B], p.y[B], p.z[B], p.m[B], theta=0.5, eps=EPS)
    x, y, z, m, kind = tb.let_export(_box(p, A))
    assert 0 < kind.sum() < len(kind)  # both superparticles and particles
    assert m.sum() == pytest.approx(p.m[B].sum(), rel=1e-13)
    for c, pc in ((x, p.x), (y, p.y), (z, p.z)):
        assert (m * c).sum() == pytest.approx((p.m[B] * pc[B]).sum(), rel=1e-12, abs=1e-15)


def test_let_with_theta_zero_is_the_remote_particles_and_gives_the_direct_sum(orc):
    p = ics.plummer(2500, 13)
    A, B = _split(p)
    tb = orc.Tree(p.x[B], p.y[B], p.z[B], p.m[B], theta=0.0, eps=EPS)
    x, y, z, m, kind = tb.let_export(_box(p, A), theta=0.0)
    assert not kind.any() and len(x) == B.sum()
    got = np.sort(np.stack([x, y, z, m], 1), axis=0)
    want = np.sort(np.stack([p.x[B], p.y[B], p.z[B], p.m[B]], 1), axis=0)
    assert np.array_equal(got, want)
    # the tree of A plus the imported particles, theta = 0: the direct sum
    ta = orc.Tree(np.r_[p.x[A], x], np.r_[p.y[A], y], np.r_[p.z[A], z], np.r_[p.m[A], m],
                  theta=0.0, eps=EPS)
    fa = [f[:A.sum()] for f in ta.force()]
    idx = np.nonzero(A)[0]
    ex = orc.direct_sum(p.x, p.y, p.z, p.m, EPS, targets=idx)
    assert _rms_rel(fa, ex) < 1e-12


def test_split_tree_force_matches_whole_system_at_the_method_error(orc):
    p = ics.plummer(6000, 14)
    A, B = _split(p)
    idx = np.nonzero(A)[0]
    ex = orc.direct_sum(p.x, p.y, p.z, p.m, EPS, targets=idx)
    whole = orc.Tree(p.x, p.y, p.z, p.m, theta=0.5, eps=EPS, n_grp=64)
    fw = [f[idx] for f in whole.force()]
    tb = orc.Tree(p.x[B], p.y[B], p.z[B], p.m[B], theta=0.5, eps=EPS)
    x, y, z, m, _ = tb.let_export(_box(p, A))
    ta = orc.Tree(np.r_[p.x[A], x], np.r_[p.y[A], y], np.r_[p.z[A], z], np.r_[p.m[A], m],
                  theta=0.5, eps=EPS, n_grp=64)
    fa = [f[:A.sum()] for f in ta.force()]
    e_whole, e_split = _rms_rel(fw, ex), _rms_rel(fa, ex)
    assert e_split < 2.0 * e_whole and e_split < 3e-3
    assert _rms_rel(fa, fw) < 3e-3
