"""GPU parity of the local essential tree export (reading R16 of the
oracle): the exported superparticles and particles equal the oracle's bit
for bit and in order, and a tree over the local particles plus the
imported elements gives the oracle's forces on the same input."""
import numpy as np
import pytest

import ics
from test_gpu_parity import env, rms_rel_acc  # noqa: F401 (fixture)

pytestmark = pytest.mark.gpu

EPS = 1.0 / 256


@pytest.mark.parametrize("theta", [0.0, 0.5, 0.8])
def test_let_export_and_split_force(env, theta):
    torch, afd, orc = env
    p = ics.plummer(20000 + 3, 81)
    A = p.x < 0.0
    B = ~A
    box = [p.x[A].min(), p.y[A].min(), p.z[A].min(), p.x[A].max(), p.y[A].max(), p.z[A].max()]
    dev = torch.device("cuda:0")
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    gb = afd.Gravity(afd.Config(eps=EPS, theta=0.5, n_grp=64), 0, torch.cuda.current_stream())
    afd.afd_tree_build(gb.ctx, T(p.x[B]), T(p.y[B]), T(p.z[B]), T(p.m[B]))
    x, y, z, m, kind = afd.afd_let_export(gb.ctx, box, theta)
    got = [v.cpu().numpy() for v in (x, y, z, m)]
    tb = orc.Tree(p.x[B], p.y[B], p.z[B], p.m[B], theta=0.5, eps=EPS, n_grp=64)
    want = tb.let_export(box, theta=theta)
    for g_, w_ in zip(got, want[:4]):
        assert np.array_equal(g_, w_)
    assert np.array_equal(kind.cpu().numpy(), want[4])
    # capped export: the first elements only, same total
    _, _, _, m2, _ = afd.afd_let_export(gb.ctx, box, theta, cap=7)
    assert np.array_equal(m2.cpu().numpy(), want[3][:7])
    gb.close()
    # the receiving side: a tree over A's particles followed by the imports
    na = int(A.sum())
    X = [np.r_[p.x[A], got[0]], np.r_[p.y[A], got[1]], np.r_[p.z[A], got[2]],
         np.r_[p.m[A], got[3]]]
    ga = afd.Gravity(afd.Config(eps=EPS, theta=0.5, n_grp=64), 0, torch.cuda.current_stream())
    acc = torch.empty(len(X[0]), 4, dtype=torch.float32, device=dev)
    ga.force_all(*(T(v) for v in X), acc, afd.AFD_MAKE_LIST)
    a = acc.cpu().numpy().astype(np.float64)[:na]
    ta = orc.Tree(*X, theta=0.5, eps=EPS, n_grp=64)
    ref = [f[:na] for f in ta.force()]
    assert rms_rel_acc(a, ref) <= 1e-6
    ga.close()
