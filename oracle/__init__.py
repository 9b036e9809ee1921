"""FP64 CPU oracle for the multiwalk / indirect-index Barnes-Hut path of
"Accelerated FDPS" (arXiv 1907.02290).

TEST INFRASTRUCTURE. Only the test suite, ``__graft_entry__.smoke()`` and
``bench.py`` (its cpu_baseline leg and its ``--impl reference`` arm) may import
this package. It shares no code with the CUDA path and never imports it.

The arithmetic lives in ``afdps_oracle.c`` (plain C, FP64, built with
``-ffp-contract=off``); this module only compiles it and marshals numpy arrays.
Each wrapper names the paper passage its C function follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "afdps_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libafdps_oracle.so")
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)
_I32 = ctypes.POINTER(ctypes.c_int32)
_U64 = ctypes.POINTER(ctypes.c_uint64)
_F32 = ctypes.POINTER(ctypes.c_float)

# Learned opening criterion (readings R12-R15 of afdps_oracle.c): features,
# hidden units and the length of the flat parameter vector
# mu[8] isd[8] W1[32][8] b1[32] W2[32][32] b2[32] w3[32] b3[1].
MAC_NF = 8
MAC_NH = 32
MAC_NP = 2 * MAC_NF + MAC_NH * MAC_NF + MAC_NH + MAC_NH * MAC_NH + MAC_NH + MAC_NH + 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available). Returns the path."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
            "-fPIC", "-shared", _SRC, "-o", _LIB_PATH + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        L.afo_direct_sum.argtypes = [ctypes.c_int64, _D, _D, _D, _D, ctypes.c_double,
                                     ctypes.c_int64, _I64, _D, _D, _D, _D]
        L.afo_root_cell.argtypes = [ctypes.c_int64, _D, _D, _D, _D]
        L.afo_root_cell.restype = ctypes.c_int
        L.afo_morton_keys.argtypes = [ctypes.c_int64, _D, _D, _D, _D, _U64]
        L.afo_radix_sort.argtypes = [ctypes.c_int64, _U64, _U64, _I64]
        L.afo_build.argtypes = [ctypes.c_int64, _D, _D, _D, _D, ctypes.c_int, ctypes.c_int,
                                ctypes.c_double, ctypes.c_double, ctypes.c_int]
        L.afo_build.restype = ctypes.c_void_p
        L.afo_update.argtypes = [ctypes.c_void_p, _D, _D, _D, _D]
        L.afo_update.restype = ctypes.c_int
        L.afo_force.argtypes = [ctypes.c_void_p, _D, _D, _D, _D]
        L.afo_force_groups.argtypes = [ctypes.c_void_p, ctypes.c_int64, _I64, _D, _D, _D, _D]
        L.afo_free.argtypes = [ctypes.c_void_p]
        L.afo_sizes.argtypes = [ctypes.c_void_p, _I64]
        L.afo_get_root.argtypes = [ctypes.c_void_p, _D]
        L.afo_get_order.argtypes = [ctypes.c_void_p, _U64, _I64]
        L.afo_get_cells.argtypes = [ctypes.c_void_p, _I32, _I64, _I64, _I64, _I64, _I32, _I64]
        L.afo_get_moments.argtypes = [ctypes.c_void_p, _D, _D, _D]
        L.afo_get_groups.argtypes = [ctypes.c_void_p, _I64, _I64, _I64, _D, _I32]
        L.afo_get_lists.argtypes = [ctypes.c_void_p, _I64, _I32, _I64, _I32]
        L.afo_leapfrog.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64,
                                   _D, _D, _D, _D, _D, _D, _D, _D, _D, _D, _D,
                                   ctypes.c_double, ctypes.c_int, ctypes.c_int, _I64]
        L.afo_leapfrog.restype = ctypes.c_int
        L.afo_num_threads.restype = ctypes.c_int
        L.afo_build_mac.argtypes = L.afo_build.argtypes + [_F32, ctypes.c_double,
                                                          ctypes.c_double, ctypes.c_double, _F32]
        L.afo_build_mac.restype = ctypes.c_void_p
        L.afo_lg2_batch.argtypes = [ctypes.c_int64, _F32, _F32]
        L.afo_mac_features.argtypes = [_F32, _F32, _F32, ctypes.c_float, ctypes.c_float, _F32,
                                       ctypes.c_int64, ctypes.c_float, ctypes.c_float, _F32]
        L.afo_mlp_forward_batch.argtypes = [_F32, ctypes.c_int64, _F32, _F32]
        L.afo_mac_label.argtypes = [ctypes.c_int64, _D, _D, _D, _D, ctypes.c_int64, _D, _D, _D,
                                    _D, ctypes.c_double, _D, _D, ctypes.c_double, ctypes.c_int]
        L.afo_mac_label.restype = ctypes.c_double
        L.afo_pair_features_batch.argtypes = [ctypes.c_void_p, ctypes.c_int64, _I64, _F32]
        L.afo_pair_label_batch.argtypes = [ctypes.c_void_p, ctypes.c_int64, _I64, _D]
        L.afo_band_pairs.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int64, _I64]
        L.afo_band_pairs.restype = ctypes.c_int64
        L.afo_relist.argtypes = [ctypes.c_void_p]
        L.afo_relist_band.argtypes = [ctypes.c_void_p, _I64, _I32, _I64]
        L.afo_mlp_forward_bound_batch.argtypes = [_F32, ctypes.c_int64, _F32, _F32, _D]
        L.afo_rn16.argtypes = [ctypes.c_float]
        L.afo_rn16.restype = ctypes.c_float
        L.afo_let_export.argtypes = [ctypes.c_void_p, _D, ctypes.c_double, ctypes.c_int64, _D, _D,
                                     _D, _D, _I32]
        L.afo_let_export.restype = ctypes.c_int64
        L.afo_nbr_lists.argtypes = [ctypes.c_void_p, _D, ctypes.c_double]
        L.afo_nbr_lists.restype = ctypes.c_int
        L.afo_sph_density.argtypes = [ctypes.c_void_p, _D, _D, _D]
        L.afo_sph_density_direct.argtypes = [ctypes.c_int64, _D, _D, _D, _D, _D,
                                             ctypes.c_int64, _I64, _D, _D]
        L.afo_get_nbr.argtypes = [ctypes.c_void_p, _I64, _I32, _F32, _F32]
        L.afo_nbr_total.argtypes = [ctypes.c_void_p]
        L.afo_nbr_total.restype = ctypes.c_int64
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(lib().afo_num_threads())


def direct_sum(x, y, z, m, eps, targets=None):
    """Softened O(N^2) direct sum (the exact target; reading R1).
    Returns (ax, ay, az, pot) for ``targets`` (default: all particles)."""
    x, y, z, m = map(_f64, (x, y, z, m))
    n = x.shape[0]
    tgt = np.arange(n, dtype=np.int64) if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    out = [np.zeros(tgt.shape[0]) for _ in range(4)]
    lib().afo_direct_sum(n, _p(x, _D), _p(y, _D), _p(z, _D), _p(m, _D), float(eps),
                         tgt.shape[0], _p(tgt, _I64), *(_p(o, _D) for o in out))
    return tuple(out)


def density_direct(x, y, z, m, h, targets=None):
    """Density and smooth neighbour number of reading R18 summed over every
    particle (the definition, no tree) for the targets (all by default)."""
    x, y, z, m, h = map(_f64, (x, y, z, m, h))
    n = x.shape[0]
    tgt = np.arange(n, dtype=np.int64) if targets is None else np.ascontiguousarray(
        targets, dtype=np.int64)
    rho, nnb = np.zeros(tgt.shape[0]), np.zeros(tgt.shape[0])
    lib().afo_sph_density_direct(n, _p(x, _D), _p(y, _D), _p(z, _D), _p(m, _D), _p(h, _D),
                                 tgt.shape[0], _p(tgt, _I64), _p(rho, _D), _p(nnb, _D))
    return rho, nnb


def root_cell(x, y, z):
    """Root cell (Section 4.3; reading R2): (cx, cy, cz, L)."""
    x, y, z = map(_f64, (x, y, z))
    root = np.zeros(4)
    rc = lib().afo_root_cell(x.shape[0], _p(x, _D), _p(y, _D), _p(z, _D), _p(root, _D))
    if rc != 0:
        raise ValueError("non-finite coordinate")
    return root


def morton_keys(x, y, z, root):
    """Morton keys (Section 4.3 step 1; reading R3)."""
    x, y, z = map(_f64, (x, y, z))
    root = _f64(root)
    keys = np.zeros(x.shape[0], dtype=np.uint64)
    lib().afo_morton_keys(x.shape[0], _p(x, _D), _p(y, _D), _p(z, _D), _p(root, _D),
                          _p(keys, _U64))
    return keys


def radix_sort(keys):
    """LSD radix sort of key-index pairs (Section 4.3 step 2, Section 6.2).
    Returns (sorted keys, permutation)."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    ks = np.zeros_like(keys)
    perm = np.zeros(keys.shape[0], dtype=np.int64)
    lib().afo_radix_sort(keys.shape[0], _p(keys, _U64), _p(ks, _U64), _p(perm, _I64))
    return ks, perm


@dataclass
class Cells:
    level: np.ndarray
    first: np.ndarray
    count: np.ndarray
    parent: np.ndarray
    skip: np.ndarray
    n_child: np.ndarray
    child: np.ndarray  # (n_cells, 8), -1 where the octant is empty


class Tree:
    """One construction step of the tree method (Section 4.2, 4.3) kept for
    reuse steps. Wraps the C ``afo_tree``; arrays are copied out on request."""

    def __init__(self, x, y, z, m, *, n_leaf=16, n_grp=64, theta=0.5, eps=1.0 / 256,
                 quad=False, mac=None, amag=None):
        """``mac``: dict(params, theta_lo, theta_hi, tau) of the learned
        criterion (R14; params are FP16-rounded, see ``fp16_round``);
        ``amag``: reference |a| per particle (caller order, FP32). The
        learned criterion is used when both are given; with ``amag`` alone
        the tree only carries the reference magnitudes (for features and
        labels)."""
        self._args = dict(n_leaf=n_leaf, n_grp=n_grp, theta=theta, eps=eps, quad=quad)
        x, y, z, m = map(_f64, (x, y, z, m))
        self.n = x.shape[0]
        w = lo = hi = tau = None
        if mac is not None:
            w = np.ascontiguousarray(mac["params"], dtype=np.float32)
            assert w.shape == (MAC_NP,)
            lo, hi, tau = float(mac["theta_lo"]), float(mac["theta_hi"]), float(mac["tau"])
        a = None if amag is None else np.ascontiguousarray(amag, dtype=np.float32)
        self._amag = a
        h = lib().afo_build_mac(self.n, _p(x, _D), _p(y, _D), _p(z, _D), _p(m, _D),
                                int(n_leaf), int(n_grp), float(theta), float(eps), int(quad),
                                None if w is None else _p(w, _F32), lo or 0.0, hi or 0.0,
                                tau or 0.0, None if a is None else _p(a, _F32))
        if not h:
            raise ValueError("non-finite particle data")
        self._h = ctypes.c_void_p(h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().afo_free(h)
            self._h = None

    def sizes(self):
        s = np.zeros(5, dtype=np.int64)
        lib().afo_sizes(self._h, _p(s, _I64))
        return {"n": int(s[0]), "n_cells": int(s[1]), "n_groups": int(s[2]),
                "n_epj": int(s[3]), "n_spj": int(s[4])}

    def root(self):
        r = np.zeros(4)
        lib().afo_get_root(self._h, _p(r, _D))
        return r

    def order(self):
        keys = np.zeros(self.n, dtype=np.uint64)
        perm = np.zeros(self.n, dtype=np.int64)
        lib().afo_get_order(self._h, _p(keys, _U64), _p(perm, _I64))
        return keys, perm

    def cells(self) -> Cells:
        nc = self.sizes()["n_cells"]
        lv = np.zeros(nc, np.int32)
        f, c, p, s = (np.zeros(nc, np.int64) for _ in range(4))
        nch = np.zeros(nc, np.int32)
        ch = np.zeros(nc * 8, np.int64)
        lib().afo_get_cells(self._h, _p(lv, _I32), _p(f, _I64), _p(c, _I64), _p(p, _I64),
                            _p(s, _I64), _p(nch, _I32), _p(ch, _I64))
        return Cells(lv, f, c, p, s, nch, ch.reshape(nc, 8))

    def moments(self):
        """(M, COM (n_cells,3), Q (n_cells,6) as xx yy zz xy xz yz)."""
        nc = self.sizes()["n_cells"]
        M = np.zeros(nc)
        com = np.zeros(nc * 3)
        q = np.zeros(nc * 6)
        lib().afo_get_moments(self._h, _p(M, _D), _p(com, _D), _p(q, _D))
        return M, com.reshape(nc, 3), q.reshape(nc, 6)

    def groups(self):
        ng = self.sizes()["n_groups"]
        f, c, cell = (np.zeros(ng, np.int64) for _ in range(3))
        box = np.zeros(ng * 6)
        self_in = np.zeros(ng, np.int32)
        lib().afo_get_groups(self._h, _p(f, _I64), _p(c, _I64), _p(cell, _I64), _p(box, _D),
                             _p(self_in, _I32))
        return {"first": f, "count": c, "cell": cell, "box": box.reshape(ng, 6),
                "self_in": self_in}

    def lists(self):
        """CSR lists: (epj_off, epj, spj_off, spj)."""
        s = self.sizes()
        ng = s["n_groups"]
        eo = np.zeros(ng + 1, np.int64)
        so = np.zeros(ng + 1, np.int64)
        e = np.zeros(s["n_epj"], np.int32)
        sp = np.zeros(s["n_spj"], np.int32)
        lib().afo_get_lists(self._h, _p(eo, _I64), _p(e, _I32), _p(so, _I64), _p(sp, _I32))
        return eo, e, so, sp

    def relist_band(self, spj_off, spj):
        """Make the learned-criterion lists again, taking another
        implementation's decisions (its SPJ lists: CSR offsets per group and
        cell ids in this tree's numbering) for the pairs whose network output
        lies within the rounding bound of R13 from tau -- the only pairs two
        correct FP32 implementations may decide differently. Returns
        (band pairs visited, those decided otherwise than by this oracle);
        ``lists()`` then equals the other implementation's lists iff it agrees
        on every other pair."""
        off = np.ascontiguousarray(spj_off, dtype=np.int64)
        idx = np.ascontiguousarray(spj, dtype=np.int32)
        assert off.shape[0] == self.sizes()["n_groups"] + 1 and idx.shape[0] == off[-1]
        cnt = np.zeros(2, np.int64)
        lib().afo_relist_band(self._h, _p(off, _I64), _p(idx if idx.size else np.zeros(1, np.int32),
                                                         _I32), _p(cnt, _I64))
        return int(cnt[0]), int(cnt[1])

    def update(self, x, y, z, m):
        """Reusing step (Section 4.2): new particle data, same topology/lists."""
        x, y, z, m = map(_f64, (x, y, z, m))
        if lib().afo_update(self._h, _p(x, _D), _p(y, _D), _p(z, _D), _p(m, _D)) != 0:
            raise ValueError("non-finite particle data")

    def let_export(self, box, theta=None):
        """LET of reading R16 for a remote domain box (min xyz, max xyz):
        (x, y, z, m, kind) with kind 0 for particles, 1 for superparticles."""
        th = self._args["theta"] if theta is None else theta
        b = _f64(box)
        n = int(lib().afo_let_export(self._h, _p(b, _D), float(th), 0, None, None, None, None,
                                     None))
        out = [np.zeros(max(n, 1)) for _ in range(4)]
        kind = np.zeros(max(n, 1), np.int32)
        lib().afo_let_export(self._h, _p(b, _D), float(th), n, *(_p(o, _D) for o in out),
                             _p(kind, _I32))
        return (*(o[:n] for o in out), kind[:n])

    def neighbour_lists(self, h, skin=0.0):
        """Neighbour lists of reading R17 (Section 2, short-range walk) for
        search radii ``h`` (caller order) and margin ``skin``; they replace
        earlier ones and survive ``update``. Returns (off, idx): CSR lists of
        Morton positions per group."""
        self._nbr_h = _f64(h)
        if lib().afo_nbr_lists(self._h, _p(self._nbr_h, _D), float(skin)) != 0:
            raise ValueError("search radii must be finite and positive, skin finite and >= 0")
        off, idx, _, _ = self.neighbour_data()
        return off, idx

    def neighbour_data(self):
        """(off, idx, cell tight boxes (n_cells, 6), group search boxes
        (n_groups, 6)); boxes FP32, min x y z then max x y z."""
        s = self.sizes()
        total = int(lib().afo_nbr_total(self._h))
        if total < 0:
            raise RuntimeError("no neighbour lists")
        off = np.zeros(s["n_groups"] + 1, np.int64)
        idx = np.zeros(max(total, 1), np.int32)
        tb = np.zeros((max(s["n_cells"], 1), 6), np.float32)
        sb = np.zeros((max(s["n_groups"], 1), 6), np.float32)
        lib().afo_get_nbr(self._h, _p(off, _I64), _p(idx, _I32), _p(tb, _F32), _p(sb, _F32))
        return off, idx[:total], tb[:s["n_cells"]], sb[:s["n_groups"]]

    def density(self, h):
        """Density and smooth neighbour number of reading R18 over the
        neighbour lists (current positions), caller order."""
        hh = _f64(h)
        rho, nnb = np.zeros(self.n), np.zeros(self.n)
        lib().afo_sph_density(self._h, _p(hh, _D), _p(rho, _D), _p(nnb, _D))
        return rho, nnb

    def relist(self):
        """Lists made again on the current topology and moments (a list
        construction after reusing steps, without a new tree)."""
        lib().afo_relist(self._h)

    def force(self):
        """FP64 force on the saved lists, caller order: (ax, ay, az, pot)."""
        out = [np.zeros(self.n) for _ in range(4)]
        lib().afo_force(self._h, *(_p(o, _D) for o in out))
        return tuple(out)

    def force_groups(self, groups):
        """FP64 force for the particles of the listed groups only (caller
        order); other entries are NaN."""
        sel = np.ascontiguousarray(groups, dtype=np.int64)
        out = [np.full(self.n, np.nan) for _ in range(4)]
        lib().afo_force_groups(self._h, sel.shape[0], _p(sel, _I64), *(_p(o, _D) for o in out))
        return tuple(out)

    def band_pairs(self, theta_lo, theta_hi):
        """(group, cell) pairs left to the network by R14 (int64, (n, 2))."""
        n = int(lib().afo_band_pairs(self._h, float(theta_lo), float(theta_hi), 0, None))
        out = np.zeros((max(n, 1), 2), dtype=np.int64)
        lib().afo_band_pairs(self._h, float(theta_lo), float(theta_hi), n, _p(out, _I64))
        return out[:n]

    def pair_features(self, pairs):
        """FP32 features of R12 for (group, cell) pairs; needs ``amag``."""
        pr = np.ascontiguousarray(pairs, dtype=np.int64).reshape(-1, 2)
        f = np.zeros((pr.shape[0], MAC_NF), dtype=np.float32)
        lib().afo_pair_features_batch(self._h, pr.shape[0], _p(pr, _I64), _p(f, _F32))
        return f

    def pair_labels(self, pairs):
        """FP64 training targets of R15 for (group, cell) pairs."""
        pr = np.ascontiguousarray(pairs, dtype=np.int64).reshape(-1, 2)
        out = np.zeros(pr.shape[0])
        lib().afo_pair_label_batch(self._h, pr.shape[0], _p(pr, _I64), _p(out, _D))
        return out

    def interactions(self):
        """Sum over groups of n_i * (n_epj + n_spj) (self pair included)."""
        g = self.groups()
        eo, _, so, _ = self.lists()
        return int(np.sum(g["count"] * ((eo[1:] - eo[:-1]) + (so[1:] - so[:-1]))))


def leapfrog(x, y, z, vx, vy, vz, m, *, dt, n_steps, n_reuse, n_leaf=16, n_grp=64,
             theta=0.5, eps=1.0 / 256, quad=False):
    """Kick-drift-kick leapfrog with list reuse (reading R11). Evaluation 0
    (the initial force) is a construction step; evaluation k is one when
    k % n_reuse == 0. Returns new (x, y, z, vx, vy, vz, ax, ay, az, pot)."""
    arrs = [np.array(a, dtype=np.float64, copy=True) for a in (x, y, z, vx, vy, vz)]
    m = _f64(m)
    t = Tree(*arrs[:3], m, n_leaf=n_leaf, n_grp=n_grp, theta=theta, eps=eps, quad=quad)
    acc = [np.ascontiguousarray(a) for a in t.force()]
    h = ctypes.c_void_p(t._h.value)
    t._h = None  # ownership moves to the C loop
    counter = np.array([1], dtype=np.int64)
    rc = lib().afo_leapfrog(ctypes.byref(h), arrs[0].shape[0], *(_p(a, _D) for a in arrs),
                            _p(m, _D), *(_p(a, _D) for a in acc), float(dt), int(n_steps),
                            int(n_reuse), _p(counter, _I64))
    lib().afo_free(h)
    if rc != 0:
        raise ValueError("non-finite particle data")
    return (*arrs, *acc)


# ---------------------------------------------------------------------------
# Learned opening criterion (not in the paper; readings R12-R15).
# ---------------------------------------------------------------------------

def lg2(x):
    """The deterministic FP32 log2 of R12."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.zeros_like(x)
    lib().afo_lg2_batch(x.size, _p(x, _F32), _p(out, _F32))
    return out


def mac_features(bmin, bmax, com, s2, M, Q, count, eps2, amin):
    """R12 features from raw FP32 inputs (one pair)."""
    b0, b1, c = (np.ascontiguousarray(v, dtype=np.float32) for v in (bmin, bmax, com))
    q = np.ascontiguousarray(Q, dtype=np.float32)
    f = np.zeros(MAC_NF, dtype=np.float32)
    lib().afo_mac_features(_p(b0, _F32), _p(b1, _F32), _p(c, _F32), float(np.float32(s2)),
                           float(np.float32(M)), _p(q, _F32), int(count),
                           float(np.float32(eps2)), float(np.float32(amin)), _p(f, _F32))
    return f


def mac_label(xi, ai, xj, mj, M, com, Q, eps, quad):
    """R15 target for group particles xi (n_i, 3) with reference magnitudes
    ai and a cell of particles xj (n_j, 3), mj with monopole M at com and
    quadrupole Q."""
    xi, xj = np.asarray(xi, np.float64).reshape(-1, 3), np.asarray(xj, np.float64).reshape(-1, 3)
    cols_i = [np.ascontiguousarray(xi[:, k]) for k in range(3)]
    cols_j = [np.ascontiguousarray(xj[:, k]) for k in range(3)]
    ai, mj, com, Q = map(_f64, (ai, mj, com, Q))
    return float(lib().afo_mac_label(xi.shape[0], *(_p(c, _D) for c in cols_i), _p(ai, _D),
                                     xj.shape[0], *(_p(c, _D) for c in cols_j), _p(mj, _D),
                                     float(M), _p(com, _D), _p(Q, _D), float(eps), int(quad)))


def fp16_round(params):
    """Parameters as the criterion stores them (R13): FP16 values in FP32."""
    return np.asarray(params, dtype=np.float32).astype(np.float16).astype(np.float32)


def mlp_forward(params, feats):
    """R13 network per feature row: FP16 inputs and first-layer activations,
    FP32 sums (bias, then fused multiply-adds in input order)."""
    p = np.ascontiguousarray(params, dtype=np.float32)
    f = np.ascontiguousarray(feats, dtype=np.float32).reshape(-1, MAC_NF)
    out = np.zeros(f.shape[0], dtype=np.float32)
    lib().afo_mlp_forward_batch(_p(p, _F32), f.shape[0], _p(f, _F32), _p(out, _F32))
    return out


def rn16(v):
    """RN16 of R13: the nearest FP16 value (ties to even) of an FP32 value."""
    return float(lib().afo_rn16(float(np.float32(v))))


def mlp_forward_bound(params, feats):
    """R13 network per feature row and, per row, the bound of R13 on the
    difference between its output and any other FP32 summation order's (the
    layers' sums in another order, a first-layer activation rounded to FP16
    from the other sum)."""
    p = np.ascontiguousarray(params, dtype=np.float32)
    f = np.ascontiguousarray(feats, dtype=np.float32).reshape(-1, MAC_NF)
    out = np.zeros(f.shape[0], dtype=np.float32)
    bound = np.zeros(f.shape[0], dtype=np.float64)
    lib().afo_mlp_forward_bound_batch(_p(p, _F32), f.shape[0], _p(f, _F32), _p(out, _F32),
                                      _p(bound, _D))
    return out, bound


def mlp_unpack(params):
    """Split the flat vector into (mu, isd, W1, b1, W2, b2, w3, b3)."""
    p = np.asarray(params)
    sizes = [MAC_NF, MAC_NF, MAC_NH * MAC_NF, MAC_NH, MAC_NH * MAC_NH, MAC_NH, MAC_NH, 1]
    parts, o = [], 0
    for s in sizes:
        parts.append(p[o:o + s])
        o += s
    mu, isd, W1, b1, W2, b2, w3, b3 = parts
    return mu, isd, W1.reshape(MAC_NH, MAC_NF), b1, W2.reshape(MAC_NH, MAC_NH), b2, w3, b3


def mlp_loss(params, feats, labels):
    """Mean squared error of the R13 network in FP64 (no FP16 rounding)."""
    mu, isd, W1, b1, W2, b2, w3, b3 = mlp_unpack(np.asarray(params, np.float64))
    X = (np.asarray(feats, np.float64) - mu) * isd
    H1 = np.maximum(X @ W1.T + b1, 0.0)
    H2 = np.maximum(H1 @ W2.T + b2, 0.0)
    y = H2 @ w3 + b3[0]
    return float(np.mean((y - np.asarray(labels, np.float64)) ** 2))


def mlp_loss_grad(params, feats, labels):
    """FP64 backward pass of ``mlp_loss`` (chain rule through both ReLU
    layers; the derivative of ReLU at 0 is taken as 0). Returns (loss, grad)
    with grad laid out like params (zero for mu and isd, which are not
    trained)."""
    mu, isd, W1, b1, W2, b2, w3, b3 = mlp_unpack(np.asarray(params, np.float64))
    X = (np.asarray(feats, np.float64) - mu) * isd
    Z1 = X @ W1.T + b1
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ W2.T + b2
    H2 = np.maximum(Z2, 0.0)
    y = H2 @ w3 + b3[0]
    r = y - np.asarray(labels, np.float64)
    B = X.shape[0]
    dy = 2.0 * r / B
    g_w3 = H2.T @ dy
    g_b3 = np.array([dy.sum()])
    dZ2 = np.outer(dy, w3) * (Z2 > 0.0)
    g_W2 = dZ2.T @ H1
    g_b2 = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ W2) * (Z1 > 0.0)
    g_W1 = dZ1.T @ X
    g_b1 = dZ1.sum(axis=0)
    grad = np.concatenate([np.zeros(2 * MAC_NF), g_W1.ravel(), g_b1, g_W2.ravel(), g_b2,
                           g_w3, g_b3])
    return float(np.mean(r * r)), grad
