"""GB300 (sm_103a) multiwalk, indirect-index Barnes-Hut gravity.

Thin ctypes binding over ``libafdps.so`` (C ABI in ``include/afdps.h``). The
functions keep the C names and only marshal arguments: torch tensors become
device pointers, a torch CUDA stream becomes a ``cudaStream_t``. Every step of
the computation runs in the library's CUDA kernels; there is no fallback. If
the library has not been built, importing the binding raises.

Build it with ``python -m paper_1907_02290_gb300.build`` (or
``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

AFD_MAKE_LIST = 0
AFD_MAKE_LIST_FOR_REUSE = 1
AFD_REUSE_LIST = 2

EXPORT = {
    "root": (0, np.float64), "keys": (1, np.uint64), "perm": (2, np.uint32),
    "cell_level": (3, np.uint32), "cell_first": (4, np.uint32), "cell_count": (5, np.uint32),
    "cell_skip": (6, np.uint32), "cell_parent": (7, np.uint32), "cell_child": (8, np.uint32),
    "cell_mass": (9, np.float64), "cell_com": (10, np.float64), "cell_quad": (11, np.float64),
    "group_first": (12, np.uint32), "group_count": (13, np.uint32),
    "group_box": (14, np.float64), "group_self": (15, np.uint32),
    "epj_off": (16, np.uint64), "epj_idx": (17, np.uint32),
    "spj_off": (18, np.uint64), "spj_idx": (19, np.uint32),
    "nbr_off": (20, np.uint64), "nbr_idx": (21, np.uint32),
    "cell_tbox": (22, np.float32), "group_sbox": (23, np.float32),
}


class AfdError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {afd_error_string(status)} (status {status})")


class afd_config(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("theta", ctypes.c_double),
                ("n_leaf", ctypes.c_int32), ("n_grp", ctypes.c_int32),
                ("multipole", ctypes.c_int32), ("far_precision", ctypes.c_int32),
                ("mac", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_lib = None
_VP = ctypes.c_void_p
_I64 = ctypes.c_int64
_D = ctypes.c_double


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libafdps.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "(there is no CPU fallback)")
    L = ctypes.CDLL(path)
    sig = {
        "afd_create": ([ctypes.POINTER(_VP), ctypes.POINTER(afd_config), ctypes.c_int, _VP], ctypes.c_int),
        "afd_destroy": ([_VP], None),
        "afd_set_stream": ([_VP, _VP], ctypes.c_int),
        "afd_set_systems": ([_VP, _VP, ctypes.c_int, _VP], ctypes.c_int),
        "afd_tree_build": ([_VP, _VP, _VP, _VP, _VP, _I64], ctypes.c_int),
        "afd_make_interaction_lists": ([_VP, ctypes.c_int], ctypes.c_int),
        "afd_reuse_lists": ([_VP, _VP, _VP, _VP, _VP], ctypes.c_int),
        "afd_calc_force": ([_VP, _VP], ctypes.c_int),
        "afd_calc_force_all": ([_VP, _VP, _VP, _VP, _VP, _I64, _VP, ctypes.c_int], ctypes.c_int),
        "afd_calc_force_all_host": ([_VP, _VP, _VP, _VP, _VP, _I64, _VP, ctypes.c_int], ctypes.c_int),
        "afd_kick_drift": ([_VP] + [_VP] * 7 + [_I64, _D, _D], ctypes.c_int),
        "afd_kick": ([_VP] + [_VP] * 4 + [_I64, _D], ctypes.c_int),
        "afd_leapfrog": ([_VP] + [_VP] * 7 + [_I64, _VP, _D, ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "afd_energy": ([_VP] + [_VP] * 5 + [_I64, _VP], ctypes.c_int),
        "afd_sync": ([_VP], ctypes.c_int),
        "afd_stats": ([_VP, _VP], ctypes.c_int),
        "afd_export": ([_VP, ctypes.c_int, _VP, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
        "afd_last_force_ms": ([_VP, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
        "afd_error_string": ([ctypes.c_int], ctypes.c_char_p),
        "afd_root_cell_static": ([_VP, _VP, _VP, _VP, _I64, _VP, _VP, _VP], ctypes.c_int),
        "afd_fp32_peak": ([ctypes.c_int, _VP, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "afd_pipe_rates": ([ctypes.c_int, _VP, _VP], ctypes.c_int),
        "afd_system_stats": ([_VP, _VP, _VP], ctypes.c_int),
        "afd_graph_capture_step": ([_VP] + [_VP] * 8 + [_D], ctypes.c_int),
        "afd_graph_launch": ([_VP], ctypes.c_int),
        "afd_autotune_n_grp": ([_VP, _VP, _VP, _VP, _VP, _I64, _VP, ctypes.c_int, ctypes.c_int, _VP,
                                _VP], ctypes.c_int),
        "afd_set_launch": ([_VP, ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "afd_set_walk_limits": ([_VP, _I64, ctypes.c_int32, _I64], ctypes.c_int),
        "afd_calc_force_materialized": ([_VP, _VP, _VP], ctypes.c_int),
        "afd_let_export": ([_VP, _VP, _D, _I64, _VP, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
        "afd_make_neighbour_lists": ([_VP, _VP, _D], ctypes.c_int),
        "afd_calc_density": ([_VP, _VP, _VP, _VP], ctypes.c_int),
        "afd_neighbour_stats": ([_VP, _VP], ctypes.c_int),
        "afd_partition_work": ([_VP, _I64, ctypes.c_int, _VP], ctypes.c_int),
        "afd_set_work_share": ([_VP, ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "afd_get_work_share": ([_VP, _VP], ctypes.c_int),
        "afd_get_launch": ([_VP, _VP, _VP], ctypes.c_int),
        "afd_autotune_launch": ([_VP, _VP, ctypes.c_int, _VP], ctypes.c_int),
        "afd_mac_set": ([_VP, _VP, _D, _D, _D], ctypes.c_int),
        "afd_mac_set_reference": ([_VP, _VP, _I64], ctypes.c_int),
        "afd_mac_samples": ([_VP, _D, _D, _D, ctypes.c_uint64, _I64, _VP, _VP, _VP, _VP],
                            ctypes.c_int),
        "afd_mac_info": ([_VP, _VP], ctypes.c_int),
        "afd_mlp_forward": ([_VP, _VP, _I64, _VP, _VP], ctypes.c_int),
        "afd_mlp_loss_grad": ([_VP, _VP, _VP, _I64, _VP, _VP, _VP], ctypes.c_int),
        "afd_mlp_train": ([_VP, _VP, _I64, ctypes.c_int, ctypes.c_int, _D, ctypes.c_uint64, _VP,
                           _VP, _VP], ctypes.c_int),
        "afd_direct_sum": ([_VP, _VP, _VP, _VP, _I64, _VP, _I64, _D, _VP, _VP], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _check(status: int, where: str):
    if status != 0:
        raise AfdError(status, where)


def _dptr(t, dtype=None, n=None, what="tensor"):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{what} must be {dtype}, got {t.dtype}")
    if n is not None and t.numel() < n:
        raise ValueError(f"{what} holds {t.numel()} elements, needs {n}")
    return _VP(t.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        return None
    return _VP(stream.cuda_stream)


# ---------------------------------------------------------------- C names


def afd_error_string(status: int) -> str:
    return lib().afd_error_string(int(status)).decode()


def afd_create(cfg: afd_config, device: int = 0, stream=None):
    h = _VP()
    _check(lib().afd_create(ctypes.byref(h), ctypes.byref(cfg), int(device), _stream_ptr(stream)),
           "afd_create")
    return h


def afd_destroy(ctx):
    lib().afd_destroy(ctx)


def afd_set_stream(ctx, stream):
    _check(lib().afd_set_stream(ctx, _stream_ptr(stream)), "afd_set_stream")


def afd_set_systems(ctx, sys_off, n_grp=None):
    """Declare independent systems: particles [sys_off[s], sys_off[s+1])."""
    off = np.ascontiguousarray(sys_off, dtype=np.int64)
    grp = None if n_grp is None else np.ascontiguousarray(n_grp, dtype=np.int32)
    _check(lib().afd_set_systems(ctx, _VP(off.ctypes.data), int(off.shape[0] - 1),
                                 None if grp is None else _VP(grp.ctypes.data)),
           "afd_set_systems")


def afd_tree_build(ctx, x, y, z, m):
    import torch
    n = x.numel()
    p = [_dptr(a, torch.float64, n, nm) for a, nm in zip((x, y, z, m), "xyzm")]
    _check(lib().afd_tree_build(ctx, *p, n), "afd_tree_build")


def afd_make_interaction_lists(ctx, mode=AFD_MAKE_LIST_FOR_REUSE):
    _check(lib().afd_make_interaction_lists(ctx, int(mode)), "afd_make_interaction_lists")


def afd_reuse_lists(ctx, x, y, z, m):
    import torch
    n = x.numel()
    p = [_dptr(a, torch.float64, n, nm) for a, nm in zip((x, y, z, m), "xyzm")]
    _check(lib().afd_reuse_lists(ctx, *p), "afd_reuse_lists")


def afd_calc_force(ctx, acc4):
    import torch
    _check(lib().afd_calc_force(ctx, _dptr(acc4, torch.float32, None, "acc4")), "afd_calc_force")


def afd_calc_force_all(ctx, x, y, z, m, acc4, mode):
    import torch
    n = x.numel()
    p = [_dptr(a, torch.float64, n, nm) for a, nm in zip((x, y, z, m), "xyzm")]
    _check(lib().afd_calc_force_all(ctx, *p, n, _dptr(acc4, torch.float32, 4 * n, "acc4"),
                                    int(mode)), "afd_calc_force_all")


def afd_calc_force_all_host(ctx, x, y, z, m, acc4, mode):
    """Host-array variant: x, y, z, m float64 and acc4 float32 (n, 4) CPU
    tensors or numpy arrays (pinned memory gives the fastest copies)."""
    def hp(a, dtype):
        if hasattr(a, "data_ptr"):
            if a.is_cuda or not a.is_contiguous():
                raise ValueError("host arrays must be contiguous CPU tensors")
            return _VP(a.data_ptr())
        if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be contiguous with the right dtype")
        return _VP(a.ctypes.data)
    n = len(x)
    p = [hp(a, np.float64) for a in (x, y, z, m)]
    _check(lib().afd_calc_force_all_host(ctx, *p, n, hp(acc4, np.float32), int(mode)),
           "afd_calc_force_all_host")


def afd_kick_drift(ctx, x, y, z, vx, vy, vz, acc4, dt_kick, dt_drift):
    import torch
    n = x.numel()
    p = [_dptr(a, torch.float64, n) for a in (x, y, z, vx, vy, vz)]
    _check(lib().afd_kick_drift(ctx, *p, _dptr(acc4, torch.float32, 4 * n), n, float(dt_kick),
                                float(dt_drift)), "afd_kick_drift")


def afd_kick(ctx, vx, vy, vz, acc4, dt_kick):
    import torch
    n = vx.numel()
    p = [_dptr(a, torch.float64, n) for a in (vx, vy, vz)]
    _check(lib().afd_kick(ctx, *p, _dptr(acc4, torch.float32, 4 * n), n, float(dt_kick)),
           "afd_kick")


def afd_leapfrog(ctx, x, y, z, vx, vy, vz, m, acc4, dt, n_steps, n_reuse):
    import torch
    n = x.numel()
    p = [_dptr(a, torch.float64, n) for a in (x, y, z, vx, vy, vz, m)]
    _check(lib().afd_leapfrog(ctx, *p, n, _dptr(acc4, torch.float32, 4 * n), float(dt),
                              int(n_steps), int(n_reuse)), "afd_leapfrog")


def afd_energy(ctx, vx, vy, vz, m, acc4):
    import torch
    n = vx.numel()
    out = (ctypes.c_double * 2)()
    p = [_dptr(a, torch.float64, n) for a in (vx, vy, vz, m)]
    _check(lib().afd_energy(ctx, *p, _dptr(acc4, torch.float32, 4 * n), n,
                            ctypes.cast(out, _VP)), "afd_energy")
    return float(out[0]), float(out[1])


def afd_set_walk_limits(ctx, iter_cap=0, stack_cap=0, arena_chunks_max=0):
    """Limits of the walks' bounded loops (0: defaults); for error-path tests."""
    _check(lib().afd_set_walk_limits(ctx, int(iter_cap), int(stack_cap), int(arena_chunks_max)),
           "afd_set_walk_limits")


def afd_sync(ctx):
    _check(lib().afd_sync(ctx), "afd_sync")


def afd_stats(ctx) -> dict:
    out = (ctypes.c_int64 * 10)()
    _check(lib().afd_stats(ctx, ctypes.cast(out, _VP)), "afd_stats")
    keys = ("n", "n_cells", "n_groups", "n_epj", "n_spj", "interactions", "saved", "max_level",
            "launches", "n_units")
    return dict(zip(keys, (int(v) for v in out)))


def afd_export(ctx, what: str) -> np.ndarray:
    item, dtype = EXPORT[what]
    nbytes = ctypes.c_size_t(0)
    _check(lib().afd_export(ctx, item, None, ctypes.byref(nbytes)), "afd_export")
    arr = np.zeros(nbytes.value // np.dtype(dtype).itemsize, dtype=dtype)
    if nbytes.value:
        _check(lib().afd_export(ctx, item, _VP(arr.ctypes.data), ctypes.byref(nbytes)),
               "afd_export")
    return arr


def afd_last_force_ms(ctx) -> float:
    v = ctypes.c_float(0.0)
    _check(lib().afd_last_force_ms(ctx, ctypes.byref(v)), "afd_last_force_ms")
    return float(v.value)


def afd_root_cell_static(x, y, z, m, root_out, nonfinite_out, stream=None):
    """Root cell without any device allocation (for callers that cannot
    allocate): root_out float64 (4,) and nonfinite_out int32 (1,) CUDA
    tensors receive the result; queued on ``stream``."""
    import torch
    n = x.numel()
    p = [_dptr(a, torch.float64, n, nm) for a, nm in zip((x, y, z, m), "xyzm")]
    _check(lib().afd_root_cell_static(*p, n, _dptr(root_out, torch.float64, 4, "root_out"),
                                      _dptr(nonfinite_out, torch.int32, 1, "nonfinite_out"),
                                      _stream_ptr(stream)), "afd_root_cell_static")


def afd_system_stats(ctx, n_sys):
    """Per-system (interactions, list entries) of the current lists."""
    inter = np.zeros(n_sys, np.int64)
    entries = np.zeros(n_sys, np.int64)
    _check(lib().afd_system_stats(ctx, _VP(inter.ctypes.data), _VP(entries.ctypes.data)),
           "afd_system_stats")
    return inter, entries


def afd_graph_capture_step(ctx, x, y, z, vx, vy, vz, m, acc4, dt):
    import torch
    n = x.numel()
    p = [_dptr(a, torch.float64, n) for a in (x, y, z, vx, vy, vz, m)]
    _check(lib().afd_graph_capture_step(ctx, *p, _dptr(acc4, torch.float32, 4 * n), float(dt)),
           "afd_graph_capture_step")


def afd_graph_launch(ctx):
    _check(lib().afd_graph_launch(ctx), "afd_graph_launch")


def afd_autotune_n_grp(ctx, x, y, z, m, acc4, candidates, n_reuse, n_sys=1):
    """Autotune n_grp per system; returns the chosen sizes (installed)."""
    import torch
    n = x.numel()
    p = [_dptr(a, torch.float64, n, nm) for a, nm in zip((x, y, z, m), "xyzm")]
    cand = np.ascontiguousarray(candidates, dtype=np.int32)
    best = np.zeros(n_sys, np.int32)
    _check(lib().afd_autotune_n_grp(ctx, *p, n, _VP(cand.ctypes.data), int(cand.shape[0]),
                                    int(n_reuse), _dptr(acc4, torch.float32, 4 * n, "acc4"),
                                    _VP(best.ctypes.data)), "afd_autotune_n_grp")
    return best


def afd_calc_force_materialized(ctx, acc4):
    """Non-indirect ablation; returns (copy ms, force ms)."""
    import torch
    ms = np.zeros(2, dtype=np.float32)
    _check(lib().afd_calc_force_materialized(ctx, _dptr(acc4, torch.float32, what="acc4"),
                                             _VP(ms.ctypes.data)), "afd_calc_force_materialized")
    return float(ms[0]), float(ms[1])


def afd_let_export(ctx, box, theta, cap=None):
    """Local essential tree for a remote domain box: (x, y, z, m, kind)
    device tensors (float64, float64, float64, float64, int32 viewed u32)."""
    import torch
    b = np.ascontiguousarray(box, dtype=np.float64)
    n = ctypes.c_int64(0)
    if cap is None:
        _check(lib().afd_let_export(ctx, _VP(b.ctypes.data), float(theta), 0, None, None, None,
                                    None, None, ctypes.byref(n)), "afd_let_export")
        cap = int(n.value)
    dev = torch.device("cuda", torch.cuda.current_device())
    out = [torch.empty(max(cap, 1), dtype=torch.float64, device=dev) for _ in range(4)]
    kind = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    _check(lib().afd_let_export(ctx, _VP(b.ctypes.data), float(theta), int(cap),
                                *(_VP(o.data_ptr()) for o in out), _VP(kind.data_ptr()),
                                ctypes.byref(n)), "afd_let_export")
    k = min(int(n.value), cap)
    return (*(o[:k] for o in out), kind[:k])


def afd_make_neighbour_lists(ctx, h, skin=0.0):
    """Neighbour lists for search radii h (CUDA float64, caller order) and
    margin skin (short-range walk, Section 2)."""
    import torch
    n = afd_stats(ctx)["n"]
    _check(lib().afd_make_neighbour_lists(ctx, _dptr(h, torch.float64, n, "h"), float(skin)),
           "afd_make_neighbour_lists")


def afd_calc_density(ctx, h, rho, nnb=None):
    """Gather density (and smooth neighbour number) over the neighbour
    lists into rho / nnb (CUDA float32, caller order)."""
    import torch
    n = afd_stats(ctx)["n"]
    _check(lib().afd_calc_density(ctx, _dptr(h, torch.float64, n, "h"),
                                  _dptr(rho, torch.float32, n, "rho"),
                                  None if nnb is None else _dptr(nnb, torch.float32, n, "nnb")),
           "afd_calc_density")


def afd_neighbour_stats(ctx) -> dict:
    out = (ctypes.c_int64 * 2)()
    _check(lib().afd_neighbour_stats(ctx, ctypes.cast(out, _VP)), "afd_neighbour_stats")
    return {"entries": int(out[0]), "pairs": int(out[1])}


def afd_partition_work(work, parts) -> np.ndarray:
    """Contiguous balanced parts of a host work array: bounds (parts + 1)."""
    w = np.ascontiguousarray(work, dtype=np.uint64)
    bounds = np.zeros(int(parts) + 1, dtype=np.int64)
    _check(lib().afd_partition_work(_VP(w.ctypes.data) if w.size else None, w.size, int(parts),
                                    _VP(bounds.ctypes.data)), "afd_partition_work")
    return bounds


def afd_set_work_share(ctx, part, parts):
    _check(lib().afd_set_work_share(ctx, int(part), int(parts)), "afd_set_work_share")


def afd_get_work_share(ctx) -> dict:
    out = (ctypes.c_int64 * 5)()
    _check(lib().afd_get_work_share(ctx, ctypes.cast(out, _VP)), "afd_get_work_share")
    return dict(zip(("part", "parts", "g0", "g1", "interactions"), (int(v) for v in out)))


def afd_set_launch(ctx, warps_per_block, chunk):
    _check(lib().afd_set_launch(ctx, int(warps_per_block), int(chunk)), "afd_set_launch")


def afd_get_launch(ctx):
    w, c = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().afd_get_launch(ctx, ctypes.byref(w), ctypes.byref(c)), "afd_get_launch")
    return int(w.value), int(c.value)


def afd_autotune_launch(ctx, acc4, reps=5):
    """Time the force kernel over (chunk, warps) in {32, 64} x {2, 4, 8} on
    the current lists and install the fastest; returns (warps, chunk, ms
    table of shape (2, 3))."""
    import torch
    ms = np.zeros(6, dtype=np.float32)
    _check(lib().afd_autotune_launch(ctx, _dptr(acc4, torch.float32, what="acc4"), int(reps),
                                     _VP(ms.ctypes.data)), "afd_autotune_launch")
    w, c = afd_get_launch(ctx)
    return w, c, ms.reshape(2, 3)


def afd_fp32_peak(device: int = 0, stream=None) -> float:
    """Measured FP32 FMA rate of the device in TFLOP/s."""
    v = ctypes.c_double(0.0)
    _check(lib().afd_fp32_peak(int(device), _stream_ptr(stream), ctypes.byref(v)), "afd_fp32_peak")
    return float(v.value)


def afd_pipe_rates(device: int = 0, stream=None) -> dict:
    """Measured packed/scalar FP32 FMA, MUFU rsqrt and packed FP16 FMA rates."""
    out = np.zeros(4)
    _check(lib().afd_pipe_rates(int(device), _stream_ptr(stream), _VP(out.ctypes.data)),
           "afd_pipe_rates")
    return {"f32x2_fma_tflops": float(out[0]), "f32_fma_tflops": float(out[1]),
            "rsqrt_tops": float(out[2]), "f16x2_fma_tflops": float(out[3])}


# ---------------------------------------------------------------- learned criterion

AFD_MAC_FEATURES = 8
AFD_MAC_HIDDEN = 32
AFD_MAC_PARAMS = 1393


def _host_f32(a, n, what):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.size != n:
        raise ValueError(f"{what} must hold {n} floats, got {a.size}")
    return a


def afd_mac_set(ctx, params, theta_lo, theta_hi, tau):
    """Install the network (host floats; None removes it)."""
    if params is None:
        _check(lib().afd_mac_set(ctx, None, 0.0, 0.0, 0.0), "afd_mac_set")
        return
    p = _host_f32(params, AFD_MAC_PARAMS, "params")
    _check(lib().afd_mac_set(ctx, _VP(p.ctypes.data), float(theta_lo), float(theta_hi),
                             float(tau)), "afd_mac_set")


def afd_mac_set_reference(ctx, amag):
    import torch
    _check(lib().afd_mac_set_reference(ctx, _dptr(amag, torch.float32, what="amag"),
                                       amag.numel()), "afd_mac_set_reference")


def afd_mac_samples(ctx, theta_lo, theta_hi, keep, seed, feat, label, pair=None):
    """Fill feat (cap x 8), label (cap) and optionally pair (cap x 2 int32
    tensor viewed as u32); returns the total number of kept pairs."""
    import torch
    cap = label.numel()
    n = ctypes.c_int64(0)
    _check(lib().afd_mac_samples(ctx, float(theta_lo), float(theta_hi), float(keep), int(seed),
                                 cap, _dptr(feat, torch.float32, 8 * cap, "feat"),
                                 _dptr(label, torch.float32, cap, "label"),
                                 _dptr(pair, torch.int32, 2 * cap, "pair"), ctypes.byref(n)),
           "afd_mac_samples")
    return int(n.value)


def afd_mac_info(ctx) -> dict:
    out = np.zeros(5, dtype=np.int64)
    _check(lib().afd_mac_info(ctx, _VP(out.ctypes.data)), "afd_mac_info")
    return {"learned": int(out[0]), "evaluations": int(out[1]), "accepted": int(out[2]),
            "reference": int(out[3]), "rounds": int(out[4])}


def afd_mlp_forward(params, feat, out, stream=None):
    import torch
    p = _host_f32(params, AFD_MAC_PARAMS, "params")
    n = out.numel()
    _check(lib().afd_mlp_forward(_VP(p.ctypes.data), _dptr(feat, torch.float32, 8 * n, "feat"), n,
                                 _dptr(out, torch.float32, n, "out"), _stream_ptr(stream)),
           "afd_mlp_forward")


def afd_mlp_loss_grad(params, feat, label, stream=None):
    """(loss, grad as numpy float32 array of AFD_MAC_PARAMS)."""
    import torch
    p = _host_f32(params, AFD_MAC_PARAMS, "params")
    n = label.numel()
    grad = np.zeros(AFD_MAC_PARAMS, dtype=np.float32)
    loss = ctypes.c_float(0.0)
    _check(lib().afd_mlp_loss_grad(_VP(p.ctypes.data), _dptr(feat, torch.float32, 8 * n, "feat"),
                                   _dptr(label, torch.float32, n, "label"), n,
                                   _VP(grad.ctypes.data), ctypes.byref(loss), _stream_ptr(stream)),
           "afd_mlp_loss_grad")
    return float(loss.value), grad


def afd_mlp_train(feat, label, epochs, batch, lr, seed, stream=None):
    """(params as numpy float32, per-epoch loss as numpy float32)."""
    import torch
    n = label.numel()
    params = np.zeros(AFD_MAC_PARAMS, dtype=np.float32)
    hist = np.zeros(int(epochs), dtype=np.float32)
    _check(lib().afd_mlp_train(_dptr(feat, torch.float32, 8 * n, "feat"),
                               _dptr(label, torch.float32, n, "label"), n, int(epochs), int(batch),
                               float(lr), int(seed), _VP(params.ctypes.data),
                               _VP(hist.ctypes.data), _stream_ptr(stream)), "afd_mlp_train")
    return params, hist


def afd_direct_sum(x, y, z, m, targets, eps, out, stream=None):
    """out: (n_t, 4) float64 CUDA tensor; targets: int32 CUDA tensor (u32)."""
    import torch
    n = x.numel()
    nt = targets.numel()
    _check(lib().afd_direct_sum(_dptr(x, torch.float64, n, "x"), _dptr(y, torch.float64, n, "y"),
                                _dptr(z, torch.float64, n, "z"), _dptr(m, torch.float64, n, "m"),
                                n, _dptr(targets, torch.int32, nt, "targets"), nt, float(eps),
                                _dptr(out, torch.float64, 4 * nt, "out"), _stream_ptr(stream)),
           "afd_direct_sum")


# ---------------------------------------------------------------- convenience


@dataclass
class Config:
    eps: float = 1.0 / 256
    theta: float = 0.5
    n_leaf: int = 16
    n_grp: int = 64
    multipole: int = 0
    far_precision: int = 0
    mac: int = 0

    def c(self) -> afd_config:
        return afd_config(float(self.eps), float(self.theta), int(self.n_leaf), int(self.n_grp),
                          int(self.multipole), int(self.far_precision), int(self.mac), 0)


class Gravity:
    """Owns one library context; methods forward to the C entry points."""

    def __init__(self, cfg: Config, device: int = 0, stream=None):
        self.cfg = cfg
        self.ctx = afd_create(cfg.c(), device, stream)

    def close(self):
        if self.ctx is not None and self.ctx.value:
            afd_destroy(self.ctx)
        self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def force_all(self, x, y, z, m, acc4, mode=AFD_MAKE_LIST_FOR_REUSE):
        afd_calc_force_all(self.ctx, x, y, z, m, acc4, mode)

    def stats(self):
        return afd_stats(self.ctx)

    def export(self, what):
        return afd_export(self.ctx, what)

    def neighbour_lists(self, h, skin=0.0):
        afd_make_neighbour_lists(self.ctx, h, skin)

    def density(self, h, rho, nnb=None):
        afd_calc_density(self.ctx, h, rho, nnb)
