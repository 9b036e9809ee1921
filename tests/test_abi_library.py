"""The C-ABI library without a GPU: it builds, loads, exports every entry
point include/afdps.h declares, and validates arguments on the host. No
compute call is made here."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "afdps.h")
PKG = os.path.join(ROOT, "paper_1907_02290_gb300")


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char \*)\s*(afd_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1907_02290_gb300 import build

    return build.build()


def test_header_declares_the_boundary():
    names = declared()
    for required in ("afd_create", "afd_destroy", "afd_tree_build", "afd_make_interaction_lists",
                     "afd_reuse_lists", "afd_calc_force", "afd_calc_force_all",
                     "afd_error_string", "afd_export"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (afd_\w+)$", out, re.M))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(libpath)
    for n in declared():
        assert getattr(lib, n)


def test_host_side_validation_without_gpu(libpath):
    import paper_1907_02290_gb300 as afd

    L = afd.lib()
    assert afd.afd_error_string(0) == "ok"
    assert "saved" in afd.afd_error_string(-4)
    h = ctypes.c_void_p()
    for bad in (afd.Config(n_grp=0), afd.Config(n_grp=2048), afd.Config(eps=-1.0),
                afd.Config(theta=float("nan")), afd.Config(n_leaf=0), afd.Config(multipole=2),
                afd.Config(mac=2)):
        assert L.afd_create(ctypes.byref(h), ctypes.byref(bad.c()), 0, None) == -1
    assert L.afd_create(None, None, 0, None) == -1
    assert L.afd_calc_force(None, None) == -1
    assert L.afd_stats(None, None) == -1
    # learned criterion: argument checks happen before any device work
    assert L.afd_mac_set(None, None, 0.0, 0.0, 0.0) == -1
    assert L.afd_mac_set_reference(None, None, 0) == -1
    assert L.afd_mac_info(None, None) == -1
    assert L.afd_mlp_forward(None, None, 0, None, None) == -1
    assert L.afd_mlp_loss_grad(None, None, None, 0, None, None, None) == -1
    assert L.afd_mlp_train(None, None, 0, 1, 1, 1e-3, 0, None, None, None) == -1
    assert L.afd_direct_sum(None, None, None, None, 10, None, 0, 0.0, None, None) == 0
    assert L.afd_direct_sum(None, None, None, None, 10, None, 5, -1.0, None, None) == -1
    assert afd.afd_error_string(-12).startswith("no reference accelerations")


def test_work_partition_is_contiguous_covering_and_balanced(libpath):
    """afd_partition_work (host only): bounds run from 0 to n without going
    back, every part's work is within one element of total / parts, each
    bound is the first index whose prefix reaches its share, and all-zero
    work is split by count."""
    import numpy as np

    import paper_1907_02290_gb300 as afd

    gen = np.random.default_rng(3)
    for n, parts in ((1, 1), (7, 2), (1000, 8), (14270, 8), (5, 9), (300, 3)):
        w = gen.integers(0, 10**6, n).astype(np.uint64)
        w[gen.random(n) < 0.1] = 0
        b = afd.afd_partition_work(w, parts)
        assert b[0] == 0 and b[-1] == n and np.all(np.diff(b) >= 0)
        pre = np.concatenate([[0], np.cumsum(w.astype(np.float64))])
        tot = pre[-1]
        share = np.array([pre[b[p + 1]] - pre[b[p]] for p in range(parts)])
        assert np.all(np.abs(share - tot / parts) <= w.max() + 1e-6 * tot)
        for p in range(1, parts):
            k = b[p]
            assert pre[k] * parts >= tot * p and (k == 0 or pre[k - 1] * parts < tot * p)
    assert list(afd.afd_partition_work(np.zeros(4, np.uint64), 3)) == [0, 2, 3, 4]
    assert list(afd.afd_partition_work(np.zeros(0, np.uint64), 3)) == [0, 0, 0, 0]
    L = afd.lib()
    assert L.afd_partition_work(None, 3, 2, None) == -1
    assert L.afd_set_work_share(None, 0, 1) == -1


C_CLIENT = r"""
/* A plain C99 client of the library: only include/afdps.h, no C++ and no
 * Python. Without a GPU it exercises the host-side calls. */
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "afdps.h"

int main(void) {
  if (strcmp(afd_error_string(AFD_OK), "ok") != 0) return 1;
  afd_config bad;
  memset(&bad, 0, sizeof(bad));
  bad.n_grp = 0; /* invalid */
  afd_ctx *ctx = NULL;
  if (afd_create(&ctx, &bad, 0, NULL) != AFD_ERR_ARG) return 2;
  if (afd_calc_force(NULL, NULL) != AFD_ERR_ARG) return 3;
  const uint64_t work[6] = {4, 4, 4, 4, 4, 4};
  int64_t bounds[4];
  if (afd_partition_work(work, 6, 3, bounds) != AFD_OK) return 4;
  if (bounds[0] != 0 || bounds[1] != 2 || bounds[2] != 4 || bounds[3] != 6) return 5;
  printf("c client ok\n");
  return 0;
}
"""


def test_plain_c_client_compiles_links_and_runs(libpath, tmp_path):
    """The boundary is a C ABI: a C99 program that includes only the header
    compiles with -Werror, links against the shared library and runs its
    host-side calls."""
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    libdir = os.path.dirname(libpath)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I",
                    os.path.join(ROOT, "include"), str(src), "-o", str(exe), "-L", libdir,
                    "-l:" + os.path.basename(libpath), "-Wl,-rpath," + libdir],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, (out.returncode, out.stderr)
    assert "c client ok" in out.stdout


def test_product_path_never_touches_the_oracle():
    """The package and its sources neither import nor link the oracle."""
    for dirpath, _, files in os.walk(PKG):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "afdps_oracle" not in text and "afo_" not in text, f


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_1907_02290_gb300 as afd

    monkeypatch.setattr(afd, "_lib", None)
    monkeypatch.setattr(afd._build, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        afd.lib()


def test_self_checking_variant_compiles(tmp_path):
    """The AFD_CHECK=1 variant (index checks in the kernels) still builds."""
    from concurrent.futures import ThreadPoolExecutor

    from paper_1907_02290_gb300 import build

    def compile_one(name):
        src = os.path.join(PKG, "csrc", name)
        cmd = [build.nvcc(), "-c", src, "-o", str(tmp_path / (name + ".o")), "-I",
               os.path.join(ROOT, "include")] + build.ARCH + \
            ["-O1", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
             "-DAFD_CHECK=1"]
        return subprocess.run(cmd, capture_output=True, text=True)

    with ThreadPoolExecutor(3) as ex:
        res = list(ex.map(compile_one, ["afd_force.cu", "afd_walk.cu", "afd_tree.cu"]))
    for r in res:
        assert r.returncode == 0, r.stderr[-2000:]
