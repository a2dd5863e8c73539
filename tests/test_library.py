"""The C-ABI library builds for sm_103a, loads, and exports every entry point of include/hodlr.h.

No compute calls: this runs on machines without a GPU.
"""
import ctypes
import os
import re
import subprocess

import pytest

import synth
from paper_2303_10102_gb300 import build as pbuild
from paper_2303_10102_gb300 import lib as plib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hodlr.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hodlr_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def so_path():
    return pbuild.build()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ["hodlr_create", "hodlr_build", "hodlr_nll", "hodlr_grad", "hodlr_fisher",
                     "hodlr_batch_nll_grad", "hodlr_perm", "hodlr_last_error", "hodlr_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(so_path):
    out = subprocess.run(["nm", "-D", "--defined-only", so_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (hodlr_[a-z_0-9]+)\b", out))
    missing = [n for n in declared_symbols() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(so_path)
    for n in declared_symbols():
        assert getattr(lib, n) is not None
    assert set(plib.SIGNATURES) == set(declared_symbols())


def test_build_targets_sm_103a_only():
    assert "arch=compute_103a,code=sm_103a" in pbuild.FLAGS
    assert sum("arch=" in f for f in pbuild.FLAGS) == 1


@pytest.mark.parametrize("name", ["C0", "C1", "C2", "C2L", "C4"])
def test_workspace_plan(so_path, name):
    w = synth.workload(name)
    lib = plib.load()
    m = plib.Model(w.dim, (ctypes.c_int * 2)(w.G, w.G if w.dim == 2 else 1), w.nvar, w.nu, 1)
    o = plib.Opts(w.leaf, w.cap, w.c - w.cap, w.tol, 1, 0.0)
    n = lib.hodlr_workspace_size(ctypes.byref(m), ctypes.byref(o))
    assert n > 0
    assert n < 280 * 2 ** 30, n / 2 ** 30          # fits one GB300 (FP32 bulk)


def test_workspace_plan_rejects_bad_options(so_path):
    lib = plib.load()
    m = plib.Model(3, (ctypes.c_int * 2)(8, 8), 1, 1.5, 0)
    o = plib.Opts(16, 4, 0, 0.0, 1, 0.0)
    assert lib.hodlr_workspace_size(ctypes.byref(m), ctypes.byref(o)) == 0
    m = plib.Model(1, (ctypes.c_int * 2)(64, 1), 2, 1.5, 0)
    o = plib.Opts(15, 4, 0, 0.0, 1, 0.0)                # leaf not a multiple of nvar
    assert lib.hodlr_workspace_size(ctypes.byref(m), ctypes.byref(o)) == 0


@pytest.mark.parametrize("name", ["C0", "C1", "C2", "C2L", "C4"])
def test_tree_order_bit_exact_at_full_size(so_path, name):
    """a1 (KD / Morton ordering and the cluster tree, Sec. 5.2 and Sec. 3.2.2): the library's host
    plan (hodlr_plan, no device work; the closed-form Morton rank and halving walk that the
    device kernel runs) equals the oracle's tree (a sort of the Morton keys) bit for bit at the
    workloads' full sizes, up to N = 2^21."""
    from oracle.tree import Tree
    import numpy as np
    w = synth.workload(name)
    lib = plib.load()
    m = plib.Model(w.dim, (ctypes.c_int * 2)(w.G, w.G if w.dim == 2 else 1), w.nvar, w.nu, 0)
    o = plib.Opts(w.leaf, w.cap, w.c - w.cap, w.tol, 1, 0.0)
    dims = np.zeros(6, dtype=np.int64)
    P64 = ctypes.POINTER(ctypes.c_int64)
    assert lib.hodlr_plan(ctypes.byref(m), ctypes.byref(o), dims.ctypes.data_as(P64), None) == 0
    t = Tree(w.dim, w.G, w.nvar, w.leaf)
    assert dims[0] == t.N and dims[1] == t.tau and dims[5] == 2 ** t.tau
    perm = np.zeros(t.N, dtype=np.int64)
    assert lib.hodlr_plan(ctypes.byref(m), ctypes.byref(o), dims.ctypes.data_as(P64), perm.ctypes.data_as(P64)) == 0
    assert np.array_equal(perm, np.asarray(t.perm, dtype=np.int64))


@pytest.mark.parametrize("dim,G,nvar,leaf", [(1, 99, 1, 32), (1, 1000, 1, 64), (1, 40961, 1, 64),
                                               (1, 4097, 2, 128), (2, 23, 1, 64), (2, 45, 2, 128),
                                               (2, 3, 1, 2), (2, 100, 1, 64), (2, 129, 2, 32), (2, 1000, 1, 256)])
def test_uneven_trees_match_the_oracle_bit_exactly(so_path, dim, G, nvar, leaf):
    """Median splits of a size that is not leaf x 2^tau (Sec. 3.2.2 index sets) give leaves whose
    sizes differ by one, and 2-D grids of a side that is not a power of two give Morton ranks
    that are not the keys themselves: the library's plan equals the oracle's tree order bit for
    bit."""
    import numpy as np
    from oracle.tree import Tree
    lib = plib.load()
    dims = np.zeros(6, dtype=np.int64)
    P64 = ctypes.POINTER(ctypes.c_int64)
    m = plib.Model(dim, (ctypes.c_int * 2)(G, G if dim == 2 else 1), nvar, 1.5, 0)
    o = plib.Opts(leaf, 8, 4, 0.0, 1, 0.0)
    t = Tree(dim, G, nvar, leaf)
    perm = np.zeros(t.N, dtype=np.int64)
    assert lib.hodlr_plan(ctypes.byref(m), ctypes.byref(o), dims.ctypes.data_as(P64), perm.ctypes.data_as(P64)) == 0
    sizes = [hi - lo for lo, hi in t.leaves()]
    assert dims[0] == t.N and dims[1] == t.tau and dims[5] == 2 ** t.tau and dims[2] == max(sizes)
    assert np.array_equal(perm, np.asarray(t.perm, dtype=np.int64))


def test_plan_rejects_bad_models(so_path):
    import numpy as np
    lib = plib.load()
    dims = np.zeros(6, dtype=np.int64)
    P64 = ctypes.POINTER(ctypes.c_int64)
    o = plib.Opts(32, 8, 4, 0.0, 1, 0.0)
    bad = plib.Model(3, (ctypes.c_int * 2)(16, 16), 1, 1.5, 0)
    assert lib.hodlr_plan(ctypes.byref(bad), ctypes.byref(o), dims.ctypes.data_as(P64), None) == -1   # EINVAL


def test_create_argument_errors_before_device_work(so_path):
    """hodlr_create reports bad arguments without touching the device: null pointers, an unknown
    model or precision, and a workspace that is not 256-byte aligned (all HODLR_EINVAL)."""
    lib = plib.load()
    h = ctypes.c_void_p()
    m = plib.Model(1, (ctypes.c_int * 2)(256, 1), 1, 1.5, 0)
    o = plib.Opts(32, 8, 4, 0.0, 1, 0.0)
    assert lib.hodlr_create(None, ctypes.byref(m), ctypes.byref(o), None, ctypes.c_void_p(256), 1 << 20) == -1
    assert lib.hodlr_create(ctypes.byref(h), None, ctypes.byref(o), None, ctypes.c_void_p(256), 1 << 20) == -1
    for bad in (plib.Model(3, (ctypes.c_int * 2)(16, 16), 1, 1.5, 0),      # dim
                plib.Model(1, (ctypes.c_int * 2)(256, 1), 3, 1.5, 0),      # nvar
                plib.Model(1, (ctypes.c_int * 2)(256, 1), 1, 2.5, 0),      # nu
                plib.Model(1, (ctypes.c_int * 2)(256, 1), 1, 1.5, 7)):     # precision
        assert lib.hodlr_create(ctypes.byref(h), ctypes.byref(bad), ctypes.byref(o), None, ctypes.c_void_p(256),
                                1 << 20) == -1
        assert not h.value
    assert lib.hodlr_create(ctypes.byref(h), ctypes.byref(m), ctypes.byref(o), None, ctypes.c_void_p(257),
                            1 << 30) == -1
    assert lib.hodlr_create(ctypes.byref(h), ctypes.byref(m), ctypes.byref(o), None, None, 1 << 30) == -1
    assert not h.value


def test_autotune_table_and_argument_errors(so_path):
    """The tuner's table is host data: empty until a context tunes, readable without a GPU."""
    import numpy as np
    lib = plib.load()
    n = ctypes.c_int(-1)
    assert lib.hodlr_autotune_clear() == 0
    assert lib.hodlr_autotune_table(None, 0, ctypes.byref(n)) == 0 and n.value == 0
    assert lib.hodlr_autotune_table(None, 4, ctypes.byref(n)) == -1
    assert lib.hodlr_autotune_table(None, 0, None) == -1
    assert lib.hodlr_autotune(None, 1) == -1
    assert plib.autotune_table() == []


def test_slice_plan_argument_errors(so_path):
    """hodlr_dgemm_slices_plan validates its plan on the host (no device work)."""
    lib = plib.load()
    for bad in [(2, 0, 1), (-2, 0, 1), (0, 3, 1), (1, 2, 1), (1, 0, 0)]:
        assert lib.hodlr_dgemm_slices_plan(*bad) == -1, bad
    for good in [(0, 0, 1), (0, 2, 1), (1, 1, 4), (-1, 0, 1)]:
        assert lib.hodlr_dgemm_slices_plan(*good) == 0, good
    assert lib.hodlr_dgemm_slices_plan(-1, 0, 1) == 0
