"""The C-ABI library builds, loads and exports every symbol include/sg.h declares.

CPU only: no kernel is launched.  The host-side parts of the library (GLL
nodes/weights, workspace size queries, argument validation) are checked
against the oracle and the header.
"""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sg.h")


@pytest.fixture(scope="module")
def sg():
    from paper_2009_10863_gb300 import build as b
    b.build()
    import paper_2009_10863_gb300 as sgmod
    sgmod.lib()
    return sgmod


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sg_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported_and_bound(sg):
    names = _declared()
    assert len(names) >= 18
    L = ctypes.CDLL(sg.LIB_PATH)
    for n in names:
        assert hasattr(L, n), "missing export " + n
    bound = {s[0] for s in sg.SIGNATURES}
    assert set(names) == bound


def test_version_and_error_strings(sg):
    L = sg.lib()
    assert L.sg_version() == 1
    h = ctypes.c_void_p()
    assert L.sg_op_create(ctypes.byref(h), 0, 1, 1, 3, 0.0, 0) == sg.ERR_INVALID
    assert b"element" in L.sg_last_error()
    assert L.sg_op_create(ctypes.byref(h), 2, 2, 2, 9, 0.0, 0) == sg.ERR_INVALID
    assert L.sg_op_create(ctypes.byref(h), 2, 2, 2, 3, -1.0, 0) == sg.ERR_INVALID
    assert L.sg_op_create(ctypes.byref(h), 2, 2, 2, 3, 0.0, 7) == sg.ERR_INVALID


@pytest.mark.parametrize("p", range(1, 9))
def test_library_gll_matches_oracle(sg, p):
    """The library's Newton/barycentric GLL nodes and weights agree with the
    oracle's numpy root-finding implementation."""
    from oracle.gll import gll_nodes_weights
    L = sg.lib()
    h = ctypes.c_void_p()
    assert L.sg_op_create(ctypes.byref(h), 2, 3, 1, p, 1.0, 0) == 0
    assert L.sg_op_size(h) == (2 * p + 1) * (3 * p + 1) * (p + 1)
    x = (ctypes.c_double * (p + 1))()
    w = (ctypes.c_double * (p + 1))()
    assert L.sg_op_gll(h, x, w) == 0
    xo, wo = gll_nodes_weights(p)
    assert np.allclose(np.array(x[:]), xo, atol=1e-15)
    assert np.allclose(np.array(w[:]), wo, atol=1e-15)
    assert L.sg_op_destroy(h) == 0


def test_workspace_queries(sg):
    L = sg.lib()
    n = 12345
    ring = L.sg_guess_workspace_bytes(n, 8, sg.EXTRAP, sg.F64)
    proj = L.sg_guess_workspace_bytes(n, 8, sg.PROJ_QR, sg.F64)
    ring32 = L.sg_guess_workspace_bytes(n, 8, sg.EXTRAP, sg.F32)
    assert ring >= 8 * 8 * n and proj >= 17 * 8 * n and proj > 2 * ring * 0.9
    assert ring32 < ring
    assert L.sg_guess_workspace_bytes(n, 17, sg.EXTRAP, sg.F64) == 0
    assert L.sg_guess_workspace_bytes(n, 8, 9, sg.F64) == 0
    assert L.sg_guess_workspace_bytes(0, 8, sg.EXTRAP, sg.F64) == 0


def test_argument_errors_without_a_device(sg):
    """Entry points reject bad arguments before any device work (so this runs
    on a host without a GPU) and say why."""
    L = sg.lib()
    VP = ctypes.c_void_p
    assert L.sg_pcg_solve_async(None, VP(16), VP(32), 1e-10, 10, 0, VP(256), None) == sg.ERR_INVALID
    assert b"NULL" in L.sg_last_error()
    assert L.sg_pcg_result(None, VP(256), None, None) == sg.ERR_INVALID
    assert L.sg_ir_solve_ru(None, None, VP(16), VP(32), 1e-10, 0.1, 5, 100, VP(256), None, None, None,
                            None) == sg.ERR_INVALID
    h = ctypes.c_void_p()
    assert L.sg_guess_create(ctypes.byref(h), 1000, 8, sg.PROJ_ENERGY, -1, 1e-10, None, VP(256),
                             sg.F64) == sg.ERR_INVALID
    assert b"operator" in L.sg_last_error()
    assert L.sg_guess_create(ctypes.byref(h), 1000, 8, 7, -1, 1e-10, None, VP(256), sg.F64) == sg.ERR_INVALID
    n = 4321
    assert L.sg_guess_workspace_bytes(n, 8, sg.PROJ_ENERGY, sg.F64) == L.sg_guess_workspace_bytes(n, 8, sg.PROJ_QR,
                                                                                                   sg.F64)
    assert L.sg_guess_workspace_bytes(n, 8, 7, sg.F64) == 0


def test_layer_knob_and_deviceless_operator(sg):
    """sg_op_set_layers validates its arguments; on a host without a CUDA
    device an operator still answers the host queries but refuses launches."""
    L = sg.lib()
    assert L.sg_op_set_layers(None, 1) == sg.ERR_INVALID
    h = ctypes.c_void_p()
    assert L.sg_op_create(ctypes.byref(h), 2, 2, 3, 4, 1.0, sg.F64) == 0
    assert L.sg_op_set_layers(h, -1) == sg.ERR_INVALID
    assert b"zl" in L.sg_last_error()
    for zl in (0, 1, 2, 7):
        assert L.sg_op_set_layers(h, zl) == 0
    assert L.sg_op_size(h) == (2 * 4 + 1) * (2 * 4 + 1) * (3 * 4 + 1)
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        VP = ctypes.c_void_p
        assert L.sg_sem_apply(h, VP(256), VP(512), None) == sg.ERR_STATE
        assert b"without a CUDA device" in L.sg_last_error()
    assert L.sg_op_destroy(h) == 0


def test_noalloc_constants_match_header(sg):
    text = open(HEADER).read()
    assert int(re.search(r"#define SG_NOALLOC_MAX_NODES (\d+)", text).group(1)) == sg.NOALLOC_MAX_NODES
    assert int(re.search(r"#define SG_NOALLOC_SCRATCH_BYTES \(?(\d+)", text).group(1)) == sg.NOALLOC_SCRATCH_BYTES


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("p", range(1, 9))
def test_noalloc_scratch_holds_every_accepted_operator(sg, p, dtype):
    """Every operator the allocation-free PCG accepts (at most
    NOALLOC_MAX_NODES nodes) fits its static scratch array: for degree p and
    both dtypes, the cubic mesh and the thinnest column mesh (the most reduction
    partials) just below the node limit.  The workspace query is evaluated on
    this host (no device: one SM assumed); the bound adds the partials of the
    largest update grid a GPU with 152 SMs uses (8 CTAs per SM, 4 doubles each)."""
    L = sg.lib()
    es = 8 if dtype == 0 else 4
    meshes = []
    e = 1
    while ((p * (e + 1) + 1) ** 3) <= sg.NOALLOC_MAX_NODES:
        e += 1
    meshes.append((e, e, e))
    ez = (sg.NOALLOC_MAX_NODES // (p + 1) ** 2 - 1) // p
    meshes.append((1, 1, ez))
    for E in meshes:
        h = ctypes.c_void_p()
        assert L.sg_op_create(ctypes.byref(h), *E, p, 1.0, dtype) == sg.OK
        n = L.sg_op_size(h)
        assert 0 < n <= sg.NOALLOC_MAX_NODES
        ws = int(L.sg_pcg_workspace_bytes(h))
        assert ws >= 5 * es * n
        assert ws + 8 * 152 * 4 * 8 <= sg.NOALLOC_SCRATCH_BYTES, (E, ws)
        L.sg_op_destroy(h)
