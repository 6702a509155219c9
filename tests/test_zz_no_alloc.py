"""The allocation-free PCG entry point against the workspace one, through the C ABI.

sg_pcg_solve_noalloc serves callers that cannot allocate device memory: its
scratch is a static array inside the library, so the caller passes only the
operator, b and x.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_10863_gb300 import build as b
    b.build()
    import paper_2009_10863_gb300 as sgmod
    sgmod.lib()
    return sgmod


def _noalloc(sg, op, b, x, tol, maxit=10000):
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = sg.lib().sg_pcg_solve_noalloc(op.h, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                       float(tol), int(maxit), sg.STOP_REL_B, ctypes.byref(it),
                                       ctypes.byref(rr), stream)
    return rc, it.value, rr.value


def _problem(sg, E, p, lam, seed, dtype="f64"):
    op = sg.Op(*E, p, lam, dtype)
    rng = np.random.default_rng(seed)
    xs = torch.tensor(rng.standard_normal(op.n), dtype=op.dtype, device="cuda")
    b = op.apply(xs)
    x0 = torch.tensor(0.1 * rng.standard_normal(op.n), dtype=op.dtype, device="cuda")
    return op, b, x0


def test_noalloc_matches_workspace_pcg_two_calls(sg):
    cases = [((4, 4, 4), 3, 0.0, 1), ((3, 4, 5), 5, 50.0, 2)]   # two calls in a row
    for E, p, lam, seed in cases:
        op, b, x0 = _problem(sg, E, p, lam, seed)
        x_ref = x0.clone()
        it_ref, rel_ref = op.pcg(b, x_ref, 1e-10)
        x_new = x0.clone()
        rc, it_new, rel_new = _noalloc(sg, op, b, x_new, 1e-10)
        torch.cuda.synchronize()
        assert rc == sg.OK
        assert abs(it_new - it_ref) <= 1
        assert rel_new <= 1e-10 * 1.0000001
        d = float(torch.linalg.vector_norm(x_new - x_ref)) / float(torch.linalg.vector_norm(x_ref))
        assert d <= 1e-10


def test_noalloc_largest_accepted_size_against_oracle(sg):
    """A solve near the array's capacity: 7x7x7 elements of degree 7 (125,000
    nodes, FP64: five PCG vectors of 1 MB each) against the FP64 oracle's PCG
    from the same guess -- iterations +-1 and the solution to 1e-10 -- on two
    calls in a row."""
    from oracle.sem import SemOperator
    from oracle.pcg import pcg as opcg
    E, p, lam = (7, 7, 7), 7, 10.0
    ref = SemOperator(*E, p, lam)
    assert ref.n <= sg.NOALLOC_MAX_NODES and ref.n > 0.9 * sg.NOALLOC_MAX_NODES
    op = sg.Op(*E, p, lam, "f64")
    rng = np.random.default_rng(5)
    for call in range(2):
        xs = rng.standard_normal(ref.n) * ref.interior
        b = ref.apply(xs)
        x0 = 0.1 * rng.standard_normal(ref.n) * ref.interior
        x = torch.tensor(x0, dtype=torch.float64, device="cuda")
        bd = torch.tensor(b, dtype=torch.float64, device="cuda")
        rc, it, rr = _noalloc(sg, op, bd, x, 1e-10)
        torch.cuda.synchronize()
        assert rc == sg.OK
        xo, ito, _, _ = opcg(ref.apply, ref.diagonal(), b, x0, 1e-10, interior=ref.interior)
        assert abs(it - ito) <= 1, "call %d: %d vs %d iterations" % (call, it, ito)
        xg = x.cpu().numpy()
        assert np.linalg.norm(xg - xo) <= 1e-10 * np.linalg.norm(xo) * (1 if it == ito else 10)
        assert np.linalg.norm(b - ref.apply(xg)) <= 1.0000001e-10 * np.linalg.norm(b)


def test_noalloc_fp32_and_size_limit(sg):
    op, b, x0 = _problem(sg, (4, 4, 4), 3, 1.0, 3, "f32")
    x_ref = x0.clone()
    it_ref, _ = op.pcg(b, x_ref, 1e-5)
    x_new = x0.clone()
    rc, it_new, _ = _noalloc(sg, op, b, x_new, 1e-5)
    assert rc == sg.OK and abs(it_new - it_ref) <= 1
    d = float(torch.linalg.vector_norm(x_new - x_ref)) / float(torch.linalg.vector_norm(x_ref))
    assert d <= 1e-5
    # above the stated maximum: rejected with a clear message, x untouched
    big = sg.Op(16, 16, 16, 7, 0.0, "f64")
    xb = big.zeros()
    rc, _, _ = _noalloc(sg, big, big.zeros(), xb, 1e-8)
    assert rc == sg.ERR_INVALID
    assert b"maximum" in sg.lib().sg_last_error()
