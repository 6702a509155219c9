"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Every comparison feeds both sides the same seeded inputs.  Tolerances:
FP64 operator 1e-13 (relative 2-norm; rounding order only), guesses 1e-12,
solutions 1e-10, PCG iterations +-1; FP32 paths 1e-5 relative.
"""
import numpy as np
import pytest

from oracle.sem import SemOperator
from oracle.pcg import pcg as opcg, REL_B, INITRESID, RHS
from oracle import extrap as oex
from oracle.proj import ProjectionQR, ProjectionClassic, ProjectionEnergy
from oracle.sequence import run_sequence
from synthetic import Modes, random_vectors, noise, CONFIGS, BATCHED

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


def dev(a, dtype=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dtype, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().double().cpu().numpy()


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


MESHES = [((1, 1, 1), 1, 0.0), ((2, 2, 2), 1, 1.0), ((4, 4, 4), 3, 0.0), ((3, 5, 2), 2, 3.5),
          ((5, 3, 4), 4, 0.0), ((2, 3, 2), 5, 1e3), ((4, 3, 3), 6, 0.0), ((5, 4, 3), 7, 1e5),
          ((9, 3, 2), 7, 0.0), ((2, 2, 3), 8, 2.0), ((1, 2, 1), 7, 1.0)]


# ---------------------------------------------------------------- operator
@pytest.mark.parametrize("E,p,lam", MESHES)
def test_sem_apply_f64(sg, E, p, lam):
    ref = SemOperator(*E, p, lam)
    op = sg.Op(*E, p, lam, "f64")
    x = random_vectors(p * 100 + sum(E), 1, ref.n)[0]      # boundary entries nonzero on purpose
    want = ref.apply(x)
    got = host(op.apply(dev(x)))
    assert rel(got, want) <= 1e-13
    assert np.max(np.abs(got - want)) <= 1e-12 * max(1.0, np.max(np.abs(want)))
    assert np.all(got[~ref.interior] == 0.0)


@pytest.mark.parametrize("E,p,lam", MESHES[2::2])
def test_sem_apply_f32(sg, E, p, lam):
    ref = SemOperator(*E, p, lam)
    op = sg.Op(*E, p, lam, "f32")
    x = np.float32(random_vectors(p + 7, 1, ref.n)[0]).astype(np.float64)
    want = ref.apply(x)
    got = host(op.apply(dev(x, torch.float32)))
    assert rel(got, want) <= 1e-5
    assert np.all(got[~ref.interior] == 0.0)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_sem_apply_layers_per_cta(sg, dtype):
    """The operator with 1, 2, 3 and all element layers per CTA (the z-carry
    between layers, the ring of staged planes, and the single-layer FP64 PCG
    step that stages the old p and q in idle ring slots) against the oracle."""
    E, p, lam = (3, 2, 7), 7, 30.0
    ref = SemOperator(*E, p, lam)
    op = sg.Op(*E, p, lam, dtype)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    x = random_vectors(17, 1, ref.n)[0]
    if dtype == "f32":
        x = np.float32(x).astype(np.float64)
    want = ref.apply(x)
    tol = 1e-13 if dtype == "f64" else 1e-5
    for zl in (1, 2, 3, 7, 0):
        op.set_layers(zl)
        assert rel(host(op.apply(dev(x, tdt))), want) <= tol, "zl = %d" % zl


@pytest.mark.parametrize("zl", [1, 2, 4])
def test_pcg_layers_per_cta(sg, zl):
    """FP64 PCG with the operator on 1, 2 and 4 element layers per CTA: the
    solution and the iteration count match the oracle's."""
    ref, rng, xs = _problem((3, 2, 6), 5, 20.0, seed=8)
    b = ref.apply(xs)
    x0 = np.zeros(ref.n)
    xo, ito, _, _ = opcg(ref.apply, ref.diagonal(), b, x0, 1e-10, interior=ref.interior)
    op = sg.Op(3, 2, 6, 5, 20.0, "f64")
    op.set_layers(zl)
    x = dev(x0)
    it, _ = op.pcg(dev(b), x, 1e-10)
    assert abs(it - ito) <= 1
    assert rel(host(x), xo) <= 1e-10


@pytest.mark.parametrize("E,p,lam", MESHES[::3])
def test_diagonal(sg, E, p, lam):
    ref = SemOperator(*E, p, lam)
    op = sg.Op(*E, p, lam, "f64")
    assert rel(host(op.diagonal()), ref.diagonal()) <= 1e-14


def test_sem_apply_full_size_fp64_helmholtz(sg):
    """16^3 elements, p = 7, lambda = 1e5: the FP64 Helmholtz operator at full size."""
    c = CONFIGS["helmholtz_16x16x16_p7"]
    ref = SemOperator(*c["E"], c["p"], c["lam"])
    op = sg.Op(*c["E"], c["p"], c["lam"], "f64")
    cx, cy, cz = ref.coords_1d()
    x = Modes(c["seed"], c["modes"], c["kmax"]).field(cx, cy, cz, 0.3)
    x = x + 1e-3 * random_vectors(9, 1, ref.n)[0]
    want = ref.apply(x)
    got = host(op.apply(dev(x)))
    assert rel(got, want) <= 1e-13


def test_sem_apply_full_size_fp32_poisson(sg):
    """32^3 elements, p = 7 Poisson in FP32 (the mixed-precision operator)."""
    c = CONFIGS["poisson_32x32x32_p7"]
    ref = SemOperator(*c["E"], c["p"], c["lam"])
    op = sg.Op(*c["E"], c["p"], c["lam"], "f32")
    # a random field: a smooth one cancels strongly in A x (||A x|| << sum |terms|),
    # which measures FP32 rounding, not the kernel's indexing
    x = np.float32(random_vectors(31, 1, ref.n)[0]).astype(np.float64)
    want = ref.apply(x)
    got = host(op.apply(dev(x, torch.float32)))
    assert rel(got, want) <= 1e-5
    assert np.max(np.abs(got - want)) <= 1e-5 * np.max(np.abs(want))


# ---------------------------------------------------------------- PCG
def _problem(E=(4, 4, 4), p=3, lam=0.0, seed=3):
    ref = SemOperator(*E, p, lam)
    rng = np.random.default_rng(seed)
    xs = rng.standard_normal(ref.n) * ref.interior
    return ref, rng, xs


@pytest.mark.parametrize("tol", [1e-6, 1e-10])
@pytest.mark.parametrize("E,p,lam", [((4, 4, 4), 3, 0.0), ((3, 4, 5), 5, 50.0), ((5, 3, 2), 7, 1e4)])
def test_pcg_matches_oracle(sg, tol, E, p, lam):
    ref, rng, xs = _problem(E, p, lam)
    b = ref.apply(xs) + 0.01 * rng.standard_normal(ref.n) * ref.interior
    x0 = 0.1 * rng.standard_normal(ref.n) * ref.interior
    xo, ito, relo, _ = opcg(ref.apply, ref.diagonal(), b, x0, tol, interior=ref.interior)
    op = sg.Op(*E, p, lam, "f64")
    x = dev(x0)
    it, relg = op.pcg(dev(b), x, tol)
    assert abs(it - ito) <= 1
    assert relg <= tol * 1.0000001
    assert rel(host(x), xo) <= max(1e-10, 10 * tol)
    if it == ito:
        assert rel(host(x), xo) <= 1e-10


@pytest.mark.parametrize("crit", [REL_B, INITRESID, RHS])
def test_pcg_criteria(sg, crit):
    ref, rng, xs = _problem((3, 3, 3), 4, 2.0, seed=5)
    b = ref.apply(xs)
    x0 = xs + 1e-4 * rng.standard_normal(ref.n) * ref.interior
    _, ito, _, _ = opcg(ref.apply, ref.diagonal(), b, x0, 1e-8, criterion=crit, interior=ref.interior)
    op = sg.Op(3, 3, 3, 4, 2.0, "f64")
    x = dev(x0)
    it, _ = op.pcg(dev(b), x, 1e-8, criterion=crit)
    assert abs(it - ito) <= 1


def test_pcg_edge_cases(sg):
    ref, rng, xs = _problem((2, 3, 2), 3, 1.0, seed=6)
    op = sg.Op(2, 3, 2, 3, 1.0, "f64")
    b = ref.apply(xs)
    # exact initial guess: 0 iterations
    x = dev(xs)
    it, r = op.pcg(dev(b), x, 1e-10)
    assert it == 0 and r < 1e-12
    # b = 0: 0 iterations, x = 0 is returned for x0 = 0
    x = op.zeros()
    it, r = op.pcg(op.zeros(), x, 1e-10)
    assert it == 0 and float(x.abs().max()) == 0.0
    # maxit cap -> NOT_CONVERGED with exactly maxit iterations
    x = op.zeros()
    it, r = op.pcg(dev(b), x, 1e-14, maxit=3)
    assert it == 3 and r > 1e-14
    with pytest.raises(sg.SGError):
        op.pcg(dev(b), op.zeros(), 1e-14, maxit=3, raise_on_maxit=True)
    # boundary entries of the initial guess are zeroed
    x0 = xs + 5.0 * (~ref.interior)
    x = dev(x0)
    op.pcg(dev(b), x, 1e-10)
    assert np.all(host(x)[~ref.interior] == 0.0)


def test_pcg_single_element_all_boundary(sg):
    """One element of degree 1: every node is a Dirichlet node (n = 8)."""
    op = sg.Op(1, 1, 1, 1, 0.0, "f64")
    x = op.zeros()
    it, r = op.pcg(op.zeros(), x, 1e-10)
    assert it == 0
    y = op.apply(dev(np.arange(8.0)))
    assert float(y.abs().max()) == 0.0


# ---------------------------------------------------------------- extrapolation
@pytest.mark.parametrize("method,s,m", [("extrap", 4, 2), ("extrap", 8, 2), ("extrap", 8, 3),
                                        ("extrap", 6, 5), ("spextrap", 8, 2), ("spextrap", 12, 3),
                                        ("last", 4, 0), ("extrap", 1, 0)])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_extrap_sequence(sg, method, s, m, dtype):
    n = 3001                                   # ragged: not a multiple of the vector width
    tdt = torch.float64 if dtype == "f64" else torch.float32
    g = sg.Guess(n, s, method, m=m, dtype=dtype)
    hist = random_vectors(11, s + 5, n)
    if dtype == "f32":
        hist = np.float32(hist).astype(np.float64)
    ringh = []
    tolr = 1e-12 if dtype == "f64" else 1e-5
    for k in range(s + 5):
        x0 = torch.full((n,), 7.0, dtype=tdt, device="cuda")
        g.form(None, x0)
        if k == 0:
            assert float((x0 - 7.0).abs().max()) == 0.0      # no history: x0 untouched
        else:
            if method == "last":
                want = ringh[-1]
            else:
                beta = oex.startup_coeffs(len(ringh), s, m, sparse=(method == "spextrap"))
                want = oex.extrap_guess(ringh, beta)
            assert rel(host(x0), want) <= tolr
        # in-place protocol on even steps, copy on odd steps
        if k % 2 == 0:
            slot = g.next_slot()
            slot.copy_(dev(hist[k], tdt))
            g.update(slot)
        else:
            g.update(dev(hist[k], tdt))
        ringh.append(hist[k])
        keep = 1 if method == "last" else s
        ringh = ringh[-keep:]


def test_extrap_inplace_guess_into_next_slot(sg):
    """Guess formed straight into the slot that holds the oldest solution."""
    n, s, m = 1000, 4, 2
    g = sg.Guess(n, s, "extrap", m=m)
    hist = random_vectors(12, 6, n)
    for k in range(4):
        g.update(dev(hist[k]))
    slot = g.next_slot()
    g.form(None, slot)
    want = oex.extrap_guess(list(hist[:4]), oex.lsq_coeffs(4, 2))
    assert rel(host(slot), want) <= 1e-12


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("method", ["extrap", "qr", "energy"])
def test_guess_checkpoint_restore(sg, method, dtype):
    """A history exported after six updates of an s = 4 handle (the ring has
    wrapped) and restored into a fresh handle (its own workspace) forms the same
    guesses, bit for bit, as the original over three further steps.  Images of
    another kind of handle, truncated images, forged ring positions and (for
    projection) images built under another operator are refused before
    anything is copied: the refusing handle keeps forming its own guesses."""
    E, p, lam = (3, 2, 2), 4, 3.0
    tdt = torch.float64 if dtype == "f64" else torch.float32
    op = sg.Op(*E, p, lam, dtype)
    rng = np.random.default_rng(41)
    mask = host(op.apply(dev(np.ones(op.n), tdt))) != 0.0
    xs = [dev(rng.standard_normal(op.n) * mask, tdt) for _ in range(9)]
    bs = [dev(rng.standard_normal(op.n) * mask, tdt) for _ in range(3)]
    kw = dict(m=2) if method == "extrap" else dict(eps_rel=1e-4 if dtype == "f32" else 1e-10, op=op)
    g = sg.Guess(op.n, 4, method, dtype=dtype, **kw)
    for x in xs[:6]:
        g.update(x.clone())
    image = g.export()
    h = sg.Guess(op.n, 4, method, dtype=dtype, **kw)
    h.restore(image)
    for k in range(3):
        x0g, x0h = op.zeros(), op.zeros()
        g.form(bs[k], x0g)
        h.form(bs[k], x0h)
        assert torch.equal(x0g, x0h), "guess %d" % k
        g.update(xs[6 + k].clone())
        h.update(xs[6 + k].clone())
    assert g.info()[0] == h.info()[0]

    # refusals leave the target handle as it was
    other = sg.Guess(op.n, 3, method, dtype=dtype, **kw)
    for x in xs[:2]:
        other.update(x.clone())
    before = op.zeros()
    other.form(bs[0], before)
    bad = [image[:-8]]                                   # truncated
    forged = image.copy()
    forged[36:40] = np.frombuffer(np.int32(99).tobytes(), np.uint8)   # ring position 'next'
    bad.append(forged)
    for img in [image] + bad:
        with pytest.raises(sg.SGError):
            other.restore(img)
    with pytest.raises(sg.SGError):
        h.restore(forged)
    after = op.zeros()
    other.form(bs[0], after)
    assert torch.equal(before, after)
    if method != "extrap":                               # another operator (lambda)
        op2 = sg.Op(*E, p, 2 * lam, dtype)
        k = sg.Guess(op.n, 4, method, dtype=dtype, eps_rel=kw["eps_rel"], op=op2)
        with pytest.raises(sg.SGError):
            k.restore(image)


def test_zero_guess(sg):
    g = sg.Guess(100, 4, "zero")
    x0 = torch.ones(100, dtype=torch.float64, device="cuda")
    g.form(None, x0)
    assert float(x0.abs().max()) == 0.0


# ---------------------------------------------------------------- projection
def _proj_sequence(sg, klass, method, M, E=(3, 3, 2), p=3, lam=2.0, steps=10, dtype="f64", xscale=1.0,
                   bounded=False):
    ref = SemOperator(*E, p, lam)
    op = sg.Op(*E, p, lam, dtype)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    # the rejection threshold must sit above the storage precision's noise:
    # an in-span vector leaves ||b~|| / ||A x|| ~ 1e-7 after CGS2 in FP32
    eps = 1e-10 if dtype == "f64" else 1e-4
    g = sg.Guess(ref.n, M, method, eps_rel=eps, op=op, dtype=dtype)
    o = klass(M, eps, ref.apply)
    rng = np.random.default_rng(21)
    base = rng.standard_normal((3, ref.n)) * ref.interior
    tolr = 1e-12 if dtype == "f64" else 2e-4
    prev = []
    for k in range(steps):
        b = ref.apply(rng.standard_normal(ref.n) * ref.interior) * xscale
        x0 = torch.full((ref.n,), 3.0, dtype=tdt, device="cuda")
        g.form(dev(b, tdt), x0)
        want = o.form(b, np.full(ref.n, 3.0))
        assert rel(host(x0), want) <= tolr, "guess at step %d" % k
        if k == 6:   # a combination of earlier solutions (rejected when in the window)
            x = 0.5 * prev[-1] + 0.25 * prev[-2]
        else:
            c2 = np.cos(0.07 * k + 1.0) if bounded else 0.1 * k   # bounded: long runs stay well conditioned
            x = (np.cos(0.3 * k) * base[0] + np.sin(0.2 * k) * base[1] + c2 * base[2]
                 + 1e-3 * rng.standard_normal(ref.n) * ref.interior) * xscale
        if dtype == "f32":
            x = np.float32(x).astype(np.float64)
        g.update(dev(x, tdt))
        o.update(x)
        prev.append(x)
        d, R = g.info()
        assert d == o.d, "d at step %d" % k
        if method in ("qr", "energy") and dtype == "f64":
            Ro = o.R[:d, :d]
            assert np.allclose(R[:d, :d], Ro, rtol=1e-10, atol=1e-10 * np.abs(Ro).max())


@pytest.mark.parametrize("M", [1, 2, 3, 5])
def test_proj_qr_sequence(sg, M):
    _proj_sequence(sg, ProjectionQR, "qr", M)


def test_proj_qr_long_sequence(sg):
    """40 steps of QR(4): 36 Givens downdates in the factored form, whose
    column scales are carried from step to step."""
    _proj_sequence(sg, ProjectionQR, "qr", 4, steps=40)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_proj_qr_very_long_sequence(sg, dtype):
    """300 steps of QR(3): the column scales of the factored downdate are
    carried through 297 downdates and the guesses stay on the oracle's."""
    _proj_sequence(sg, ProjectionQR, "qr", 3, steps=300, dtype=dtype, bounded=True)


@pytest.mark.parametrize("method,klass", [("qr", ProjectionQR), ("energy", ProjectionEnergy)])
def test_proj_sequence_tiny_values(sg, method, klass):
    """Solutions of size ~1e-100 give column scales ~1e100, outside the range
    the factored downdate keeps; the downdate then runs in the plain form."""
    _proj_sequence(sg, klass, method, 3, xscale=1e-100)


def test_proj_sequence_tiny_values_f32(sg):
    """FP32 storage keeps scales within 2^+-40: solutions of size ~1e-15
    (scales ~1e15) send every downdate through the plain form."""
    _proj_sequence(sg, ProjectionQR, "qr", 3, xscale=1e-15, dtype="f32")


def test_proj_qr_sequence_f32(sg):
    _proj_sequence(sg, ProjectionQR, "qr", 4, dtype="f32")


@pytest.mark.parametrize("M", [1, 3, 4])
def test_proj_classic_sequence(sg, M):
    _proj_sequence(sg, ProjectionClassic, "classic", M)


@pytest.mark.parametrize("M", [1, 2, 3, 5])
def test_proj_energy_sequence(sg, M):
    """Energy-norm projection (A-orthonormal X~) against the oracle: guesses to
    1e-12, history size and R through insertions, a rejected dependent vector
    and Givens downdates."""
    _proj_sequence(sg, ProjectionEnergy, "energy", M)


def test_proj_energy_sequence_f32(sg):
    _proj_sequence(sg, ProjectionEnergy, "energy", 4, dtype="f32")


def test_proj_energy_full_size_galerkin(sg):
    """16^3 p = 7 FP64 Helmholtz, ENERGY(6) after 8 updates (two downdates): the
    guess is the A-orthogonal projection of the solution onto the window, so its
    residual is orthogonal to every window solution (x_j . (b - A x0) = 0), and
    an in-span right-hand side gives back its solution."""
    E, p, lam, M = (16, 16, 16), 7, 1e5, 6
    op = sg.Op(*E, p, lam, "f64")
    g = sg.Guess(op.n, M, "energy", eps_rel=1e-10, op=op)
    cx, cy, cz = op.coords_1d()
    inner = [(c > 0) & (c < 1) for c in (cx, cy, cz)]
    mask = np.einsum('k,j,i->kji', inner[2], inner[1], inner[0]).reshape(-1).astype(np.float64)
    rng = np.random.default_rng(31)
    xs = [dev(rng.standard_normal(op.n) * mask) for _ in range(M + 2)]
    for x in xs:
        g.update(x)
    assert g.info()[0] == M
    b = op.apply(dev(rng.standard_normal(op.n) * mask))
    x0 = op.zeros()
    g.form(b, x0)
    r = b - op.apply(x0)
    for xj in xs[2:]:
        assert abs(float(xj @ r)) <= 1e-10 * float(xj.norm() * b.norm())
    xin = 0.7 * xs[-1] - 0.4 * xs[-3]
    g.form(op.apply(xin), x0)
    assert rel(host(x0), host(xin)) <= 1e-10


def test_proj_rejects_dependent_vector(sg):
    ref = SemOperator(3, 2, 2, 3, 1.0)
    op = sg.Op(3, 2, 2, 3, 1.0, "f64")
    g = sg.Guess(ref.n, 4, "qr", eps_rel=1e-8, op=op)
    rng = np.random.default_rng(2)
    xs = rng.standard_normal((2, ref.n)) * ref.interior
    for x in xs:
        g.update(dev(x))
    assert g.info()[0] == 2
    g.update(dev(0.3 * xs[0] - 2.0 * xs[1]))
    assert g.info()[0] == 2
    # b in the span -> the guess is the exact solution
    xin = 1.5 * xs[0] + 0.25 * xs[1]
    x0 = op.zeros()
    g.form(dev(ref.apply(xin)), x0)
    assert rel(host(x0), xin) <= 1e-12


def test_proj_full_size(sg):
    """QR(8) at 16^3 elements, p = 7 (1.44M nodes): ten updates, guesses vs the oracle."""
    c = CONFIGS["helmholtz_16x16x16_p7"]
    ref = SemOperator(*c["E"], c["p"], c["lam"])
    op = sg.Op(*c["E"], c["p"], c["lam"], "f64")
    cx, cy, cz = ref.coords_1d()
    modes = Modes(c["seed"], 12, c["kmax"])
    g = sg.Guess(ref.n, 8, "qr", eps_rel=1e-10, op=op)
    o = ProjectionQR(8, 1e-10, ref.apply)
    rng = np.random.default_rng(5)
    for k in range(10):
        x = modes.field(cx, cy, cz, 0.01 * k) * ref.interior + 1e-6 * rng.standard_normal(ref.n) * ref.interior
        g.update(dev(x))
        o.update(x)
    b = ref.apply(modes.field(cx, cy, cz, 0.1) * ref.interior)
    x0 = op.zeros()
    g.form(dev(b), x0)
    assert g.info()[0] == o.d == 8
    assert rel(host(x0), o.form(b, np.zeros(ref.n))) <= 1e-12


def test_headline_sequence_full_size(sg):
    """The 16^3 p = 7 Helmholtz sequence with EXTRAP(2,8) and 1e-10, run as
    the bench runs it (right-hand sides with the bench's noise, guess formed in
    the next ring slot, PCG as one graph launch) for 18 steps, so that the
    steady-state guess from a full ring of 8 solutions is compared 10 times:
    every guess equals the oracle's extrapolation of the GPU's earlier
    solutions, and at three sampled steps (one during start-up, two with a full
    ring) the oracle's PCG from the same guess takes the same number of
    iterations (+-1) to the same solution."""
    c = CONFIGS["helmholtz_16x16x16_p7"]
    s, m, tol = c["s"], 2, c["tol"]
    ref = SemOperator(*c["E"], c["p"], c["lam"])
    op = sg.Op(*c["E"], c["p"], c["lam"], "f64")
    cx, cy, cz = ref.coords_1d()
    modes = Modes(c["seed"], c["modes"], c["kmax"])
    g = sg.Guess(op.n, s, "extrap", m=m)
    diag = ref.diagonal()
    sols = []
    full_ring = 0
    for k in range(1, 19):
        b = ref.apply(modes.field(cx, cy, cz, c["dt"] * k) * ref.interior)
        b = b + c["noise"] * np.sqrt(np.mean(b * b)) * noise(c["seed"], k, ref.n) * (b != 0)
        x = g.next_slot()
        g.form(dev(b), x)
        x0 = host(x)
        if sols:
            beta = oex.startup_coeffs(len(sols), s, m)
            assert rel(x0, oex.extrap_guess(sols[-s:], beta)) <= 1e-12, "guess at step %d" % k
            full_ring += len(sols) >= s
        it, _ = op.pcg(dev(b), x, tol)
        xk = host(x)
        if k in (4, 12, 18):
            xo, ito, _, _ = opcg(ref.apply, diag, b, x0, tol, interior=ref.interior)
            assert abs(it - ito) <= 1, "iterations at step %d" % k
            assert rel(xk, xo) <= (1e-10 if it == ito else 10 * tol)
        g.update(x)
        sols.append(xk)
    assert full_ring == 10


# ---------------------------------------------------------------- whole sequence
def _gpu_sequence(sg, c, method, s, m, rhs, dtype="f64"):
    op = sg.Op(*c["E"], c["p"], c["lam"], dtype)
    g = sg.Guess(op.n, s, method, m=m, eps_rel=c["tol"], op=op)
    out = []
    for b in rhs:
        bd = dev(b)
        x = g.next_slot() if method in ("extrap", "last", "spextrap") else op.zeros()
        if x is None:
            x = op.zeros()
        if method == "zero":
            x.zero_()
        g.form(bd, x)
        it, r = op.pcg(bd, x, c["tol"])
        g.update(x)
        out.append((it, r, host(x)))
    return out


@pytest.mark.parametrize("method,mcode", [("zero", 0), ("last", 1), ("extrap", 2), ("qr", 3)])
def test_c1_sequence_end_to_end(sg, method, mcode):
    """The 4^3-element, p = 3 Poisson sequence (20 steps, s = 4, tol 1e-8)."""
    c = CONFIGS["poisson_4x4x4_p3"]
    ref = SemOperator(*c["E"], c["p"], c["lam"])
    cx, cy, cz = ref.coords_1d()
    modes = Modes(c["seed"], c["modes"], c["kmax"])
    rhs = [ref.apply(modes.field(cx, cy, cz, c["dt"] * k) * ref.interior) for k in range(1, c["steps"] + 1)]
    o = run_sequence(ref, rhs, mcode, c["s"], m=2, tol=c["tol"], keep=True)
    gres = _gpu_sequence(sg, c, method, c["s"], 2, rhs)
    for k, (rec, (it, r, x)) in enumerate(zip(o, gres)):
        assert abs(it - rec["iters"]) <= 1, "step %d: %d vs %d" % (k, it, rec["iters"])
        assert r <= c["tol"] * 1.000001
        assert rel(x, rec["x"]) <= 1e-6
    # the better guesses must cut iterations versus the zero guess
    if method in ("extrap", "qr"):
        assert sum(t[0] for t in gres[8:]) < sum(rec["iters"] for rec in run_sequence(ref, rhs, 0, 4, tol=c["tol"])[8:])


# ---------------------------------------------------------------- mixed precision
@pytest.mark.parametrize("method", ["restart", "replace"])
@pytest.mark.parametrize("E,p,lam", [((4, 4, 4), 3, 0.0), ((3, 4, 5), 5, 50.0), ((4, 4, 3), 7, 0.0)])
def test_fp32_ir_reaches_fp64_tolerance(sg, E, p, lam, method):
    """FP32 operator/PCG wrapped in FP64 refinement (restarted, or with residual
    replacement) meets ||b - A x|| <= 1e-10 ||b|| measured with the FP64 oracle
    operator; error vs the FP64 oracle solution is reported and bounded."""
    ref, rng, xs = _problem(E, p, lam, seed=8)
    b = ref.apply(xs)
    ms = sg.MixedSolver(*E, p, lam)
    x = ms.op64.zeros()
    outer, inner, relg = ms.solve(dev(b), x, 1e-10, inner_tol=1e-5, method=method)
    xg = host(x)
    rel_oracle = np.linalg.norm(b - ref.apply(xg)) / np.linalg.norm(b)
    assert relg <= 1e-10 and rel_oracle <= 1.01e-10
    assert outer >= 2 and inner > 0
    xo, _, _, _ = opcg(ref.apply, ref.diagonal(), b, np.zeros(ref.n), 1e-13, interior=ref.interior)
    assert rel(xg, xo) <= 1e-7


@pytest.mark.parametrize("method", ["restart", "replace"])
def test_fp32_ir_full_size_c3(sg, method):
    """One mixed-precision solve on the full 32^3 p = 7 Poisson mesh (11.4M
    nodes, the FP32 operator's multi-layer CTAs and the FP64 residual pass at
    that size), from the EXTRAP-free zero guess: the FP64 residual measured with
    the oracle operator meets 1e-10, and the solution agrees with the smooth
    manufactured one to the accuracy the system's conditioning allows."""
    c = CONFIGS["poisson_32x32x32_p7"]
    ref = SemOperator(*c["E"], c["p"], c["lam"])
    cx, cy, cz = ref.coords_1d()
    xs = Modes(c["seed"], c["modes"], c["kmax"]).field(cx, cy, cz, 0.37) * ref.interior
    b = ref.apply(xs)
    ms = sg.MixedSolver(*c["E"], c["p"], c["lam"])
    x = ms.op64.zeros()
    outer, inner, relg = ms.solve(dev(b), x, 1e-10, method=method)
    xg = host(x)
    rel_oracle = np.linalg.norm(b - ref.apply(xg)) / np.linalg.norm(b)
    assert relg <= 1e-10 and rel_oracle <= 1.01e-10
    assert outer >= 2 and inner > 0
    assert rel(xg, xs) <= 1e-7


def test_residual_replacement_keeps_the_krylov_space(sg):
    """On a 12^3 p = 7 Poisson problem, FP32 PCG with FP64 residual replacement
    (updates every 10x residual drop) needs fewer FP32 iterations than restarted
    refinement (inner 1e-4); both reach 1e-10 in FP64, and neither is below the
    FP64 PCG iteration count."""
    E, p = (12, 12, 12), 7
    op = sg.Op(*E, p, 0.0, "f64")
    cx, cy, cz = op.coords_1d()
    f = Modes(3, 8, 4).field(cx, cy, cz, 0.3)
    b = op.apply(dev(f))
    ms = sg.MixedSolver(*E, p, 0.0)
    it64, _ = op.pcg(b, op.zeros(), 1e-10)
    res = {}
    for method in ("restart", "replace"):
        x = ms.op64.zeros()
        o, inner, relg = ms.solve(b, x, 1e-10, method=method)
        assert relg <= 1e-10
        assert op.residual_norm(b, x) <= 1e-10
        res[method] = inner
    assert res["replace"] < res["restart"]
    assert min(res.values()) >= 0.9 * it64


def test_residual_replacement_edge_cases(sg):
    ref, rng, xs = _problem((3, 3, 3), 4, 2.0, seed=9)
    ms = sg.MixedSolver(3, 3, 3, 4, 2.0)
    b = dev(ref.apply(xs))
    x = dev(xs)                                   # exact guess: no update
    o, inner, relg = ms.solve(b, x, 1e-10, method="replace")
    assert o == 0 and inner == 0 and relg <= 1e-10
    x = ms.op64.zeros()                           # b = 0
    o, inner, relg = ms.solve(ms.op64.zeros(), x, 1e-10, method="replace")
    assert o == 0 and float(x.abs().max()) == 0.0
    x = ms.op64.zeros()                           # update limit -> NOT_CONVERGED, best iterate kept
    o, inner, relg = ms.solve(b, x, 1e-10, inner_tol=0.5, max_outer=1, method="replace")
    assert o == 1 and relg > 1e-10
    bn = b.clone()                                # non-finite residual: breakdown, reported, no hang
    bn[bn.numel() // 2] = float("nan")            # the centre node (interior)
    with pytest.raises(sg.SGError):
        ms.solve(bn, ms.op64.zeros(), 1e-10, method="replace")
    with pytest.raises(ValueError):
        ms.solve(b, x, 1e-10, method="nope")


def test_convert_roundtrip(sg):
    x = dev(random_vectors(5, 1, 1001)[0])
    y = torch.empty(1001, dtype=torch.float32, device="cuda")
    sg.convert(x, y)
    z = torch.empty_like(x)
    sg.convert(y, z)
    assert np.array_equal(host(y), np.float32(host(x)).astype(np.float64))
    assert np.array_equal(host(z), host(y))


# ---------------------------------------------------------------- batched sequences
def test_batched_ir_solves_every_system(sg):
    """Four systems of different sizes and lambda in one persistent launch per
    CG iteration: each meets 1e-10 with the FP64 oracle operator, and agrees
    with the FP64 oracle solution."""
    meshes = [(2, 2, 2, 0.0), (2, 1, 1, 1e3), (1, 2, 2, 1e3), (1, 1, 1, 1e3)]
    bs = sg.BatchSolver(meshes)
    refs, bvs, xvs, xos = [], [], [], []
    for k, (ex, ey, ez, lam) in enumerate(meshes):
        ref, rng, xs = _problem((ex, ey, ez), 7, lam, seed=20 + k)
        b = ref.apply(xs)
        refs.append((ref, b))
        bvs.append(dev(b))
        xvs.append(torch.zeros(ref.n, dtype=torch.float64, device="cuda"))
        xo, _, _, _ = opcg(ref.apply, ref.diagonal(), b, np.zeros(ref.n), 1e-13, interior=ref.interior)
        xos.append(xo)
    outer, inner, relres = bs.solve(bvs, xvs, 1e-10)
    for k, (ref, b) in enumerate(refs):
        xg = host(xvs[k])
        assert relres[k] <= 1e-10 and outer[k] >= 1 and inner[k] > 0
        assert np.linalg.norm(b - ref.apply(xg)) / np.linalg.norm(b) <= 1.01e-10
        assert rel(xg, xos[k]) <= 1e-7
    # a second solve from the converged solutions: no outer step is needed
    outer2, inner2, relres2 = bs.solve(bvs, xvs, 1e-10)
    assert outer2 == [0, 0, 0, 0] and max(relres2) <= 1e-10


def _c4_problems():
    probs = []
    for c in BATCHED:
        ref = SemOperator(*c["E"], c["p"], c["lam"])
        cx, cy, cz = ref.coords_1d()
        xs = Modes(c["seed"], 8, 4).field(cx, cy, cz, 0.25) * ref.interior
        probs.append((c, ref, xs, ref.apply(xs)))
    return probs


def test_batched_full_size_c4_several_items_per_cta(sg):
    """The four batched systems (24^3 Poisson, 20^3 / 16^3 / 12^3 Helmholtz, p = 7;
    19.7M nodes in all) in the persistent kernel, first with the default
    two-layer work items, then with the autotuner's shape.  Every shape the
    tuner can pick gives more work items than the grid has CTAs (at least 1728
    items against at most 4 CTAs x SMs), so CTAs run several items one after
    another (the shared-memory hand-over between items).  Each system's FP64
    residual, measured with the oracle operator, meets 1e-10, and its solution
    agrees with the manufactured one."""
    probs = _c4_problems()
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    for zl in (2, 4):
        items = sum(-(-c["E"][0] // 2) * -(-c["E"][1] // 2) * -(-c["E"][2] // zl) for c, *_ in probs)
        assert items > 4 * nsm
    solver = sg.BatchSolver([(c["E"][0], c["E"][1], c["E"][2], c["lam"]) for c, *_ in probs])
    bvs = [dev(b) for _, _, _, b in probs]
    for tuned in (False, True):
        if tuned:
            zl, bps, ms = solver.tune()
            assert zl in (1, 2, 3, 4) and 1 <= bps <= 4
        xvs = [torch.zeros(ref.n, dtype=torch.float64, device="cuda") for _, ref, _, _ in probs]
        outer, inner, relres = solver.solve(bvs, xvs, 1e-10)
        for k, (c, ref, xs, b) in enumerate(probs):
            xg = host(xvs[k])
            assert relres[k] <= 1e-10 and outer[k] >= 1 and inner[k] > 0
            assert np.linalg.norm(b - ref.apply(xg)) / np.linalg.norm(b) <= 1.01e-10, "system %d" % k
            assert rel(xg, xs) <= 1e-7, "system %d" % k


def test_batched_tuner_then_mixed_convergence(sg):
    meshes = [(3, 2, 2, 0.0), (2, 2, 2, 1e3)]
    bs = sg.BatchSolver(meshes)
    zl, bps, ms = bs.tune()
    assert zl in (1, 2, 3, 4) and bps >= 1 and ms > 0
    refs, bvs, xvs = [], [], []
    for k, (ex, ey, ez, lam) in enumerate(meshes):
        ref, rng, xs = _problem((ex, ey, ez), 7, lam, seed=30 + k)
        b = ref.apply(xs)
        refs.append((ref, b, xs))
        bvs.append(dev(b))
        # system 0 starts at its exact solution: it must stay put while 1 iterates
        xvs.append(dev(xs) if k == 0 else torch.zeros(ref.n, dtype=torch.float64, device="cuda"))
    outer, inner, relres = bs.solve(bvs, xvs, 1e-10)
    assert outer[0] == 0 and inner[0] == 0 and outer[1] >= 1
    for k, (ref, b, xs) in enumerate(refs):
        xg = host(xvs[k])
        assert np.linalg.norm(b - ref.apply(xg)) / np.linalg.norm(b) <= 1.01e-10


# ---------------------------------------------------------------- failure detection (no GPU fault)
def test_bounded_grid_barrier_wait_expires_and_context_survives(sg):
    """The grid barrier of the batched kernel waits a bounded time: when a CTA
    never arrives the wait expires, the kernel returns and SG_ERR_TIMEOUT is
    reported; afterwards the device keeps working."""
    import ctypes
    scratch = torch.zeros(16, dtype=torch.uint8, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert sg.lib().sg_selftest_barrier(0, 1 << 20, ctypes.c_void_p(scratch.data_ptr()), st) == sg.OK
    rc = sg.lib().sg_selftest_barrier(1, 1 << 14, ctypes.c_void_p(scratch.data_ptr()), st)
    assert rc == sg.ERR_TIMEOUT and b"expired" in sg.lib().sg_last_error()
    # the context is intact: a regular solve still works
    ref, rng, xs = _problem((2, 2, 2), 3, 1.0, seed=40)
    op = sg.Op(2, 2, 2, 3, 1.0, "f64")
    x = op.zeros()
    it, r = op.pcg(dev(ref.apply(xs)), x, 1e-10)
    assert r <= 1e-10 and it > 0


def test_nonfinite_input_reports_breakdown(sg):
    """A NaN in the right-hand side ends PCG with SG_ERR_BREAKDOWN (host-side fault injection)."""
    ref, rng, xs = _problem((2, 2, 2), 3, 1.0, seed=41)
    op = sg.Op(2, 2, 2, 3, 1.0, "f64")
    b = ref.apply(xs)
    b[np.flatnonzero(ref.interior)[5]] = np.nan
    with pytest.raises(sg.SGError) as ei:
        op.pcg(dev(b), op.zeros(), 1e-10)
    assert ei.value.code == sg.ERR_BREAKDOWN


@pytest.mark.parametrize("method", ["extrap", "qr"])
def test_largest_history(sg, method):
    """s = SG_MAX_HISTORY = 16 (the largest history) against the oracle."""
    s = 16
    if method == "extrap":
        n = 5001
        g = sg.Guess(n, s, "extrap", m=3)
        hist = random_vectors(13, s + 2, n)
        for k in range(s + 2):
            g.update(dev(hist[k]))
        x0 = torch.zeros(n, dtype=torch.float64, device="cuda")
        g.form(None, x0)
        want = oex.extrap_guess(list(hist[2:]), oex.lsq_coeffs(s, 3))
        assert rel(host(x0), want) <= 1e-12
    else:
        ref = SemOperator(3, 3, 3, 3, 5.0)
        op = sg.Op(3, 3, 3, 3, 5.0, "f64")
        g = sg.Guess(ref.n, s, "qr", eps_rel=1e-12, op=op)
        o = ProjectionQR(s, 1e-12, ref.apply)
        rng = np.random.default_rng(17)
        for k in range(s + 3):
            x = rng.standard_normal(ref.n) * ref.interior
            g.update(dev(x))
            o.update(x)
        assert g.info()[0] == o.d == s
        b = ref.apply(rng.standard_normal(ref.n) * ref.interior)
        x0 = op.zeros()
        g.form(dev(b), x0)
        assert rel(host(x0), o.form(b, np.zeros(ref.n))) <= 1e-12


# ---------------------------------------------------------------- device-driven PCG iterations
def _pcg_problem(seed=50):
    ref, rng, xs = _problem((4, 3, 3), 5, 20.0, seed=seed)
    b = ref.apply(xs) + 0.01 * rng.standard_normal(ref.n) * ref.interior
    x0 = 0.1 * rng.standard_normal(ref.n) * ref.interior
    return ref, b, x0


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_pcg_graph_launch_and_async_paths_agree(sg, dtype):
    """The iteration graph (default), the host-launched chunks (taken while kernel
    timing is on) and the asynchronous entry run the same kernels in the same
    order: identical iterates and iteration counts; the FP64 one against the oracle."""
    ref, b, x0 = _pcg_problem()
    tdt = torch.float64 if dtype == "f64" else torch.float32
    tol = 1e-10 if dtype == "f64" else 1e-5
    op = sg.Op(4, 3, 3, 5, 20.0, dtype)
    bd = dev(b, tdt)
    xg = dev(x0, tdt)
    itg, _ = op.pcg(bd, xg, tol, true_residual=False)
    sg.profile_enable(True)
    try:
        xl = dev(x0, tdt)
        itl, _ = op.pcg(bd, xl, tol, true_residual=False)
    finally:
        sg.profile_enable(False)
    xa = dev(x0, tdt)
    op.pcg_async(bd, xa, tol)
    ita = op.pcg_result()
    assert itg == itl == ita and itg > 3
    assert torch.equal(xg, xl) and torch.equal(xg, xa)
    if dtype == "f64":
        xo, ito, _, _ = opcg(ref.apply, ref.diagonal(), b, x0, tol, interior=ref.interior)
        assert abs(itg - ito) <= 1
        assert rel(host(xg), xo) <= 1e-10


def test_pcg_async_edge_cases(sg):
    ref, rng, xs = _problem((2, 3, 2), 3, 1.0, seed=51)
    op = sg.Op(2, 3, 2, 3, 1.0, "f64")
    b = dev(ref.apply(xs))
    x = dev(xs)                                   # exact guess: 0 iterations
    op.pcg_async(b, x, 1e-10)
    assert op.pcg_result() == 0
    x = op.zeros()                                # b = 0
    op.pcg_async(op.zeros(), x, 1e-10)
    assert op.pcg_result() == 0 and float(x.abs().max()) == 0.0
    x = op.zeros()                                # maxit
    op.pcg_async(b, x, 1e-14, maxit=3)
    assert op.pcg_result() == 3
    with pytest.raises(sg.SGError):
        op.pcg_async(b, op.zeros(), 1e-14, maxit=3)
        op.pcg_result(raise_on_maxit=True)
    bn = ref.apply(xs)                            # NaN right-hand side
    bn[np.flatnonzero(ref.interior)[3]] = np.nan
    op.pcg_async(dev(bn), op.zeros(), 1e-10)
    with pytest.raises(sg.SGError) as ei:
        op.pcg_result()
    assert ei.value.code == sg.ERR_BREAKDOWN
    x = op.zeros()                                # a normal solve afterwards
    op.pcg_async(b, x, 1e-10)
    assert op.pcg_result() > 0
    assert op.residual_norm(b, x) <= 1e-10


def test_pcg_graph_cache_over_many_workspaces(sg):
    """More workspaces than the per-operator graph cache holds (8): every solve
    is right, and re-used workspaces hit the cache."""
    import ctypes
    ref, b, x0 = _pcg_problem(seed=52)
    op = sg.Op(4, 3, 3, 5, 20.0, "f64")
    nb = int(sg.lib().sg_pcg_workspace_bytes(op.h))
    wss = [torch.empty(nb, dtype=torch.uint8, device="cuda") for _ in range(11)]
    bd = dev(b)
    ref_x, ref_it = None, None
    for rnd in range(2):
        for ws in wss:
            x = dev(x0)
            it = ctypes.c_int(0)
            rc = sg.lib().sg_pcg_solve(op.h, ctypes.c_void_p(bd.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                       1e-10, 10000, 0, ctypes.c_void_p(ws.data_ptr()), ctypes.byref(it), None,
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
            assert rc == 0
            if ref_x is None:
                ref_x, ref_it = x.clone(), it.value
            assert it.value == ref_it and torch.equal(x, ref_x)
