"""Pins of the FP64 oracle against what the paper and mathematics fix.

None of these checks re-types the oracle's own formulas: they compare it with
library FFTs at integer nodes, closed-form sums, the paper's printed grid
formula, closed-form solutions of the wave equation (physics), brute-force
operator matrices and the adjoint identity.  Each pin is chosen so that a
plausible slip in the oracle (a dropped factor, a flipped sign, a transposed
index, the printed "2k" weight) fails at least one of them.
"""
import json
import os

import numpy as np
import pytest

import oracle
import phantoms as ph

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


# ---------------------------------------------------------------------------
# Eq. (dft): direct nonuniform DFT
# ---------------------------------------------------------------------------

def test_nudft_integer_nodes_equal_library_fft():
    """At integer nodes Eq. (dft) is the classical DFT (the paper's remark on
    evenly spaced nodes); nodes beyond +-N/2 alias with period N."""
    rng = np.random.default_rng(1)
    N = 64
    g = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    nu = np.array([0, 1, -1, 5, -32, 31, 64 + 3, -64 - 7, 2 * 64 + 10], dtype=float)
    ref = np.fft.fft(g)[np.mod(nu.astype(int), N)]
    assert np.max(np.abs(oracle.nudft(g, nu) - ref)) < 1e-11 * np.abs(ref).max()


def test_nudft_impulse_closed_form():
    rng = np.random.default_rng(2)
    N, n0 = 50, 17
    g = np.zeros(N, complex)
    g[n0] = 1.0
    nu = rng.uniform(-80, 80, 40)
    ref = np.exp(-2j * np.pi * nu * n0 / N)
    assert np.max(np.abs(oracle.nudft(g, nu) - ref)) < 1e-13


def test_nudft_geometric_closed_form():
    """g_n = r^n sums to a geometric series: (1 - q^N) / (1 - q), q = r e^{-2 pi i nu/N}."""
    N = 96
    r = 0.97 * np.exp(0.3j)
    g = r ** np.arange(N)
    nu = np.array([0.25, -3.7, 10.5, 47.9, -120.3])
    q = r * np.exp(-2j * np.pi * nu / N)
    ref = (1 - q ** N) / (1 - q)
    assert np.max(np.abs(oracle.nudft(g, nu) - ref) / np.abs(ref)) < 1e-12


def test_nudft_adjoint_identity():
    rng = np.random.default_rng(3)
    N = 40
    g = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    h = rng.standard_normal(30) + 1j * rng.standard_normal(30)
    nu = rng.uniform(-60, 60, 30)
    lhs = np.vdot(h, oracle.nudft(g, nu))
    rhs = np.vdot(oracle.nudft_adjoint(h, nu, N), g)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


# ---------------------------------------------------------------------------
# Eq. (fft-1a) and Eq. (fft-1): uniform DFTs against the library FFT
# ---------------------------------------------------------------------------

def test_lateral_dft_2d_equals_library_fft():
    g = ph.Geometry(dim=2, nx=24, nt=20, nz=16)
    p = ph.random_data(4, g)
    assert _rel(oracle.lateral_dft(g, p), np.fft.fft(p, axis=0)) < 1e-13


def test_lateral_dft_3d_equals_library_fft():
    g = ph.Geometry(dim=3, nx=12, ny=10, nt=16, nz=8)
    p = ph.random_data(5, g)
    assert _rel(oracle.lateral_dft(g, p), np.fft.fft2(p, axes=(0, 1))) < 1e-13


@pytest.mark.parametrize("dim", [2, 3])
def test_inverse_dft_equals_library_ifft(dim):
    g = ph.Geometry(dim=dim, nx=10, ny=6 if dim == 3 else 1, nt=8, nz=12)
    rng = np.random.default_rng(6)
    F = rng.standard_normal(g.image_shape) + 1j * rng.standard_normal(g.image_shape)
    ref = np.fft.ifftn(F).real
    assert _rel(oracle.image_from_spectrum(g, F), ref) < 1e-13


# ---------------------------------------------------------------------------
# Nodes and weight: the paper's printed unit-grid case (Eq. dft-2d)
# ---------------------------------------------------------------------------

def test_nodes_on_paper_grid_match_printed_formula():
    cases = json.load(open(os.path.join(GOLDEN, "kb_constants.json")))["paper_grid_node"]["cases"]
    N = 32
    # unit grid of the paper: X = 1, spacing 1/N everywhere, unit sound speed
    g = ph.Geometry(dim=2, nx=N, nt=N, nz=N, dx=1.0 / N, dt=1.0 / N, dz=1.0 / N)
    for k, l, expect in cases:
        assert abs(oracle.node(g, k, 0, l) - expect) < 1e-12


def test_nodes_scale_with_sound_speed_and_steps():
    """nu and the weight depend on c and dt only through c*dt (the travel-time
    substitution tau = c t of Eq. inv)."""
    a = ph.Geometry(dim=3, nx=16, ny=8, nt=32, nz=16, dx=1.0, dy=2.0, dt=1.0, c=1.0, dz=1.0)
    b = ph.Geometry(dim=3, nx=16, ny=8, nt=32, nz=16, dx=1.0, dy=2.0, dt=0.25, c=4.0, dz=1.0)
    for (kx, ky, l) in [(3, 2, 5), (-8, 1, -3), (0, 0, 7), (5, -4, -8)]:
        assert abs(oracle.node(a, kx, ky, l) - oracle.node(b, kx, ky, l)) < 1e-12
        assert abs(oracle.weight(a, kx, ky, l) - oracle.weight(b, kx, ky, l)) < 1e-12


def test_weight_zero_on_l0_row_and_even_in_frequency():
    g = ph.Geometry(dim=2, nx=16, nt=32, nz=16)
    for k in range(-8, 8):
        assert oracle.weight(g, k, 0, 0) == 0.0
        for l in range(1, 8):
            assert oracle.weight(g, k, 0, l) == pytest.approx(oracle.weight(g, -k, 0, -l), rel=1e-15)
            assert oracle.node(g, k, 0, l) == pytest.approx(-oracle.node(g, -k, 0, -l), rel=1e-15)


def test_integer_node_column_equals_weighted_fft():
    """P4: with nt = 2 nz and unit steps the k = 0 nodes are nu = 2l (integers),
    so that column of the spectrum is weight x library FFT of the lateral sum."""
    g = ph.Geometry(dim=2, nx=16, nt=64, nz=32)
    p = ph.random_data(7, g)
    F = oracle.spectrum(g, p)
    row0 = np.fft.fft(p.sum(axis=0))
    for li in range(g.nz):
        l = li if li < g.nz // 2 else li - g.nz
        ref = oracle.weight(g, 0, 0, l) * row0[(2 * l) % g.nt]
        assert abs(F[0, li] - ref) < 1e-11 * np.abs(row0).max()


def test_spectrum_is_hermitian_except_nyquist_row():
    """P7: real data give fhat(-k,-l) = conj fhat(k,l); only the l = -nz/2 row
    (whose partner is not on the grid) breaks it, so the inverse DFT is real
    up to that row."""
    g = ph.Geometry(dim=2, nx=16, nt=48, nz=20)
    p = ph.random_data(8, g)
    F = oracle.spectrum(g, p)
    idx_k = (-np.arange(g.nx)) % g.nx
    idx_l = (-np.arange(g.nz)) % g.nz
    Fm = np.conj(F[idx_k][:, idx_l])
    mask = np.ones(g.nz, bool)
    mask[g.nz // 2] = False
    assert np.max(np.abs(F[:, mask] - Fm[:, mask])) < 1e-11 * np.abs(F).max()
    F0 = F.copy()
    F0[:, g.nz // 2] = 0
    z = np.fft.ifft2(F0)
    assert np.abs(z.imag).max() < 1e-12 * np.abs(z.real).max()


def test_spectrum_rows_match_full_spectrum():
    g = ph.Geometry(dim=3, nx=8, ny=6, nt=16, nz=10, dx=1.0, dy=1.5, dz=0.8)
    p = ph.random_data(9, g)
    F = oracle.spectrum(g, p)
    kx = np.array([0, 3, -4, -1])
    ky = np.array([0, -3, 2, 1])
    rows = oracle.spectrum_rows(g, p, kx, ky)
    for r in range(len(kx)):
        assert _rel(rows[r], F[kx[r] % g.nx, ky[r] % g.ny]) < 1e-12


# ---------------------------------------------------------------------------
# Linearity and the adjoint
# ---------------------------------------------------------------------------

def test_reconstruction_is_linear():
    g = ph.Geometry(dim=2, nx=16, nt=32, nz=16)
    a, b = ph.random_data(10, g), ph.random_data(11, g)
    lhs = oracle.reconstruct(g, 2.0 * a - 0.5 * b)
    rhs = 2.0 * oracle.reconstruct(g, a) - 0.5 * oracle.reconstruct(g, b)
    assert _rel(lhs, rhs) < 1e-13


@pytest.mark.parametrize("dim", [2, 3])
def test_adjoint_dot_product(dim):
    g = ph.Geometry(dim=dim, nx=12, ny=8 if dim == 3 else 1, nt=24, nz=10, dz=0.7, dt=0.9, c=1.3)
    p = ph.random_data(12, g)
    h = ph.random_image(13, g)
    lhs = np.vdot(oracle.reconstruct(g, p), h)
    rhs = np.vdot(p, oracle.adjoint(g, h))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_adjoint_is_the_dense_transpose():
    """Brute force on a tiny grid: assemble the operator matrix column by
    column from unit data, assemble the adjoint matrix from unit images, and
    require exact transposition."""
    g = ph.Geometry(dim=2, nx=6, nt=10, nz=6)
    nd, ni = g.nx * g.nt, g.nx * g.nz
    A = np.empty((ni, nd))
    for j in range(nd):
        e = np.zeros(nd)
        e[j] = 1
        A[:, j] = oracle.reconstruct(g, e.reshape(g.data_shape)).ravel()
    B = np.empty((nd, ni))
    for j in range(ni):
        e = np.zeros(ni)
        e[j] = 1
        B[:, j] = oracle.adjoint(g, e.reshape(g.image_shape)).ravel()
    assert np.max(np.abs(A.T - B)) < 1e-13 * np.abs(A).max()


# ---------------------------------------------------------------------------
# Physics: closed-form solutions of the wave equation (Sec. 2, Eq. inv)
# ---------------------------------------------------------------------------

def _fit(f, truth):
    """Best-fit scale and correlation of f against truth with its per-column
    depth mean removed (the l = 0 row of the spectrum is zero by the weight)."""
    tr = truth - truth.mean(axis=-1, keepdims=True)
    s = float((f * tr).sum() / (tr * tr).sum())
    corr = float((f * tr).sum() / np.linalg.norm(f) / np.linalg.norm(tr))
    return s, corr


def test_physics_2d_fcirc_wide_aperture():
    """Exact data of the paper's circular object (Sec. 5.1) on a wide line
    aperture must reconstruct to the object itself: unit scale, right place."""
    g = ph.Geometry(dim=2, nx=512, nt=1024, nz=128)
    discs = [(256.0, 40.0, 10.0, 1.0)]
    f = oracle.reconstruct(g, ph.fcirc_2d(g, discs))
    s, corr = _fit(f, ph.fcirc_2d_image(g, discs))
    assert 0.95 < s < 1.05 and corr > 0.95
    ix, iz = np.unravel_index(np.argmax(f), f.shape)
    assert abs(ix - 256) <= 1 and abs(iz - 40) <= 1


def test_physics_2d_general_grid():
    """Same object on a grid with c != 1, dt != dx and dz != dx: pins the node
    scaling c dt nt / 2pi and the weight factor c dt / dz.  The depth step is
    kept >= c dt so that the image band stays inside the data band (Appendix:
    sampling condition)."""
    g = ph.Geometry(dim=2, nx=400, nt=1200, nz=100, dx=1.0, dt=0.5, c=1.5, dz=0.8)
    discs = [(200.0, 30.0, 8.0, 1.0)]
    f = oracle.reconstruct(g, ph.fcirc_2d(g, discs))
    s, corr = _fit(f, ph.fcirc_2d_image(g, discs))
    assert 0.93 < s < 1.07 and corr > 0.93
    ix, iz = np.unravel_index(np.argmax(f), f.shape)
    assert abs(ix * g.dx - 200.0) <= 1.0 and abs(iz * g.dz - 30.0) <= 1.0


def test_physics_3d_smooth_ball():
    """Smooth ball in 3-D (closed-form radial solution) reconstructs to itself
    on a planar aperture with dy != dx (pins the second lateral axis)."""
    g = ph.Geometry(dim=3, nx=128, ny=100, dy=1.25, nt=256, nz=32)
    balls = [(64.0, 62.5, 12.0, 6.0, 1.0)]
    f = oracle.reconstruct(g, ph.balls_3d(g, balls, smooth=True))
    s, corr = _fit(f, ph.balls_3d_image(g, balls, smooth=True))
    assert 0.95 < s < 1.05 and corr > 0.93
    assert np.unravel_index(np.argmax(f), f.shape) == (64, 50, 12)


def test_physics_sensitivity_of_the_pins():
    """The printed "2k" weight (lateral index in the numerator) and a flipped
    inverse transform both fail the 2-D physics pin, so the pin can tell them
    apart from the reading the oracle takes."""
    g = ph.Geometry(dim=2, nx=512, nt=1024, nz=128)
    discs = [(256.0, 40.0, 10.0, 1.0)]
    p = ph.fcirc_2d(g, discs)
    truth = ph.fcirc_2d_image(g, discs)
    F = oracle.spectrum(g, p)
    kx = np.fft.fftfreq(g.nx, 1.0 / g.nx)[:, None]
    lz = np.fft.fftfreq(g.nz, 1.0 / g.nz)[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        ratio = np.where(lz != 0, np.abs(kx * g.nz / g.nx) / np.abs(lz), 0.0)   # 2|Kx| instead of 2|Kz|
    s_bad, _ = _fit(oracle.image_from_spectrum(g, F * ratio), truth)
    assert not (0.95 < s_bad < 1.05)
    flipped = np.fft.fftn(F).real / F.size              # e^{-i} instead of e^{+i}
    s_flip, c_flip = _fit(flipped, truth)
    assert c_flip < 0.5


# ---------------------------------------------------------------------------
# The paper's window constants and Algorithm 1 against the oracle (P5)
# ---------------------------------------------------------------------------

def _kb_hat(u, K, a):
    from scipy.special import i0
    s2 = K * K - u * u
    s = np.sqrt(np.abs(s2))
    out = np.full_like(u, 2 * a / i0(a * K))
    pos, neg = s2 > 1e-300, s2 < -1e-300
    out[pos] = 2 * np.sinh(a * s[pos]) / (i0(a * K) * s[pos])
    out[neg] = 2 * np.sin(a * s[neg]) / (i0(a * K) * s[neg])
    return out


def test_paper_window_constants():
    from scipy.special import i0
    gold = json.load(open(os.path.join(GOLDEN, "kb_constants.json")))
    kr = gold["kb_ratio"]
    K, a = kr["K"], kr["alpha_over_pi"] * np.pi
    ratio = _kb_hat(np.array([float(K)]), K, a)[0] / _kb_hat(np.array([0.0]), K, a)[0]
    assert abs(ratio / kr["value"] - 1) < 0.02 + kr["rel_tol"]
    fb = gold["fourmont_bound"]
    c, K, a = fb["c"], fb["K"], fb["alpha_over_pi"] * np.pi
    bound = 30 / (np.pi * i0(K * np.pi * np.sqrt(a * a - 1) / c ** 2))
    assert abs(bound / fb["value"] - 1) < 0.05 + fb["rel_tol"]


def _nufft_fp64(g, nu, c, K, alpha):
    """Algorithm 1 in FP64 with the readings the design takes: constant
    1/(2 pi c) (Lemma), phase e^{-i pi (omega - j/c)} (Proposition), taps
    wrapped mod cN.  The e^{-i pi(...)} phase is realised by placing sample n
    at position n - N/2 (mod cN) before the FFT."""
    from scipy.special import i0
    N = len(g)
    M = int(round(c * N))
    n = np.arange(N)
    th = 2 * np.pi * n / N - np.pi
    psi = i0(K * np.sqrt(np.maximum(alpha ** 2 - th ** 2, 0))) / i0(alpha * K)
    X = np.zeros(M, complex)
    X[(n - N // 2) % M] = g / (2 * np.pi * c * psi)
    G = np.fft.fft(X)
    x = c * nu
    j0 = np.floor(x).astype(int)
    H = int(np.ceil(c * K))
    out = np.zeros(len(nu), complex)
    for t in range(-H + 1, H + 1):
        j = j0 + t
        out += _kb_hat((x - j) / c, K, alpha) * G[j % M]
    return out * np.exp(-1j * np.pi * nu)


@pytest.mark.parametrize("alpha_over_pi,limit", [(3.0, 3e-8), (3.0 * (1 - 1e-3), 1e-10)])
def test_algorithm1_within_paper_bound_of_oracle(alpha_over_pi, limit):
    """The NUFFT of Algorithm 1 (c = 2, K = 3) agrees with the oracle's direct
    sums within the paper's error bound (3e-8 at alpha = 3 pi), including
    nodes far beyond +-N/2 (wrapped taps)."""
    rng = np.random.default_rng(14)
    N = 128
    g = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    nu = rng.uniform(-1.6 * N / 2, 1.6 * N / 2, 300)
    exact = oracle.nudft(g, nu)
    approx = _nufft_fp64(g, nu, 2.0, 3.0, alpha_over_pi * np.pi)
    assert _rel(approx, exact) < limit


@pytest.mark.parametrize("g,box", [
    (ph.Geometry(dim=3, nx=12, ny=10, nt=20, nz=8, dx=0.9, dy=1.1, dt=0.7, c=1.3, dz=1.2), ((3, 9), (0, 10), (5, 17))),
    (ph.Geometry(dim=2, nx=14, nt=24, nz=10, dt=0.8, dz=1.1), ((0, 14), None, (0, 24))),
    (ph.Geometry(dim=2, nx=14, nt=24, nz=10), ((5, 6), None, (23, 24))),
])
def test_adjoint_box_is_the_adjoint_restricted(g, box):
    """The box-restricted adjoint (for grids too large for the full one) is
    the full oracle adjoint on that box, sample for sample."""
    h = np.random.default_rng(9).standard_normal(g.image_shape)
    full = oracle.adjoint(g, h)
    bx, by, bn = box
    got = oracle.adjoint_box(g, h, bx, by, bn)
    if g.dim == 2:
        ref = full[bx[0]:bx[1], bn[0]:bn[1]]
    else:
        ref = full[bx[0]:bx[1], by[0]:by[1], bn[0]:bn[1]]
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(full))
