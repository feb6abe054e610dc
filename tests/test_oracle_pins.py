"""Pins of the FP64 oracle against facts fixed by the mathematics of the
step (closed forms, library solves, invariants, brute force), never against
the oracle itself."""
import math

import numpy as np
import pytest

import oracle
from oracle import OracleGrid


def rand_field(nz, ny, nx, seed=0, lo=0.0, hi=1.0):
    return np.random.default_rng(seed).uniform(lo, hi, size=(nz, ny, nx))


def no_kc(g):
    return np.zeros((g.ny, g.nx), np.int32)


# ---------------------------------------------------------------- advection

@pytest.mark.parametrize("cx,cy,axis,shift", [(1.0, 0.0, 2, 1), (0.0, 1.0, 1, 1),
                                              (-1.0, 0.0, 2, -1), (0.0, -1.0, 1, -1)])
def test_exact_shift_at_cfl_one(cx, cy, axis, shift):
    """Courant number 1 on one axis: one step is exactly a periodic roll."""
    g = OracleGrid(12, 10, 5, cx, cy, 0.0, 0.1, True, (0, 0, 0, 0, 3), 0, 0)
    q = rand_field(5, 10, 12, 1)
    out, _ = oracle.run(g, q, 1)
    assert np.array_equal(out, np.roll(q, shift, axis=axis))


def test_exact_shift_with_zero_diffusion():
    """r = 0 makes every sweep the identity even with k_c > 0."""
    g = OracleGrid(9, 7, 6, 1.0, 0.0, 0.0, 0.0, True, (3, 3, 0, 0, 2), 5, 3)
    q = rand_field(6, 7, 9, 2)
    out, _ = oracle.run(g, q, 3)
    assert np.array_equal(out, np.roll(q, 3, axis=2))


def test_fourier_mode_amplification():
    """q = Re exp(i(a i + b j)) is multiplied each step by
    G = 1 - cx (1 - e^{-ia}) - cy (1 - e^{-ib}) (von Neumann factor of the
    donor-cell scheme); a column-constant field is untouched by the sweeps."""
    nx, ny, nz, n = 32, 24, 4, 7
    m1, m2 = 3, 5
    a, b = 2 * np.pi * m1 / nx, 2 * np.pi * m2 / ny
    cx, cy = 0.3, 0.45
    ii, jj = np.meshgrid(np.arange(nx), np.arange(ny))
    z = np.exp(1j * (a * ii + b * jj))
    q = np.broadcast_to(z.real, (nz, ny, nx)).copy()
    g = OracleGrid(nx, ny, nz, cx, cy, 0.0, 0.2, True, (0, 0, 0, 0, 100), 3, 3)
    out, _ = oracle.run(g, q, n)
    G = 1 - cx * (1 - np.exp(-1j * a)) - cy * (1 - np.exp(-1j * b))
    exp = (G ** n * z).real
    assert np.max(np.abs(out - exp[None])) < 1e-13


# ---------------------------------------------------------------- diffusion

@pytest.mark.parametrize("nz", [1, 2, 3, 8, 33])
def test_dct_eigenmode(nz):
    """cos(pi m (k+1/2)/nz) is an eigenvector of the zero-flux operator; one
    implicit solve divides it by 1 + 4 r sin^2(pi m / (2 nz))."""
    r = 0.37
    k = np.arange(nz)
    for m in range(nz):
        v = np.cos(np.pi * m * (k + 0.5) / nz)
        lam = 1.0 / (1.0 + 4 * r * np.sin(np.pi * m / (2 * nz)) ** 2)
        assert np.max(np.abs(oracle.thomas(v, r) - lam * v)) < 1e-14


def dense_operator(nz, r):
    """M = I - r L, L the second difference with zero-flux ends, built from
    face fluxes: each interior face couples its two cells."""
    M = np.eye(nz)
    for f in range(nz - 1):
        M[f, f] += r
        M[f + 1, f + 1] += r
        M[f, f + 1] -= r
        M[f + 1, f] -= r
    return M


@pytest.mark.parametrize("nz", range(1, 9))
def test_thomas_against_dense_solve(nz):
    rng = np.random.default_rng(nz)
    for _ in range(5):
        r = rng.uniform(0, 3)
        d = rng.normal(size=nz)
        M = dense_operator(nz, r)
        x = d.copy()
        for kc in range(1, 4):
            x = oracle.thomas(x, r)
            ref = np.linalg.solve(np.linalg.matrix_power(M, kc), d)
            # both solves are backward stable; cond(M) <= 1 + 4r
            tol = 64 * np.finfo(float).eps * (1 + 4 * r) ** kc * np.abs(d).max()
            assert np.max(np.abs(x - ref)) < tol


def test_inverse_is_nonnegative_with_unit_row_sums():
    nz, r = 11, 0.8
    Minv = np.stack([oracle.thomas(e, r) for e in np.eye(nz)], axis=1)
    assert Minv.min() >= 0.0
    assert np.max(np.abs(Minv.sum(axis=1) - 1.0)) < 1e-14
    assert np.max(np.abs(Minv.sum(axis=0) - 1.0)) < 1e-14


def test_sweeps_use_the_columns_own_kc():
    """k_c is per column: a column with k_c = 3 equals three solves, a column
    with k_c = 0 is the advected column unchanged."""
    g = OracleGrid(4, 3, 7, 0.0, 0.0, 0.0, 0.25)
    q = rand_field(7, 3, 4, 5)
    kc = np.zeros((3, 4), np.int32)
    kc[1, 2] = 3
    out = oracle.step(g, q, kc)
    x = q[:, 1, 2]
    for _ in range(3):
        x = np.linalg.solve(dense_operator(7, 0.25), x)
    assert np.max(np.abs(out[:, 1, 2] - x)) < 1e-14
    mask = np.ones((3, 4), bool)
    mask[1, 2] = False
    assert np.array_equal(out[:, mask], q[:, mask])


def solves(col, r, n):
    """n implicit solves of one column by dense linear algebra."""
    return np.linalg.solve(np.linalg.matrix_power(dense_operator(col.size, r), n), col)


def test_array_kc_gives_each_column_its_own_number_of_solves():
    """k_c from an array (the lognormal workloads' source): with no advection,
    column (i, j) after one step is M^-k_c(i,j) applied to it, for every k_c
    from 0 to 4 on a non-square grid (a transposed lookup lands elsewhere)."""
    nx, ny, nz, r = 5, 4, 6, 0.3
    kc = np.fromfunction(lambda j, i: (i + 2 * j) % 5, (ny, nx), dtype=int).astype(np.int32)
    g = OracleGrid(nx, ny, nz, 0.0, 0.0, 0.0, r, kc_disk=False, kc=kc)
    assert np.array_equal(oracle.kc_field(g, 0), kc)
    q = rand_field(nz, ny, nx, 21)
    out, _ = oracle.run(g, q, 1)
    for j in range(ny):
        for i in range(nx):
            exp = solves(q[:, j, i], r, int(kc[j, i]))
            assert np.max(np.abs(out[:, j, i] - exp)) < 1e-14
    assert np.array_equal(out[:, kc == 0], q[:, kc == 0])


def test_run_from_t0_takes_the_load_rule_at_t0():
    """A run that starts at global step t0 uses k_c(t0): the disk rolled by
    t0 (vy, vx) cells (the motion pinned above), not k_c(0)."""
    nx, ny, nz, r, t0 = 12, 10, 5, 0.2, 4
    g = OracleGrid(nx, ny, nz, 0.0, 0.0, 0.0, r, True, (2, 3, 1, 2, 3), 3, 0)
    kc_t0 = np.roll(oracle.kc_field(g, 0), (2 * t0, t0), axis=(0, 1))
    assert not np.array_equal(kc_t0, oracle.kc_field(g, 0))
    q = rand_field(nz, ny, nx, 22)
    out, _ = oracle.run(g, q, 1, t0=t0)
    for j in range(ny):
        for i in range(nx):
            exp = solves(q[:, j, i], r, int(kc_t0[j, i]))
            assert np.max(np.abs(out[:, j, i] - exp)) < 1e-14


def test_per_step_kc_arrays_are_taken_step_by_step():
    """Per-step k_c arrays (k_c re-draws): with no advection a column ends as
    M^-(k_1 + k_2 + k_3) of itself, in whole-grid runs and in window runs."""
    nx, ny, nz, r, n = 6, 5, 4, 0.25, 3
    rng = np.random.default_rng(23)
    kcs = rng.integers(0, 4, size=(n, ny, nx)).astype(np.int32)
    total = kcs.sum(axis=0)
    assert not np.array_equal(total, n * kcs[0])
    g = OracleGrid(nx, ny, nz, 0.0, 0.0, 0.0, r, kc_disk=False, kc=kcs[0])
    q = rand_field(nz, ny, nx, 24)
    full, _ = oracle.run(g, q, n, kc_fields=kcs)
    i0, j0, wx, wy = 4, 3, 4, 3                      # wraps around both edges
    ii, jj = np.arange(i0, i0 + wx) % nx, np.arange(j0, j0 + wy) % ny
    win = oracle.run_window(g, q, i0, j0, wx, wy, n, kc_window=kcs[:, jj][:, :, ii])
    for j in range(ny):
        for i in range(nx):
            exp = solves(q[:, j, i], r, int(total[j, i]))
            assert np.max(np.abs(full[:, j, i] - exp)) < 1e-14
    for b, j in enumerate(jj):
        for a, i in enumerate(ii):
            exp = solves(q[:, j, i], r, int(total[j, i]))
            assert np.max(np.abs(win[:, b, a] - exp)) < 1e-14


# ---------------------------------------------------------------- full step

def test_mass_conserved():
    g = OracleGrid(20, 14, 9, 0.35, 0.4, 0.0, 0.3, True, (5, 5, 1, 2, 4), 7, 1)
    q = rand_field(9, 14, 20, 7)
    m0 = math.fsum(q.ravel())
    out, mass = oracle.run(g, q, 12)
    assert abs(math.fsum(out.ravel()) - m0) < 1e-13 * m0
    assert np.max(np.abs(mass - m0)) < 1e-13 * m0


def test_mass_conserved_with_vertical_advection():
    g = OracleGrid(8, 6, 10, 0.2, -0.3, 0.4, 0.5, True, (2, 2, 0, 0, 2), 2, 1)
    q = rand_field(10, 6, 8, 8)
    m0 = math.fsum(q.ravel())
    out, _ = oracle.run(g, q, 9)
    assert abs(math.fsum(out.ravel()) - m0) < 1e-13 * m0


def test_vertical_shift_with_closed_ends():
    """cz = 1: every level moves up one cell; the bottom cell receives
    nothing and the top cell keeps what it cannot send through the closed
    top face."""
    g = OracleGrid(3, 2, 6, 0.0, 0.0, 1.0, 0.0)
    q = rand_field(6, 2, 3, 9)
    out = oracle.step(g, q, np.zeros((2, 3), np.int32))
    exp = np.zeros_like(q)
    exp[1:] = q[:-1]
    exp[-1] += q[-1]
    assert np.max(np.abs(out - exp)) < 1e-15


def test_separable_product_mode():
    """Uniform k_c: Fourier(x, y) x cosine(z) evolves by G^n (1+4 r s^2)^(-k_c n)."""
    nx, ny, nz, n, kc, r = 16, 8, 12, 5, 3, 0.15
    a = 2 * np.pi * 2 / nx
    m = 2
    ii = np.arange(nx)
    k = np.arange(nz)
    z = np.exp(1j * a * ii)
    col = np.cos(np.pi * m * (k + 0.5) / nz)
    q = (col[:, None, None] * np.broadcast_to(z.real, (ny, nx))[None]).copy()
    g = OracleGrid(nx, ny, nz, 0.6, 0.0, 0.0, r, True, (0, 0, 0, 0, 100), kc, kc)
    out, _ = oracle.run(g, q, n)
    G = 1 - 0.6 * (1 - np.exp(-1j * a))
    lam = 1.0 / (1.0 + 4 * r * np.sin(np.pi * m / (2 * nz)) ** 2)
    exp = col[:, None, None] * (G ** n * z).real[None, None, :] * lam ** (kc * n)
    assert np.max(np.abs(out - exp)) < 1e-13


def test_monotone_bounds():
    """cx, cy >= 0, cx + cy <= 1 and a nonnegative M^{-1} with unit row sums:
    the field's min never falls and its max never rises."""
    g = OracleGrid(15, 13, 7, 0.45, 0.3, 0.0, 0.9, True, (4, 4, 1, 1, 5), 6, 2)
    q = rand_field(7, 13, 15, 11, -1.0, 2.0)
    lo, hi = q.min(), q.max()
    for t in range(6):
        q, _ = oracle.run(g, q, 1, t0=t)
        assert q.min() >= lo - 1e-15 and q.max() <= hi + 1e-15
        lo, hi = q.min(), q.max()


# ---------------------------------------------------------------- load rule

def test_disk_counts_lattice_points():
    """A static disk of radius 12 covers 441 cells (lattice points in a
    circle of radius 12, counted here by brute force); the 64x64 plain-FP64
    workload therefore has mean k_c (441*8 + 3655*1)/4096."""
    g = OracleGrid(64, 64, 4, kc_disk=True, disk=(24, 40, 0, 0, 12), k_in=8, k_out=1)
    kc = oracle.kc_field(g, 0)
    brute = sum(1 for a in range(-12, 13) for b in range(-12, 13) if a * a + b * b <= 144)
    assert brute == 441
    assert int((kc == 8).sum()) == brute
    assert kc[40, 24] == 8 and kc[40, 36] == 8 and kc[40, 37] == 1
    assert abs(kc.mean() - (441 * 8 + 3655) / 4096) < 1e-15


def test_disk_moves_and_wraps():
    """The disk moves (vx, vy) cells per step with periodic wrap, so k_c(t)
    is k_c(0) rolled by t*(vy, vx), including across the domain edge."""
    g = OracleGrid(40, 30, 2, kc_disk=True, disk=(35, 3, 1, 2, 6), k_in=9, k_out=2)
    k0 = oracle.kc_field(g, 0)
    for t in (1, 7, 45):
        assert np.array_equal(oracle.kc_field(g, t), np.roll(k0, (2 * t, t), axis=(0, 1)))
    assert int((k0 == 9).sum()) == 113   # lattice points within radius 6


def test_window_matches_full_run():
    """The window run equals the periodic run on every column whose upwind
    cone stays inside the window (and is NaN elsewhere)."""
    g = OracleGrid(24, 20, 6, 0.5, 0.5, 0.0, 0.1, True, (20, 18, 1, 1, 5), 6, 1)
    q = rand_field(6, 20, 24, 12)
    n = 4
    full, _ = oracle.run(g, q, n)
    i0, j0, wx, wy = 18, 15, 12, 10          # wraps around both edges
    w = oracle.run_window(g, q, i0, j0, wx, wy, n)
    ii = np.arange(i0, i0 + wx) % 24
    jj = np.arange(j0, j0 + wy) % 20
    ref = full[:, jj][:, :, ii]
    assert np.array_equal(w[:, n:, n:], ref[:, n:, n:])
    assert np.isnan(w[:, :n, :]).all() and np.isnan(w[:, :, :n]).all()


def test_compensated_sum_matches_exact_rounding():
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.normal(size=10000) * 1e8, rng.normal(size=10000)])
    rng.shuffle(x)
    assert oracle.compensated_sum(x) == math.fsum(x)


# ---------------------------------------------------------------- Jacobi dynamics
# The Sec. IV "3D Jacobi solver" phase read as one weighted Jacobi sweep of
# the 7-point stencil per step (periodic x/y, zero-flux z by mirror ghosts).

def jac_grid(nx, ny, nz, nu, r=0.1, kc=(0, 0)):
    return OracleGrid(nx, ny, nz, 0.0, 0.0, 0.0, r, True, (0, 0, 0, 0, 10 ** 6), kc[0], kc[1],
                      dynamics=1, nu=nu)


@pytest.mark.parametrize("a,b,c,nu", [(1, 0, 0, 1 / 7), (2, 3, 1, 1 / 7), (0, 0, 2, 1 / 6),
                                      (5, 1, 4, 0.05), (6, 7, 9, 1 / 7)])
def test_jacobi_fourier_mode_is_an_eigenvector(a, b, c, nu):
    """cos(2 pi a i/nx) cos(2 pi b j/ny) cos(pi c (k + 1/2)/nz) is an eigenvector
    of the sweep (periodic x/y; the mirror ghosts make the half-integer
    cosine the zero-flux eigenvector in z) with eigenvalue
    1 - nu (6 - 2 cos(2 pi a/nx) - 2 cos(2 pi b/ny) - 2 cos(pi c/nz))."""
    nx, ny, nz = 12, 14, 10
    g = jac_grid(nx, ny, nz, nu)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    q = (np.cos(2 * np.pi * a * i / nx) * np.cos(2 * np.pi * b * j / ny)
         * np.cos(np.pi * c * (k + 0.5) / nz))
    lam = 1 - nu * (6 - 2 * np.cos(2 * np.pi * a / nx) - 2 * np.cos(2 * np.pi * b / ny)
                    - 2 * np.cos(np.pi * c / nz))
    assert np.max(np.abs(oracle.jacobi(g, q) - lam * q)) <= 1e-13


@pytest.mark.parametrize("nu", [1 / 7, 1 / 6, 0.05])
def test_jacobi_conserves_mass_and_keeps_bounds(nu):
    """Every cell hands nu of its value to each of its six neighbour slots
    (a mirror slot hands it back to itself): the total is conserved, and with
    non-negative weights every new value lies between the old extremes."""
    g = jac_grid(9, 8, 7, nu)
    q = rand_field(7, 8, 9, 11, -1.0, 2.0)
    out = oracle.jacobi(g, q)
    assert abs(out.sum() - q.sum()) <= 1e-12 * np.abs(q).sum()
    assert out.min() >= q.min() - 1e-15 and out.max() <= q.max() + 1e-15


def test_jacobi_unit_impulse_spreads_to_the_six_neighbours():
    """A unit value at an interior cell becomes 1 - 6 nu there and nu at each
    face neighbour; at the top face and x = 0 the mirror keeps one more nu at
    the cell and the periodic wrap sends one to x = nx - 1."""
    nu = 0.1
    nx, ny, nz = 6, 5, 4
    g = jac_grid(nx, ny, nz, nu)
    q = np.zeros((nz, ny, nx))
    q[1, 2, 3] = 1.0
    out = oracle.jacobi(g, q)
    want = np.zeros_like(q)
    want[1, 2, 3] = 1 - 6 * nu
    for (k, j, i) in ((0, 2, 3), (2, 2, 3), (1, 1, 3), (1, 3, 3), (1, 2, 2), (1, 2, 4)):
        want[k, j, i] = nu
    assert np.allclose(out, want, atol=1e-16, rtol=0)
    q = np.zeros((nz, ny, nx))
    q[nz - 1, 0, 0] = 1.0
    out = oracle.jacobi(g, q)
    want = np.zeros_like(q)
    want[nz - 1, 0, 0] = 1 - 6 * nu + nu
    for (k, j, i) in ((nz - 2, 0, 0), (nz - 1, 1, 0), (nz - 1, ny - 1, 0), (nz - 1, 0, 1),
                      (nz - 1, 0, nx - 1)):
        want[k, j, i] = nu
    assert np.allclose(out, want, atol=1e-16, rtol=0)


def test_jacobi_step_with_sweeps_conserves_mass():
    """Jacobi sweep then k_c implicit solves (unit column sums of M^-1): the
    global sum is invariant over many steps, to FP64 roundoff."""
    g = OracleGrid(20, 16, 12, 0.0, 0.0, 0.0, 0.3, True, (5, 5, 1, 2, 5), 7, 1, dynamics=1,
                   nu=1 / 7)
    q = rand_field(12, 16, 20, 5)
    _, mass = oracle.run(g, q, 12)
    assert np.max(np.abs(mass - q.sum())) <= 1e-12 * q.sum()


def test_jacobi_window_run_matches_full_run_inside():
    """Window runs (used to check full-size fields column by column): after s
    steps the columns at least s cells from every window edge equal the full
    run, and the rest are NaN (the sweep reads both sides in x and y)."""
    g = OracleGrid(16, 14, 6, 0.0, 0.0, 0.0, 0.2, True, (4, 4, 1, 0, 4), 5, 1, dynamics=1,
                   nu=1 / 7)
    q = rand_field(6, 14, 16, 9)
    s = 2
    full, _ = oracle.run(g, q, s)
    w = oracle.run_window(g, q, 3, 2, 9, 8, s)
    inner = w[:, s:8 - s, s:9 - s]
    assert np.array_equal(inner, full[:, 2 + s:2 + 8 - s, 3 + s:3 + 9 - s])
    assert np.isnan(w[:, :, 0]).all() and np.isnan(w[:, :, 8]).all()
    assert np.isnan(w[:, 0, :]).all() and np.isnan(w[:, 7, :]).all()
