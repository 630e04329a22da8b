"""Pins of the oracle to facts the paper and the mathematics fix (CPU only).

Each test is chosen so that a plausible mistake in the oracle (a dropped term,
a wrong sign, factor or index, a transposed operand) fails it:

* the generalized fundamental solution satisfies Delta_S G = 1/(4 pi) away
  from its pole (Sec. 1.1, Eq. lap_G) - pins G's normalisation;
* the constant-density identity (I + 2K) zeta_k = 2 area(Omega_k)/(4 pi) at
  every node (Sec. 4.1 read with the jump relation Eq. jump and Green's
  identity, Eq. green2) - pins the kernel's sign, its 1/2pi, its diagonal and
  the row/column orientation, against an independent closed-form area; with the
  islands traversed the other way it becomes 2 zeta_k - 2 area(Omega_k)/(4 pi);
* the rows of an island-constant density from each curve's orientation and winding
  number (the planar form of the same identity, both orientations, the island around
  the pole included) - pins the exact rows the float operator adds;
* the diagonal entry equals the limit of the off-diagonal kernel (Appendix A);
* the planar Cauchy form (Sec. 3, Eq. dlpC and cont_kern, sign of the Cauchy
  term corrected) agrees entry by entry with the 3D form;
* exact harmonic solutions G(x, p) - G(x, q) are reproduced, with the exact
  multipliers (net source strength per island) - pins E, F, D and evaluation;
* spectral convergence of the trapezoidal rule (Sec. 5);
* a point vortex in the ocean of one circular island (Sec. 6, Example 2) against its
  closed form by a planar image;
* the unbordered operator has exactly M - 1 null vectors of the form
  sum c_k zeta_k with sum c_k area_k = 0 (Sec. 4.1), the bordered one none;
* rotation invariance of the solution under the choice of pole (Sec. 3);
* the reference quadtree: a hand-derived example and brute-force invariants,
  and completeness of the U/V/W/X lists;
* the stereographic projection (Sec. 3) at points whose images are known in closed
  form: the south pole, the equator, and a point at colatitude theta;
* the row-by-row matvec (the oracle's direct O(N^2) product, which the GPU parity
  tests sample) equals the dense bordered matrix times the vector, on a ragged case;
* the exact data of the paper's first and third examples, (1/2) sum Re 1/(xi - xi_k), is
  Laplace-Beltrami harmonic and has its closed-form value at the south pole, and the
  bordered solve reproduces it off the curves of an elliptical-island geometry.
"""
import json
import os

import numpy as np
import pytest

import workloads as wl
from helpers import cap_area, curve_point, max_rel

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TWO_PI = 2 * np.pi


def _three_islands(n=128, seed=7):
    return wl.star_caps(seed, 3, n, r0=[0.4, 0.3, 0.25], amp=[0.2, 0.1, 0.25], kfreq=[5, 3, 4])


# ---- Green's function --------------------------------------------------------

def test_green_laplace_beltrami(oracle):
    """Delta_S G(., x0) = 1/(4 pi) away from x0, by central differences of the
    spherical-coordinate Laplace-Beltrami operator (Sec. 1.2)."""
    x0 = np.array([0.3, -0.2, 0.9])
    x0 /= np.linalg.norm(x0)

    def Gs(th, ph):
        x = np.array([np.cos(ph) * np.sin(th), np.sin(ph) * np.sin(th), np.cos(th)])
        return oracle.green(x, x0)

    th, ph, e = 1.9, 2.4, 1e-4
    f0 = Gs(th, ph)
    d2ph = (Gs(th, ph + e) - 2 * f0 + Gs(th, ph - e)) / e ** 2
    fth = lambda t: np.sin(t) * (Gs(t + e / 2, ph) - Gs(t - e / 2, ph)) / e
    dth = (fth(th + e / 2) - fth(th - e / 2)) / e
    lap = d2ph / np.sin(th) ** 2 + dth / np.sin(th)
    assert abs(lap - 1 / (4 * np.pi)) < 1e-6


def test_green_special_values(oracle):
    x = np.array([0.0, 0.6, 0.8])
    # antipodal points: |x - y| = 2
    assert abs(oracle.green(x, -x) - (-np.log(2) / (4 * np.pi))) < 1e-15
    y = np.array([0.6, 0.0, 0.8])
    assert oracle.green(x, y) == oracle.green(y, x)
    # |x - y| = 1: G = log2 / 4pi
    z = np.array([0.0, 0.0, 1.0])
    w = np.array([np.sqrt(3) / 2, 0.0, 0.5])
    assert abs(oracle.green(z, w) - np.log(2) / (4 * np.pi)) < 1e-15


# ---- stereographic projection ---------------------------------------------------

def test_projection_closed_forms(oracle):
    """xi = (x1 + i x2)/(1 - x3) (Sec. 3), projecting from the north pole: the south
    pole maps to 0; a point at colatitude theta and longitude phi maps to
    cot(theta/2) e^{i phi}, so the equator goes to the unit circle at its own
    longitude.  Dividing by 1 + x3 moves the south pole to infinity and inverts the
    radii; swapping x1 and x2 reflects the angles about the diagonal."""
    th = np.array([0.05, 0.3, 1.0, np.pi / 2, 2.2, 3.0, 3.1])
    ph = np.array([0.1, 2.0, -1.3, 0.7, 4.0, 5.5, -2.9])
    x = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], axis=1)
    xi = oracle.project(np.vstack([x, [[0.0, 0.0, -1.0]]]))
    assert np.all(xi[-1] == 0.0)
    z = xi[:-1, 0] + 1j * xi[:-1, 1]
    want = np.exp(1j * ph) / np.tan(th / 2)
    assert np.max(np.abs(z - want) / np.abs(want)) < 1e-13  # 1 - cos(theta) rounds near the pole
    eq = np.isclose(th, np.pi / 2)
    assert abs(abs(z[eq][0]) - 1.0) < 1e-15
    assert abs(np.angle(z[eq][0]) - 0.7) < 1e-15


# ---- the double-layer operator --------------------------------------------------

@pytest.mark.parametrize("op", [0, 1])
def test_apply_rows_equal_dense_matrix_product(oracle, op):
    """The row-by-row matvec (every column of a row, node columns then multiplier
    columns for op 0; the density block I + 2K for op 1) equals the dense bordered
    matrix of Eq. (matrix_eqns) times the vector, on islands of 17, 23 and 30 nodes:
    node rows, the constraint rows of Eq. (disc_constr) and the row of Eq. (sum_ak)."""
    g = wl.star_caps(21, 3, [17, 23, 30], r0=[0.4, 0.3, 0.25], amp=[0.2, 0.1, 0.25],
                     kfreq=[5, 3, 4])
    A = oracle.matrix(g)
    N, n = g.N, g.N + g.M
    v = np.random.default_rng(3).standard_normal(n if op == 0 else N)
    ref = A @ v if op == 0 else A[:N, :N] @ v
    rows = np.arange(len(ref))[::-1].copy()       # any row order
    out = oracle.apply_rows(g, v, rows, op=op)
    assert np.max(np.abs(out - ref[rows])) < 1e-13 * np.max(np.abs(ref))
    # a subset of rows, each computed alone
    sub = np.array([0, 16, 17, 39, 69] + ([N, N + 1, N + 2] if op == 0 else []))
    assert np.max(np.abs(oracle.apply_rows(g, v, sub, op=op) - ref[sub])) < 1e-13 * np.max(np.abs(ref))
    assert np.allclose(oracle.apply(g, v, op), ref, rtol=0, atol=1e-13 * np.max(np.abs(ref)))


def test_cap_area_closed_form():
    # circular cap: area = 2 pi (1 - cos r0)
    assert abs(cap_area(0.3, 0.0, 3) - TWO_PI * (1 - np.cos(0.3))) < 1e-14


def test_constant_density_identity(oracle):
    g = _three_islands(128)
    A = oracle.matrix(g)
    N = g.N
    K2 = A[:N, :N]
    isl = g.island_of_node()
    for k in range(g.M):
        zeta = (isl == k).astype(float)
        y = K2 @ zeta
        ak = cap_area(g.r0[k], g.amp[k], g.kfreq[k]) / (4 * np.pi)
        assert np.max(np.abs(y - 2 * ak)) < 1e-11, k


def test_constant_density_identity_other_pole(oracle):
    """The same identity with the pole left where the generator put it."""
    g = wl.star_caps(11, 2, 256, r0=[0.35, 0.2], amp=[0.15, 0.3], kfreq=[2, 6], pole=None)
    A = oracle.matrix(g)
    isl = g.island_of_node()
    for k in range(2):
        y = A[:g.N, :g.N] @ (isl == k).astype(float)
        ak = cap_area(g.r0[k], g.amp[k], g.kfreq[k]) / (4 * np.pi)
        assert np.max(np.abs(y - 2 * ak)) < 1e-10


def test_constant_density_identity_reversed_orientation(oracle):
    """Islands traversed the other way flip the double layer's normal, so
    (I + 2K) zeta_k = 2 zeta_k - 2 area(Omega_k)/(4 pi): the island-constant rows the
    float operator adds exactly (orientation o_k = +1 there) are pinned here."""
    import dataclasses
    g = _three_islands(128)
    ptr = np.asarray(g.island_ptr)
    idx = np.concatenate([np.arange(ptr[k], ptr[k + 1])[::-1] for k in range(g.M)])
    x, dx, d2x = (np.asarray(a).reshape(g.N, 3) for a in (g.x, g.dx, g.d2x))
    gr = dataclasses.replace(g, x=x[idx].copy(), dx=-dx[idx], d2x=d2x[idx].copy())
    K2 = oracle.matrix(gr)[:g.N, :g.N]
    isl = g.island_of_node()
    for k in range(g.M):
        zeta = (isl == k).astype(float)
        ak = cap_area(g.r0[k], g.amp[k], g.kfreq[k]) / (4 * np.pi)
        assert np.max(np.abs(K2 @ zeta - (2 * zeta - 2 * ak))) < 1e-11, k


def test_diagonal_is_limit_of_kernel(oracle):
    """K_ii from Appendix A equals lim_{tau->0} of the off-diagonal kernel."""
    g = wl.star_caps(3, 1, 64, r0=[0.4], amp=[0.2], kfreq=[5], pole=None)
    c, e1, e2 = g.centres[0], g.e1[0], g.e2[0]
    for t0 in (0.0, 0.7, 2.1, 4.4):
        x0, dx0, d2x0 = curve_point(c, e1, e2, 0.4, 0.2, 5, t0)

        def pair(tau):
            x1, dx1, d2x1 = curve_point(c, e1, e2, 0.4, 0.2, 5, t0 + tau)
            geo = wl.Geometry(M=1, island_ptr=np.array([0, 2]), x=np.stack([x0, x1]),
                              dx=np.stack([dx0, dx1]), d2x=np.stack([d2x0, d2x1]),
                              centres=g.centres, r0=g.r0, amp=g.amp, kfreq=g.kfreq,
                              e1=g.e1, e2=g.e2)
            A = oracle.matrix(geo)
            return A[0, 1] / (2 * np.pi), (A[0, 0] - 1) / (2 * np.pi)  # h = 2pi/2

        kb = lambda tau: 0.5 * (pair(tau)[0] + pair(-tau)[0])
        tau = 2e-3
        lim = (4 * kb(tau / 2) - kb(tau)) / 3
        diag = pair(tau)[1]
        assert abs(lim - diag) < 1e-7 * abs(diag) + 1e-12, (t0, lim, diag)


def test_planar_cauchy_form_agrees(oracle):
    """Entries in the stereographic plane (Sec. 3): with w_j = h xi'_j,
    K_ij = (1/2pi) Im(w_j / (xi_j - xi_i)) + beta_j, beta_j = -(h/2pi) Im(conj(xi_j) xi'_j/(1+|xi_j|^2)),
    K_ii = (h/4pi) Im(xi''_i/xi'_i) + beta_i (Eq. cont_kern)."""
    g = _three_islands(64)
    A = oracle.matrix(g)
    N = g.N
    h = np.repeat(TWO_PI / g.nodes_per_island, g.nodes_per_island)
    X, DX, D2X = g.x, g.dx, g.d2x
    w = 1 - X[:, 2]
    z = X[:, 0] + 1j * X[:, 1]
    zp = DX[:, 0] + 1j * DX[:, 1]
    zpp = D2X[:, 0] + 1j * D2X[:, 1]
    wp, wpp = -DX[:, 2], -D2X[:, 2]
    xi = z / w
    xip = zp / w - z * wp / w ** 2
    xipp = zpp / w - 2 * zp * wp / w ** 2 - z * wpp / w ** 2 + 2 * z * wp ** 2 / w ** 3
    beta = -(h / TWO_PI) * np.imag(np.conj(xi) * xip / (1 + np.abs(xi) ** 2))
    dz = xi[None, :] - xi[:, None]
    np.fill_diagonal(dz, 1.0)
    Kp = (1 / TWO_PI) * np.imag((h * xip)[None, :] / dz) + beta[None, :]
    np.fill_diagonal(Kp, (h / (4 * np.pi)) * np.imag(xipp / xip) + beta)
    K = (A[:N, :N] - np.eye(N)) / 2
    assert np.max(np.abs(K - Kp)) < 1e-12 * np.max(np.abs(K))
    # the sign of the Cauchy term as printed, 1/(xi_i - xi_j), does not agree
    Kbad = (1 / TWO_PI) * np.imag((h * xip)[None, :] / (-dz)) + beta[None, :]
    np.fill_diagonal(Kbad, np.diag(Kp))
    assert np.max(np.abs(K - Kbad)) > 1e-3


def _planar(g):
    """xi, xi', xi'' (Sec. 3), the weights h, dself_i = (h/4pi) Im(xi''/xi') and beta."""
    h = np.repeat(TWO_PI / g.nodes_per_island, g.nodes_per_island)
    X, DX, D2X = (np.asarray(a).reshape(g.N, 3) for a in (g.x, g.dx, g.d2x))
    w = 1 - X[:, 2]
    z, zp, zpp = (A[:, 0] + 1j * A[:, 1] for A in (X, DX, D2X))
    wp, wpp = -DX[:, 2], -D2X[:, 2]
    xi = z / w
    xip = zp / w - z * wp / w ** 2
    xipp = zpp / w - 2 * zp * wp / w ** 2 - z * wpp / w ** 2 + 2 * z * wp ** 2 / w ** 3
    dself = (h / (4 * np.pi)) * np.imag(xipp / xip)
    beta = -(h / TWO_PI) * np.imag(np.conj(xi) * xip / (1 + np.abs(xi) ** 2))
    return h, xi, xip, dself, beta


@pytest.mark.parametrize("reverse", [False, True])
def test_island_constant_rows_from_orientation_and_winding(oracle, reverse):
    """The rows the float operator adds exactly for a density constant on island k:
    with o_k = 2 x (the planar double layer of 1_k at one of its own nodes) and n_k =
    (its value at a node of another island), rounded, 2K 1_k = (o_k - 2 n_k) 1_k +
    (2 n_k + 2 beta . 1_k) 1 -- for the island around the pole (n_k != 0) too, and with
    the islands traversed the other way."""
    import dataclasses
    g = _three_islands(128)
    if reverse:
        ptr = np.asarray(g.island_ptr)
        idx = np.concatenate([np.arange(ptr[k], ptr[k + 1])[::-1] for k in range(g.M)])
        x, dx, d2x = (np.asarray(a).reshape(g.N, 3) for a in (g.x, g.dx, g.d2x))
        g = dataclasses.replace(g, x=x[idx].copy(), dx=-dx[idx], d2x=d2x[idx].copy())
    ptr = np.asarray(g.island_ptr)
    h, xi, xip, dself, beta = _planar(g)
    K2 = oracle.matrix(g)[:g.N, :g.N] - np.eye(g.N)  # 2K
    enclosing = 0
    for k in range(g.M):
        sl = slice(ptr[k], ptr[k + 1])
        i0, i1 = ptr[k], ptr[(k + 1) % g.M]
        d0 = xi[sl] - xi[i0]
        d0[0] = 1.0
        t0 = (h * xip)[sl] / d0
        t0[0] = 0.0
        on = np.imag(t0.sum()) / TWO_PI + dself[i0]
        off = np.imag(((h * xip)[sl] / (xi[sl] - xi[i1])).sum()) / TWO_PI
        o, n = np.sign(on), np.rint(off)
        assert abs(2 * on - o) < 1e-9 and abs(off - n) < 1e-9
        enclosing += n != 0
        one = np.zeros(g.N)
        one[sl] = 1.0
        ref = (o - 2 * n) * one + (2 * n + 2 * beta[sl].sum())
        assert np.max(np.abs(K2 @ one - ref)) < 1e-10, k
    assert enclosing == 1  # the island around the pole (c_1 at the north pole)


# ---- the bordered system ------------------------------------------------------

def test_point_vortex_in_cap_ocean_by_planar_image(oracle):
    """Sec. 6, Example 2, on a geometry with a closed form: one circular island around the
    north pole is |xi| > R = cot(r0/2) in the plane, the ocean the disk |xi| < R.  For a
    vortex at nu, psi = Gamma (G(., v) - H) with H the harmonic function on the disk equal
    to G(., v) on |xi| = R: with |x - v|^2 = 4 |xi - nu|^2 / ((1 + |xi|^2)(1 + |nu|^2)) and,
    on the circle, |xi - nu| = |nu| |xi - nu*| / R (nu* = R^2 / conj(nu), outside the disk),
    H = (1/4pi) [log 2 - log 4 - log|xi - nu*|^2 - log(|nu|^2/R^2) + log(1 + R^2) + log(1 + |nu|^2)]."""
    r0, gam = 0.6, 1.7
    g = wl.star_caps(3, 1, 256, r0=[r0], amp=[0.0], kfreq=[2])
    th, ph = r0 + 0.9, 0.4
    v = np.array([[np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)]])
    t = wl.targets_off_islands(g, 64, seed=7)
    psi = oracle.point_vortices(g, v, [gam], t)
    R = 1.0 / np.tan(r0 / 2)
    xi_t = t[:, 0] / (1 - t[:, 2]) + 1j * t[:, 1] / (1 - t[:, 2])
    nu = (v[0, 0] + 1j * v[0, 1]) / (1 - v[0, 2])
    nus = R * R / np.conj(nu)
    H = (np.log(2.0) - np.log(4.0) - np.log(np.abs(xi_t - nus) ** 2) - np.log(np.abs(nu) ** 2 / R ** 2)
         + np.log(1 + R * R) + np.log(1 + np.abs(nu) ** 2)) / (4 * np.pi)
    exact = gam * (oracle.green_sum(t, v, [1.0]) - H)
    assert np.all(np.abs(xi_t) < R)  # the targets lie in the ocean
    assert max_rel(psi, exact) < 1e-10

def _solve_error(oracle, g, src, gam, T=64):
    data = oracle.green_sum(g.x, src, gam)
    sig, a = oracle.solve(g, data)
    tg = wl.targets_off_islands(g, T, seed=123)
    u = oracle.evaluate(g, sig, a, tg)
    uex = oracle.green_sum(tg, src, gam)
    return max_rel(u, uex), sig, a


def test_exact_solution_single_island(oracle):
    g = wl.config_geometry("C1")
    src, gam, _ = wl.pair_sources(g, 0)
    err, sig, a = _solve_error(oracle, g, src, gam)
    assert err < 1e-11
    assert abs(a[0]) < 1e-13


def test_exact_solution_multiply_connected_and_multipliers(oracle):
    g = _three_islands(128)
    src, gam, isl = wl.pair_sources(g, 0, 1)
    err, sig, a = _solve_error(oracle, g, src, gam)
    assert err < 1e-10
    assert np.max(np.abs(a - np.array([1.0, -1.0, 0.0]))) < 1e-10
    # the discrete constraints hold
    ptr = g.island_ptr
    for k in range(1, 3):
        assert abs(sig[ptr[k]:ptr[k + 1]].sum()) < 1e-9


def test_spectral_convergence(oracle):
    errs = []
    for n in (24, 48, 96):
        g = wl.star_caps(21, 2, n, r0=[0.35, 0.25], amp=[0.2, 0.2], kfreq=[3, 4])
        src, gam, _ = wl.pair_sources(g, 0, 1)
        errs.append(_solve_error(oracle, g, src, gam, T=32)[0])
    assert errs[1] < errs[0] / 30
    assert errs[2] < max(errs[1] / 30, 1e-12)


def test_null_space_of_unbordered_operator(oracle):
    g = _three_islands(64)
    N = g.N
    A = oracle.matrix(g)
    K2 = A[:N, :N]
    U, s, Vt = np.linalg.svd(K2)
    assert s[-1] < 1e-10 and s[-2] < 1e-10 and s[-3] > 1e-3
    isl = g.island_of_node()
    Z = np.stack([(isl == k).astype(float) for k in range(3)], axis=1)
    areas = np.array([cap_area(g.r0[k], g.amp[k], g.kfreq[k]) for k in range(3)])
    for v in Vt[-2:]:
        coef, res, *_ = np.linalg.lstsq(Z, v, rcond=None)
        assert np.linalg.norm(Z @ coef - v) < 1e-6
        assert abs(coef @ areas) < 1e-6 * np.linalg.norm(coef)
    sb = np.linalg.svd(A, compute_uv=False)
    assert sb[-1] > 1e-3


def test_rotation_invariance(oracle):
    g0 = wl.star_caps(9, 2, 96, r0=[0.3, 0.2], amp=[0.2, 0.1], kfreq=[4, 2], pole=None)
    R = wl.rotation_to_pole(g0.centres[1])
    g1 = wl.star_caps(9, 2, 96, r0=[0.3, 0.2], amp=[0.2, 0.1], kfreq=[4, 2], pole=None)
    g1 = wl.rotated(g1, R)
    src, gam, _ = wl.pair_sources(g0, 0, 1)
    s0, a0 = oracle.solve(g0, oracle.green_sum(g0.x, src, gam))
    src1 = wl.apply_rotation(R, src)
    s1, a1 = oracle.solve(g1, oracle.green_sum(g1.x, src1, gam))
    assert np.max(np.abs(s0 - s1)) < 1e-11
    assert np.max(np.abs(a0 - a1)) < 1e-11


def test_preconditioner_clusters_spectrum(oracle):
    """Sec. 5: the block preconditioner P = [[I, 2E], [F, D]] makes P^-1 A better
    conditioned than A (Table 1 reports bounded cond(P^-1 A))."""
    g = _three_islands(64)
    A = oracle.matrix(g)
    P = oracle.preconditioner_matrix(A, g.N)
    B = np.linalg.solve(P, A)
    assert np.linalg.cond(B) < np.linalg.cond(A)


# ---- reference quadtree --------------------------------------------------------

def test_tree_hand_example(oracle):
    with open(os.path.join(GOLDEN, "tree_hand_example.json")) as f:
        ref = json.load(f)
    t = oracle.tree(np.array(ref["xi"], dtype=float), leaf=ref["leaf"], depth=ref["depth"])
    assert t.perm.tolist() == ref["perm"]
    assert [int(k) for k in t.keys] == ref["keys_sorted"]
    assert t.nbox == len(ref["boxes"])
    for b, (lev, ix, iy, beg, end) in enumerate(ref["boxes"]):
        assert (t.level[b], t.ix[b], t.iy[b], t.begin[b], t.end[b]) == (lev, ix, iy, beg, end)


def _check_tree_invariants(t, xi, leaf, D):
    N = len(xi)
    assert sorted(t.perm.tolist()) == list(range(N))
    keys = t.keys.astype(np.uint64)
    assert np.all(keys[1:] >= keys[:-1])
    # ties broken by original index (stable)
    same = keys[1:] == keys[:-1]
    assert np.all(t.perm[1:][same] > t.perm[:-1][same])
    for b in range(t.nbox):
        n = t.end[b] - t.begin[b]
        assert n > 0
        if t.nchild[b] == 0:
            assert n <= leaf or t.level[b] == D
        else:
            ch = range(t.first_child[b], t.first_child[b] + t.nchild[b])
            assert t.begin[ch[0]] == t.begin[b] and t.end[ch[-1]] == t.end[b]
            for c0, c1 in zip(ch, list(ch)[1:]):
                assert t.end[c0] == t.begin[c1]
            for c in ch:
                assert t.parent[c] == b and t.level[c] == t.level[b] + 1
                assert t.ix[c] >> 1 == t.ix[b] and t.iy[c] >> 1 == t.iy[b]
        # every node of the box has the box's cell at its level
        l = int(t.level[b])
        sl = slice(t.begin[b], t.end[b])
        cx = np.floor((xi[t.perm[sl], 0] - t.xmin) / t.L * 2.0 ** D).astype(np.int64) >> (D - l)
        cy = np.floor((xi[t.perm[sl], 1] - t.ymin) / t.L * 2.0 ** D).astype(np.int64) >> (D - l)
        assert np.all(np.minimum(cx, (1 << l) - 1) == t.ix[b])
        assert np.all(np.minimum(cy, (1 << l) - 1) == t.iy[b])


def test_tree_invariants_multi_island(oracle):
    g = wl.config_geometry("C2", nodes=128)
    xi = oracle.project(g.x)
    t = oracle.tree(xi, leaf=16)
    _check_tree_invariants(t, xi, 16, 30)
    assert t.level.max() >= 6


def _touch(t, a, b):
    la, lb = t.level[a], t.level[b]
    if la > lb:
        a, b, la, lb = b, a, lb, la
    s = lb - la
    return (t.ix[b] <= (t.ix[a] + 1) << s and t.ix[b] + 1 >= t.ix[a] << s and
            t.iy[b] <= (t.iy[a] + 1) << s and t.iy[b] + 1 >= t.iy[a] << s)


def test_interaction_lists_cover_every_pair_once(oracle):
    """For every target leaf and source leaf, exactly one of: P2P (U), M2L from an
    ancestor-or-self's V box containing the source, M2P from a W box containing it,
    P2L (X) of an ancestor-or-self.  Brute force over all leaf pairs."""
    g = wl.star_caps(4, 3, 48, r0=[0.3, 0.2, 0.25], amp=[0.2, 0.3, 0.1], kfreq=[3, 5, 2])
    xi = oracle.project(g.x)
    t = oracle.tree(xi, leaf=4, lists=True)
    nb = t.nbox
    lst = {k: [set(getattr(t, k + "_idx")[getattr(t, k + "_ptr")[b]:getattr(t, k + "_ptr")[b + 1]].tolist())
               for b in range(nb)] for k in "UVWX"}

    def anc(b):
        out = []
        while b >= 0:
            out.append(b)
            b = t.parent[b]
        return out

    leaves = [b for b in range(nb) if t.nchild[b] == 0]
    for tl in leaves:
        A = anc(tl)
        for sl in leaves:
            SA = set(anc(sl))
            cnt = (sl in lst["U"][tl])
            cnt += sum(len(lst["V"][a] & SA) for a in A)
            cnt += len(lst["W"][tl] & SA)
            cnt += sum(sl in lst["X"][a] for a in A)
            assert cnt == 1, (tl, sl, cnt)
    # U symmetric, W/X duals
    for b in leaves:
        for u in lst["U"][b]:
            assert b in lst["U"][u]
        for w in lst["W"][b]:
            assert b in lst["X"][w]
    assert sum(len(v) for v in lst["V"]) > 0 and sum(len(w) for w in lst["W"]) > 0


# ---- the elliptical islands of the first and third examples ------------------------------

def test_dipole_data_is_harmonic_with_known_values(oracle):
    """(1/2) sum_k Re 1/(xi - xi_k) (Sec. 6, Eq. exact_bcs): Delta_S psi = 0 away from the
    sources (central differences of the spherical-coordinate operator), and at the south
    pole (xi = 0) psi = (1/2) sum_k Re(-1/xi_k)."""
    src = np.array([[0.3, -0.4, 0.5], [-0.6, 0.1, -0.2]])
    src /= np.linalg.norm(src, axis=1)[:, None]

    def psi(th, ph):
        x = np.array([[np.cos(ph) * np.sin(th), np.sin(ph) * np.sin(th), np.cos(th)]])
        return oracle.dipole_data(x, src)[0]

    th, ph, e = 2.2, 0.9, 1e-4
    f0 = psi(th, ph)
    d2ph = (psi(th, ph + e) - 2 * f0 + psi(th, ph - e)) / e ** 2
    fth = lambda t: np.sin(t) * (psi(t + e / 2, ph) - psi(t - e / 2, ph)) / e
    dth = (fth(th + e / 2) - fth(th - e / 2)) / e
    assert abs(d2ph / np.sin(th) ** 2 + dth / np.sin(th)) < 1e-5 * abs(f0)
    xk = (src[:, 0] + 1j * src[:, 1]) / (1 - src[:, 2])
    sp = oracle.dipole_data(np.array([[0.0, 0.0, -1.0]]), src)[0]
    assert abs(sp - 0.5 * np.sum(np.real(-1.0 / xk))) < 1e-15 * np.sum(np.abs(1 / xk))
    # a source at the north pole adds nothing
    both = np.vstack([src, [[0.0, 0.0, 1.0]]])
    assert oracle.dipole_data(np.array([[0.5, 0.5, 0.0]]) / np.sqrt(0.5), both)[0] == \
        oracle.dipole_data(np.array([[0.5, 0.5, 0.0]]) / np.sqrt(0.5), src)[0]


def test_ellipse_islands_exact_solution(oracle):
    """Fifteen elliptical islands (the first example's M): the dense solve reproduces the
    exact solution off the curves, with zero multipliers (no net source in any island)."""
    g = wl.ellipse_islands(1, 15, 128)
    data = oracle.dipole_data(g.x, g.centres[1:])
    sig, a = oracle.solve(g, data)
    t = wl.targets_off_islands(g, 75, seed=2)
    u = oracle.evaluate(g, sig, a, t)
    ue = oracle.dipole_data(t, g.centres[1:])
    assert max_rel(u, ue) < 1e-8
    assert np.max(np.abs(a)) < 1e-9 * np.max(np.abs(sig))
