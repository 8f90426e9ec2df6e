"""Pins of the predictor oracle (oracle/predictors.py) against closed forms,
special cases and the paper's own inequality -- nothing here re-types the
function under test."""
import numpy as np
import pytest
from scipy.special import factorial

from synth import LatticeSpec, offset_blocks, excitation
from oracle import dense, ports, predictors as pr


def test_xi_definition_eq20():
    za = 54.1 + 29.9j
    assert abs(pr.xi(za * (1 + 0.013 - 0.002j), za) - (0.013 - 0.002j)) < 1e-15


def test_s_of_single_port_is_reflection_coefficient():
    """1x1: S = (Z - Z0)/(Z + Z0), Eq. 19's reflection coefficient."""
    for z in (50.0 + 0j, 73.1 + 42.5j, 12.0 - 80.0j):
        s = pr.s_from_z(np.array([[z]]), 50.0)
        assert abs(s[0, 0] - ports.reflection(z, 50.0)) < 1e-15
        assert abs(pr.z_from_s(s, 50.0)[0, 0] - z) < 1e-12


def test_s_to_z_special_cases_and_round_trip():
    n = 7
    # Matched ports (S = 0) give Z_p = Z0 I.
    assert np.allclose(pr.z_from_s(np.zeros((n, n)), 50.0), 50.0 * np.eye(n), atol=1e-13)
    # Uncoupled ports: diagonal S from diagonal Z, entry by entry Eq. 19.
    zd = np.diag(np.linspace(20, 90, n) + 1j * np.linspace(-30, 30, n))
    sd = pr.s_from_z(zd, 50.0)
    assert np.allclose(np.diag(sd), ports.reflection(np.diag(zd), 50.0), atol=1e-15)
    assert np.abs(sd - np.diag(np.diag(sd))).max() < 1e-15
    # A reciprocal Z_p from a solved lattice: S symmetric, and back to Z_p.
    spec = LatticeSpec(3, 2, 5, 0.5, 1)
    z = dense.assemble(offset_blocks(spec), 3, 2)
    zp = ports.port_impedance_matrix(z, 3, 2, 5)
    s = pr.s_from_z(zp, 50.0)
    assert np.abs(s - s.T).max() < 1e-12
    assert np.abs(pr.z_from_s(s, 50.0) - zp).max() < 1e-10 * np.abs(zp).max()


def test_column_coupling_closed_form_and_sign():
    """Gamma(psi) = exp(a e^{j psi}) = sum_{n>=0} a^n e^{j n psi} / n!, so
    C_n = a^n / n! for n >= 0 and 0 for n < 0 (pins the e^{-j n psi} kernel)."""
    a = 0.7
    q = 64
    psi = pr.psi_samples(q)
    c = pr.column_coupling(np.exp(a * np.exp(1j * psi)), 6)
    n = np.arange(-6, 7)
    expect = np.where(n >= 0, a ** np.abs(n) / factorial(np.abs(n)), 0.0)
    assert np.abs(c - expect).max() < 1e-15


def test_column_coupling_recovers_trig_polynomial():
    rng = np.random.default_rng(3)
    coef = rng.standard_normal(11) + 1j * rng.standard_normal(11)  # n = -5..5
    q = 16
    psi = pr.psi_samples(q)
    gamma = sum(coef[k] * np.exp(1j * (k - 5) * psi) for k in range(11))
    assert np.abs(pr.column_coupling(gamma, 5) - coef).max() < 1e-13


def test_theta_form_is_the_substitution():
    """Eq. 30 with kd = pi (d = lambda/2): sampling Gamma^(theta) at
    theta = asin(psi / kd) equals sampling Gamma(psi)."""
    kd = np.pi
    g_psi = lambda p: 0.2 * np.exp(1j * p) - 0.05 * np.exp(-2j * p) + 0.1
    c1 = pr.column_coupling(g_psi(pr.psi_samples(32)), 4)
    c2 = pr.column_coupling_theta(lambda t: g_psi(kd * np.sin(t)), 4, 32, kd)
    assert np.abs(c1 - c2).max() < 1e-14
    assert abs(c1[4 + 1] - 0.2) < 1e-14 and abs(c1[4 - 2] + 0.05) < 1e-14


def test_border_set_and_closest_element():
    assert len(pr.border_elements(6, 4)) == 2 * 6 + 2 * 4 - 4
    assert len(pr.border_elements(5, 1)) == 5
    # 5x5: centre (2,2); the four edge midpoints are at distance 2; the one on
    # the centre's row with the smaller index is (0, 2) -> 10.
    assert pr.closest_border_element(5, 5) == 10
    # 6x4: centre (3,2); (3,3) on the top row is at distance 1 -> 21.
    assert pr.closest_border_element(6, 4) == 21
    assert pr.centre_index(6, 4) == 15


def test_border_bound_holds_when_growing_the_array():
    """Eq. 23: growing the array from (N-2)x(N-2) to NxN changes the centre
    element's broadside Z_a by at most sum_{n in E_B} |Z_p,cn|."""
    for n in (3, 5):
        za = []
        for m in (n - 2, n):
            spec = LatticeSpec(m, m, 6, 0.5, 2)
            z = dense.assemble(offset_blocks(spec), m, m)
            v = excitation(spec, [(0.0, 0.0)])
            i = dense.solve(z, v)
            za.append(ports.active_impedance(i, v)[0, m // 2, m // 2])
            zp = ports.port_impedance_matrix(z, m, m, 6)
        bound = pr.border_bound(zp, n, n)
        assert abs(za[1] - za[0]) <= bound
        assert pr.xi_z(zp, n, n) <= pr.xi_z_max(zp, n, n) + 1e-15


def test_s_ideal_structure_and_xi_s_limit():
    kd = np.pi
    s = pr.s_ideal(5, 4, 0.1 + 0.05j, -0.2 + 0.1j, kd)
    assert np.abs(s - s.T).max() == 0
    assert np.allclose(np.diag(s), 0.1 + 0.05j)
    c = pr.centre_index(5, 4)
    assert s[c, c + 1] == -0.2 + 0.1j                      # nearest neighbour: s1 itself
    assert abs(abs(s[0, 3]) * 9 - abs(-0.2 + 0.1j)) < 1e-15  # distance 3: |s1| / 9
    # Without coupling S_ideal is diagonal, Z is diagonal and xi_S vanishes.
    assert pr.xi_s(5, 5, 0.1, 0.0, kd) == 0.0
    assert 0 < pr.xi_s(5, 5, 0.1, 0.05, kd) < 1


def test_row_phase_excitation_is_the_e_plane_scan():
    """Eq. 29 against the scan excitation: the inter-element phase of an
    E-plane scan (phi = 0) at angle theta is psi = -k d sin(theta) in the
    e^{-j k d sin(theta) m_x} convention of the scan phase."""
    spec = LatticeSpec(5, 3, 4, 0.6, 0)
    thetas = [0.0, 20.0, 47.5]
    kd = 2 * np.pi * spec.d
    psi = [-kd * np.sin(np.radians(t)) for t in thetas]
    v_row = pr.row_phase_excitation(spec.nx, spec.ny, spec.b, psi, port_basis=2)
    v_scan = excitation(spec, [(t, 0.0) for t in thetas], port_basis=2)
    assert np.abs(v_row - v_scan).max() < 1e-13


def test_xi_z_invariants():
    """Eqs. 24-25: invariant under scaling Z_p; when the centre's coupling
    decays with distance the closest border element is also the largest
    (xi_Z = its maximum); a far border element made dominant separates them."""
    nx, ny = 5, 5
    n = nx * ny
    c = pr.centre_index(nx, ny)
    mx, my = np.arange(n) % nx, np.arange(n) // nx
    dist = np.hypot(mx - mx[c], my - my[c])
    zp = np.where(dist > 0, (0.3 - 0.2j) / np.maximum(dist, 1) ** 2, 60 + 20j).astype(np.complex128)
    zp = np.tile(zp, (n, 1))  # row c is what the predictors read
    j = pr.closest_border_element(nx, ny)
    assert pr.xi_z(zp, nx, ny) == pr.xi_z_max(zp, nx, ny)
    assert abs(pr.xi_z(zp, nx, ny) - abs(0.3 - 0.2j) / (dist[j] ** 2 * abs(60 + 20j))) < 1e-15
    assert abs(pr.xi_z(3.7j * zp, nx, ny) - pr.xi_z(zp, nx, ny)) < 1e-15
    corner = 0
    zp[c, corner] = 10.0
    assert pr.xi_z_max(zp, nx, ny) == 10.0 / abs(60 + 20j) > pr.xi_z(zp, nx, ny)


def test_s_ideal_phase_hand_values():
    """S_ideal's off-neighbour entries (reading of Eq. 36 in the module
    docstring): s1 dist^-2 exp(-j k d (dist - 1)).  With k d chosen so that
    the extra distance is a quarter turn the phase factor is exactly -j, so
    the entries are written out by hand: a sign error in the phase flips
    them, a wrong power of the distance rescales them."""
    s1 = -0.2 + 0.1j  # s1 * (-j) = 0.1 + 0.2j
    # 3 x 3 lattice; element e = mx + 3 my.  Diagonal neighbour (0,0)-(1,1):
    # dist sqrt(2), k d (sqrt(2) - 1) = pi / 2.
    kd = (np.pi / 2) / (np.sqrt(2.0) - 1.0)
    s = pr.s_ideal(3, 3, 0.3, s1, kd)
    assert abs(s[0, 4] - (0.1 + 0.2j) / 2) < 1e-15
    assert abs(s[4, 0] - (0.1 + 0.2j) / 2) < 1e-15
    # Two cells along x, (0,0)-(2,0): dist 2, k d = pi / 2 -> phase -j, |.| = |s1| / 4.
    s = pr.s_ideal(3, 3, 0.3, s1, np.pi / 2)
    assert abs(s[0, 2] - (0.1 + 0.2j) / 4) < 1e-15
    # (0,0)-(2,2): dist 2 sqrt(2), phase exp(-j (pi/2)(2 sqrt 2 - 1)); with k d = pi / (2 sqrt 2 - 1)
    # the phase is exp(-j pi) = -1, |.| = |s1| / 8.
    s = pr.s_ideal(3, 3, 0.3, s1, np.pi / (2 * np.sqrt(2.0) - 1.0))
    assert abs(s[0, 8] - (0.2 - 0.1j) / 8) < 1e-15
    # Nearest neighbours carry s1 itself whatever k d is; the diagonal is s_cc.
    assert s[4, 5] == s1 and s[4, 1] == s1 and s[4, 4] == 0.3


def test_z_from_s_satisfies_its_defining_relation():
    """Eq. 31: Z_p (I - S) = Z0 (I + S) (the factors commute), for a
    generic S, and s_from_z inverts it."""
    rng = np.random.default_rng(3)
    n = 7
    s = 0.2 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    z = pr.z_from_s(s, 50.0)
    eye = np.eye(n)
    assert np.abs(z @ (eye - s) - 50.0 * (eye + s)).max() < 1e-12
    assert np.abs(pr.s_from_z(z, 50.0) - s).max() < 1e-13


@pytest.mark.parametrize("nx,ny,s_cc,s1,kd", [(3, 3, 0.5, 0.02 + 0.01j, np.pi),
                                                (5, 4, -0.3 + 0.2j, 0.05 - 0.02j, 2.2),
                                                (4, 5, 0.1j, 0.03, 3.9)])
def test_xi_s_against_a_neumann_series(nx, ny, s_cc, s1, kd):
    """xi_S (Eq. 36) by a second route: with S = s_cc I + T the converted
    matrix is Z0 (I + S)(I - S)^{-1} = Z0 (-I + (2/c) sum_n (T/c)^n),
    c = 1 - s_cc, a convergent series here (||T / c|| < 1); its entries
    [c, j] and [c, c], at the hand-counted centre and closest border
    element, give xi_S.  Catches a swapped S <-> Z conversion, the wrong
    border element or the wrong denominator."""
    s = pr.s_ideal(nx, ny, s_cc, s1, kd)
    t = s - s_cc * np.eye(nx * ny)
    c = 1.0 - s_cc
    assert np.linalg.norm(t / c, 2) < 0.5
    acc = np.eye(nx * ny, dtype=np.complex128)
    term = np.eye(nx * ny, dtype=np.complex128)
    for _ in range(80):
        term = term @ (t / c)
        acc = acc + term
    z = 50.0 * (-np.eye(nx * ny) + (2.0 / c) * acc)
    cen = {(3, 3): 4, (5, 4): 12, (4, 5): 10}[(nx, ny)]      # (floor(Nx/2), floor(Ny/2))
    # Closest border element: 3x3 -> (0,1) (distance 1, centre row, smaller index than (2,1));
    # 5x4 -> (2,3), one row above the centre (2,2); 4x5 -> (3,2), one column right of (2,2).
    j = {(3, 3): 3, (5, 4): 17, (4, 5): 11}[(nx, ny)]
    assert pr.centre_index(nx, ny) == cen and pr.closest_border_element(nx, ny) == j
    want = abs(z[cen, j]) / abs(z[cen, cen])
    assert abs(pr.xi_s(nx, ny, s_cc, s1, kd, 50.0) - want) < 1e-12 * want
