"""Error predictors for approximating the centre element's active impedance
(Sec. II-E, the part after the active reflection coefficient).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain complex128 numpy,
written from the paper's definitions:

  * xi (Eq. 20):  Z~_a = Z_a,c (1 + xi), the relative error of an
    approximation Z~_a of the centre element's active impedance;
  * border bound (Eq. 23): |dZ_a,c| <= sum over the
    border set E_B of |Z_p,cn|;
  * xi_Z: max over E_B of |Z_p,cj| / |Z_p,cc| (Eq. 24), and its predictor (Eq. 25)
    with j the border element closest to the centre;
  * column coupling C_n (Eq. 28): the n-th Fourier coefficient of the
    active reflection coefficient over the inter-element phase psi (the
    excitation of Eq. 29), and its scan-angle form (Eq. 30) through
    psi = k d sin(theta);
  * S -> Z (Eq. 31): Z_p = Z0 (I + S)(I - S)^{-1}, and its inverse;
  * xi_S (Eq. 36): the xi_Z predictor evaluated on Z0 (I + S_ideal)(I -
    S_ideal)^{-1} for an idealised scattering matrix S_ideal.

Readings (where the paper leaves a choice):
  * E_B is the outermost ring of the Nx x Ny array (the elements that were
    added when growing it from (Nx-2) x (Ny-2));
  * "closest to c" is the Euclidean lattice distance; ties go to the element
    on the centre's row (the E-plane neighbour direction, x), then the
    smallest element index;
  * the Fourier integral is evaluated by the trapezoidal rule on Q uniform
    samples psi_q = -pi + 2 pi q / Q; the integrand is 2 pi periodic, so the
    rule is exact for trigonometric polynomials of degree < Q;
  * S_ideal: diagonal S_cc; off the diagonal |S_ij| = |s1| / dist_ij^2 with
    the free-space phase of the extra distance, S_ij = s1 dist_ij^-2
    exp(-j k d (dist_ij - 1)), dist_ij the Euclidean element distance in
    units of the spacing d and s1 the nearest-neighbour coupling of the
    centre element; xi_S's denominator is the cc entry of the same
    converted matrix.
"""
import numpy as np


def xi(za_approx, za_centre):
    """Eq. 20 solved for xi: xi = Z~_a / Z_a,c - 1."""
    return np.asarray(za_approx, dtype=np.complex128) / np.asarray(za_centre, dtype=np.complex128) - 1.0


def centre_index(nx, ny):
    """Element index e = mx + Nx*my of the centre (floor(Nx/2), floor(Ny/2))."""
    return (nx // 2) + nx * (ny // 2)


def border_elements(nx, ny):
    """Indices of E_B: elements with mx in {0, Nx-1} or my in {0, Ny-1}."""
    out = []
    for my in range(ny):
        for mx in range(nx):
            if mx in (0, nx - 1) or my in (0, ny - 1):
                out.append(mx + nx * my)
    return out


def closest_border_element(nx, ny):
    """j in E_B closest to the centre (Euclidean lattice distance); ties: on
    the centre's row first, then the smallest index."""
    cx, cy = nx // 2, ny // 2
    best = None
    for e in border_elements(nx, ny):
        mx, my = e % nx, e // nx
        key = ((mx - cx) ** 2 + (my - cy) ** 2, 0 if my == cy else 1, e)
        if best is None or key < best:
            best = key
    return best[2]


def border_bound(zp, nx, ny):
    """Right-hand side of the border bound (Eq. 23): sum over n in E_B of |Z_p,cn|."""
    c = centre_index(nx, ny)
    return float(sum(abs(zp[c, n]) for n in border_elements(nx, ny)))


def xi_z_max(zp, nx, ny):
    """Eq. 24: max over j in E_B of |Z_p,cj| / |Z_p,cc|."""
    c = centre_index(nx, ny)
    return max(abs(zp[c, j]) for j in border_elements(nx, ny)) / abs(zp[c, c])


def xi_z(zp, nx, ny):
    """Eq. 25: |Z_p,cj| / |Z_p,cc| with j the border element closest to c."""
    c = centre_index(nx, ny)
    j = closest_border_element(nx, ny)
    return abs(zp[c, j]) / abs(zp[c, c])


def z_from_s(s, z0=50.0):
    """Eq. 31: Z_p = Z0 (I + S)(I - S)^{-1}."""
    s = np.asarray(s, dtype=np.complex128)
    eye = np.eye(s.shape[0], dtype=np.complex128)
    return z0 * (eye + s) @ np.linalg.inv(eye - s)


def s_from_z(zp, z0=50.0):
    """Eq. 31 solved for S: S = (Z_p - Z0 I)(Z_p + Z0 I)^{-1}."""
    zp = np.asarray(zp, dtype=np.complex128)
    eye = np.eye(zp.shape[0], dtype=np.complex128)
    return (zp - z0 * eye) @ np.linalg.inv(zp + z0 * eye)


def psi_samples(q):
    """psi_q = -pi + 2 pi q / Q, q = 0 .. Q-1."""
    return -np.pi + 2.0 * np.pi * np.arange(q) / q


def column_coupling(gamma, nmax):
    """Eq. 28 by the trapezoidal rule: C_n = (1/Q) sum_q Gamma(psi_q)
    exp(-j n psi_q) for n = -nmax .. nmax; gamma = Gamma at psi_samples(Q)."""
    gamma = np.asarray(gamma, dtype=np.complex128)
    psi = psi_samples(len(gamma))
    n = np.arange(-nmax, nmax + 1)
    return (gamma[None, :] * np.exp(-1j * n[:, None] * psi[None, :])).sum(axis=1) / len(gamma)


def theta_of_psi(psi, kd):
    """Eq. 30's substitution: theta = asin(psi / (k d)) (radians), defined
    where |psi| <= k d (d >= lambda/2 covers the whole psi range)."""
    return np.arcsin(np.asarray(psi, dtype=np.float64) / kd)


def column_coupling_theta(gamma_of_theta, nmax, q, kd):
    """Eq. 30: C_n from an ARC given as a function of scan angle theta,
    sampled at theta(psi_q)."""
    psi = psi_samples(q)
    return column_coupling(np.array([gamma_of_theta(t) for t in theta_of_psi(psi, kd)]), nmax)


def row_phase_excitation(nx, ny, b, psi, port_basis=0):
    """Eq. 29: unit-amplitude voltages with inter-element phase psi along x
    (E-plane scan, psi_y = 0): V[q][my][mx][port_basis] = exp(j mx psi_q)."""
    psi = np.asarray(psi, dtype=np.float64)
    v = np.zeros((len(psi), ny, nx, b), dtype=np.complex128)
    mx = np.arange(nx)
    for q, p in enumerate(psi):
        v[q, :, :, port_basis] = np.exp(1j * mx * p)[None, :]
    return v


def s_ideal(nx, ny, s_cc, s1, kd):
    """Idealised scattering matrix (reading in the module docstring)."""
    n = nx * ny
    mx = np.arange(n) % nx
    my = np.arange(n) // nx
    dist = np.sqrt((mx[:, None] - mx[None, :]) ** 2 + (my[:, None] - my[None, :]) ** 2)
    s = np.empty((n, n), dtype=np.complex128)
    off = dist > 0
    s[off] = s1 * dist[off] ** -2 * np.exp(-1j * kd * (dist[off] - 1.0))
    s[~off] = s_cc
    return s


def xi_s(nx, ny, s_cc, s1, kd, z0=50.0):
    """Eq. 36: |[Z0 (I + S_ideal)(I - S_ideal)^{-1}]_cj| / |[...]_cc|."""
    z = z_from_s(s_ideal(nx, ny, s_cc, s1, kd), z0)
    c = centre_index(nx, ny)
    j = closest_border_element(nx, ny)
    return abs(z[c, j]) / abs(z[c, c])
