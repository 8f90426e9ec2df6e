"""Port quantities from the solved currents (Sec. II-E).

Each element has one delta-gap port on basis `port_basis`; its port current
is that entry of I and its port voltage that entry of V.
"""
import numpy as np


def port_currents(i, port_basis=0):
    """I_p [nrhs][Ny][Nx]."""
    return np.asarray(i)[..., port_basis]


def active_impedance(i, v, port_basis=0):
    """Z_a = diag(I_p)^{-1} Z_p I_p (Eqs. 16-17).  Under voltage excitation
    Z_p I_p = V_p (Eq. 18 relates port voltages to port currents), so this is
    Z_a,e = V_p,e / I_p,e element by element."""
    ip = np.asarray(i)[..., port_basis].astype(np.complex128)
    vp = np.asarray(v)[..., port_basis].astype(np.complex128)
    return vp / ip


def reflection(za, z0=50.0):
    """Active reflection coefficient, Eq. 19, with a real reference Z0."""
    return (za - z0) / (za + z0)


def port_impedance_matrix(z, nx, ny, b, port_basis=0):
    """Passive port impedance Z_p (Eq. 18): with unit current at port j and
    zero current at the other ports, Z_p,ij is the voltage at port i.
    Eliminating the non-port unknowns gives Y_p = [Z^{-1}]_{ports,ports} and
    Z_p = Y_p^{-1}.  Returns (N_el x N_el)."""
    ports = np.arange(nx * ny) * b + port_basis
    zinv = np.linalg.inv(z)
    return np.linalg.inv(zinv[np.ix_(ports, ports)])


def active_impedance_from_zp(zp, ip):
    """Eq. 17 written out: Z_a = diag(I_p)^{-1} Z_p I_p, for ip [nrhs][N_el]."""
    ip = np.asarray(ip, dtype=np.complex128)
    return (ip @ zp.T) / ip


def named_elements(nx, ny):
    """(mx, my) of the centre (floor(Nx/2), floor(Ny/2)), edge (0, floor(Ny/2))
    and corner (0, 0) elements."""
    return {"centre": (nx // 2, ny // 2), "edge": (0, ny // 2), "corner": (0, 0)}


def rrmse(z_solver, z_direct):
    """Relative rms error (Sec. IV-A, Eq. 39), read as
    sqrt(mean(|a - b|^2 / |b|^2)) -- the printed formula lacks the squares."""
    a = np.asarray(z_solver).ravel()
    d = np.asarray(z_direct).ravel()
    return float(np.sqrt(np.mean(np.abs(a - d) ** 2 / np.abs(d) ** 2)))
