"""Synthetic multilevel block-Toeplitz problems shaped like the paper's arrays.

The paper's impedance matrices come from RWG meshes of real antennas, which
are not available; these lattices stand in for them (same structure: an
Nx x Ny regular array of identical elements, b basis functions per element,
element-pair blocks that depend only on the lattice offset, Sec. II-A).

Units are wavelengths (lambda = 1, k = 2*pi).  For seed s the generator draws,
in this order, u_i in [0,1)^2 (b pairs, x then y per basis), w_i ~ U(0.5, 1)
and alpha_i ~ U(0, pi).  Basis i of element (mx, my) sits at
(mx*d, my*d) + d*u_i.  The coupling between observation basis i of element m
and source basis j of element n, with lattice offset Delta = m - n, is

    Z_Delta[i][j] = w_i w_j cos(alpha_i - alpha_j) exp(-1j k r) / (4 pi r),
    r = max(|Delta*d + p_i - p_j|, a),  a = 0.01,

plus a self-loading of 50+30j ohm on every diagonal entry of Z_0.  The
construction is reciprocal: Z_{-Delta} = Z_Delta^T exactly (Sec. II-D states
the MoM matrix is symmetric).

Block layout: complex array [2Ny-1][2Nx-1][b][b], offset (dx, dy) at index
(dy + Ny - 1, dx + Nx - 1), rows = observation basis.
Vector layout: complex array [nrhs][Ny][Nx][b]; element e = mx + Nx*my and
global unknown e*b + i, as in the two-level ordering of Eq. (2).
"""
from dataclasses import dataclass

import numpy as np

from .rng import SplitMix64

K_WAVENUMBER = 2.0 * np.pi
R_FLOOR = 0.01
SELF_LOAD = 50.0 + 30.0j


@dataclass(frozen=True)
class LatticeSpec:
    nx: int
    ny: int
    b: int
    d: float = 0.5
    seed: int = 0

    @property
    def n_el(self):
        return self.nx * self.ny

    @property
    def n(self):
        return self.nx * self.ny * self.b


def element_geometry(b, d, seed=0):
    """Basis positions p (b,2), weights w (b,) and orientations alpha (b,)."""
    g = SplitMix64(seed)
    u = g.uniform(2 * b).reshape(b, 2)
    w = g.uniform(b, 0.5, 1.0)
    alpha = g.uniform(b, 0.0, np.pi)
    return d * u, w, alpha


def offset_blocks(spec, dtype=np.complex128):
    """All (2Nx-1)(2Ny-1) offset blocks of the lattice, layout [2Ny-1][2Nx-1][b][b].

    Entries are computed in float64; with dtype=complex64 they are rounded once
    at the end (the rounded values then define the problem).
    """
    nx, ny, b, d = spec.nx, spec.ny, spec.b, spec.d
    p, w, alpha = element_geometry(b, d, spec.seed)
    coef = np.outer(w, w) * np.cos(alpha[:, None] - alpha[None, :])
    pij = p[:, None, :] - p[None, :, :]  # (b, b, 2): p_i - p_j
    dxs = np.arange(-(nx - 1), nx, dtype=np.float64) * d
    out = np.empty((2 * ny - 1, 2 * nx - 1, b, b), dtype=dtype)
    for iy, dy in enumerate(range(-(ny - 1), ny)):
        rx = dxs[:, None, None] + pij[None, :, :, 0]
        ry = dy * d + pij[None, :, :, 1]
        r = np.maximum(np.sqrt(rx * rx + ry * ry), R_FLOOR)
        blk = coef[None] * np.exp(-1j * K_WAVENUMBER * r) / (4.0 * np.pi * r)
        if dy == 0:
            blk[nx - 1] += SELF_LOAD * np.eye(b)
        out[iy] = blk
    return out


def offset_blocks_torch(spec, device="cuda", dtype=None):
    """The same offset blocks as offset_blocks(), evaluated with torch on
    `device` (float64 arithmetic, same formula and geometry draw) -- for
    workloads whose host generation would be too slow.  Values agree with
    the numpy version to float64 rounding of the elementary functions.
    Returns a [2Ny-1][2Nx-1][b][b] tensor (complex64 unless dtype given)."""
    import torch
    dtype = dtype or torch.complex64
    nx, ny, b, d = spec.nx, spec.ny, spec.b, spec.d
    p, w, alpha = element_geometry(b, d, spec.seed)
    dev = torch.device(device)
    p = torch.as_tensor(p, dtype=torch.float64, device=dev)
    w = torch.as_tensor(w, dtype=torch.float64, device=dev)
    al = torch.as_tensor(alpha, dtype=torch.float64, device=dev)
    coef = torch.outer(w, w) * torch.cos(al[:, None] - al[None, :])
    pij = p[:, None, :] - p[None, :, :]
    dxs = torch.arange(-(nx - 1), nx, dtype=torch.float64, device=dev) * d
    out = torch.empty((2 * ny - 1, 2 * nx - 1, b, b), dtype=dtype, device=dev)
    eye = torch.eye(b, dtype=torch.float64, device=dev)
    for iy, dy in enumerate(range(-(ny - 1), ny)):
        rx = dxs[:, None, None] + pij[None, :, :, 0]
        ry = dy * d + pij[None, :, :, 1]
        r = torch.clamp(torch.sqrt(rx * rx + ry * ry), min=R_FLOOR)
        amp = coef[None] / (4.0 * np.pi * r)
        ph = -K_WAVENUMBER * r
        re, im = amp * torch.cos(ph), amp * torch.sin(ph)
        if dy == 0:
            re[nx - 1] += SELF_LOAD.real * eye
            im[nx - 1] += SELF_LOAD.imag * eye
        out[iy] = torch.complex(re, im).to(dtype)
    return out


def margin_geometry(spec, bm=2):
    """Basis positions, weights and orientations of a synthetic array margin:
    bm basis functions in every cell of the ring around the lattice (cells
    (mx, my), -1 <= mx <= Nx, -1 <= my <= Ny, on the ring's boundary), drawn
    from seed + 1.  Returns (pos [nm, 2], w [nm], alpha [nm])."""
    nx, ny, d = spec.nx, spec.ny, spec.d
    u, w1, a1 = element_geometry(bm, d, spec.seed + 1)
    cells = [(mx, my) for my in range(-1, ny + 1) for mx in range(-1, nx + 1)
             if mx in (-1, nx) or my in (-1, ny)]
    pos = np.array([[mx * d + u[i, 0], my * d + u[i, 1]] for (mx, my) in cells for i in range(bm)])
    w = np.tile(w1, len(cells))
    alpha = np.tile(a1, len(cells))
    return pos, w, alpha


def margin_blocks(spec, bm=2, dtype=np.complex128):
    """Margin blocks of the reciprocal synthetic MoM matrix Z = [Z_A, Z_B^T;
    Z_B, Z_C] (Sec. II-A's margin partition): Z_B [nm][N] couples margin
    basis m to lattice unknown e*b + i, Z_C [nm][nm] the margin bases among
    themselves, both with the lattice kernel w w' cos(alpha - alpha')
    e^{-jkr} / (4 pi r) (r floored at 0.01) and 50+30j ohm self-loading on
    Z_C's diagonal."""
    nx, ny, b, d = spec.nx, spec.ny, spec.b, spec.d
    mp, mw, ma = margin_geometry(spec, bm)
    p, w, alpha = element_geometry(b, d, spec.seed)
    ex = np.arange(nx * ny) % nx
    ey = np.arange(nx * ny) // nx
    lp = np.stack([(ex[:, None] * d + p[None, :, 0]).ravel(), (ey[:, None] * d + p[None, :, 1]).ravel()], axis=1)
    lw = np.tile(w, nx * ny)
    la = np.tile(alpha, nx * ny)

    def kernel(p1, w1, a1, p2, w2, a2):
        r = np.sqrt(((p1[:, None, :] - p2[None, :, :]) ** 2).sum(-1))
        r = np.maximum(r, R_FLOOR)
        coef = np.outer(w1, w2) * np.cos(a1[:, None] - a2[None, :])
        return coef * np.exp(-1j * K_WAVENUMBER * r) / (4.0 * np.pi * r)

    zb = kernel(mp, mw, ma, lp, lw, la)
    zc = kernel(mp, mw, ma, mp, mw, ma) + SELF_LOAD * np.eye(len(mp))
    return zb.astype(dtype), zc.astype(dtype)


def scan_phase(nx, ny, d, theta_deg, phi_deg):
    """Progressive port phase a[my][mx] = exp(-j k d sin(theta) (mx cos(phi) + my sin(phi)))."""
    th = np.deg2rad(theta_deg)
    ph = np.deg2rad(phi_deg)
    mx = np.arange(nx)[None, :]
    my = np.arange(ny)[:, None]
    return np.exp(-1j * K_WAVENUMBER * d * np.sin(th) * (mx * np.cos(ph) + my * np.sin(ph)))


def excitation(spec, angles, port_basis=0):
    """Delta-gap port excitation V [nrhs][Ny][Nx][b]: the scan phase on basis
    `port_basis` of each element, zero elsewhere.  `angles` is a list of
    (theta_deg, phi_deg); (0, 0) is broadside (all ports 1)."""
    nx, ny, b = spec.nx, spec.ny, spec.b
    v = np.zeros((len(angles), ny, nx, b), dtype=np.complex128)
    for q, (th, ph) in enumerate(angles):
        v[q, :, :, port_basis] = scan_phase(nx, ny, spec.d, th, ph)
    return v


def config_c1():
    """4x4 lattice, spacing 0.5, b = 32, one broadside RHS, complex128 blocks."""
    return LatticeSpec(4, 4, 32, 0.5, 0), [(0.0, 0.0)]


def config_c2():
    """32x32 lattice, spacing 0.5, b = 128, blocks stored complex64, 2 RHS:
    broadside and a 45 degree E-plane (x) scan."""
    return LatticeSpec(32, 32, 128, 0.5, 0), [(0.0, 0.0), (45.0, 0.0)]


def config_c3_angles():
    """8 x 8 scan grid: theta_p = p*60/7 (p = 0..7), phi_q = q*90/8 (q = 0..7),
    RHS index p*8 + q."""
    return [(p * 60.0 / 7.0, q * 90.0 / 8.0) for p in range(8) for q in range(8)]
