"""Seeded synthetic workloads: species tables, geometry and initial densities.

This module only builds inputs (grids, species parameters, external
potentials, starting densities).  It holds none of the method's arithmetic and
is the one module that both the CUDA path's tests/benchmarks and the CPU
oracle's tests draw inputs from.  numpy only; no torch, no CUDA.

Geometry is expressed as the external potential beta*mu_ext (the paper defines
the problem geometry through mu_ext, Sec. "Theory"): V_i(x) = +inf where the
voxel centre x lies strictly inside the contact distance of a hard obstacle
(distance < R_obstacle + R_i, minimum image on the periodic box), else the
smooth potential of the workload (0 for pure hard geometry).

Grid points sit at x_j = j h_d, j = 0..N_d-1; the box is [0, N_d h_d) periodic.
Arrays are float64, shaped (S, Nz, Ny, Nx) with x fastest.
"""

from dataclasses import dataclass, field

import numpy as np

# Species of the workloads: (name, radius nm, valence)
NA = ("Na+", 0.095, 1.0)
CL = ("Cl-", 0.181, -1.0)
CA = ("Ca2+", 0.099, 2.0)
O_HALF = ("O-1/2", 0.14, -0.5)


@dataclass
class Workload:
    name: str
    shape: tuple                 # (Nz, Ny, Nx)
    h: tuple                     # (hx, hy, hz), nm
    species: list                # names
    radius: np.ndarray           # nm
    z: np.ndarray                # valences
    bulk_molar: np.ndarray       # mol/L
    V: np.ndarray                # (S, Nz, Ny, Nx) beta*mu_ext, +inf = excluded
    temperature_K: float = 298.15
    eps_r: float = 78.5
    mixing: float = None         # fixed Picard mixing, or None for line search
    max_it: int = 50
    tol: float = 0.0
    n_fixed: np.ndarray = None   # particles of fixed-number species (0: species in the bath)
    notes: dict = field(default_factory=dict)

    @property
    def nspecies(self):
        return len(self.radius)

    def initial_rho_nm3(self, per_nm3_bulk):
        """Bulk density on accessible voxels, 0 on excluded ones (per_nm3_bulk: (S,) nm^-3); a
        fixed-number species starts uniform over its accessible voxels with its particle number."""
        acc = ~np.isinf(self.V)
        rho = np.where(acc, np.asarray(per_nm3_bulk, dtype=np.float64)[:, None, None, None], 0.0)
        if self.n_fixed is not None:
            dv = self.h[0] * self.h[1] * self.h[2]
            for i, n in enumerate(self.n_fixed):
                if n > 0:
                    rho[i] = np.where(acc[i], n / (np.count_nonzero(acc[i]) * dv), 0.0)
        return rho


def grid_coordinates(shape, h):
    nz, ny, nx = shape
    hx, hy, hz = h
    x = (np.arange(nx) * hx)[None, None, :]
    y = (np.arange(ny) * hy)[None, :, None]
    z = (np.arange(nz) * hz)[:, None, None]
    return z, y, x


def _min_image(d, length):
    return d - length * np.round(d / length)


def sphere_exclusion(shape, h, radius_species, centres, radii):
    """V (S, Nz, Ny, Nx): +inf where min-image distance to any centre < R_obs + R_i."""
    zc, yc, xc = grid_coordinates(shape, h)
    L = (shape[2] * h[0], shape[1] * h[1], shape[0] * h[2])
    S = len(radius_species)
    V = np.zeros((S,) + tuple(shape), dtype=np.float64)
    for (cx, cy, cz), ro in zip(centres, radii):
        dx = _min_image(xc - cx, L[0])
        dy = _min_image(yc - cy, L[1])
        dz = _min_image(zc - cz, L[2])
        r2 = dx * dx + dy * dy + dz * dz
        for i in range(S):
            V[i][r2 < (ro + radius_species[i]) ** 2] = np.inf
    return V


def _species(table):
    names = [t[0] for t in table]
    radius = np.array([t[1] for t in table])
    z = np.array([t[2] for t in table])
    return names, radius, z


def centred_sphere(n=32, h=0.1, molar=0.1, sphere_radius=0.5, mixing=0.1, max_it=50):
    """Two species Na+/Cl- at `molar` each, one neutral hard sphere at the box centre."""
    names, radius, z = _species([NA, CL])
    shape = (n, n, n)
    hh = (h, h, h)
    c = n * h / 2.0
    V = sphere_exclusion(shape, hh, radius, [(c, c, c)], [sphere_radius])
    return Workload(name=f"nacl_sphere_{n}^3", shape=shape, h=hh, species=names, radius=radius, z=z,
                    bulk_molar=np.array([molar, molar]), V=V, mixing=mixing, max_it=max_it,
                    notes={"sphere_radius": sphere_radius})


def obstacles_3species(n=128, h=0.05, n_obstacles=16, r_lo=0.3, r_hi=0.6, seed=1, tol=1e-8, max_it=2000):
    """Na+ 0.1 M, Ca2+ 0.01 M, Cl- 0.12 M around seeded non-overlapping hard neutral spheres."""
    names, radius, z = _species([NA, CA, CL])
    shape = (n, n, n)
    hh = (h, h, h)
    L = n * h
    rng = np.random.default_rng(seed)
    centres, radii = [], []
    while len(centres) < n_obstacles:
        r = rng.uniform(r_lo, r_hi)
        c = rng.uniform(0.0, L, size=3)
        ok = True
        for c2, r2 in zip(centres, radii):
            d = _min_image(c - np.asarray(c2), L)
            if np.sqrt(np.sum(d * d)) < r + r2:
                ok = False
                break
        if ok:
            centres.append(tuple(c))
            radii.append(r)
    V = sphere_exclusion(shape, hh, radius, centres, radii)
    return Workload(name=f"3species_16obstacles_{n}^3", shape=shape, h=hh, species=names, radius=radius,
                    z=z, bulk_molar=np.array([0.1, 0.01, 0.12]), V=V, mixing=None, max_it=max_it, tol=tol,
                    notes={"centres": centres, "radii": radii, "seed": seed})


def pore_slab_4species(n=256, h=0.05, slab_half=1.0, pore_radius=0.5, pore_half=0.5, o_count=8,
                       tol=1e-6, max_it=2000):
    """Na+ 0.1 M, Ca2+ 0.001 M, Cl- 0.102 M and o_count half-charged O confined to a pore.

    A hard slab |z - z0| < slab_half (nm) across the box, pierced along z by a cylindrical hole
    of radius pore_radius about the box axis (x0, y0) = (L/2, L/2), z0 = L/2.  A bath species i
    is excluded where |z - z0| < slab_half + R_i and r_perp > pore_radius - R_i (r_perp: the
    minimum-image distance from the axis).  The O particles (fixed number, not in the bath) are
    confined to r_perp <= pore_radius - R_O and |z - z0| <= pore_half - R_O, the central
    2 pore_half of the hole.
    """
    names, radius, z = _species([NA, CA, CL, O_HALF])
    shape = (n, n, n)
    hh = (h, h, h)
    L = n * h
    zc, yc, xc = grid_coordinates(shape, hh)
    dx = _min_image(xc - L / 2.0, L)
    dy = _min_image(yc - L / 2.0, L)
    dz = _min_image(zc - L / 2.0, L)
    r_perp = np.sqrt(dx * dx + dy * dy)
    V = np.zeros((4,) + shape, dtype=np.float64)
    for i in range(3):
        excl = (np.abs(dz) < slab_half + radius[i]) & (r_perp > pore_radius - radius[i])
        V[i][np.broadcast_to(excl, shape)] = np.inf
    Ro = radius[3]
    allowed = (r_perp <= pore_radius - Ro) & (np.abs(dz) <= pore_half - Ro)
    V[3][~np.broadcast_to(allowed, shape)] = np.inf
    return Workload(name=f"pore_slab_4species_{n}^3", shape=shape, h=hh, species=names, radius=radius, z=z,
                    bulk_molar=np.array([0.1, 0.001, 0.102, 0.0]), V=V, mixing=None, max_it=max_it, tol=tol,
                    n_fixed=np.array([0.0, 0.0, 0.0, float(o_count)]),
                    notes={"slab_half_nm": slab_half, "pore_radius_nm": pore_radius, "pore_half_nm": pore_half})


def hard_wall_ionic(nxy=21, nz=161, lxy=2.0, lz=6.0, molar=1.0, tol=1e-8, max_it=2000):
    """Univalent salt at a hard, uncharged wall (Sec. "Results", the representative ionic
    calculation): cation R 0.1 nm, anion R 0.2125 nm, `molar` each, in a periodic
    lxy x lxy x lz nm cell on an nxy x nxy x nz grid (h_d = L_d / N_d) with a zero-thickness wall
    in the plane z = 0.  The cell is periodic along z, so the wall bounds the fluid from both
    sides: species i is excluded where the minimum-image distance to the plane is < R_i.
    """
    names = ["cation(0.1)", "anion(0.2125)"]
    radius = np.array([0.1, 0.2125])
    z = np.array([1.0, -1.0])
    shape = (nz, nxy, nxy)
    hh = (lxy / nxy, lxy / nxy, lz / nz)
    zc, _, _ = grid_coordinates(shape, hh)
    dist = np.abs(_min_image(zc, lz))
    V = np.zeros((2,) + shape, dtype=np.float64)
    for i in range(2):
        V[i][np.broadcast_to(dist < radius[i], shape)] = np.inf
    return Workload(name=f"hard_wall_ionic_{nxy}x{nxy}x{nz}", shape=shape, h=hh, species=names, radius=radius,
                    z=z, bulk_molar=np.array([molar, molar]), V=V, mixing=None, max_it=max_it, tol=tol,
                    notes={"cell_nm": [lxy, lxy, lz], "wall": "z = 0 plane, hard, uncharged"})


def hard_wall_hs(eta, nz=512, nxy=4, hz=0.00625, hxy=0.05, radius=0.1, tol=1e-10, max_it=5000):
    """Hard spheres of radius `radius` at bath packing fraction `eta` against a hard wall (Sec.
    "Hard sphere fluids": R 0.1 nm, packing fractions 1e-5 ... 0.4, voxels 0.05 x 0.05 x 0.00625
    nm, the effectively one-dimensional problem computed in full 3D).  The paper gives no domain
    size; here nxy x nxy x nz voxels, periodic, with a zero-thickness wall in the plane z = 0 seen
    from both sides (excluded where the minimum-image distance to the plane is < R).  The contact
    density is rho at z = R (grid index R / hz when that is an integer)."""
    rho = eta / (4.0 / 3.0 * np.pi * radius ** 3)
    shape = (nz, nxy, nxy)
    hh = (hxy, hxy, hz)
    zc, _, _ = grid_coordinates(shape, hh)
    lz = nz * hz
    dist = np.abs(_min_image(zc, lz))
    V = np.zeros((1,) + shape, dtype=np.float64)
    V[0][np.broadcast_to(dist < radius, shape)] = np.inf
    return Workload(name=f"hard_sphere_wall_eta{eta:g}_{nxy}x{nxy}x{nz}", shape=shape, h=hh, species=["HS(0.1)"],
                    radius=np.array([radius]), z=np.array([0.0]), bulk_molar=np.array([rho / 0.602214076]), V=V,
                    mixing=None, max_it=max_it, tol=tol,
                    notes={"eta": eta, "contact_index": radius / hz, "wall": "z = 0 plane, hard"})


def gaussian_random_field(shape, h, corr_len, std, seed):
    """Zero-mean periodic Gaussian field with covariance ~ exp(-r^2 / (2 l^2)), scaled to `std`."""
    rng = np.random.default_rng(seed)
    white = rng.standard_normal(shape)
    kz = 2 * np.pi * np.fft.fftfreq(shape[0], d=h[2])[:, None, None]
    ky = 2 * np.pi * np.fft.fftfreq(shape[1], d=h[1])[None, :, None]
    kx = 2 * np.pi * np.fft.fftfreq(shape[2], d=h[0])[None, None, :]
    filt = np.exp(-0.25 * (kx * kx + ky * ky + kz * kz) * corr_len * corr_len)
    g = np.real(np.fft.ifftn(np.fft.fftn(white) * filt))
    g -= g.mean()
    return g * (std / g.std())


def smooth_field_nacl(n=64, h=0.1, molar=0.5, corr_len=0.5, std=1.0, seed=2):
    """NaCl with V_i = z_i g(x), g a seeded Gaussian random field (no hard exclusion)."""
    names, radius, z = _species([NA, CL])
    shape = (n, n, n)
    hh = (h, h, h)
    g = gaussian_random_field(shape, hh, corr_len, std, seed)
    V = np.stack([zi * g for zi in z])
    return Workload(name=f"nacl_grf_{n}^3", shape=shape, h=hh, species=names, radius=radius, z=z,
                    bulk_molar=np.array([molar, molar]), V=V, mixing=None, max_it=200,
                    notes={"corr_len": corr_len, "std": std, "seed": seed})


def batch_state_points(count=64, sizes=(32, 48, 64, 96), h=0.1, c_lo=0.01, c_hi=1.0,
                       r_lo=0.3, r_hi=1.0, seed=4, max_it=100):
    """Seeded ragged batch of NaCl state points, each with a centred neutral hard sphere."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        n = int(rng.choice(sizes))
        c = float(np.exp(rng.uniform(np.log(c_lo), np.log(c_hi))))
        r = float(rng.uniform(r_lo, r_hi))
        w = centred_sphere(n=n, h=h, molar=c, sphere_radius=r, mixing=None, max_it=max_it)
        w.name = f"batch{b}_{n}^3"
        out.append(w)
    return out


def fd_voxels(shape, count=64, seed=3):
    """Seeded voxel indices (z, y, x) for finite-difference gradient checks."""
    rng = np.random.default_rng(seed)
    return [tuple(int(rng.integers(0, s)) for s in shape) for _ in range(count)]


def random_density(shape, nspecies, mean, amplitude, seed):
    """Smooth positive random densities (S, Nz, Ny, Nx) for parity tests of the convolutions."""
    rng = np.random.default_rng(seed)
    mean = np.asarray(mean, dtype=np.float64)
    out = np.empty((nspecies,) + tuple(shape))
    for i in range(nspecies):
        g = gaussian_random_field(shape, (1.0, 1.0, 1.0), 2.0, 1.0, int(rng.integers(1 << 31)))
        out[i] = mean[i] * (1.0 + amplitude * np.tanh(g))
    return out
