"""Seeded synthetic inputs for the batched patch update.

This module holds no arithmetic of the method itself (no flux, no update, no
conversion between conserved and primitive variables).  It only builds

* patch tables: periodic boxes tiled by equal patches, one box per
  refinement level, with face-neighbour ids and SoA-arena offsets
  (the paper's list of K patches, Sec. II Eq. 2, and its typical patch sizes,
  Sec. IV);
* smooth random fields: sums of 4 random Fourier modes with integer wave
  numbers in {-4..4}^d, so that every field is periodic on its box;
* Gaussian pulses and i.i.d. samples;
* the workload descriptions (pde, dimension, patch mix, halo, time stepping).

Both the CUDA path and the oracle take their inputs from here.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Same field order and sizes as the library's patch descriptor (72 bytes).
PATCH_DTYPE = np.dtype([("p", "<i4"), ("level", "<i4"), ("dx", "<f8"), ("x0", "<f8", (3,)),
                        ("offset", "<i8"), ("nbr", "<i4", (6,))])
assert PATCH_DTYPE.itemsize == 72

PDE_ADV_FLUX, PDE_ADV_NCP, PDE_EULER2D, PDE_EULER3D, PDE_WAVE3D, PDE_SRHD3D, PDE_GW59 = range(7)
SCHEME_FV, SCHEME_FD, SCHEME_FV2 = 0, 1, 2  # FV2: MUSCL-minmod reconstruction, halo 2
PDE_NQ = {0: 1, 1: 1, 2: 4, 3: 5, 4: 5, 5: 5, 6: 59}
PDE_NM = {0: 3, 1: 3, 2: 0, 3: 0, 4: 1, 5: 5, 6: 0}

SEED_BASE = 260819273


@dataclasses.dataclass
class Level:
    """A periodic box of nx x ny x nz patches of p^d voxels each."""
    n: tuple          # patches per axis (nz = 1 in 2D)
    p: int
    dx: float
    level: int = 0


@dataclasses.dataclass
class Mesh:
    dim: int
    patches: np.ndarray       # PATCH_DTYPE records
    var_stride: int           # elements between two variables of the arena
    levels: list
    level_ranges: list        # [first, last) patch index per level

    @property
    def K(self):
        return len(self.patches)

    @property
    def nvox(self):
        return int(sum(int(p) ** self.dim for p in self.patches["p"]))


def _round_up(x, m):
    return (x + m - 1) // m * m


def make_mesh(levels, dim, align=16):
    """Tile each level's periodic box by patches (x fastest), assign arena offsets."""
    recs, ranges = [], []
    off = 0
    for lev in levels:
        nx, ny, nz = lev.n if dim == 3 else (lev.n[0], lev.n[1], 1)
        first = len(recs)
        ranges.append((first, first + nx * ny * nz))
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    def pid(a, b, c):
                        return first + ((c % nz) * ny + (b % ny)) * nx + (a % nx)
                    nbr = [pid(i - 1, j, k), pid(i + 1, j, k), pid(i, j - 1, k), pid(i, j + 1, k), -1, -1]
                    if dim == 3:
                        nbr[4], nbr[5] = pid(i, j, k - 1), pid(i, j, k + 1)
                    x0 = (i * lev.p * lev.dx, j * lev.p * lev.dx, k * lev.p * lev.dx if dim == 3 else 0.0)
                    recs.append((lev.p, lev.level, lev.dx, x0, off, nbr))
                    off += _round_up(lev.p ** dim, align)
    patches = np.array(recs, dtype=PATCH_DTYPE)
    return Mesh(dim=dim, patches=patches, var_stride=_round_up(off, 32), levels=list(levels), level_ranges=ranges)


def coupled_mesh(nc, p, dx_c, lo, m, dim=3, align=16):
    """Two refinement levels with ratio 2: a periodic box of nc^dim coarse patches (level 0) and a
    finer level (level 1) that covers the coarse patches with lattice indices [lo, lo + m)^dim by
    (2m)^dim patches of the same p at dx_c / 2.  Fine patches on the border of the refined block
    have the adjacent coarse patch (outside the block) as face neighbour; the coarse level keeps
    its own periodic table (the coarse patches under the block stay in the list)."""
    coarse = make_mesh([Level((nc,) * 3 if dim == 3 else (nc, nc, 1), p, dx_c, 0)], dim, align)
    recs = [tuple(r) for r in coarse.patches.tolist()]
    off = int(coarse.patches["offset"][-1]) + _round_up(p ** dim, align)
    nf = 2 * m
    first = len(recs)
    nz = nf if dim == 3 else 1

    def cid(i, j, k):
        return ((k % nc) * nc + (j % nc)) * nc + (i % nc) if dim == 3 else (j % nc) * nc + (i % nc)

    for k in range(nz):
        for j in range(nf):
            for i in range(nf):
                def nb(di, dj, dk):
                    ii, jj, kk = i + di, j + dj, k + dk
                    if 0 <= ii < nf and 0 <= jj < nf and (dim == 2 or 0 <= kk < nf):
                        return first + ((kk if dim == 3 else 0) * nf + jj) * nf + ii
                    # coarse patch containing the neighbouring fine position
                    gi, gj = 2 * lo + ii, 2 * lo + jj
                    gk = 2 * lo + kk if dim == 3 else 0
                    return cid(gi // 2, gj // 2, gk // 2)
                nbr = [nb(-1, 0, 0), nb(1, 0, 0), nb(0, -1, 0), nb(0, 1, 0), -1, -1]
                if dim == 3:
                    nbr[4], nbr[5] = nb(0, 0, -1), nb(0, 0, 1)
                dxf = dx_c / 2
                x0 = ((2 * lo + i) * p * dxf, (2 * lo + j) * p * dxf, (2 * lo + k) * p * dxf if dim == 3 else 0.0)
                recs.append((p, 1, dxf, x0, off, nbr))
                off += _round_up(p ** dim, align)
    patches = np.array(recs, dtype=PATCH_DTYPE)
    levels = [Level((nc,) * 3 if dim == 3 else (nc, nc, 1), p, dx_c, 0),
              Level((nf,) * 3 if dim == 3 else (nf, nf, 1), p, dx_c / 2, 1)]
    return Mesh(dim=dim, patches=patches, var_stride=_round_up(off, 32), levels=levels,
                level_ranges=[(0, first), (first, len(recs))])


def coupled_fields(mesh, rng, specs):
    """Fourier fields periodic on the coarse box, evaluated at every voxel centre of both levels."""
    X = voxel_centres_any(mesh)
    L = [mesh.levels[0].n[a] * mesh.levels[0].p * mesh.levels[0].dx for a in range(mesh.dim)]
    out = np.zeros((len(specs), mesh.var_stride))
    m = np.zeros(mesh.var_stride, dtype=bool)
    for pt in mesh.patches:
        m[int(pt["offset"]):int(pt["offset"]) + int(pt["p"]) ** mesh.dim] = True
    for v, (mid, amp) in enumerate(specs):
        out[v, m] = fourier_field(rng, X[:, m], L, mesh.dim, mid, amp)
    return out


def euler_prims_coupled(mesh, seed):
    """The euler_prims recipe on a coupled mesh: fields periodic on the coarse box at every voxel."""
    rng = np.random.default_rng(seed)
    specs = [(1.0, 0.5)] + [(0.0, 0.5)] * mesh.dim + [(1.0, 0.5)]
    return coupled_fields(mesh, rng, specs)


def voxel_centres_any(mesh):
    """Voxel-centre coordinates (3, var_stride) for any patch table (patch by patch)."""
    X = np.zeros((3, mesh.var_stride))
    for pt in mesh.patches:
        p = int(pt["p"])
        pz = p if mesh.dim == 3 else 1
        z, y, x = np.meshgrid(np.arange(pz), np.arange(p), np.arange(p), indexing="ij")
        loc = [x.ravel(), y.ravel(), z.ravel()]
        o = int(pt["offset"])
        for a in range(mesh.dim):
            X[a, o:o + p * p * pz] = pt["x0"][a] + (loc[a] + 0.5) * pt["dx"]
    return X


def _level_block(mesh, li):
    """(first offset, patches, voxels per patch, contiguous?) of level li."""
    a, b = mesh.level_ranges[li]
    sel = mesh.patches[a:b]
    n = int(sel["p"][0]) ** mesh.dim
    off = sel["offset"]
    contiguous = bool(np.all(off == off[0] + n * np.arange(len(sel))))
    return int(off[0]), sel, n, contiguous


def voxel_centres(mesh):
    """Coordinates (3, var_stride) of every voxel centre (padding stays 0)."""
    X = np.zeros((3, mesh.var_stride))
    for li in range(len(mesh.levels)):
        first, sel, n, contiguous = _level_block(mesh, li)
        p = int(sel["p"][0])
        pz = p if mesh.dim == 3 else 1
        z, y, x = np.meshgrid(np.arange(pz), np.arange(p), np.arange(p), indexing="ij")
        loc = [x.ravel(), y.ravel(), z.ravel()]
        for a in range(mesh.dim):
            vals = sel["x0"][:, a][:, None] + (loc[a][None, :] + 0.5) * sel["dx"][:, None]
            if contiguous:
                X[a, first:first + n * len(sel)] = vals.ravel()
            else:
                X[a, (sel["offset"][:, None] + np.arange(n)[None, :]).ravel()] = vals.ravel()
    return X


def level_extent(mesh, li):
    lev = mesh.levels[li]
    L = [lev.n[a] * lev.p * lev.dx for a in range(mesh.dim)]
    return L


def level_slices(mesh, li):
    """Arena indices of all voxels of level li (a slice when the level is contiguous)."""
    first, sel, n, contiguous = _level_block(mesh, li)
    if contiguous:
        return slice(first, first + n * len(sel))
    return (sel["offset"][:, None] + np.arange(n)[None, :]).ravel()


def fourier_field(rng, X, L, dim, mid, amp, modes=4, kmax=4):
    """mid + amp * sum_m a_m sin(2 pi k_m.x/L + phi_m) / sum_m a_m (periodic on the box L)."""
    a = rng.uniform(0.0, 1.0, modes)
    phi = rng.uniform(0.0, 2 * math.pi, modes)
    ks = []
    while len(ks) < modes:
        k = rng.integers(-kmax, kmax + 1, dim)
        if np.any(k != 0):
            ks.append(k)
    f = np.zeros(X.shape[1])
    for m in range(modes):
        w = np.array([2 * math.pi * ks[m][ax] / L[ax] for ax in range(dim)])
        f += a[m] * np.sin(w @ X[:dim] + phi[m])
    return mid + amp * f / a.sum()


def fill_fields(mesh, rng, specs):
    """Arena (len(specs), var_stride) of Fourier fields; specs = [(mid, amp), ...] per variable."""
    X = voxel_centres(mesh)
    out = np.zeros((len(specs), mesh.var_stride))
    for li in range(len(mesh.levels)):
        idx = level_slices(mesh, li)
        L = level_extent(mesh, li)
        Xl = X[:, idx]
        for v, (mid, amp) in enumerate(specs):
            out[v, idx] = fourier_field(rng, Xl, L, mesh.dim, mid, amp)
    return out


# ------------------------------------------------------------------ workloads
@dataclasses.dataclass
class Workload:
    name: str
    pde: int
    scheme: int
    mesh: Mesh
    halo: int
    rk: int
    steps: int
    cfl: float
    sigma: float
    seed: int
    params: np.ndarray | None = None

    @property
    def nq(self):
        return PDE_NQ[self.pde]

    @property
    def nm(self):
        return PDE_NM[self.pde]


def euler2d_mesh(n=8, p=16, dx=1.0 / 128):
    return make_mesh([Level((n, n, 1), p, dx, 0)], dim=2)


def euler3d_amr_mesh(scale=1):
    """The AMR-like mix: 4096 x 8^3 + 1024 x 16^3 + 128 x 32^3 patches, dx = 1/128.

    Each level is its own periodic box.  ``scale`` > 1 divides the patch
    counts per axis (small cases for tests)."""
    s = scale
    return make_mesh([Level((16 // s, 16 // s, 16 // s), 8, 1.0 / 128, 0),
                      Level((16 // s, 8 // s, 8 // s), 16, 1.0 / 128, 1),
                      Level((max(8 // s, 1), max(4 // s, 1), max(4 // s, 1)), 32, 1.0 / 128, 2)], dim=3)


def euler_prims(mesh, seed):
    """rho, p in [0.5, 1.5]; velocities in [-0.5, 0.5]; rows (rho, u.., p)."""
    rng = np.random.default_rng(seed)
    specs = [(1.0, 0.5)] + [(0.0, 0.5)] * mesh.dim + [(1.0, 0.5)]
    return fill_fields(mesh, rng, specs)


def workload(name, scale=1):
    """Workload descriptions.

    euler2d : 2D Euler, 64 patches of 16^2, FV Rusanov, forward Euler, 10 steps, CFL 0.4.
    euler3d : 3D Euler, AMR-like patch mix, FV Rusanov, SSP-RK3, CFL 0.4.
    wave3d  : first-order wave system with c(x), FD4 + KO, RK4, 2048 patches of 16^3.
    srhd3d  : special-relativistic hydro, FV Rusanov + con2prim, SSP-RK3, 4096 patches of 16^3.
    gw59    : 59-unknown gravitational-wave stand-in, FD4 + KO, RK4, 3 levels of 24^3/16^3 patches.
    euler3d_muscl : the euler3d mix and data with the second-order FV stage (MUSCL-minmod, halo 2).
    euler3d_amr2 : 3D Euler on two coupled refinement levels: 8^3 coarse patches of 16^3 (dx 1/128) and
                   the block of coarse lattice [2, 6)^3 refined into 8^3 patches of 16^3 (dx 1/256);
                   FV Rusanov with prolongation, reflux and restriction, SSP-RK3, CFL 0.4.
    euler3d_p6 : 3D Euler on the paper's typical 6^3 cells: 32 x 32 x 16 patches of 6^3 (dx 1/192,
                 3,538,944 voxels), FV Rusanov (the generic stage), SSP-RK3, CFL 0.4.
    euler3d_p3 : the same box in 3^3 cells: 64 x 64 x 32 patches of 3^3 (131,072 patches).
    """
    if name == "euler2d":
        return Workload(name, PDE_EULER2D, SCHEME_FV, euler2d_mesh(), 1, 1, 10, 0.4, 0.0, SEED_BASE + 0)
    if name == "euler3d":
        return Workload(name, PDE_EULER3D, SCHEME_FV, euler3d_amr_mesh(scale), 1, 3, 100, 0.4, 0.0,
                        SEED_BASE + 1)
    if name == "euler3d_amr2":
        s_ = scale
        return Workload(name, PDE_EULER3D, SCHEME_FV, coupled_mesh(8 // s_, 16, 1.0 / 128, 2 // s_, 4 // s_), 1, 3,
                        20, 0.4, 0.0, SEED_BASE + 6)
    if name == "euler3d_p6":
        s_ = scale
        return Workload(name, PDE_EULER3D, SCHEME_FV, make_mesh([Level((32 // s_, 32 // s_, 16 // s_), 6,
                                                                       1.0 / 192, 0)], dim=3), 1, 3, 20, 0.4, 0.0,
                        SEED_BASE + 7)
    if name == "euler3d_p3":
        s_ = scale
        return Workload(name, PDE_EULER3D, SCHEME_FV, make_mesh([Level((64 // s_, 64 // s_, 32 // s_), 3,
                                                                       1.0 / 192, 0)], dim=3), 1, 3, 20, 0.4, 0.0,
                        SEED_BASE + 8)
    if name == "euler3d_muscl":
        return Workload(name, PDE_EULER3D, SCHEME_FV2, euler3d_amr_mesh(scale), 2, 3, 20, 0.4, 0.0,
                        SEED_BASE + 1)
    if name == "wave3d":
        s = scale
        mesh = make_mesh([Level((16 // s, 16 // s, 8 // s), 16, 1.0 / 128, 0)], dim=3)
        return Workload(name, PDE_WAVE3D, SCHEME_FD, mesh, 3, 4, 10, 0.25, 0.1, SEED_BASE + 2,
                        np.array([0.1]))
    if name == "srhd3d":
        s = scale
        mesh = make_mesh([Level((16 // s, 16 // s, 16 // s), 16, 1.0 / 256, 0)], dim=3)
        return Workload(name, PDE_SRHD3D, SCHEME_FV, mesh, 1, 3, 10, 0.4, 0.0, SEED_BASE + 3,
                        np.array([5.0 / 3.0]))
    if name == "gw59":
        s = scale
        mesh = make_mesh([Level((8 // s, 8 // s, 8 // s), 24, 1.0 / 192, 0),
                          Level((12 // s, 12 // s, 12 // s), 16, 1.0 / 192, 1),
                          Level((16 // s, 16 // s, 16 // s), 16, 1.0 / 256, 2)], dim=3)
        rng = np.random.default_rng(SEED_BASE + 4)
        C = rng.uniform(-0.1, 0.1, (11, 11))
        params = np.concatenate([[0.1], C.ravel()])
        return Workload(name, PDE_GW59, SCHEME_FD, mesh, 3, 4, 5, 0.25, 0.1, SEED_BASE + 4, params)
    raise KeyError(name)


def dyadic_field(rng, shape, bits=10, lo=-64, hi=64):
    """Values k / 2^bits with small integers k: sums, halves and differences stay exact."""
    return rng.integers(lo, hi + 1, shape).astype(np.float64) / float(2 ** bits)


def gaussian(X, centre, width, dim):
    r2 = np.zeros(X.shape[1])
    for a in range(dim):
        r2 = r2 + (X[a] - centre[a]) ** 2
    return np.exp(-r2 / (2 * width * width))


def wave_initial(mesh, seed, width=0.05):
    """Wave system: Gaussian pulse phi, Pi = 0, psi = grad phi (analytic); material
    c(x) = 1.25 + 0.75 sin(2 pi x/Lx) sin(2 pi y/Ly) sin(2 pi z/Lz) in [0.5, 2]."""
    rng = np.random.default_rng(seed)
    X = voxel_centres(mesh)
    q = np.zeros((5, mesh.var_stride))
    mat = np.zeros((1, mesh.var_stride))
    for li in range(len(mesh.levels)):
        idx = level_slices(mesh, li)
        L = level_extent(mesh, li)
        Xl = X[:, idx]
        x0 = [rng.uniform(0.25, 0.75) * L[a] for a in range(3)]
        g = gaussian(Xl, x0, width, 3)
        q[0, idx] = g
        for a in range(3):
            q[2 + a, idx] = -(Xl[a] - x0[a]) / (width * width) * g
        mat[0, idx] = 1.25 + 0.75 * (np.sin(2 * math.pi * Xl[0] / L[0]) * np.sin(2 * math.pi * Xl[1] / L[1])
                                     * np.sin(2 * math.pi * Xl[2] / L[2]))
    return q, mat


def gw59_initial(mesh, seed, amp=1e-6, width=0.05, noise=0.0):
    """Flat state (alpha = 1, everything else 0) plus a Gaussian of amplitude amp in alpha
    and phi_1 with a seeded centre per level; optional smooth noise of amplitude `noise`
    in every variable (test data that exercises the nonlinear terms)."""
    rng = np.random.default_rng(seed)
    X = voxel_centres(mesh)
    q = np.zeros((59, mesh.var_stride))
    for li in range(len(mesh.levels)):
        idx = level_slices(mesh, li)
        L = level_extent(mesh, li)
        Xl = X[:, idx]
        x0 = [rng.uniform(0.25, 0.75) * L[a] for a in range(3)]
        g = gaussian(Xl, x0, width, 3)
        q[55, idx] = 1.0 + amp * g
        q[0, idx] = amp * g
        if noise:
            for v in range(59):
                q[v, idx] += fourier_field(rng, Xl, L, 3, 0.0, noise)
    return q


def srhd_iid_prims(n, seed, wmax=10.0):
    """i.i.d. SRHD primitives (rows rho, v_x, v_y, v_z, p): rho, p log-uniform on
    [0.1, 10]; Lorentz factor uniform on [1, wmax]; isotropic direction."""
    rng = np.random.default_rng(seed)
    w = np.zeros((5, n))
    w[0] = np.exp(rng.uniform(math.log(0.1), math.log(10.0), n))
    w[4] = np.exp(rng.uniform(math.log(0.1), math.log(10.0), n))
    W = rng.uniform(1.0, wmax, n)
    speed = np.sqrt(1.0 - 1.0 / (W * W))
    nd = rng.normal(size=(3, n))
    nd /= np.linalg.norm(nd, axis=0)
    w[1:4] = speed * nd
    return w


def srhd_initial(mesh, seed, wmax=10.0):
    """Smooth SRHD primitives: ln rho and ln p are Fourier fields mapped onto
    [ln 0.1, ln 10]; W = 1 + (wmax - 1) s(x) with s a Fourier field in [0, 1];
    v = sqrt(1 - 1/W^2) n(x), n a normalised Fourier vector field."""
    rng = np.random.default_rng(seed)
    lo, hi = math.log(0.1), math.log(10.0)
    f = fill_fields(mesh, rng, [(0.5 * (lo + hi), 0.5 * (hi - lo))] * 2 + [(0.5, 0.5)] + [(0.0, 1.0)] * 3)
    w = np.zeros((5, mesh.var_stride))
    w[0] = np.exp(f[0])
    w[4] = np.exp(f[1])
    W = 1.0 + (wmax - 1.0) * f[2]
    nrm = np.sqrt(f[3] ** 2 + f[4] ** 2 + f[5] ** 2)
    nrm = np.where(nrm < 1e-12, 1.0, nrm)
    speed = np.sqrt(np.maximum(1.0 - 1.0 / (W * W), 0.0))
    for a in range(3):
        w[1 + a] = speed * f[3 + a] / nrm
    return w
