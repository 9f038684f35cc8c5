"""Seeded synthetic voxel structures shaped like the paper's workloads.

Each generator returns a ``Workload`` holding integer voxel labels
``[N_z][N_y][N_x]`` (x fastest), a per-label conductor index (-1 for a
dielectric label), a per-label relative permittivity and the voxel edge in
metres.  Nothing here computes any part of the method; the module is shared
by the tests, ``bench.py`` and the oracle-driven checks.

Background outside the grid is vacuum (eps_r = 1).  Voxel edge 1 um unless
stated.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Workload:
    name: str
    labels: np.ndarray          # int32 [nz, ny, nx]
    conductor_id: np.ndarray    # int32 [n_labels]
    eps_r: np.ndarray           # float64 [n_labels]
    voxel_size: float = 1e-6

    @property
    def shape_xyz(self):
        nz, ny, nx = self.labels.shape
        return nx, ny, nz

    @property
    def n_conductors(self) -> int:
        c = self.conductor_id
        return int(c.max() + 1) if np.any(c >= 0) else 0


def cube(a: int = 4) -> Workload:
    """An isolated a x a x a conductor cube filling its grid (config: cube,
    96 panels at a = 4)."""
    lab = np.zeros((a, a, a), np.int32)
    return Workload(f"cube{a}", lab, np.array([0], np.int32), np.array([1.0]))


def plates(nx: int = 32, ny: int = 32, nz: int = 16) -> Workload:
    """Two 24 x 24 x 2 conductor plates 4 voxels apart with an eps_r = 3.9
    slab filling the gap, on a 32 x 32 x 16 grid: plates at x,y in [4,28),
    z in [4,6) and [10,12); slab at z in [6,10)."""
    lab = np.zeros((nz, ny, nx), np.int32)            # 0 vacuum
    lab[6:10, 4:28, 4:28] = 1                          # slab
    lab[4:6, 4:28, 4:28] = 2                           # plate 0
    lab[10:12, 4:28, 4:28] = 3                         # plate 1
    return Workload("plates_32x32x16", lab, np.array([-1, -1, 0, 1], np.int32),
                    np.array([1.0, 3.9, 1.0, 1.0]))


def bus_crossing() -> Workload:
    """4 lines along y over 4 lines along x (cross-section 4 x 4, pitch 8) in
    three stacked dielectric layers eps_r 2.5 / 3.9 / 7.0 (z in [0,21),
    [21,42), [42,64)) filling a 128 x 128 x 64 grid.  Lower lines: x in
    {50,58,66,74}+[0,4), y in [16,112), z in [16,20); upper lines: y in
    {50,58,66,74}+[0,4), x in [16,112), z in [24,28)."""
    nx, ny, nz = 128, 128, 64
    lab = np.zeros((nz, ny, nx), np.int32)
    lab[0:21] = 0
    lab[21:42] = 1
    lab[42:64] = 2
    cid = [-1, -1, -1]
    eps = [2.5, 3.9, 7.0]
    c = 0
    for x0 in (50, 58, 66, 74):
        lab[16:20, 16:112, x0:x0 + 4] = 3 + c
        cid.append(c); eps.append(1.0); c += 1
    for y0 in (50, 58, 66, 74):
        lab[24:28, y0:y0 + 4, 16:112] = 3 + c
        cid.append(c); eps.append(1.0); c += 1
    return Workload("bus_crossing_128x128x64", lab, np.array(cid, np.int32),
                    np.array(eps))


def small_boxes(count: int = 16, n: int = 16, seed0: int = 0):
    """``count`` independent n^3 grids, each holding one box conductor in
    vacuum with sides drawn from U{2..12} per axis at a random position
    (seeds seed0 .. seed0+count-1).  All share one grid shape."""
    out = []
    for s in range(seed0, seed0 + count):
        rng = np.random.default_rng(s)
        size = rng.integers(2, 13, size=3)
        lo = [int(rng.integers(0, n - size[a] + 1)) for a in range(3)]
        lab = np.zeros((n, n, n), np.int32)
        lab[lo[2]:lo[2] + size[2], lo[1]:lo[1] + size[1], lo[0]:lo[0] + size[0]] = 1
        out.append(Workload(f"box{s}", lab, np.array([-1, 0], np.int32),
                            np.array([1.0, 1.0])))
    return out


def smooth_field(n: int, sigma: float, seed: int) -> np.ndarray:
    """Seeded N(0,1) field on an n^3 periodic grid, smoothed by a Gaussian of
    width ``sigma`` voxels (periodic FFT filter) and standardised; [z][y][x]."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((n, n, n))
    k = np.fft.fftfreq(n)
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    filt = np.exp(-2.0 * (np.pi * sigma) ** 2 * (kx ** 2 + ky ** 2 + kz ** 2))
    s = np.real(np.fft.ifftn(np.fft.fftn(g) * filt))
    return (s - s.mean()) / s.std()


def pillars_field(n: int = 64, seed: int = 4, layer_scale=(1.0, 1.0, 1.0)):
    """Two 8 x 8 x 48 conductor pillars (x in [12,20) and [44,52), y in
    [28,36), z in [8,56)) in a dielectric whose per-voxel permittivity is
    eps_v = s_L * (1 + 6 sigmoid(g_v)), g a smoothed seeded Gaussian field
    (sigma = 4 voxels) and L the z-third of the voxel.  Every dielectric voxel
    has its own label, so a per-label gradient is a per-voxel gradient.

    Returns (workload, base, layer_of_label) where base[v] = 1 + 6 sigmoid(g)
    and layer_of_label[label] in {0,1,2} (-1 for conductor labels)."""
    g = smooth_field(n, 4.0, seed)
    base = 1.0 + 6.0 / (1.0 + np.exp(-g))
    # z-thirds [0,21), [21,42), [42,64) at n = 64
    bounds = [0, round(n * 21 / 64), round(n * 42 / 64), n]
    layer = np.zeros((n, n, n), np.int64)
    for L in range(3):
        layer[bounds[L]:bounds[L + 1]] = L
    sc = np.asarray(layer_scale, dtype=np.float64)
    eps_vox = sc[layer] * base
    nvox = n ** 3
    lab = np.arange(nvox, dtype=np.int64).reshape(n, n, n)
    cond = np.zeros((n, n, n), bool)
    s8 = n // 8
    zlo, zhi = n // 8, n - n // 8
    for x0 in (12 * n // 64, 44 * n // 64):
        cond[zlo:zhi, 28 * n // 64:28 * n // 64 + s8, x0:x0 + s8] = True
    lab[cond & (np.arange(n)[None, None, :] < n // 2)] = nvox
    lab[cond & (np.arange(n)[None, None, :] >= n // 2)] = nvox + 1
    cid = np.full(nvox + 2, -1, np.int32)
    cid[nvox] = 0
    cid[nvox + 1] = 1
    eps = np.concatenate([eps_vox.reshape(-1), [1.0, 1.0]])
    layer_of_label = np.concatenate([layer.reshape(-1), [-1, -1]])
    base_of_label = np.concatenate([base.reshape(-1), [1.0, 1.0]])
    wl = Workload(f"pillars_field_{n}^3", lab.astype(np.int32), cid, eps)
    return wl, base_of_label, layer_of_label


def meanders(nx: int = 512, ny: int = 512, nz: int = 64, legs: int = 32) -> Workload:
    """Two interleaved meander conductors: a double-track serpentine.  The two
    tracks (width 4, spacing 4, thickness 8 at z in [28,36) for nz = 64) run
    side by side along ``legs`` legs parallel to y, y in [16, ny-16), at an x
    pitch of 16, joined by nested U-turns (the outer track turns 4 voxels
    beyond the leg ends, the inner track 4 voxels short of them, 4 voxels
    apart).  The whole grid is a dielectric with eps_r = 3.9."""
    lab = np.zeros((nz, ny, nx), np.int32)      # label 0: dielectric
    A, B = 1, 2
    z0, z1 = 28 * nz // 64, 36 * nz // 64
    ylo, yhi = 16, ny - 16
    for j in range(legs):
        x0 = 2 + 16 * j
        left, right = (A, B) if j % 2 == 0 else (B, A)
        lab[z0:z1, ylo:yhi, x0:x0 + 4] = left
        lab[z0:z1, ylo:yhi, x0 + 8:x0 + 12] = right
    for j in range(legs - 1):
        x0 = 2 + 16 * j
        left, right = (A, B) if j % 2 == 0 else (B, A)
        outer, inner = left, right          # every turn bends towards +x
        if j % 2 == 0:                      # turn at the top
            lab[z0:z1, yhi:yhi + 4, x0:x0 + 28] = outer
            lab[z0:z1, yhi - 4:yhi, x0 + 8:x0 + 12] = 0
            lab[z0:z1, yhi - 4:yhi, x0 + 16:x0 + 20] = 0
            lab[z0:z1, yhi - 8:yhi - 4, x0 + 8:x0 + 20] = inner
        else:                               # turn at the bottom
            lab[z0:z1, ylo - 4:ylo, x0:x0 + 28] = outer
            lab[z0:z1, ylo:ylo + 4, x0 + 8:x0 + 12] = 0
            lab[z0:z1, ylo:ylo + 4, x0 + 16:x0 + 20] = 0
            lab[z0:z1, ylo + 4:ylo + 8, x0 + 8:x0 + 20] = inner
    return Workload(f"meanders_{nx}x{ny}x{nz}", lab,
                    np.array([-1, 0, 1], np.int32), np.array([3.9, 1.0, 1.0]))


def coated_sphere(n: int = 20, eps_coat: float = 2.0) -> Workload:
    """PEC sphere of radius n/4 voxels coated by a dielectric shell of radius
    n/2 voxels (voxel centres strictly inside each radius), on an n^3 grid:
    the paper's Sec. III.A structure (r_c = 0.25 m, r_d = 0.5 m) at voxel
    edge 1/n m."""
    c = (np.arange(n) + 0.5) - n / 2
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    R = np.sqrt(X * X + Y * Y + Z * Z)
    lab = np.zeros((n, n, n), np.int32)
    lab[R < n / 2] = 1
    lab[R < n / 4] = 2
    return Workload(f"coated_sphere_{n}^3", lab, np.array([-1, -1, 0], np.int32),
                    np.array([1.0, eps_coat, 1.0]), voxel_size=1.0 / n)


def random_structure(shape=(7, 5, 6), seed: int = 0, n_cond: int = 2, n_diel: int = 3,
                     fill: float = 0.5) -> Workload:
    """A small seeded structure on a (nx, ny, nz) grid for parity tests: each
    voxel gets one of ``n_diel`` dielectric labels (random eps_r in [1.5, 8];
    label 0 is vacuum when ``fill`` < 1) and ``n_cond`` conductor boxes are
    carved in, kept one voxel apart so that no two conductors touch."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    lab = rng.integers(1, n_diel + 1, size=(nz, ny, nx)).astype(np.int32)
    lab[rng.random((nz, ny, nx)) > fill] = 0
    eps = np.concatenate([[1.0], 1.5 + 6.5 * rng.random(n_diel), np.ones(n_cond)])
    cid = np.concatenate([np.full(n_diel + 1, -1), np.arange(n_cond)]).astype(np.int32)
    taken = np.zeros((nz, ny, nx), bool)
    for c in range(n_cond):
        for _ in range(100):
            size = [int(rng.integers(1, max(2, d // 2) + 1)) for d in (nx, ny, nz)]
            lo = [int(rng.integers(0, d - s + 1)) for d, s in zip((nx, ny, nz), size)]
            sl = (slice(lo[2], lo[2] + size[2]), slice(lo[1], lo[1] + size[1]),
                  slice(lo[0], lo[0] + size[0]))
            grown = (slice(max(0, lo[2] - 1), lo[2] + size[2] + 1),
                     slice(max(0, lo[1] - 1), lo[1] + size[1] + 1),
                     slice(max(0, lo[0] - 1), lo[0] + size[0] + 1))
            if not taken[grown].any():
                lab[sl] = n_diel + 1 + c
                taken[sl] = True
                break
    return Workload(f"random{shape}_{seed}", lab, cid, eps)
