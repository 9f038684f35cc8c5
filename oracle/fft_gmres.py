"""FFT-accelerated product and GMRES(35) in plain FP64 on the CPU -- part of
the ORACLE, TEST INFRASTRUCTURE ONLY (see the package header: only tests,
the smoke check and the bench's CPU legs may use it).

The product of Eqs. 9-11.  For a test orientation a and a source orientation
b, the interaction of the two face grids (Sec. II.B) is a discrete
convolution over integer index offsets n:

    y_a[i] = sum_b sum_i' K_ab(i - i') x_b[i'],

where K_ab(n) is the Galerkin integral at the centre difference
n + c_a - c_b (c_o = centre of face (0,0,0) of orientation o): Eq. 5 for the
rows of conductor panels, Eq. 6 for the rows of dielectric panels, which also
add I' x (Eq. 7).  Every K_ab is evaluated directly at every offset by the
oracle's integrals (no symmetry or parity is used), placed in a circulant of
the paper's size M = 2(N + 1) per axis (Appendix B: large enough that the
circular convolution equals the linear one), and applied with scipy's FFTs.

GMRES(35) (Sec. III) solves Eq. 4 with this product from x0 = 0; the
capacitance follows Eq. 8 as in the dense oracle.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft
from scipy.sparse.linalg import LinearOperator, gmres

from . import EPS0, charge_weights, entries, face_coords, face_grid_dims, rhs_unit_potentials


def _face_origin(o: int) -> np.ndarray:
    """Centre of face (0,0,0) of orientation o: the x-face (i,j,k) sits at
    (i, j + 1/2, k + 1/2), and likewise for y and z (Sec. II.B)."""
    c = np.full(3, 0.5)
    c[o] = 0.0
    return c


class FFTProduct:
    """y = A x for the panels of ``ps`` (a PanelSet) by circulant FFTs."""

    def __init__(self, ps, rtol: float = 1e-12, workers: int | None = None):
        self.ps = ps
        self.workers = workers
        self.M = (2 * (ps.nx + 1), 2 * (ps.ny + 1), 2 * (ps.nz + 1))
        self.F = [face_grid_dims(ps.nx, ps.ny, ps.nz, o) for o in range(3)]
        self.ijk = face_coords(ps)
        Mx, My, Mz = self.M
        self.K = {}
        for kind in (0, 1):
            for a in range(3):
                for b in range(3):
                    Fa, Fb = self.F[a], self.F[b]
                    axes = [np.arange(-(Fb[t] - 1), Fa[t]) for t in range(3)]
                    nx_, ny_, nz_ = (v.ravel() for v in np.meshgrid(*axes, indexing="ij"))
                    d = np.stack([nx_, ny_, nz_], 1) + (_face_origin(a) - _face_origin(b))
                    vals = entries(kind, a, b, d, rtol=rtol)
                    circ = np.zeros((Mz, My, Mx))
                    circ[nz_ % Mz, ny_ % My, nx_ % Mx] = vals
                    self.K[(kind, a, b)] = sfft.rfftn(circ, workers=workers)

    @classmethod
    def timing_stand_in(cls, ps, workers: int | None = None):
        """The same product with every kernel spectrum replaced by one shared
        array of ones, for timing grids whose kernels are too many to
        integrate here: the FFTs, the multiply-accumulate and the scatter /
        gather do exactly the work of the real product, whose cost does not
        depend on the spectra's values.  Its results are meaningless."""
        self = cls.__new__(cls)
        self.ps = ps
        self.workers = workers
        self.M = (2 * (ps.nx + 1), 2 * (ps.ny + 1), 2 * (ps.nz + 1))
        self.F = [face_grid_dims(ps.nx, ps.ny, ps.nz, o) for o in range(3)]
        self.ijk = face_coords(ps)
        Mx, My, Mz = self.M
        ones = np.ones((Mz, My, Mx // 2 + 1), np.complex128)
        self.K = {(kind, a, b): ones for kind in (0, 1) for a in range(3) for b in range(3)}
        return self

    def __call__(self, x: np.ndarray) -> np.ndarray:
        ps = self.ps
        Mx, My, Mz = self.M
        X = []
        for b in range(3):
            grid = np.zeros((Mz, My, Mx))
            m = ps.orient == b
            ijk = self.ijk[m]
            grid[ijk[:, 2], ijk[:, 1], ijk[:, 0]] = x[m]
            X.append(sfft.rfftn(grid, workers=self.workers))
        y = np.zeros(ps.n)
        for a in range(3):
            for kind in (0, 1):
                rows = (ps.orient == a) & (ps.kind == kind)
                if not rows.any():
                    continue
                acc = self.K[(kind, a, 0)] * X[0] + self.K[(kind, a, 1)] * X[1] + self.K[(kind, a, 2)] * X[2]
                ya = sfft.irfftn(acc, s=(Mz, My, Mx), workers=self.workers)
                ijk = self.ijk[rows]
                y[rows] = ya[ijk[:, 2], ijk[:, 1], ijk[:, 0]]
        diel = ps.kind == 1
        y[diel] += ps.idiag[diel] * x[diel]
        return y


def solve_fft(ps, B: np.ndarray, tol: float = 1e-10, product: FFTProduct | None = None,
              maxiter: int = 200):
    """GMRES(35) on A X = B column by column (x0 = 0, relative residual tol).
    Returns (X, iterations per column)."""
    A = product if product is not None else FFTProduct(ps)
    op = LinearOperator((ps.n, ps.n), matvec=A, dtype=np.float64)
    X = np.zeros_like(B, dtype=np.float64)
    its = []
    for c in range(B.shape[1]):
        count = [0]

        def cb(_):
            count[0] += 1

        try:
            x, info = gmres(op, B[:, c], rtol=tol, atol=0.0, restart=35, maxiter=maxiter,
                            callback=cb, callback_type="pr_norm")
        except TypeError:           # scipy before 1.12 names the tolerance `tol`
            x, info = gmres(op, B[:, c], tol=tol, atol=0.0, restart=35, maxiter=maxiter,
                            callback=cb, callback_type="pr_norm")
        if info != 0:
            raise RuntimeError(f"GMRES did not reach {tol} (info {info})")
        X[:, c] = x
        its.append(count[0])
    return X, its


def capacitance_fft(ps, voxel_size: float = 1.0, tol: float = 1e-10, product: FFTProduct | None = None):
    """Capacitance matrix (Eq. 8) by FFT-GMRES(35).  Returns (C in farads,
    C' normalised, charges rho' [N x m], iterations per conductor)."""
    X, its = solve_fft(ps, rhs_unit_potentials(ps), tol=tol, product=product)
    Cn = charge_weights(ps).T @ X
    return EPS0 * voxel_size * Cn, Cn, X, its
