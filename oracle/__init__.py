"""ORACLE for the VoxCap hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The product library never links, imports or
executes anything here, and this package imports nothing from the product.

A plain, slow, FP64 CPU restatement of what the paper's method computes,
each function citing the passage it follows (arxiv 2004.02609):

* ``panels``         -- conductor / dielectric surface panels of a voxel grid
                        (Sec. II.A, Eqs. 3-4 and 7; Sec. II.B for the x/y/z
                        face grids).
* ``entries``        -- Galerkin integrals P' (Eq. 5) and E' (Eq. 6) of one
                        panel pair, by the C code in ``entries.c`` (closed-form
                        rectangle potential inside, adaptive quadrature outside).
* ``dense_matrix``   -- the N x N system of Eq. 4 in normalised units.
* ``capacitance``    -- unit-potential solves by LU and Eq. 8, with the
                        free-charge scaling of conductors in a dielectric.
* ``precond_apply``  -- block-diagonal-diagonal preconditioner of Eq. 14
                        (Sec. II.D) and the conventional variants used for
                        comparison in Sec. III.A.
* ``capacitance_grad`` -- dC/d(eps) by a dense adjoint solve, with the
                        limit of Eq. 7 for faces between equal
                        permittivities (``equal_eps_faces``), which carry
                        no panel but gain one as soon as a side changes.
* ``tucker_hosvd`` / ``tucker_expand`` -- Eq. 13 (truncated HOSVD, einsum).
* ``fft_gmres``      -- (module) the FFT-accelerated product of Eqs. 9-11 by
                        directly evaluated circulant kernels and scipy FFTs,
                        and GMRES(35) (Sec. III) on it: the CPU counterpart of
                        the method for grids too large for the dense LU,
                        checked against ``dense_matrix`` on small grids.

Normalised units: voxel edge 1 and G' = 1/(4 pi r).  A physical system with
voxel edge dv scales P by dv^3/eps0 and E, I by dv^2/eps0 (Appendix C); the
charges then scale as rho = (eps0/dv) rho' and C = eps0 * dv * C'.

Readings of the paper that this oracle takes:
* every panel normal is the +axis direction; side ``a`` is the voxel on the
  -axis side of the face and side ``b`` the +axis side; a dielectric panel has
  I' = (eps_a + eps_b) / (2 (eps_a - eps_b)) (Eq. 7 with the normal oriented
  from a to b) and E' is the derivative along +axis;
* outside the bounding box is vacuum (eps_r = 1, not a conductor);
* a conductor panel's free-charge factor is eps_r of its non-conductor side;
* two different conductors sharing a face is an error (short circuit).
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

EPS0 = 8.8541878128e-12   # F/m (CODATA 2018); the paper gives no value


class ShortCircuitError(ValueError):
    """Two different conductors share a voxel face."""


# --------------------------------------------------------------------------
# C entry integrals (Eqs. 5, 6)
# --------------------------------------------------------------------------
_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        lib.oracle_entry.restype = ctypes.c_double
        lib.oracle_entry.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double]
        lib.oracle_square_field.restype = ctypes.c_double
        lib.oracle_square_field.argtypes = [ctypes.c_int, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_double]
        lib.oracle_entries.restype = None
        lib.oracle_entries.argtypes = [ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_double,
                                       ctypes.c_void_p]
        _LIB = lib
    return _LIB


def entry(kind: int, test_orient: int, src_orient: int, d, rtol: float = 1e-13) -> float:
    """One Galerkin integral: kind 0 = P' (Eq. 5), kind 1 = E' (Eq. 6).

    ``d`` is the test-panel centre minus the source-panel centre (voxel units).
    """
    return _lib().oracle_entry(int(kind), int(test_orient), int(src_orient),
                               float(d[0]), float(d[1]), float(d[2]), float(rtol))


def entries(kind, test_orient, src_orient, d, rtol: float = 1e-13) -> np.ndarray:
    """Vectorised ``entry`` (OpenMP across entries in C)."""
    kind = np.ascontiguousarray(np.broadcast_to(kind, (len(d),)), dtype=np.int32)
    to = np.ascontiguousarray(np.broadcast_to(test_orient, (len(d),)), dtype=np.int32)
    so = np.ascontiguousarray(np.broadcast_to(src_orient, (len(d),)), dtype=np.int32)
    dd = np.ascontiguousarray(d, dtype=np.float64).reshape(-1, 3)
    out = np.empty(len(dd), dtype=np.float64)
    if len(dd):
        _lib().oracle_entries(len(dd), kind.ctypes.data, to.ctypes.data, so.ctypes.data,
                              dd.ctypes.data, float(rtol), out.ctypes.data)
    return out


def square_field(which: int, X: float, Y: float, Z: float) -> float:
    """Potential (which=0) or its d/dX, d/dY, d/dZ (1, 2, 3) of the unit-density
    square [-1/2,1/2]^2 in the plane Z=0, without the 1/(4 pi) factor."""
    return _lib().oracle_square_field(int(which), float(X), float(Y), float(Z))


# --------------------------------------------------------------------------
# Panels (Sec. II.A-B)
# --------------------------------------------------------------------------
@dataclass
class PanelSet:
    nx: int
    ny: int
    nz: int
    orient: np.ndarray      # int8, 0/1/2 = normal along x/y/z
    face: np.ndarray        # int32, linear index in that orientation's face grid
    kind: np.ndarray        # int8, 0 = conductor row, 1 = dielectric row
    owner: np.ndarray       # int16, conductor index (-1 for dielectric panels)
    idiag: np.ndarray       # float64, I' of Eq. 7 (0 for conductor panels)
    qscale: np.ndarray      # float64, free-charge factor eps_r (0 for dielectric)
    label_a: np.ndarray     # int32, label of the -axis side voxel (-1 = outside)
    label_b: np.ndarray     # int32, label of the +axis side voxel (-1 = outside)
    n_conductors: int
    centers: np.ndarray = field(repr=False)   # (N, 3) float64 panel centres

    @property
    def n(self) -> int:
        return len(self.orient)

    @property
    def n_cond(self) -> int:
        return int(np.count_nonzero(self.kind == 0))

    @property
    def n_diel(self) -> int:
        return int(np.count_nonzero(self.kind == 1))


def face_grid_dims(nx: int, ny: int, nz: int, orient: int):
    """Dimensions (Fx, Fy, Fz) of the face grid of one orientation: the grid
    of x-normal faces is (N_x+1) x N_y x N_z, and likewise (Sec. II.B)."""
    dims = [nx, ny, nz]
    dims[orient] += 1
    return tuple(dims)


def _sides(arr3, orient, fill):
    """Values on the -axis side (a) and +axis side (b) of every face of one
    orientation.  ``arr3`` is indexed [z][y][x]; outside the grid = ``fill``."""
    ax = 2 - orient                       # numpy axis of the face normal
    pad = [(0, 0)] * 3
    pad[ax] = (1, 1)
    p = np.pad(arr3, pad, mode="constant", constant_values=fill)
    sl_a = [slice(None)] * 3
    sl_b = [slice(None)] * 3
    sl_a[ax] = slice(0, -1)
    sl_b[ax] = slice(1, None)
    return p[tuple(sl_a)], p[tuple(sl_b)]


def panels(labels, conductor_id, eps_r) -> PanelSet:
    """Conductor and dielectric panels of a labelled voxel grid.

    labels: int array [N_z][N_y][N_x] (x fastest) of material labels;
    conductor_id[label] >= 0 marks a conductor (its index), -1 a dielectric;
    eps_r[label] the relative permittivity (ignored for conductors).

    A face whose two voxels are one conductor and one non-conductor is a
    conductor panel (Eq. 1 tested on it); a face between two non-conductors
    of different permittivity is a dielectric panel (Eq. 2, with I' of Eq. 7);
    faces inside one conductor or between equal permittivities carry no panel.
    Panel order: conductor panels first, then dielectric (Eq. 4); within each,
    orientation x < y < z (Eq. 9), then ascending face index.
    """
    labels = np.asarray(labels)
    nz, ny, nx = labels.shape
    cid = np.asarray(conductor_id, dtype=np.int64)[labels]
    eps = np.asarray(eps_r, dtype=np.float64)[labels]
    lab = labels.astype(np.int64)
    per_kind = {0: [], 1: []}
    for o in range(3):
        ca, cb = _sides(cid, o, -1)
        ea, eb = _sides(eps, o, 1.0)
        la, lb = _sides(lab, o, -1)
        ca, cb, ea, eb, la, lb = (x.reshape(-1) for x in (ca, cb, ea, eb, la, lb))
        both = (ca >= 0) & (cb >= 0)
        if np.any(both & (ca != cb)):
            raise ShortCircuitError("two different conductors share a face")
        cond = (ca >= 0) ^ (cb >= 0)
        diel = (ca < 0) & (cb < 0) & (ea != eb)
        fidx = np.nonzero(cond)[0]
        owner = np.where(ca[fidx] >= 0, ca[fidx], cb[fidx])
        qs = np.where(ca[fidx] >= 0, eb[fidx], ea[fidx])
        per_kind[0].append((o, fidx, owner, np.zeros(len(fidx)), qs, la[fidx], lb[fidx]))
        didx = np.nonzero(diel)[0]
        a, b = ea[didx], eb[didx]
        idg = (a + b) / (2.0 * (a - b))
        per_kind[1].append((o, didx, -np.ones(len(didx), np.int64), idg,
                            np.zeros(len(didx)), la[didx], lb[didx]))
    cols = {k: [] for k in ("orient", "face", "kind", "owner", "idiag", "qscale", "la", "lb")}
    for kind in (0, 1):
        for (o, f, ow, idg, qs, la, lb) in per_kind[kind]:
            cols["orient"].append(np.full(len(f), o, np.int8))
            cols["face"].append(f.astype(np.int32))
            cols["kind"].append(np.full(len(f), kind, np.int8))
            cols["owner"].append(ow.astype(np.int16))
            cols["idiag"].append(idg.astype(np.float64))
            cols["qscale"].append(qs.astype(np.float64))
            cols["la"].append(la.astype(np.int32))
            cols["lb"].append(lb.astype(np.int32))
    cat = {k: np.concatenate(v) for k, v in cols.items()}
    ncond = int(np.max(np.asarray(conductor_id)) + 1) if np.any(np.asarray(conductor_id) >= 0) else 0
    ps = PanelSet(nx, ny, nz, cat["orient"], cat["face"], cat["kind"], cat["owner"],
                  cat["idiag"], cat["qscale"], cat["la"], cat["lb"], ncond,
                  centers=np.zeros((0, 3)))
    ps.centers = panel_centers(ps)
    return ps


def face_coords(ps: PanelSet, orient=None, face=None):
    """Integer face-grid coordinates (i, j, k) of each panel."""
    orient = ps.orient if orient is None else orient
    face = ps.face if face is None else face
    out = np.zeros((len(face), 3), dtype=np.int64)
    for o in range(3):
        m = orient == o
        fx, fy, _ = face_grid_dims(ps.nx, ps.ny, ps.nz, o)
        f = face[m].astype(np.int64)
        out[m, 0] = f % fx
        out[m, 1] = (f // fx) % fy
        out[m, 2] = f // (fx * fy)
    return out


def panel_centers(ps: PanelSet) -> np.ndarray:
    """Panel centres: the x-face (i,j,k) sits at (i, j+1/2, k+1/2), etc."""
    c = face_coords(ps).astype(np.float64) + 0.5
    for o in range(3):
        m = ps.orient == o
        c[m, o] -= 0.5
    return c


# --------------------------------------------------------------------------
# Dense system (Eq. 4) and products
# --------------------------------------------------------------------------
def dense_matrix(ps: PanelSet, rtol: float = 1e-13) -> np.ndarray:
    """A = [P'; E'] + diag(0, I') in normalised units (Eqs. 4-7).

    Rows of conductor panels hold P'_kl (Eq. 5); rows of dielectric panels hold
    E'_kl (Eq. 6) plus I'_k on the diagonal (Eq. 7).  Entries depend only on
    the two orientations and the centre difference, so each distinct
    (row kind, orientations, difference) is integrated once.
    """
    n = ps.n
    c2 = np.rint(2.0 * ps.centers).astype(np.int64)       # exact half-integers
    span = int(2 * (max(ps.nx, ps.ny, ps.nz) + 2))
    W = 2 * span + 1
    kr = ps.kind.astype(np.int64)
    orr = ps.orient.astype(np.int64)
    key = np.empty((n, n), dtype=np.int64)
    for k0 in range(0, n, 2048):
        k1 = min(n, k0 + 2048)
        d = c2[k0:k1, None, :] - c2[None, :, :] + span
        kk = ((kr[k0:k1, None] * 3 + orr[k0:k1, None]) * 3 + orr[None, :])
        key[k0:k1] = ((kk * W + d[..., 0]) * W + d[..., 1]) * W + d[..., 2]
    uniq, inv = np.unique(key.reshape(-1), return_inverse=True)
    dz = uniq % W - span
    rest = uniq // W
    dy = rest % W - span
    rest //= W
    dx = rest % W - span
    rest //= W
    ol = rest % 3
    rest //= 3
    ot = rest % 3
    kd = rest // 3
    vals = entries(kd, ot, ol, np.stack([dx, dy, dz], 1) / 2.0, rtol=rtol)
    A = vals[inv].reshape(n, n)
    diel = np.nonzero(ps.kind == 1)[0]
    A[diel, diel] += ps.idiag[diel]
    return A


def matvec(A: np.ndarray, x: np.ndarray) -> np.ndarray:
    """y = A x (the product the FFT method accelerates, Eqs. 9-11)."""
    return A @ x


def rhs_unit_potentials(ps: PanelSet) -> np.ndarray:
    """B[:, i]: unit potential on conductor i, zero on the others (Sec. II.A
    before Eq. 8); V_k = A_k Phi_k with A_k = 1 in voxel units; dielectric
    rows are 0 (Eq. 4)."""
    B = np.zeros((ps.n, ps.n_conductors))
    cond = np.nonzero(ps.kind == 0)[0]
    B[cond, ps.owner[cond]] = 1.0
    return B


def charge_weights(ps: PanelSet) -> np.ndarray:
    """W[:, i]: w_i,k = A_k * eps_r(k) on conductor i's panels (Eq. 8 with the
    free-charge scaling of conductors embedded in a dielectric)."""
    W = np.zeros((ps.n, ps.n_conductors))
    cond = np.nonzero(ps.kind == 0)[0]
    W[cond, ps.owner[cond]] = ps.qscale[cond]
    return W


def capacitance(ps: PanelSet, A: np.ndarray | None = None, voxel_size: float = 1.0,
                rtol: float = 1e-13):
    """Capacitance matrix (Eq. 8) by dense LU.

    Returns (C in farads, C' normalised, charges rho' [N x m])."""
    if A is None:
        A = dense_matrix(ps, rtol=rtol)
    B = rhs_unit_potentials(ps)
    X = np.linalg.solve(A, B)
    Cn = charge_weights(ps).T @ X
    return EPS0 * voxel_size * Cn, Cn, X


# --------------------------------------------------------------------------
# Preconditioner (Eq. 14, Sec. II.D)
# --------------------------------------------------------------------------
def panel_boxes(ps: PanelSet, nv) -> np.ndarray:
    """Small-box index of every panel.  Boxes hold nv[a] voxels along axis a;
    a face at index i along its own normal axis belongs to box
    min(i // nv, n_boxes - 1) (so the far boundary faces join the last box),
    and to box j // nv along the other axes."""
    nv = np.broadcast_to(np.asarray(nv, dtype=np.int64), (3,))
    dims = np.array([ps.nx, ps.ny, ps.nz])
    nb = (dims + nv - 1) // nv
    fc = face_coords(ps)
    bc = fc // nv
    bc = np.minimum(bc, nb - 1)
    return bc[:, 0] + nb[0] * (bc[:, 1] + nb[1] * bc[:, 2])


def precond_matrix(ps: PanelSet, A: np.ndarray, nv=10, kind: str = "bdd") -> np.ndarray:
    """The dense preconditioner R of Eq. 14 (and its comparison variants).

    bdd: conductor rows -- inverse of the conductor-conductor block of each
         small box; dielectric rows -- 1/I' (the paper's proposal).
    bd:  all panels of each small box form the block (conventional
         block-diagonal).
    diag: 1/A_kk.   none: identity.
    """
    n = ps.n
    R = np.zeros((n, n))
    if kind == "none":
        return np.eye(n)
    if kind == "diag":
        return np.diag(1.0 / np.diag(A))
    box = panel_boxes(ps, nv)
    if kind == "bdd":
        sel = ps.kind == 0
        diel = np.nonzero(ps.kind == 1)[0]
        R[diel, diel] = 1.0 / ps.idiag[diel]
    elif kind == "bd":
        sel = np.ones(n, bool)
    else:
        raise ValueError(kind)
    for b in np.unique(box[sel]):
        S = np.nonzero(sel & (box == b))[0]
        R[np.ix_(S, S)] = np.linalg.inv(A[np.ix_(S, S)])
    return R


def unique_box_patterns(ps: PanelSet, nv=10) -> int:
    """Number of distinct conductor-panel patterns over the small boxes (the
    unique blocks of R_BD that need storing, Sec. II.D point (ii))."""
    nv3 = np.broadcast_to(np.asarray(nv, dtype=np.int64), (3,))
    box = panel_boxes(ps, nv3)
    dims = np.array([ps.nx, ps.ny, ps.nz])
    nb = (dims + nv3 - 1) // nv3
    fc = face_coords(ps)
    pats = set()
    cond = np.nonzero(ps.kind == 0)[0]
    for b in np.unique(box[cond]):
        S = cond[box[cond] == b]
        bz, rest = divmod(int(b), int(nb[0] * nb[1]))
        by, bx = divmod(rest, int(nb[0]))
        origin = np.array([bx, by, bz]) * nv3
        local = fc[S] - origin
        pats.add(tuple(sorted(zip(ps.orient[S].tolist(), map(tuple, local.tolist())))))
    return len(pats)


# --------------------------------------------------------------------------
# Adjoint gradient of the capacitance matrix
# --------------------------------------------------------------------------
def capacitance_grad(labels, conductor_id, eps_r, dL_dC, voxel_size: float = 1.0,
                     rtol: float = 1e-13):
    """dL/d(eps_r[label]) for L = sum_ij dL_dC[i,j] * C_ij, by one dense
    adjoint solve.

    C_ij = eps0 dv * w_i^T rho_j, A rho_j = b_j (Eqs. 4, 8).  Only I' on the
    dielectric rows (Eq. 7) and the free-charge factors w depend on eps, so
      dL/dth = eps0 dv * sum_ij G_ij [ (dw_i/dth)^T rho_j - lam_i^T (dA/dth) rho_j ],
    with A^T lam_i = w_i.

    A face between two non-conductors of equal permittivity eps carries no
    panel, but it becomes one as soon as either side changes: with eps_a =
    eps + d its I' = (2 eps + d) / (2 d) is large, the new panel's charge is
    -(r^T rho_j) / I' to first order (r: the E' row of the face against the
    existing panels, so r^T rho_j is the normal field there), and through the
    column c of the new panel (P' on conductor rows, E' on dielectric rows)
    C_ij changes by eps0 dv (lam_i^T c)(r^T rho_j) d / eps.  So such a face adds
    +eps0 dv (c^T lam_i)(r^T rho_j) / eps to dC_ij/d(eps_a) and the negative
    of that to dC_ij/d(eps_b) (Eq. 7 in the limit of equal sides; vacuum
    outside the box is a fixed eps = 1).
    Returns (grad [n_labels], C [m x m] farads).
    """
    ps = panels(labels, conductor_id, eps_r)
    A = dense_matrix(ps, rtol=rtol)
    B = rhs_unit_potentials(ps)
    W = charge_weights(ps)
    X = np.linalg.solve(A, B)
    G = np.asarray(dL_dC, dtype=np.float64)
    Mu = np.linalg.solve(A.T, W @ G)          # mu_j = sum_i G_ij lam_i
    eps_r = np.asarray(eps_r, dtype=np.float64)
    grad = np.zeros(len(eps_r))
    scale = EPS0 * voxel_size
    # free-charge factors: w_{i,k} = eps_r(non-conductor side of k)
    cond = np.nonzero(ps.kind == 0)[0]
    for k in cond:
        la, lb = ps.label_a[k], ps.label_b[k]
        other = lb if (la >= 0 and conductor_id[la] >= 0) else la
        if other < 0:
            continue                        # vacuum outside the box: fixed
        i = ps.owner[k]
        grad[other] += scale * float(G[i, :] @ X[k, :])
    # dielectric diagonal: I' = (ea+eb)/(2(ea-eb))
    diel = np.nonzero(ps.kind == 1)[0]
    for k in diel:
        la, lb = ps.label_a[k], ps.label_b[k]
        ea = eps_r[la] if la >= 0 else 1.0
        eb = eps_r[lb] if lb >= 0 else 1.0
        dIa = -eb / (ea - eb) ** 2
        dIb = ea / (ea - eb) ** 2
        t = float(Mu[k, :] @ X[k, :])
        if la >= 0:
            grad[la] -= scale * dIa * t
        if lb >= 0:
            grad[lb] -= scale * dIb * t
    # faces without a panel between equal permittivities (the limit above)
    ef = equal_eps_faces(labels, conductor_id, eps_r)
    if len(ef["orient"]):
        c2p = np.rint(2.0 * ps.centers).astype(np.int64)
        for f in range(len(ef["orient"])):
            of, cf = int(ef["orient"][f]), ef["center"][f]
            d = (np.rint(2.0 * cf).astype(np.int64) - c2p) / 2.0        # face minus panels
            r = entries(1, of, ps.orient, d, rtol=rtol)                   # E'(face <- panel l)
            c = entries(ps.kind, ps.orient, of, -d, rtol=rtol)            # A(panel k <- face)
            t = float((r @ X) @ (c @ Mu))
            e = float(ef["eps"][f])
            la, lb = int(ef["label_a"][f]), int(ef["label_b"][f])
            if la >= 0:
                grad[la] += scale * t / e
            if lb >= 0:
                grad[lb] -= scale * t / e
    C = scale * (W.T @ X)
    return grad, C


def equal_eps_faces(labels, conductor_id, eps_r) -> dict:
    """Faces between two non-conductor voxels (or a voxel and the vacuum
    outside the box) of equal permittivity: they carry no panel (Sec. II.A).
    Returns orient, face index, labels of the -axis (a) and +axis (b) sides
    (-1 outside), the common eps and the face centres."""
    labels = np.asarray(labels)
    nz, ny, nx = labels.shape
    cid = np.asarray(conductor_id, dtype=np.int64)[labels]
    eps = np.asarray(eps_r, dtype=np.float64)[labels]
    lab = labels.astype(np.int64)
    out = {k: [] for k in ("orient", "face", "label_a", "label_b", "eps")}
    for o in range(3):
        ca, cb = _sides(cid, o, -1)
        ea, eb = _sides(eps, o, 1.0)
        la, lb = _sides(lab, o, -1)
        ca, cb, ea, eb, la, lb = (x.reshape(-1) for x in (ca, cb, ea, eb, la, lb))
        idx = np.nonzero((ca < 0) & (cb < 0) & (ea == eb) & ((la >= 0) | (lb >= 0)))[0]
        out["orient"].append(np.full(len(idx), o, np.int8))
        out["face"].append(idx.astype(np.int64))
        out["label_a"].append(la[idx])
        out["label_b"].append(lb[idx])
        out["eps"].append(ea[idx])
    out = {k: np.concatenate(v) for k, v in out.items()}
    tmp = PanelSet(nx, ny, nz, out["orient"], out["face"], np.zeros(len(out["face"]), np.int8),
                   np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0), 0, centers=np.zeros((0, 3)))
    out["center"] = panel_centers(tmp)
    return out


# --------------------------------------------------------------------------
# Tucker decomposition (Eq. 13)
# --------------------------------------------------------------------------
def tucker_hosvd(X: np.ndarray, tol: float):
    """Truncated higher-order SVD: X ~ S x1 U1 x2 U2 x3 U3 (Eq. 13).

    Each mode keeps the fewest leading singular vectors whose discarded
    energy is at most (tol^2/3) ||X||_F^2, so ||X - X~||_F <= tol ||X||_F."""
    X = np.asarray(X, dtype=np.float64)
    nrm2 = float(np.sum(X * X))
    Us = []
    for mode in range(3):
        Xm = np.moveaxis(X, mode, 0).reshape(X.shape[mode], -1)
        U, s, _ = np.linalg.svd(Xm, full_matrices=False)
        tail = np.cumsum((s ** 2)[::-1])[::-1]          # tail[r] = sum_{i>=r} s_i^2
        r = len(s)
        for cand in range(1, len(s) + 1):
            rest = tail[cand] if cand < len(s) else 0.0
            if rest <= tol * tol * nrm2 / 3.0:
                r = cand
                break
        Us.append(U[:, :r].copy())
    S = np.einsum("ijk,ia,jb,kc->abc", X, Us[0], Us[1], Us[2], optimize=True)
    return S, Us[0], Us[1], Us[2]


def tucker_expand(S, U1, U2, U3) -> np.ndarray:
    """X~ = S x1 U1 x2 U2 x3 U3 (Eq. 13), FP64 einsum."""
    return np.einsum("abc,ia,jb,kc->ijk", S, U1, U2, U3, optimize=True)
