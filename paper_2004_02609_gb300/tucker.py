"""Installation stage of the Tucker enhancement (Sec. II.C, Eq. 13).

The four canonical Toeplitz tensors (parallel / orthogonal panel potentials
and their normal derivatives, normalised units) are generated once on a
D x D x D index cube by the device entry generator, compressed by a
truncated higher-order SVD to a relative Frobenius tolerance, and stored on
disk.  At set-up the library restores each of the 15 Toeplitz tensors of a
grid from these factors on the tensor cores (voxcap_tucker_expand), cropped
to the grid: see ``TuckerModel.as_ctypes`` and VoxCap(..., tucker=model).

    python -m paper_2004_02609_gb300.tucker --D 64 --tol 1e-6 --out tucker_D64.npz
"""
from __future__ import annotations

import argparse
import ctypes
from dataclasses import dataclass

import numpy as np

NAMES = ("ppar", "epar", "port", "eort")


def canonical_tensors(D: int):
    """The four canonical tensors on a D^3 cube as numpy arrays X[i, j, k]
    (mode 1 = first offset), generated on the GPU in FP64."""
    import torch
    from . import voxcap as V
    outs = [torch.empty(D * D * D, dtype=torch.float64, device="cuda") for _ in range(4)]
    torch.cuda.synchronize()
    V._check(V.lib().voxcap_canonical_tensors(D, *(V._ptr(o) for o in outs)))
    # device layout: first index fastest -> C-order array [k][j][i]
    return [o.cpu().numpy().reshape(D, D, D).transpose(2, 1, 0).copy() for o in outs]


def _leading_vectors(Xm: np.ndarray, energy_cut: float, rng) -> np.ndarray:
    """Left singular vectors of the unfolding Xm (rows x cols) whose discarded
    squared singular values sum to at most energy_cut.  Small unfoldings use
    a full SVD; large ones a randomized range finder (oversampled, one power
    iteration) followed by an SVD of the projection."""
    rows, cols = Xm.shape
    if rows * cols <= 4e7:
        U, s, _ = np.linalg.svd(Xm, full_matrices=False)
    else:
        k = min(rows, 96)
        Y = Xm @ rng.standard_normal((cols, k))
        Q, _ = np.linalg.qr(Y)
        Q, _ = np.linalg.qr(Xm @ (Xm.T @ Q))
        B = Q.T @ Xm
        Ub, s, _ = np.linalg.svd(B, full_matrices=False)
        U = Q @ Ub
    tail = np.concatenate([np.cumsum((s ** 2)[::-1])[::-1], [0.0]])
    r = next(i for i in range(1, len(s) + 1) if tail[i] <= energy_cut)
    return U[:, :r].copy()


def hosvd(X: np.ndarray, tol: float, seed: int = 0):
    """Truncated HOSVD with ||X - X~||_F <= tol ||X||_F (per-mode share tol^2/3)."""
    rng = np.random.default_rng(seed)
    nrm2 = float(np.sum(X * X))
    cut = tol * tol * nrm2 / 3.0
    Us = []
    for mode in range(3):
        Xm = np.moveaxis(X, mode, 0).reshape(X.shape[mode], -1)
        Us.append(_leading_vectors(Xm, cut, rng))
    core = np.einsum("ijk,ia,jb,kc->abc", X, Us[0], Us[1], Us[2], optimize=True)
    return core, Us


@dataclass
class TuckerModel:
    D: int
    tol: float
    cores: list      # 4 arrays [r1, r2, r3]
    factors: list    # 4 lists of 3 arrays [D, r]

    @property
    def ranks(self):
        return [tuple(c.shape) for c in self.cores]

    def nbytes(self):
        return sum(c.nbytes + sum(u.nbytes for u in us) for c, us in zip(self.cores, self.factors))

    def save(self, path):
        d = {"D": self.D, "tol": self.tol}
        for t, n in enumerate(NAMES):
            d[f"{n}_core"] = self.cores[t]
            for m in range(3):
                d[f"{n}_U{m}"] = self.factors[t][m]
        np.savez(path, **d)

    @staticmethod
    def load(path):
        z = np.load(path)
        cores = [z[f"{n}_core"] for n in NAMES]
        factors = [[z[f"{n}_U{m}"] for m in range(3)] for n in NAMES]
        return TuckerModel(int(z["D"]), float(z["tol"]), cores, factors)

    def as_ctypes(self):
        """A voxcap_tucker struct pointing at this model's arrays (keep the
        model alive while the struct is in use)."""
        from .voxcap import Tucker
        t = Tucker()
        self._keep = []
        for i in range(4):
            c = np.ascontiguousarray(self.cores[i], dtype=np.float64)
            self._keep.append(c)
            t.core[i] = c.ctypes.data
            for m in range(3):
                u = np.ascontiguousarray(self.factors[i][m], dtype=np.float64)
                self._keep.append(u)
                t.dims[i][m] = u.shape[0]
                t.ranks[i][m] = u.shape[1]
                t.factor[i][m] = u.ctypes.data
        return t


def install(D: int, tol: float) -> TuckerModel:
    """Generate and compress the canonical tensors on a D^3 cube (grids with
    max(nx, ny, nz) < D can be restored from the result)."""
    Xs = canonical_tensors(D)
    cores, factors = [], []
    for X in Xs:
        core, Us = hosvd(X, tol)
        cores.append(core)
        factors.append(Us)
    return TuckerModel(D, tol, cores, factors)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--D", type=int, default=64)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    m = install(a.D, a.tol)
    out = a.out or f"tucker_D{a.D}_tol{a.tol:g}.npz"
    m.save(out)
    print(out, "ranks", m.ranks, "bytes", m.nbytes())


if __name__ == "__main__":
    main()
