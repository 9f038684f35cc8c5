"""dC/d(eps) by the hand-written adjoint (through the C ABI) against the
oracle's dense adjoint and against central finite differences."""
import numpy as np
import pytest

import oracle as O
from paper_2004_02609_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2004_02609_gb300 import build
    build.build()


def _tiny(seed, n=(5, 4, 4)):
    """per-voxel labels with distinct permittivities plus two conductors"""
    nx, ny, nz = n
    rng = np.random.default_rng(seed)
    nv = nx * ny * nz
    lab = np.arange(nv, dtype=np.int32).reshape(nz, ny, nx)
    lab[0:2, 0:2, 0:2] = nv
    lab[2:4, 2:4, 3:5] = nv + 1
    cid = np.full(nv + 2, -1, np.int32)
    cid[nv], cid[nv + 1] = 0, 1
    eps = np.concatenate([1.5 + 4 * rng.random(nv), [1.0, 1.0]])
    return lab, cid, eps


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_gradient_matches_dense_adjoint(precision):
    from paper_2004_02609_gb300 import voxcap as V
    lab, cid, eps = _tiny(0)
    G = np.array([[1.0, 0.3], [-0.7, 2.0]])
    gref, Cref = O.capacitance_grad(lab, cid, eps, G, voxel_size=1e-6, rtol=1e-13)
    vc = V.VoxCap(lab, cid, eps, 1e-6, precision=precision, nv=3, entries="fp64")
    C, _ = vc.capacitance(tol=1e-11)
    g, _ = vc.capacitance_grad(G, tol=1e-11)
    assert np.max(np.abs(C - Cref)) < 1e-7 * np.max(np.abs(Cref))
    assert np.max(np.abs(g - gref)) < 1e-6 * np.max(np.abs(gref)), (g[:8], gref[:8])


def test_gradient_equal_permittivity_faces_by_finite_differences():
    """Faces whose two sides have equal eps carry no panel; their voxels still
    have a gradient (a panel appears as soon as one side changes): against the
    oracle's dense adjoint, which adds the equal-sides limit of Eq. 7 for
    those faces, at every voxel, and against central differences."""
    import torch
    from paper_2004_02609_gb300 import voxcap as V
    lab, cid, eps = _tiny(1, (6, 5, 4))
    nv = len(eps) - 2
    eps[: nv // 2] = 3.0          # half of the voxels share one value
    G = np.array([[0.0, 1.0], [0.0, 0.0]])
    vc = V.VoxCap(lab, cid, eps, 1e-6, precision="fp64", nv=4)
    vc.capacitance(tol=1e-12)
    g, _ = vc.capacitance_grad(G, tol=1e-12)
    gref, _ = O.capacitance_grad(lab, cid, eps, G, voxel_size=1e-6, rtol=1e-12)
    bad = np.abs(g - gref) > 1e-3 * np.abs(gref) + 1e-6 * np.max(np.abs(gref))
    assert not np.any(bad), (np.nonzero(bad)[0][:8], g[bad][:8], gref[bad][:8])
    rng = np.random.default_rng(2)
    picks = list(rng.choice(nv // 2, 5, replace=False)) + list(nv // 2 + rng.choice(nv - nv // 2, 3, replace=False))
    h = 1e-4
    for v in picks:
        ep, em = eps.copy(), eps.copy()
        ep[v] += h
        em[v] -= h
        vc.update_eps(ep)
        Cp, _ = vc.capacitance(tol=1e-12)
        vc.update_eps(em)
        Cm, _ = vc.capacitance(tol=1e-12)
        fd = (Cp[0, 1] - Cm[0, 1]) / (2 * h)
        assert abs(fd - g[v]) <= 1e-3 * np.max(np.abs(g)) + 1e-3 * abs(fd), (v, fd, g[v])


def test_autograd_layer_scalars():
    """Per-layer scalars through torch.autograd: eps_v = s_L * base_v."""
    import torch
    from paper_2004_02609_gb300 import voxcap as V
    wl, base, layer = W.pillars_field(16, seed=4)
    vc = V.VoxCap(wl.labels, wl.conductor_id, wl.eps_r, wl.voxel_size, precision="fp64", nv=4)
    lay = torch.as_tensor(layer)
    bse = torch.as_tensor(base, dtype=torch.float64)
    cond = lay < 0

    def eps_of(s):
        e = s[lay.clamp(min=0)] * bse
        return torch.where(cond, torch.ones_like(e), e)

    s = torch.tensor([1.0, 1.2, 0.9], dtype=torch.float64, requires_grad=True)
    C = V.capacitance_fn(vc, eps_of(s), tol=1e-11)
    L = C[0, 0] + 0.5 * C[0, 1]
    L.backward()
    h = 1e-4
    for k in range(3):
        sp = s.detach().clone()
        sm = s.detach().clone()
        sp[k] += h
        sm[k] -= h
        Lp = V.capacitance_fn(vc, eps_of(sp), tol=1e-11)
        Lm = V.capacitance_fn(vc, eps_of(sm), tol=1e-11)
        fd = ((Lp[0, 0] + 0.5 * Lp[0, 1]) - (Lm[0, 0] + 0.5 * Lm[0, 1])) / (2 * h)
        assert abs(fd.item() - s.grad[k].item()) <= 1e-3 * abs(fd.item())
