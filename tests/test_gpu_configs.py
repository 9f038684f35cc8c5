"""The larger configurations at full size, through the C ABI.

No dense oracle is feasible at these sizes: products are checked on sampled
rows against the oracle's integrals computed one by one, capacitances
against the plain FP64 GPU solve and the properties every capacitance matrix
has, gradients against central finite differences."""
import numpy as np
import pytest

import oracle as O
from paper_2004_02609_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2004_02609_gb300 import build
    build.build()


def _cap_properties(C):
    m = C.shape[0]
    assert np.all(np.diag(C) > 0)
    off = C[~np.eye(m, dtype=bool)]
    assert np.all(off < 0)
    assert np.all(C.sum(1) > 0)
    assert np.linalg.norm(C - C.T) <= 2e-2 * np.linalg.norm(C)


@pytest.fixture(scope="module")
def bus():
    import torch
    from paper_2004_02609_gb300 import voxcap as V
    w = W.bus_crossing()
    return w, V.VoxCap(torch.tensor(w.labels, device="cuda"), w.conductor_id, w.eps_r, w.voxel_size)


def test_bus_crossing_sampled_product(bus):
    """y = A x at full size (110,848 panels) for a sparse x, FP64 entries and
    products: sampled rows against sums of oracle integrals."""
    import torch
    from paper_2004_02609_gb300 import voxcap as V
    w, _ = bus
    vc = V.VoxCap(torch.tensor(w.labels, device="cuda"), w.conductor_id, w.eps_r, w.voxel_size,
                  entries="fp64")
    pm = vc.panel_map()
    ps = O.panels(w.labels, w.conductor_id, w.eps_r)
    assert np.array_equal(pm["face"], ps.face) and np.array_equal(pm["kind"], ps.kind)
    rng = np.random.default_rng(0)
    cols = rng.choice(vc.N, 12, replace=False)
    x = np.zeros(vc.N)
    x[cols] = rng.standard_normal(12)
    y = vc.matvec(torch.tensor(x, device="cuda")).cpu().numpy()
    rows = np.concatenate([rng.choice(ps.n_cond, 10, replace=False),
                           ps.n_cond + rng.choice(ps.n_diel, 20, replace=False), cols[:4]])
    c = ps.centers
    kind = np.repeat(ps.kind[rows], len(cols))
    to = np.repeat(ps.orient[rows], len(cols))
    so = np.tile(ps.orient[cols], len(rows))
    d = (c[rows][:, None, :] - c[cols][None, :, :]).reshape(-1, 3)
    A = O.entries(kind, to, so, d, rtol=1e-13).reshape(len(rows), len(cols))
    ref = A @ x[cols] + np.where(ps.kind[rows] == 1, ps.idiag[rows] * x[rows], 0.0)
    assert np.max(np.abs(y[rows] - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_bus_crossing_capacitance_fp32_refine_vs_fp64(bus):
    """8 conductor right-hand sides in one batch: FP32 products (FP32
    far-field entries) with FP64 refinement agree with the plain FP64 solve
    (FP64 entries) to 1e-4 (the target) and the matrix has the capacitance
    properties."""
    w, vc = bus
    C32, st = vc.capacitance(tol=1e-6)
    assert st["converged"] == 1 and C32.shape == (8, 8)
    import torch
    from paper_2004_02609_gb300 import voxcap as V
    v64 = V.VoxCap(torch.tensor(w.labels, device="cuda"), w.conductor_id, w.eps_r, w.voxel_size,
                   precision="fp64")
    C64, _ = v64.capacitance(tol=1e-9)
    assert np.max(np.abs(C32 - C64)) <= 1e-4 * np.max(np.abs(C64))
    assert np.all(np.abs(C32 - C64) <= 1e-4 * np.abs(C64) + 1e-6 * np.max(np.abs(C64)))
    _cap_properties(C64)


def test_sixteen_small_structures_batched():
    """The 16 random 16^3 box structures in one handle (shared spectra, one
    batch): each against its dense oracle solve."""
    boxes = W.small_boxes(16, 16)
    from paper_2004_02609_gb300 import voxcap as V
    vc = V.VoxCap(np.stack([b.labels for b in boxes]), boxes[0].conductor_id, boxes[0].eps_r, 1e-6)
    Cs, st = vc.capacitance(tol=1e-8)
    assert st["converged"] == 1
    for b, C in zip(boxes, Cs):
        ps = O.panels(b.labels, b.conductor_id, b.eps_r)
        Cref, _, _ = O.capacitance(ps, voxel_size=1e-6, rtol=1e-11)
        assert abs(C[0, 0] - Cref[0, 0]) <= 1e-6 * abs(Cref[0, 0])


@pytest.fixture(scope="module")
def pillars():
    from paper_2004_02609_gb300 import voxcap as V
    wl, base, layer = W.pillars_field(64, seed=4)
    vc = V.VoxCap(wl.labels, wl.conductor_id, wl.eps_r, wl.voxel_size)
    return wl, base, layer, vc


def test_pillars_gradient_by_central_differences(pillars):
    """dC/d eps per voxel (adjoint, FP32+refine forward and adjoint solves)
    against central differences with step 1e-4, on the voxels with the
    largest gradients, and the per-layer scalars through torch.autograd."""
    import torch
    from paper_2004_02609_gb300 import voxcap as V
    wl, base, layer, vc = pillars
    G = np.array([[0.0, 1.0], [0.0, 0.0]])           # L = C_01
    vc.capacitance(tol=1e-12)
    g, _ = vc.capacitance_grad(G, tol=1e-12)
    eps = wl.eps_r.copy()
    order = np.argsort(-np.abs(g))
    # the six largest gradients and two more drawn from the voxels whose
    # gradient is at least 5% of the largest: each is far above the noise of
    # the central difference (solves at 1e-12 give ~1e-8 |C| / step)
    gmax = np.abs(g[order[0]])
    rest = [v for v in order[6:] if np.abs(g[v]) >= 0.05 * gmax]
    picks = list(order[:6]) + list(np.random.default_rng(7).choice(rest, 2, replace=False))
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
        assert abs(fd - g[v]) <= 1e-3 * abs(fd), (v, fd, g[v])
    vc.update_eps(eps)
    lay = torch.as_tensor(layer)
    bse = torch.as_tensor(base, dtype=torch.float64)

    def eps_of(s):
        e = s[lay.clamp(min=0)] * bse
        return torch.where(lay < 0, torch.ones_like(e), e)

    s = torch.tensor([1.0, 1.0, 1.0], dtype=torch.float64, requires_grad=True)
    C = V.capacitance_fn(vc, eps_of(s), tol=1e-12)
    C[0, 1].backward()
    for k in range(3):
        sp, sm = s.detach().clone(), s.detach().clone()
        sp[k] += h
        sm[k] -= h
        fd = (V.capacitance_fn(vc, eps_of(sp), tol=1e-12)[0, 1] -
              V.capacitance_fn(vc, eps_of(sm), tol=1e-12)[0, 1]) / (2 * h)
        assert abs(fd.item() - s.grad[k].item()) <= 1e-3 * abs(fd.item())


def test_pillars_tucker_restored_setup(pillars):
    """Toeplitz tensors restored from Tucker factors (tol 1e-6) at 64^3: the
    capacitance matches the FP64-generated set-up to 1e-4."""
    from paper_2004_02609_gb300 import tucker as T
    from paper_2004_02609_gb300 import voxcap as V
    wl, base, layer, vc = pillars
    vc.update_eps(wl.eps_r)
    model = T.install(65, 1e-6)
    vt = V.VoxCap(wl.labels, wl.conductor_id, wl.eps_r, wl.voxel_size, tucker=model)
    Ca, _ = vc.capacitance(tol=1e-8)
    Cb, _ = vt.capacitance(tol=1e-8)
    assert np.max(np.abs(Ca - Cb)) <= 1e-4 * np.max(np.abs(Ca))
    _cap_properties(Ca)


def test_meanders_large():
    """Two interleaved meanders on 512 x 512 x 64 (1.41 M panels), 2
    right-hand sides: FP32+refine against plain FP64, and the capacitance
    matrix properties."""
    import torch
    from paper_2004_02609_gb300 import voxcap as V
    w = W.meanders()
    lab = torch.tensor(w.labels, device="cuda")
    vc = V.VoxCap(lab, w.conductor_id, w.eps_r, w.voxel_size)
    assert vc.N == 1410624
    C32, st = vc.capacitance(tol=1e-6)
    assert st["converged"] == 1
    vc.close()
    v64 = V.VoxCap(lab, w.conductor_id, w.eps_r, w.voxel_size, precision="fp64")
    C64, _ = v64.capacitance(tol=1e-8)
    assert np.max(np.abs(C32 - C64)) <= 1e-4 * np.max(np.abs(C64))
    _cap_properties(C64)


def test_meanders_tucker_restored_matches_generated():
    """512 x 512 x 64 meanders with the Toeplitz tensors restored from Tucker
    factors at tolerance 1e-6 (installed on a 514^3 index cube, Eq. 13) on the
    tensor cores, against tensors generated directly: every C entry within
    1e-4 of the largest."""
    import torch
    from paper_2004_02609_gb300 import tucker as T
    from paper_2004_02609_gb300 import voxcap as V
    w = W.meanders()
    lab = torch.tensor(w.labels, device="cuda")
    model = T.install(max(w.labels.shape) + 2, 1e-6)
    vt = V.VoxCap(lab, w.conductor_id, w.eps_r, w.voxel_size, tucker=model)
    Ct, st = vt.capacitance(tol=1e-6)
    assert st["converged"] == 1
    vt.close()
    vg = V.VoxCap(lab, w.conductor_id, w.eps_r, w.voxel_size)
    Cg, _ = vg.capacitance(tol=1e-6)
    assert np.max(np.abs(Ct - Cg)) <= 1e-4 * np.max(np.abs(Cg))
    _cap_properties(Ct)
