"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bars: panel maps bit-exact; single entries within 1e-12 relative; products
within 1e-12 relative l2 in FP64 and 2e-6 in FP32; preconditioner within
1e-10 where its blocks are inverted in FP64 and 1e-5 where they are inverted
in FP32; capacitance entries within 1e-4 relative (the targets of the hot
path)."""
import numpy as np
import pytest

import oracle as O
from paper_2004_02609_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2004_02609_gb300 import build
    build.build()


def _V():
    from paper_2004_02609_gb300 import voxcap as V
    return V


def make(w, **kw):
    """A handle on workload w; FP64 entries unless asked otherwise (these
    tests hold the operator to FP64 parity with the oracle)."""
    kw.setdefault("entries", "fp64")
    return _V().VoxCap(w.labels, w.conductor_id, w.eps_r, w.voxel_size, **kw)


SMALL = [W.cube(4), W.random_structure((7, 5, 6), 0), W.random_structure((9, 6, 5), 1),
         W.random_structure((5, 8, 7), 2, n_cond=3), W.coated_sphere(12, 3.0),
         W.plates(12, 10, 8)]
SMALL[5].name = "plates_12x10x8"


_DENSE = {}


def dense(w, rtol=1e-13):
    """Oracle panels and dense matrix of a workload, assembled once per module."""
    key = (w.name, w.labels.tobytes(), w.eps_r.tobytes(), rtol)
    if key not in _DENSE:
        ps = O.panels(w.labels, w.conductor_id, w.eps_r)
        _DENSE[key] = (ps, O.dense_matrix(ps, rtol=rtol))
    return _DENSE[key]


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("w", SMALL, ids=lambda w: w.name)
def test_panel_map_bit_exact(w):
    ps = O.panels(w.labels, w.conductor_id, w.eps_r)
    vc = make(w)
    pm = vc.panel_map()
    assert vc.N == ps.n
    for k in ("orient", "face", "kind", "owner"):
        assert np.array_equal(pm[k], getattr(ps, k).astype(pm[k].dtype)), k
    assert np.array_equal(pm["idiag"], ps.idiag)
    assert np.array_equal(pm["qscale"], ps.qscale)


def _entry_cases():
    rng = np.random.default_rng(7)
    cases = []
    for _ in range(400):
        to, so = (int(v) for v in rng.integers(0, 3, 2))
        R = [1, 2, 3, 5, 9, 17, 33, 60][int(rng.integers(0, 8))]
        d = rng.integers(-R, R + 1, 3).astype(float)
        if to != so:
            d[to] -= 0.5
            d[so] += 0.5
        cases.append((int(rng.integers(0, 2)), to, so, d))
    # every near-field configuration around the origin
    for to in range(3):
        for so in range(3):
            for dx in range(-2, 3):
                for dy in range(-2, 3):
                    for dz in range(-2, 3):
                        d = np.array([dx, dy, dz], float)
                        if to != so:
                            d[to] -= 0.5
                            d[so] += 0.5
                        for kind in (0, 1):
                            cases.append((kind, to, so, d))
    return cases


def test_entries_match_oracle():
    V = _V()
    cases = _entry_cases()
    kind = np.array([c[0] for c in cases])
    to = np.array([c[1] for c in cases])
    so = np.array([c[2] for c in cases])
    d = np.array([c[3] for c in cases])
    got = V.entries(kind, to, so, d)
    ref = O.entries(kind, to, so, d, rtol=1e-14)
    scale = np.maximum(np.abs(ref), 1e-6 * np.abs(ref).max())
    err = np.abs(got - ref) / scale
    worst = int(np.argmax(err))
    assert err.max() < 2e-12, (cases[worst], got[worst], ref[worst])


def test_toeplitz_tables_sampled():
    """The 15 block-Toeplitz tensors of a grid hold the integrals of their
    index offsets (Appendix B): sampled entries against the oracle."""
    w = W.random_structure((9, 7, 6), 3)
    vc = make(w)
    rng = np.random.default_rng(11)
    te = [0, 1, 2, 0, 0, 1, 0, 1, 2, 0, 0, 1, 1, 2, 2]
    so = [0, 1, 2, 1, 2, 2, 0, 1, 2, 1, 2, 2, 0, 0, 1]
    for t in range(15):
        T = vc.toeplitz(t)
        dz, dy, dx = T.shape
        idx = [(int(rng.integers(0, dx)), int(rng.integers(0, dy)), int(rng.integers(0, dz)))
               for _ in range(12)] + [(0, 0, 0)]
        for (ex, ey, ez) in idx:
            d = np.array([ex, ey, ez], float)
            if te[t] != so[t]:
                d[te[t]] += 0.5
                d[so[t]] += 0.5
            ref = O.entry(1 if t >= 6 else 0, te[t], so[t], d, rtol=1e-14)
            got = T[ez, ey, ex]
            assert abs(got - ref) <= 2e-12 * max(abs(ref), 1e-8), (t, ex, ey, ez, got, ref)


def test_far_field_fp32_tables():
    """Entries generated with FP32 far-field sums (the FP32+refine default):
    near-field closed forms (gap <= 1 voxel) still within 2e-12 of the oracle,
    far-field entries within 1e-6 relative."""
    w = W.random_structure((9, 7, 6), 3)
    vc = make(w, entries="far32")
    ref_vc = make(w, entries="fp64")
    te = [0, 1, 2, 0, 0, 1, 0, 1, 2, 0, 0, 1, 1, 2, 2]
    so = [0, 1, 2, 1, 2, 2, 0, 1, 2, 1, 2, 2, 0, 0, 1]
    worst_far = 0.0
    for t in range(15):
        T, R = vc.toeplitz(t), ref_vc.toeplitz(t)
        dz, dy, dx = T.shape
        ez, ey, ex = np.meshgrid(np.arange(dz), np.arange(dy), np.arange(dx), indexing="ij")
        e = [ex, ey, ez]
        if te[t] == so[t]:
            a1, a2 = [a for a in range(3) if a != te[t]]
            gap = np.maximum(e[te[t]], np.maximum(e[a1] - 1, e[a2] - 1))
        else:
            ga = 3 - te[t] - so[t]
            gap = np.maximum(e[te[t]], np.maximum(e[so[t]], e[ga] - 1))
        near = gap <= 1
        rel = np.abs(T - R) / np.maximum(np.abs(R), 1e-8)
        assert rel[near].max() <= 2e-12, t
        worst_far = max(worst_far, rel[~near].max())
    assert worst_far <= 1e-6, worst_far
    # sampled far entries against the oracle itself
    rng = np.random.default_rng(5)
    for t in (0, 3, 6, 9, 12):
        T = vc.toeplitz(t)
        dz, dy, dx = T.shape
        for _ in range(6):
            ex, ey, ez = (int(rng.integers(2, dx)), int(rng.integers(2, dy)), int(rng.integers(2, dz)))
            d = np.array([ex, ey, ez], float)
            if te[t] != so[t]:
                d[te[t]] += 0.5
                d[so[t]] += 0.5
            ref = O.entry(1 if t >= 6 else 0, te[t], so[t], d, rtol=1e-14)
            assert abs(T[ez, ey, ex] - ref) <= 1e-6 * abs(ref) + 1e-14, (t, ex, ey, ez)


@pytest.mark.parametrize("w", [SMALL[1], SMALL[3], SMALL[5]], ids=lambda w: w.name)
def test_far_field_fp32_products_and_capacitance(w):
    """With FP32 far-field entries the FP32 products stay within the FP32 bar
    (2e-6) of the exact dense operator, and the FP32+refine capacitance within
    1e-6 of max|C| of the oracle's."""
    import torch
    vc = make(w, entries="far32")
    ps, A = dense(w)
    X = np.random.default_rng(0).standard_normal((2, ps.n))
    y32 = vc.matvec(torch.tensor(X, device="cuda").float()).cpu().numpy()
    for r in range(2):
        assert rel_l2(y32[r], A @ X[r]) < 2e-6
    Cref, _, _ = O.capacitance(ps, A=A, voxel_size=w.voxel_size)
    C, st = vc.capacitance(tol=1e-8)
    assert st["converged"] == 1
    assert np.abs(C - Cref).max() < 1e-6 * np.abs(Cref).max()


@pytest.mark.parametrize("w", SMALL[1:4] + [SMALL[5]], ids=lambda w: w.name)
@pytest.mark.parametrize("pad_mode", [0, 1, 2])
def test_matvec_matches_dense(w, pad_mode):
    import torch
    nx, ny, nz = w.shape_xyz
    try:
        vc = make(w, pad_mode=pad_mode)
    except Exception as e:     # 2(N+1) not 2/3/5/7-smooth: pad_mode 1 is refused
        assert pad_mode == 1 and "smooth" in str(e)
        return                 # the refusal itself is the checked behaviour
    ps, A = dense(w)
    rng = np.random.default_rng(0)
    X = rng.standard_normal((3, ps.n))
    ref = (A @ X.T).T
    refT = (A.T @ X.T).T
    x64 = torch.tensor(X, device="cuda")
    y64 = vc.matvec(x64).cpu().numpy()
    for r in range(3):
        assert rel_l2(y64[r], ref[r]) < 1e-12
    yT = vc.matvec(x64, adjoint=True).cpu().numpy()
    for r in range(3):
        assert rel_l2(yT[r], refT[r]) < 1e-12
    y32 = vc.matvec(x64.float()).cpu().numpy()
    for r in range(3):
        assert rel_l2(y32[r], ref[r]) < 2e-6


@pytest.mark.parametrize("shape", [(6, 4, 5), (12, 3, 17), (24, 10, 6)])
def test_matvec_every_radix(shape):
    """Grids whose padded lengths need every radix of the FFT engine
    (16, 10, 12 / 28, 8, 36 / 56, 24, 16: factors 2, 3, 4, 5, 7, 8, 9, 16):
    forward and transposed products against the dense oracle, FP64 and FP32."""
    import torch
    w = W.random_structure(shape, 9, n_cond=2)
    vc = make(w)
    radices = {p for M in vc.fft_lengths() for p in (2, 3, 5, 7, 9, 16) if M % p == 0}
    ps, A = dense(w)
    X = np.random.default_rng(3).standard_normal((2, ps.n))
    x64 = torch.tensor(X, device="cuda")
    y = vc.matvec(x64).cpu().numpy()
    yT = vc.matvec(x64, adjoint=True).cpu().numpy()
    y32 = vc.matvec(x64.float()).cpu().numpy()
    for r in range(2):
        assert rel_l2(y[r], A @ X[r]) < 1e-12
        assert rel_l2(yT[r], A.T @ X[r]) < 1e-12
        assert rel_l2(y32[r], A @ X[r]) < 2e-6
    assert radices
    # every variant the autotuner may pick: both z radix orders, z tiles 4..16,
    # y tiles 4..16 (forward and inverse)
    x32 = x64.float()
    for order in (0, 1):
        for tile in (2, 3, 4):
            for yt in (-1, 2, 3):
                vc.set_product_tiles(order, tile, yt, yt)
                f = vc.matvec(x32).cpu().numpy()
                t = vc.matvec(x32, adjoint=True).cpu().numpy()
                for r in range(2):
                    assert rel_l2(f[r], A @ X[r]) < 2e-6, (order, tile, yt)
                    assert rel_l2(t[r], A.T @ X[r]) < 2e-6, (order, tile, yt)
    assert vc.set_product_tiles()[0] in (0, 1)


def _blob(n, axis):
    """A grid of n voxels along `axis` (2 or 3 across) holding a small
    structure near one end: a 2-voxel conductor with a one-voxel dielectric
    (eps_r 4) cap, in vacuum.  The padded length along `axis` is 2^a * 9 for
    the n used below; every panel pair stays within a few voxels, where the
    oracle's integrals are fast and accurate."""
    shape = [3, 3, 3]
    shape[axis] = n
    nx, ny, nz = shape
    lab = np.zeros((nz, ny, nx), np.int32)
    sl = [slice(0, 2)] * 3
    sl[2 - axis] = slice(1, 3)
    lab[tuple(sl)] = 2
    cap = list(sl)
    cap[2 - axis] = slice(3, 4)
    lab[tuple(cap)] = 1
    return W.Workload(f"blob{n}_{'xyz'[axis]}", lab, np.array([-1, -1, 0], np.int32), np.array([1.0, 4.0, 1.0]))


@pytest.mark.parametrize("n,axis", [(17, 2), (35, 2), (64, 2), (35, 1), (64, 1), (128, 1), (260, 1), (515, 1),
                                    (17, 0), (64, 0), (128, 0), (260, 0), (515, 0)])
def test_matvec_compiled_plans(n, axis):
    """The compiled-plan FP32 passes (path 1) on every compiled length (x and
    y: 36, 72, 144, 288, 576, 1152 with two or three radix stages; z: 36, 72,
    144), forward (compiled x, y and z passes) and transposed (compiled y
    passes), in every launch variant, and the FP64 products (compiled y
    passes) at 1e-12,
    against the dense oracle; and the generic passes (path 0) on the same
    handle.  The full padded transforms run although the structure is small."""
    import torch
    w = _blob(n, axis)
    vc = make(w)
    M = vc.fft_lengths()[axis]
    assert M in (36, 72, 144, 288, 576, 1152), M
    ps, A = dense(w)
    X = np.random.default_rng(11).standard_normal((2, ps.n))
    x32 = torch.tensor(X, device="cuda", dtype=torch.float32)
    res = {}
    for path in (1, 15, 0):                     # 15: every launch variant of the compiled passes
        assert vc.set_product_path(path) == path
        f = vc.matvec(x32).cpu().numpy()
        t = vc.matvec(x32, adjoint=True).cpu().numpy()
        res[path] = (f, t)
        for r in range(2):
            assert rel_l2(f[r], A @ X[r]) < 2e-6, (path, r)
            assert rel_l2(t[r], A.T @ X[r]) < 2e-6, (path, r)
    # the variants differ in tiling only: same arithmetic per line, same bits
    assert np.array_equal(res[1][0], res[15][0]) and np.array_equal(res[1][1], res[15][1])
    # FP64 products: the compiled y passes on these lengths
    x64 = torch.tensor(X, device="cuda", dtype=torch.float64)
    f = vc.matvec(x64).cpu().numpy()
    t = vc.matvec(x64, adjoint=True).cpu().numpy()
    for r in range(2):
        assert rel_l2(f[r], A @ X[r]) < 1e-12, ("fp64", r)
        assert rel_l2(t[r], A.T @ X[r]) < 1e-12, ("fp64", r)
    p = vc.set_product_path(-1)
    assert p == 0 or (p & 1 and p < 16)


@pytest.mark.parametrize("shape", [(17, 16, 17), (35, 17, 16)])
def test_matvec_compiled_plans_every_axis(shape):
    """Compiled x, y and z passes together (every padded length 36 or 72):
    forward and transposed FP32 products against the dense oracle, two
    columns, on two conductors in opposite corners of the grid, one with a
    dielectric cap."""
    import torch
    nx, ny, nz = shape
    lab = np.zeros((nz, ny, nx), np.int32)
    lab[2:5, 2:5, 2:5] = 2                      # conductor 0
    lab[2:5, 2:5, 5:7] = 1                      # dielectric cap, eps_r 4
    lab[nz - 5:nz - 2, ny - 5:ny - 2, nx - 5:nx - 2] = 3    # conductor 1, far corner
    w = W.Workload(f"corners{shape}", lab, np.array([-1, -1, 0, 1], np.int32), np.array([1.0, 4.0, 1.0, 1.0]))
    vc = make(w)
    assert all(M in (36, 72) for M in vc.fft_lengths()), vc.fft_lengths()
    ps, A = dense(w)
    X = np.random.default_rng(13).standard_normal((2, ps.n))
    x32 = torch.tensor(X, device="cuda", dtype=torch.float32)
    for path in (1, 15, 0):
        assert vc.set_product_path(path) == path
        for rep in range(2):
            f = vc.matvec(x32).cpu().numpy()
            t = vc.matvec(x32, adjoint=True).cpu().numpy()
            for r in range(2):
                assert rel_l2(f[r], A @ X[r]) < 2e-6, (path, rep, r)
                assert rel_l2(t[r], A.T @ X[r]) < 2e-6, (path, rep, r)


def test_matvec_paper_padding_equals_smooth_padding():
    """Any padded length >= 2N+1 gives the same linear convolution (Appendix B):
    the paper's 2(N+1) and the smooth length agree to rounding."""
    import torch
    w = W.random_structure((4, 6, 9), 5)        # 2(N+1) = 10, 14, 20: smooth
    a = make(w, pad_mode=0)
    b = make(w, pad_mode=1)
    assert b.fft_lengths() == (10, 14, 20)
    x = torch.randn(a.N, dtype=torch.float64, device="cuda")
    assert rel_l2(a.matvec(x).cpu(), b.matvec(x).cpu()) < 1e-13


@pytest.mark.parametrize("kind,nv,bar64", [
    ("bdd", (3, 2, 4), 1e-5),    # blocks <= 224 panels: inverted in FP32 in shared memory
    ("bd", (3, 2, 4), 1e-5),
    ("bd", (9, 7, 4), 1e-10),    # two blocks of ~530 panels: FP64 Gauss-Jordan path
    ("diag", (3, 2, 4), 1e-10),
    ("none", (3, 2, 4), 1e-10)])
def test_preconditioner_matches_dense(kind, nv, bar64):
    """R r (Eq. 14) against the oracle's dense preconditioner.  Blocks of up
    to 224 panels are inverted in FP32 (a preconditioner only steers GMRES),
    so their FP64 apply carries the FP32 inverse's error; larger blocks are
    inverted in FP64."""
    import torch
    w = W.random_structure((9, 7, 8), 4, n_cond=3)
    vc = make(w, precond=kind, nv=nv)
    ps, A = dense(w)
    R = O.precond_matrix(ps, A, nv=np.array(nv), kind=kind)
    r = np.random.default_rng(1).standard_normal((2, ps.n))
    z = vc.matvec(torch.tensor(r, device="cuda"), r_only=True).cpu().numpy()
    for c in range(2):
        assert rel_l2(z[c], R @ r[c]) < bar64
    z32 = vc.matvec(torch.tensor(r, device="cuda").float(), r_only=True).cpu().numpy()
    for c in range(2):
        assert rel_l2(z32[c], R @ r[c]) < 1e-5


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine", "fp32_refine_fast"])
@pytest.mark.parametrize("w", [SMALL[0], SMALL[1], SMALL[3], SMALL[4]], ids=lambda w: w.name)
def test_capacitance_matches_oracle(w, precision):
    """fp32_refine_fast: the fast refinement option (FP32 Gram-Schmidt
    arithmetic, FP32 residuals for early sweeps) meets the same bars."""
    ps, A = dense(w)
    Cref, _, _ = O.capacitance(ps, A=A, voxel_size=w.voxel_size)
    fast = precision.endswith("_fast")
    vc = make(w, precision=precision.replace("_fast", ""), fast_refine=int(fast))
    C, st = vc.capacitance(tol=1e-8)
    assert st["converged"] == 1
    err = np.abs(C - Cref) / np.abs(Cref).max()
    assert err.max() < 1e-6, (C, Cref)
    assert np.all(np.abs(C - Cref) <= 1e-4 * np.abs(Cref) + 1e-9 * np.abs(Cref).max())


def test_solve_residual_and_dense_solution():
    import torch
    w = SMALL[2]
    ps, A = dense(w)
    rng = np.random.default_rng(2)
    B = rng.standard_normal((2, ps.n))
    Xref = np.linalg.solve(A, B.T).T
    for precision, fast in (("fp64", 0), ("fp32_refine", 0), ("fp32_refine", 1)):
        vc = make(w, precision=precision, fast_refine=fast)
        X, st = vc.solve(torch.tensor(B, device="cuda"), tol=1e-10)
        X = X.cpu().numpy()
        for c in range(2):
            assert np.linalg.norm(A @ X[c] - B[c]) <= 1e-9 * np.linalg.norm(B[c])
            assert rel_l2(X[c], Xref[c]) < 1e-6
        assert st["converged"] == 1


def test_batched_structures_match_oracle():
    """Several same-shape structures in one handle (one batch, shared
    spectra) give each structure's own capacitance."""
    boxes = W.small_boxes(6, 12, seed0=3)
    labels = np.stack([b.labels for b in boxes])
    V = _V()
    vc = V.VoxCap(labels, boxes[0].conductor_id, boxes[0].eps_r, 1e-6)
    Cs, st = vc.capacitance(tol=1e-8)
    for b, C in zip(boxes, Cs):
        ps = O.panels(b.labels, b.conductor_id, b.eps_r)
        Cref, _, _ = O.capacitance(ps, voxel_size=1e-6, rtol=1e-12)
        assert abs(C[0, 0] - Cref[0, 0]) <= 1e-6 * abs(Cref[0, 0])
