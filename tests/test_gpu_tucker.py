"""Tucker restoration (Eq. 13) on the tensor cores, through the C ABI:
against the oracle's FP64 einsum of the same factors, within the truncation
bound of the compression, and end to end against FP64-generated tensors."""
import numpy as np
import pytest

import oracle as O
from paper_2004_02609_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2004_02609_gb300 import build
    build.build()


@pytest.mark.parametrize("shape", [((7, 9, 5), (150, 70, 40)), ((40, 12, 33), (129, 64, 65)),
                                   ((1, 1, 1), (3, 5, 2)), ((17, 35, 8), (300, 260, 17))])
def test_tucker_expand_matches_einsum(shape):
    """TF32 hi/lo split with FP32 accumulation: ~2^-21 relative per product."""
    import torch
    from paper_2004_02609_gb300 import voxcap as V
    (r1, r2, r3), (D1, D2, D3) = shape
    rng = np.random.default_rng(r1 * 31 + D1)
    S = rng.standard_normal((r1, r2, r3))
    Us = [rng.standard_normal((D, r)) / np.sqrt(r) for D, r in ((D1, r1), (D2, r2), (D3, r3))]
    ref = O.tucker_expand(S, *Us)
    got = V.tucker_expand(*(torch.tensor(a, device="cuda") for a in [S] + Us))
    assert got.shape == ref.shape
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < 2e-6, err
    assert np.max(np.abs(got - ref)) < 2e-5 * np.max(np.abs(ref))


@pytest.fixture(scope="module")
def model():
    from paper_2004_02609_gb300 import tucker as T
    return T.install(28, 1e-6)


def test_compression_bound_and_restore(model):
    """HOSVD truncation: ||X - X~|| <= tol ||X||; the oracle einsum of the
    stored factors is the reference for the device restore."""
    from paper_2004_02609_gb300 import tucker as T
    Xs = T.canonical_tensors(28)
    for t, X in enumerate(Xs):
        Xr = O.tucker_expand(model.cores[t], *model.factors[t])
        assert np.linalg.norm(Xr - X) <= 1e-6 * np.linalg.norm(X) * 1.0001
    # canonical tensors are the integrals of their offsets (oracle, sampled)
    rng = np.random.default_rng(0)
    for _ in range(10):
        i, j, k = (int(v) for v in rng.integers(0, 28, 3))
        assert abs(Xs[0][i, j, k] - O.entry(0, 2, 2, (j, k, i))) <= 2e-12 * abs(Xs[0][i, j, k])
        ref = O.entry(1, 0, 1, (i + 0.5, j + 0.5, k))
        assert abs(Xs[3][i, j, k] - ref) <= 2e-12 * max(abs(ref), 1e-8)


def test_setup_from_tucker_matches_generated(model):
    """A handle restored from Tucker factors: its 15 Toeplitz tensors agree
    with the FP64-generated ones within the compression tolerance, and its
    capacitance within 1e-4."""
    from paper_2004_02609_gb300 import voxcap as V
    w = W.random_structure((26, 20, 14), 6, n_cond=2)
    a = V.VoxCap(w.labels, w.conductor_id, w.eps_r, w.voxel_size, nv=6)
    b = V.VoxCap(w.labels, w.conductor_id, w.eps_r, w.voxel_size, nv=6, tucker=model)
    for t in range(15):
        Ta, Tb = a.toeplitz(t), b.toeplitz(t)
        assert Ta.shape == Tb.shape
        assert np.linalg.norm(Ta - Tb) <= 5e-6 * np.linalg.norm(Ta), t
    Ca, _ = a.capacitance(tol=1e-9)
    Cb, _ = b.capacitance(tol=1e-9)
    assert np.max(np.abs(Ca - Cb)) <= 1e-4 * np.max(np.abs(Ca))


def test_tucker_rejects_too_small_cube(model):
    from paper_2004_02609_gb300 import voxcap as V
    w = W.random_structure((30, 8, 8), 1)
    with pytest.raises(V.VoxCapError):
        V.VoxCap(w.labels, w.conductor_id, w.eps_r, w.voxel_size, tucker=model)
