"""The oracle's CPU FFT-GMRES(35) (oracle/fft_gmres.py) checked against the
dense oracle: the circulant FFT product of Eqs. 9-11 equals the dense
Galerkin matrix of Eq. 4 on small grids of every kind of panel pair, and the
capacitance it yields by GMRES(35) equals the dense LU's."""
import numpy as np
import pytest

import oracle as O
from oracle import fft_gmres as F
from paper_2004_02609_gb300 import workloads as W

CASES = [W.random_structure((7, 5, 6), 0), W.random_structure((5, 8, 7), 2, n_cond=3),
         W.plates(12, 10, 8), W.coated_sphere(8, 3.0)]
CASES[2].name = "plates_12x10x8"


@pytest.mark.parametrize("w", CASES, ids=lambda w: w.name)
def test_fft_product_equals_dense(w):
    ps = O.panels(w.labels, w.conductor_id, w.eps_r)
    A = O.dense_matrix(ps, rtol=1e-12)
    prod = F.FFTProduct(ps, rtol=1e-12)
    X = np.random.default_rng(0).standard_normal((3, ps.n))
    for x in X:
        y = prod(x)
        ref = A @ x
        assert np.linalg.norm(y - ref) <= 1e-12 * np.linalg.norm(ref)


def test_fft_product_is_not_symmetric_where_the_paper_says_so():
    """E' blocks make A nonsymmetric (Eq. 4): the FFT product's transpose
    action differs from its action, as the dense matrix's does."""
    w = CASES[0]
    ps = O.panels(w.labels, w.conductor_id, w.eps_r)
    prod = F.FFTProduct(ps, rtol=1e-12)
    rng = np.random.default_rng(1)
    u, v = rng.standard_normal(ps.n), rng.standard_normal(ps.n)
    assert abs(u @ prod(v) - v @ prod(u)) > 1e-6 * abs(u @ prod(v))


@pytest.mark.parametrize("w", [CASES[1], CASES[2]], ids=lambda w: w.name)
def test_fft_gmres_capacitance_equals_dense_lu(w):
    ps = O.panels(w.labels, w.conductor_id, w.eps_r)
    C, Cn, X, its = F.capacitance_fft(ps, voxel_size=w.voxel_size, tol=1e-12)
    Cref, _, Xref = O.capacitance(ps, voxel_size=w.voxel_size, rtol=1e-12)
    assert np.max(np.abs(C - Cref)) <= 1e-9 * np.max(np.abs(Cref))
    assert all(0 <= k < 35 * 200 for k in its) and sum(its) > 0   # a zero column needs none
