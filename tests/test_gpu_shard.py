"""Conductor columns of the capacitance matrix solved apart (the unit of the
multi-GPU sharding) against the whole batch, through the C ABI."""
import numpy as np
import pytest

from paper_2004_02609_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2004_02609_gb300 import build
    build.build()


@pytest.mark.parametrize("precision", ["fp32_refine", "fp64"])
def test_column_blocks_assemble_the_matrix_bit_for_bit(precision):
    """Column blocks of every 2- and 3-way split of 3 conductors, each solved
    in its own batch, equal the columns of the full batched solve exactly:
    a column's solve does not depend on its batch."""
    from paper_2004_02609_gb300 import shard
    from paper_2004_02609_gb300 import voxcap as V
    w = W.random_structure((9, 7, 6), 4, n_cond=3)
    vc = V.VoxCap(w.labels, w.conductor_id, w.eps_r, w.voxel_size, nv=4, precision=precision)
    C, st = vc.capacitance(tol=1e-8)
    assert st["converged"] == 1 and C.shape == (3, 3)
    for world in (2, 3):
        parts = [shard.column_range(3, r, world) for r in range(world)]
        got = np.concatenate([vc.capacitance_columns(j0, j1, tol=1e-8)[0] for j0, j1 in parts], axis=1)
        assert np.array_equal(got, C), (world, np.max(np.abs(got - C)))
