"""voxcap_matvec_noalloc against voxcap_matvec, through the C ABI.

The no-allocation entry point serves callers that cannot allocate device
memory while they run (a fixed memory budget, memory owned by another
allocator, or loops that cannot take cudaMalloc's implicit synchronisation).
It must give the same products as voxcap_matvec, call after call, from its
fixed library scratch, and leave the device's memory pool untouched.  This
file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_2004_02609_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _cudart():
    """The CUDA runtime the library is linked against (already loaded with it)."""
    for name in ("libcudart.so.13", "/usr/local/cuda/lib64/libcudart.so.13", "libcudart.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.skip("CUDA runtime library not found for the memory-pool query")


def _pool_bytes():
    """(used, reserved) bytes of the current device's default stream-ordered
    pool, where every device allocation of the library comes from."""
    import torch
    rt = _cudart()
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), ctypes.c_int(torch.cuda.current_device())) == 0
    used, reserved = ctypes.c_uint64(), ctypes.c_uint64()
    assert rt.cudaMemPoolGetAttribute(pool, 7, ctypes.byref(used)) == 0        # UsedMemCurrent
    assert rt.cudaMemPoolGetAttribute(pool, 5, ctypes.byref(reserved)) == 0    # ReservedMemCurrent
    return used.value, reserved.value


def test_matvec_noalloc_matches_matvec_twice():
    """A handle that has never run voxcap_matvec gives, on two no-allocation
    calls in a row, the products another handle of the same structure gives
    through voxcap_matvec, and the pool's used and reserved bytes stay the
    same across those calls."""
    import torch
    from paper_2004_02609_gb300 import build
    build.build()
    from paper_2004_02609_gb300 import voxcap as V
    L = V.lib()
    w = W.random_structure((9, 7, 6), 3, n_cond=2)
    ref_h = V.VoxCap(w.labels, w.conductor_id, w.eps_r, w.voxel_size, nv=4)
    fresh = V.VoxCap(w.labels, w.conductor_id, w.eps_r, w.voxel_size, nv=4)
    tol = {torch.float64: 1e-12, torch.float32: 2e-6}
    for dtype, code in ((torch.float64, V.F64), (torch.float32, V.F32)):
        x = torch.randn(2, ref_h.N, dtype=dtype, device="cuda")
        for flags in (0, V.MV_PRECOND, V.MV_ADJOINT):
            ref = torch.empty_like(x)
            assert L.voxcap_matvec(ref_h._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(ref.data_ptr()),
                                   2, code, flags) == 0
            ys = [torch.full_like(x, float("nan")) for _ in range(2)]
            torch.cuda.synchronize()
            before = _pool_bytes()
            for y in ys:                # two calls in a row share the scratch
                rc = L.voxcap_matvec_noalloc(fresh._h, ctypes.c_void_p(x.data_ptr()),
                                             ctypes.c_void_p(y.data_ptr()), 2, code, flags)
                assert rc == 0, L.voxcap_last_error()
            torch.cuda.synchronize()
            assert _pool_bytes() == before
            for y in ys:
                for c in range(2):
                    assert _rel(y[c].double().cpu().numpy(), ref[c].double().cpu().numpy()) < tol[dtype]


def test_matvec_noalloc_rejects_oversized_requests():
    import torch
    from paper_2004_02609_gb300 import voxcap as V
    L = V.lib()
    w = W.plates()
    vc = V.VoxCap(w.labels, w.conductor_id, w.eps_r, w.voxel_size)
    nrhs = 64
    x = torch.zeros(nrhs, vc.N, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    rc = L.voxcap_matvec_noalloc(vc._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                 nrhs, V.F64, 0)
    assert rc == -1
    assert b"16777216" in L.voxcap_last_error()
