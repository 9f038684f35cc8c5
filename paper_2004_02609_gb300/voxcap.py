"""Python binding of libvoxcap.so (include/voxcap.h).

Argument marshalling only: every step runs in the library's CUDA kernels.
PyTorch provides device memory and the current stream.  Importing this
module does not need a GPU; constructing a ``VoxCap`` does, and fails
loudly if the compiled library is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvoxcap.so")

OK = 0
ERR_NOT_CONVERGED = -6
F32, F64 = 0, 1
MV_PRECOND, MV_ADJOINT, MV_RONLY = 1, 2, 4
FP64, FP32_REFINE = 0, 1
PRECOND = {"bdd": 0, "bd": 1, "diag": 2, "none": 3}
ENTRIES = {"auto": 0, "fp64": 1, "far32": 2}
EPS0 = 8.8541878128e-12

# exported symbols, in header order (checked by the CPU tests)
SYMBOLS = ["voxcap_default_opts", "voxcap_last_error", "voxcap_setup", "voxcap_destroy",
           "voxcap_num_panels", "voxcap_panel_map", "voxcap_matvec", "voxcap_solve",
           "voxcap_capacitance", "voxcap_capacitance_columns", "voxcap_capacitance_grad", "voxcap_update_eps",
           "voxcap_entries", "voxcap_fft_length", "voxcap_toeplitz", "voxcap_launch_count",
           "voxcap_matvec_noalloc", "voxcap_tucker_expand", "voxcap_canonical_tensors",
           "voxcap_set_product_tiles", "voxcap_setup_times", "voxcap_set_product_path"]


class Tucker(ctypes.Structure):
    _fields_ = [("dims", (ctypes.c_int * 3) * 4), ("ranks", (ctypes.c_int * 3) * 4),
                ("core", ctypes.c_void_p * 4), ("factor", (ctypes.c_void_p * 3) * 4)]


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("restart", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("max_iters", ctypes.c_int),
                ("max_sweeps", ctypes.c_int), ("nv", ctypes.c_int * 3),
                ("precond", ctypes.c_int), ("pad_mode", ctypes.c_int),
                ("entries", ctypes.c_int), ("tucker", ctypes.POINTER(Tucker)),
                ("fast_refine", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("sweeps", ctypes.c_int),
                ("matvecs", ctypes.c_int), ("converged", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class VoxCapError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"voxcap error {code}: {msg}")
        self.code = code


_LIB = None


def lib():
    """Load libvoxcap.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} not found: run paper_2004_02609_gb300/build.py "
                              "(or __graft_entry__.build()) first")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        P = ctypes.POINTER
        L.voxcap_default_opts.argtypes = [P(Opts)]
        L.voxcap_default_opts.restype = None
        L.voxcap_last_error.restype = ctypes.c_char_p
        L.voxcap_setup.argtypes = [vp, i32, i32, i32, i32, vp, vp, i32, dbl, P(Opts), vp,
                                   P(vp)]
        L.voxcap_destroy.argtypes = [vp]
        L.voxcap_destroy.restype = None
        L.voxcap_num_panels.argtypes = [vp, i32, P(i64), P(i64), P(i32), P(i64), P(i64)]
        L.voxcap_panel_map.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp]
        L.voxcap_matvec.argtypes = [vp, vp, vp, i32, i32, i32]
        L.voxcap_solve.argtypes = [vp, vp, i32, dbl, vp, P(Stats)]
        L.voxcap_capacitance.argtypes = [vp, dbl, vp, vp, P(Stats)]
        L.voxcap_capacitance_columns.argtypes = [vp, dbl, i32, i32, vp, P(Stats)]
        L.voxcap_capacitance_grad.argtypes = [vp, vp, dbl, vp, P(Stats)]
        L.voxcap_update_eps.argtypes = [vp, vp]
        L.voxcap_entries.argtypes = [i32, vp, vp, vp, vp, vp]
        L.voxcap_fft_length.argtypes = [vp, P(i32), P(i32), P(i32)]
        L.voxcap_toeplitz.argtypes = [vp, i32, vp, P(i32)]
        L.voxcap_matvec_noalloc.argtypes = [vp, vp, vp, i32, i32, i32]
        L.voxcap_tucker_expand.argtypes = [vp, i32, i32, i32, vp, i32, vp, i32, vp, i32, vp]
        L.voxcap_canonical_tensors.argtypes = [i32, vp, vp, vp, vp]
        L.voxcap_set_product_tiles.argtypes = [vp, i32, i32, i32, i32, P(i32)]
        L.voxcap_set_product_path.argtypes = [vp, i32, P(i32)]
        L.voxcap_setup_times.argtypes = [vp, vp]
        L.voxcap_launch_count.argtypes = []
        L.voxcap_launch_count.restype = ctypes.c_int64
        _LIB = L
    return _LIB


def _check(rc, allow=()):
    if rc != OK and rc not in allow:
        msg = lib().voxcap_last_error().decode(errors="replace")
        raise VoxCapError(rc, msg)
    return rc


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().voxcap_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if k == "nv":
            v = (v, v, v) if np.isscalar(v) else tuple(v)
            o.nv = (ctypes.c_int * 3)(*v)
        elif k == "precond" and isinstance(v, str):
            o.precond = PRECOND[v]
        elif k == "tucker":
            if v is not None:
                t = v.as_ctypes()
                o._tucker_ref = (v, t)
                o.tucker = ctypes.pointer(t)
        elif k == "precision" and isinstance(v, str):
            o.precision = {"fp64": FP64, "fp32_refine": FP32_REFINE}[v]
        elif k == "entries" and isinstance(v, str):
            o.entries = ENTRIES[v]
        else:
            setattr(o, k, v)
    return o


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class VoxCap:
    """One handle: a voxel structure (or a batch of same-shape structures)
    set up for FFT-accelerated capacitance extraction on the current GPU.

    labels: int array [nz, ny, nx] or [n_struct, nz, ny, nx] (numpy or torch,
    host or CUDA); conductor_id / eps_r: per-label arrays; voxel_size in m."""

    def __init__(self, labels, conductor_id, eps_r, voxel_size=1e-6, **opts):
        import torch
        L = lib()
        if isinstance(labels, torch.Tensor):
            lab = labels.to(torch.int32).contiguous()
            keep = lab
            ptr = ctypes.c_void_p(lab.data_ptr())
            shape = tuple(lab.shape)
        else:
            lab = np.ascontiguousarray(labels, dtype=np.int32)
            keep = lab
            ptr = ctypes.c_void_p(lab.ctypes.data)
            shape = lab.shape
        if len(shape) == 3:
            shape = (1,) + tuple(shape)
        S, nz, ny, nx = shape
        self.cid = np.ascontiguousarray(conductor_id, dtype=np.int32)
        self.eps = np.ascontiguousarray(eps_r, dtype=np.float64)
        self.n_labels = len(self.cid)
        self.voxel_size = float(voxel_size)
        self.shape = (nx, ny, nz)
        self.n_struct = S
        o = default_opts(**opts)
        self.opts = o
        h = ctypes.c_void_p()
        rc = L.voxcap_setup(ptr, nx, ny, nz, S, self.cid.ctypes.data, self.eps.ctypes.data,
                            self.n_labels, self.voxel_size, ctypes.byref(o), _stream(),
                            ctypes.byref(h))
        del keep
        _check(rc)
        self._h = h
        nc, nd, m, nt, off = (ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int(),
                              ctypes.c_int64(), ctypes.c_int64())
        self.structs = []
        for s in range(S):
            _check(L.voxcap_num_panels(h, s, ctypes.byref(nc), ctypes.byref(nd),
                                       ctypes.byref(m), ctypes.byref(nt), ctypes.byref(off)))
            self.structs.append(dict(n_cond=nc.value, n_diel=nd.value, n_conductors=m.value,
                                     offset=off.value))
        self.N = nt.value

    def close(self):
        if getattr(self, "_h", None):
            lib().voxcap_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- queries ----
    @property
    def n_conductors(self):
        return self.structs[0]["n_conductors"]

    def set_product_tiles(self, z_order=-1, z_tile_log2=4, y_fwd_log2=-1, y_inv_log2=-1):
        """Force the launch variant of the FP32 products (z radix order 0/1,
        tile widths as log2; -1 = default y width), re-run the autotuner
        (z_order=-1) or only query (z_order=-2); returns the choice in force
        as a 4-tuple."""
        out = (ctypes.c_int * 4)()
        _check(lib().voxcap_set_product_tiles(self._h, z_order, z_tile_log2, y_fwd_log2, y_inv_log2, out))
        return tuple(out)

    def setup_times(self):
        """Wall seconds of the set-up phases: plans, panels, Toeplitz tensors
        (generated or Tucker-restored), spectra, preconditioner, tuning."""
        out = np.zeros(6, np.float64)
        _check(lib().voxcap_setup_times(self._h, out.ctypes.data))
        return dict(zip(("plans", "panels", "toeplitz", "spectra", "precond", "tuning"), out.tolist()))

    def set_product_path(self, path=-1):
        """FP32 product kernels: 0 generic, 1 compiled radix plans where the
        padded lengths have one (plus variant bits 2: persistent z pass, 4 /
        8: persistent forward / inverse y pass), -1 re-tune, -2 query; returns
        the path in force with its variant bits."""
        out = ctypes.c_int()
        _check(lib().voxcap_set_product_path(self._h, int(path), ctypes.byref(out)))
        return out.value

    def fft_lengths(self):
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().voxcap_fft_length(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def panel_map(self, s=0):
        d = self.structs[s]
        n = d["n_cond"] + d["n_diel"]
        out = dict(orient=np.zeros(n, np.int8), face=np.zeros(n, np.int32),
                   kind=np.zeros(n, np.int8), owner=np.zeros(n, np.int16),
                   idiag=np.zeros(n, np.float64), qscale=np.zeros(n, np.float64))
        _check(lib().voxcap_panel_map(self._h, s, *(out[k].ctypes.data for k in
                                                   ("orient", "face", "kind", "owner", "idiag", "qscale"))))
        return out

    def toeplitz(self, t):
        dims = (ctypes.c_int * 3)()
        _check(lib().voxcap_toeplitz(self._h, t, None, dims))
        out = np.zeros(dims[0] * dims[1] * dims[2], np.float64)
        _check(lib().voxcap_toeplitz(self._h, t, out.ctypes.data, dims))
        return out.reshape(dims[2], dims[1], dims[0])     # [ez][ey][ex]

    # ---- compute ----
    def matvec(self, x, precondition=False, adjoint=False, r_only=False):
        """y = A x (or R A x, A^T x, R x) for a CUDA tensor x of shape [N] or
        [nrhs, N] (each row one column of the N x nrhs operand)."""
        import torch
        assert x.is_cuda
        x2 = x.reshape(-1, self.N).contiguous()
        y = torch.empty_like(x2)
        dt = {torch.float32: F32, torch.float64: F64}[x2.dtype]
        fl = (MV_PRECOND if precondition else 0) | (MV_ADJOINT if adjoint else 0) | \
            (MV_RONLY if r_only else 0)
        _check(lib().voxcap_matvec(self._h, _ptr(x2), _ptr(y), x2.shape[0], dt, fl))
        return y.reshape(x.shape)

    def matvec_noalloc(self, x, precondition=False, adjoint=False, r_only=False):
        """matvec through voxcap_matvec_noalloc: same result, no device
        allocation inside the call (fixed 16 MiB library scratch)."""
        import torch
        assert x.is_cuda
        x2 = x.reshape(-1, self.N).contiguous()
        y = torch.empty_like(x2)
        dt = {torch.float32: F32, torch.float64: F64}[x2.dtype]
        fl = (MV_PRECOND if precondition else 0) | (MV_ADJOINT if adjoint else 0) | \
            (MV_RONLY if r_only else 0)
        _check(lib().voxcap_matvec_noalloc(self._h, _ptr(x2), _ptr(y), x2.shape[0], dt, fl))
        return y.reshape(x.shape)

    def solve(self, B, tol=1e-6, allow_unconverged=False):
        """X with A X = B (B: CUDA float64 [nrhs, N] or [N])."""
        import torch
        B2 = B.reshape(-1, self.N).to(torch.float64).contiguous()
        X = torch.empty_like(B2)
        st = Stats()
        rc = lib().voxcap_solve(self._h, _ptr(B2), B2.shape[0], float(tol), _ptr(X), ctypes.byref(st))
        _check(rc, allow=(ERR_NOT_CONVERGED,) if allow_unconverged else ())
        return X.reshape(B.shape), st.as_dict()

    def capacitance(self, tol=1e-6, return_charges=False, allow_unconverged=False):
        """Capacitance matrices in farads: [m, m] for one structure, a list for
        a batch of structures."""
        import torch
        ms = [d["n_conductors"] for d in self.structs]
        C = np.zeros(sum(m * m for m in ms), np.float64)
        st = Stats()
        rho = None
        rptr = None
        if return_charges:
            rho = torch.empty((max(ms), self.N), dtype=torch.float64, device="cuda")
            rptr = _ptr(rho)
        rc = lib().voxcap_capacitance(self._h, float(tol), C.ctypes.data, rptr, ctypes.byref(st))
        _check(rc, allow=(ERR_NOT_CONVERGED,) if allow_unconverged else ())
        out, o = [], 0
        for m in ms:
            out.append(C[o:o + m * m].reshape(m, m))
            o += m * m
        res = out[0] if len(out) == 1 else out
        if return_charges:
            return res, st.as_dict(), rho
        return res, st.as_dict()

    def capacitance_columns(self, j0, j1, tol=1e-6, allow_unconverged=False):
        """Columns j0..j1-1 of the capacitance matrix (farads, [m, j1-j0]) of
        a single structure: the solves of those conductors only."""
        m = self.structs[0]["n_conductors"]
        C = np.zeros(self.n_struct * m * (j1 - j0), np.float64)
        st = Stats()
        rc = lib().voxcap_capacitance_columns(self._h, float(tol), int(j0), int(j1), C.ctypes.data,
                                              ctypes.byref(st))
        _check(rc, allow=(ERR_NOT_CONVERGED,) if allow_unconverged else ())
        out = C.reshape(self.n_struct, m, j1 - j0)
        return (out[0] if self.n_struct == 1 else list(out)), st.as_dict()

    def capacitance_grad(self, dL_dC, tol=1e-6):
        """dL/d eps_r[label] for L = sum(dL_dC * C), after capacitance()."""
        G = np.ascontiguousarray(np.concatenate([np.asarray(g, np.float64).reshape(-1) for g in
                                                 (dL_dC if isinstance(dL_dC, list) else [dL_dC])]))
        out = np.zeros(self.n_labels, np.float64)
        st = Stats()
        _check(lib().voxcap_capacitance_grad(self._h, G.ctypes.data, float(tol), out.ctypes.data,
                                             ctypes.byref(st)))
        return out, st.as_dict()

    def update_eps(self, eps_r):
        self.eps = np.ascontiguousarray(eps_r, dtype=np.float64)
        _check(lib().voxcap_update_eps(self._h, self.eps.ctypes.data))
        nc, nd, m, nt, off = (ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int(),
                              ctypes.c_int64(), ctypes.c_int64())
        for s in range(self.n_struct):
            _check(lib().voxcap_num_panels(self._h, s, ctypes.byref(nc), ctypes.byref(nd),
                                           ctypes.byref(m), ctypes.byref(nt), ctypes.byref(off)))
            self.structs[s] = dict(n_cond=nc.value, n_diel=nd.value, n_conductors=m.value,
                                   offset=off.value)
        self.N = nt.value


def tucker_expand(core, U1, U2, U3):
    """X = core x1 U1 x2 U2 x3 U3 on the tensor cores (voxcap_tucker_expand);
    torch CUDA float64 inputs, returns X[i, j, k] (numpy)."""
    import torch
    r1, r2, r3 = core.shape
    D1, D2, D3 = U1.shape[0], U2.shape[0], U3.shape[0]
    args = [t.contiguous().to(torch.float64) for t in (core, U1, U2, U3)]
    out = torch.empty(D1 * D2 * D3, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    _check(lib().voxcap_tucker_expand(_ptr(args[0]), r1, r2, r3, _ptr(args[1]), D1, _ptr(args[2]), D2,
                                      _ptr(args[3]), D3, _ptr(out)))
    return out.cpu().numpy().reshape(D3, D2, D1).transpose(2, 1, 0)


def launch_count() -> int:
    """Kernel launches issued by the library in this process so far."""
    return int(lib().voxcap_launch_count())


def entries(kind, test_orient, src_orient, d):
    """Galerkin integrals of panel pairs by the device entry generator
    (kind 0: P' of Eq. 5, 1: E' of Eq. 6); d = test centre - source centre."""
    import torch
    n = len(d)
    k = torch.as_tensor(np.broadcast_to(kind, (n,)).astype(np.int32), device="cuda")
    to = torch.as_tensor(np.broadcast_to(test_orient, (n,)).astype(np.int32), device="cuda")
    so = torch.as_tensor(np.broadcast_to(src_orient, (n,)).astype(np.int32), device="cuda")
    dd = torch.as_tensor(np.ascontiguousarray(d, dtype=np.float64).reshape(n, 3), device="cuda")
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    _check(lib().voxcap_entries(n, _ptr(k), _ptr(to), _ptr(so), _ptr(dd), _ptr(out)))
    return out.cpu().numpy()


def capacitance_fn(handle: "VoxCap", eps_r, tol: float = 1e-8):
    """Differentiable capacitance: C(eps_r) through torch.autograd.

    ``eps_r`` is a float64 torch tensor [n_labels] (requires_grad as needed);
    the forward pass updates the handle's permittivities and extracts C (farads,
    [m, m]); the backward pass is the library's batched adjoint solve
    (voxcap_capacitance_grad)."""
    import torch

    class _Cap(torch.autograd.Function):
        @staticmethod
        def forward(ctx, eps):
            e = eps.detach().to("cpu", torch.float64).numpy()
            if not np.array_equal(e, handle.eps):
                handle.update_eps(e)
            C, _ = handle.capacitance(tol=tol)
            return torch.as_tensor(np.asarray(C), dtype=torch.float64, device=eps.device)

        @staticmethod
        def backward(ctx, gC):
            g, _ = handle.capacitance_grad(gC.detach().to("cpu", torch.float64).numpy(), tol=tol)
            return torch.as_tensor(g, dtype=torch.float64, device=gC.device)

    return _Cap.apply(eps_r)
