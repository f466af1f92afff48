"""Thin Python binding of the kitrt C ABI (include/kitrt.h).

Argument marshalling only: every step of the M_N path runs in the library's CUDA kernels. Device
arrays are torch CUDA tensors (the library reads their data pointers); work is enqueued on
torch's current stream. There is no CPU fallback: if the library cannot be loaded, every call
raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

KITRT_OK = 0
STATUS_NAMES = {0: "ok", 1: "EINVAL", 2: "ENOTREALIZABLE", 3: "ENOCONVERGE", 4: "ECHOL",
                5: "ELINESEARCH", 6: "ECUDA", 7: "ENOMEM", 8: "ETIMEOUT", 9: "ESCRATCH"}
MODES = {"fp64": 0, "mixed_tf32": 1, "mixed_bf16": 2, "learned": 3}
BCS = {"neumann": 0, "vacuum": 1}


class KitrtError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)} ({_lib().kitrt_status_string(code).decode()})")


class Params(C.Structure):
    _fields_ = [("degree", C.c_int32), ("quad_order", C.c_int32), ("mode", C.c_int32),
                ("bc", C.c_int32), ("tau", C.c_double), ("max_iter", C.c_int32),
                ("max_halvings", C.c_int32), ("armijo_c1", C.c_double), ("polish", C.c_int32),
                ("cfl", C.c_double), ("fallback_tol", C.c_double), ("order", C.c_int32),
                ("reg_gamma", C.c_double), ("reg_keep_mass", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("closures", C.c_int64), ("evaluations", C.c_int64), ("max_evals", C.c_int32),
                ("failed", C.c_int32), ("fallbacks", C.c_int64), ("dt", C.c_double),
                ("launches", C.c_int64), ("restarts", C.c_int64), ("proposals", C.c_int64),
                ("handovers", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Work(C.Structure):
    _fields_ = [("nmom", C.c_int32), ("nmom2", C.c_int32), ("nquad_folded", C.c_int32),
                ("gaunt_nnz", C.c_int32), ("sweep_fp64_flops", C.c_double), ("exps", C.c_double),
                ("tensor_flops", C.c_double), ("newton_flops", C.c_double),
                ("sweep_fp64_ops", C.c_double), ("sweep_grid", C.c_int32),
                ("sweep_items", C.c_int32)]


class ProfileEntry(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int64), ("units", C.c_int64),
                ("total_ms", C.c_double)]


_LIB = None
_vp = C.c_void_p
_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)

# name -> (restype, argtypes); kept in the order of include/kitrt.h
SIGNATURES = {
    "kitrt_status_string": (C.c_char_p, [C.c_int32]),
    "kitrt_default_params": (C.c_int32, [C.POINTER(Params)]),
    "kitrt_mesh_create": (C.c_int32, [_dp, C.c_int32, _ip, C.c_int32, C.POINTER(_vp)]),
    "kitrt_mesh_destroy": (C.c_int32, [_vp]),
    "kitrt_mesh_geometry": (C.c_int32, [_vp, _ip, _dp, _dp, _dp, _dp, _ip, _dp]),
    "kitrt_mn_init": (C.c_int32, [_vp, C.POINTER(Params), C.POINTER(_vp)]),
    "kitrt_mn_destroy": (C.c_int32, [_vp]),
    "kitrt_mn_sizes": (C.c_int32, [_vp, _ip, _ip, _ip]),
    "kitrt_mn_work": (C.c_int32, [_vp, C.POINTER(Work)]),
    "kitrt_mn_quadrature": (C.c_int32, [_vp, _dp, _dp, _dp]),
    "kitrt_isotropic_alpha": (C.c_int32, [_vp, _vp, _vp, _vp]),
    "kitrt_closure": (C.c_int32, [_vp, _vp, _vp, _vp, _vp, C.POINTER(Stats)]),
    "kitrt_closure_batch": (C.c_int32, [_vp, _vp, _vp, _vp, C.c_int32, _vp, C.POINTER(Stats)]),
    "kitrt_hessian": (C.c_int32, [_vp, _vp, _vp, _vp]),
    "kitrt_ansatz": (C.c_int32, [_vp, _vp, _vp, _vp]),
    "kitrt_step": (C.c_int32, [_vp, _vp, _vp, _vp, _vp, _vp, C.c_double, C.c_int32, _vp, _vp,
                               C.POINTER(Stats)]),
    "kitrt_mn_set_density": (C.c_int32, [_vp, _vp, _vp]),
    "kitrt_dose_accumulate": (C.c_int32, [_vp, _vp, C.c_double, C.c_double, _vp, _vp]),
    "kitrt_adjoint": (C.c_int32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, C.c_int32, _vp, C.c_double,
                                  C.c_int32, C.c_int32, _vp, _vp, _vp, _vp]),
    "kitrt_mlp_param_count": (C.c_int32, [C.c_int32, C.c_int32, C.c_int32]),
    "kitrt_mlp_work_floats": (C.c_int32, [C.c_int32, C.c_int32, C.c_int32]),
    "kitrt_mlp_forward": (C.c_int32, [C.c_int32, C.c_int32, C.c_int32, _vp, _vp, _vp, C.c_int32,
                                      _vp, _vp]),
    "kitrt_mlp_loss_grad": (C.c_int32, [C.c_int32, C.c_int32, C.c_int32, _vp, _vp, _vp, C.c_int32,
                                        _vp, _vp, _vp, _vp]),
    "kitrt_mlp_adam": (C.c_int32, [C.c_int32, _vp, _vp, _vp, _vp, C.c_int32, C.c_float, C.c_float,
                                   C.c_float, C.c_float, _vp]),
    "kitrt_mn_set_mlp": (C.c_int32, [_vp, _vp, _vp, C.c_int32, _vp]),
    "kitrt_vmf_moments": (C.c_int32, [_vp, _vp, _vp, _vp, C.c_int32, C.c_int32, _vp, _vp]),
    "kitrt_closure_noalloc": (C.c_int32, [_vp, _vp, _vp, _vp, C.c_int32, _vp]),
    "kitrt_mn_reset": (C.c_int32, [_vp]),
    "kitrt_sn_step": (C.c_int32, [_vp, _vp, _vp, C.c_int32, _vp, _vp, _vp, _dp, C.c_double,
                                  C.c_int32, _vp]),
    "kitrt_gather_rows": (C.c_int32, [_vp, _vp, C.c_int32, C.c_int32, _vp, _vp]),
    "kitrt_scatter_rows": (C.c_int32, [_vp, _vp, C.c_int32, C.c_int32, _vp, _vp]),
    "kitrt_scatter_add_rows": (C.c_int32, [_vp, _vp, C.c_int32, C.c_int32, _vp, _vp]),
    "kitrt_profile_enable": (C.c_int32, [_vp, C.c_int32]),
    "kitrt_profile_read": (C.c_int32, [_vp, C.POINTER(ProfileEntry), C.c_int32, _ip]),
}


def library_path() -> str:
    return _build.LIB


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"kitrt CUDA library not built ({path}); run "
                               "`python -m paper_2205_08417_gb300.build`")
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _check(rc: int, where: str):
    if rc != KITRT_OK:
        raise KitrtError(rc, where)


def _dev(t, dtype=None):
    """Data pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("kitrt expects contiguous CUDA tensors")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"kitrt expects {dtype}, got {t.dtype}")
    return C.c_void_p(t.data_ptr())


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _np_d(a):
    return a.ctypes.data_as(_dp)


def _np_i(a):
    return a.ctypes.data_as(_ip)


class Mesh:
    """Triangle mesh handle (kitrt_mesh_create)."""

    def __init__(self, xy: np.ndarray, tri: np.ndarray):
        self._xy = np.ascontiguousarray(xy, dtype=np.float64)
        self._tri = np.ascontiguousarray(tri, dtype=np.int32)
        h = C.c_void_p()
        _check(_lib().kitrt_mesh_create(_np_d(self._xy), self._xy.shape[0], _np_i(self._tri),
                                        self._tri.shape[0], C.byref(h)), "kitrt_mesh_create")
        self.handle = h
        self.ncells = int(self._tri.shape[0])

    def geometry(self):
        Cc = self.ncells
        area, perim = np.zeros(Cc), np.zeros(Cc)
        cen, nbr, nrm = np.zeros((Cc, 2)), np.zeros((Cc, 3), np.int32), np.zeros((Cc, 3, 2))
        nc = C.c_int32()
        mr = C.c_double()
        _check(_lib().kitrt_mesh_geometry(self.handle, C.byref(nc), C.byref(mr), _np_d(area),
                                          _np_d(perim), _np_d(cen), _np_i(nbr), _np_d(nrm)),
               "kitrt_mesh_geometry")
        return dict(area=area, perim=perim, centroid=cen, nbr=nbr, nrm=nrm,
                    min_inradius=mr.value)

    def close(self):
        if getattr(self, "handle", None):
            _lib().kitrt_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MNSolver:
    """M_N solver handle (kitrt_mn_init) bound to a Mesh."""

    def __init__(self, mesh: Mesh, degree: int, quad_order: int, mode: str = "fp64",
                 bc: str = "neumann", **opts):
        p = Params()
        _check(_lib().kitrt_default_params(C.byref(p)), "kitrt_default_params")
        p.degree = degree
        p.quad_order = quad_order
        p.mode = MODES[mode]
        p.bc = BCS[bc]
        for k, v in opts.items():
            setattr(p, k, v)
        self.params = p
        self.mesh = mesh
        h = C.c_void_p()
        _check(_lib().kitrt_mn_init(mesh.handle, C.byref(p), C.byref(h)), "kitrt_mn_init")
        self.handle = h
        n, Q, Qf = C.c_int32(), C.c_int32(), C.c_int32()
        _check(_lib().kitrt_mn_sizes(h, C.byref(n), C.byref(Q), C.byref(Qf)), "kitrt_mn_sizes")
        self.n, self.Q, self.Qf = n.value, Q.value, Qf.value

    def work(self):
        w = Work()
        _check(_lib().kitrt_mn_work(self.handle, C.byref(w)), "kitrt_mn_work")
        return {k: getattr(w, k) for k, _ in w._fields_}

    def quadrature(self):
        w = np.zeros(self.Qf)
        om = np.zeros((self.Qf, 2))
        m = np.zeros((self.Qf, self.n))
        _check(_lib().kitrt_mn_quadrature(self.handle, _np_d(w), _np_d(om), _np_d(m)),
               "kitrt_mn_quadrature")
        return w, om, m

    def isotropic_alpha(self, u):
        import torch
        alpha = torch.empty_like(u)
        _check(_lib().kitrt_isotropic_alpha(self.handle, _dev(u, torch.float64),
                                            _dev(alpha, torch.float64), _stream()),
               "kitrt_isotropic_alpha")
        return alpha

    def closure(self, u, alpha, status=None, stats: bool = False, check: bool = True):
        import torch
        st = Stats()
        rc = _lib().kitrt_closure(self.handle, _dev(u, torch.float64), _dev(alpha, torch.float64),
                                  _dev(status, torch.int32), _stream(),
                                  C.byref(st) if stats else None)
        if check:
            _check(rc, "kitrt_closure")
        return (rc, st.as_dict()) if stats else rc

    def closure_batch(self, u, alpha, status=None, stats: bool = False, check: bool = True):
        """Closure of the first u.shape[0] rows (at most the mesh's cell count)."""
        import torch
        st = Stats()
        rc = _lib().kitrt_closure_batch(self.handle, _dev(u, torch.float64), _dev(alpha, torch.float64),
                                        _dev(status, torch.int32), int(u.shape[0]), _stream(),
                                        C.byref(st) if stats else None)
        if check:
            _check(rc, "kitrt_closure_batch")
        return (rc, st.as_dict()) if stats else rc

    def vmf_moments(self, centres, kappa, weight):
        """Moments of von Mises-Fisher mixtures (device FP64 tensors [count, lobes, 3],
        [count, lobes], [count, lobes]) on this solver's quadrature."""
        import torch
        count, lobes = kappa.shape
        u = torch.empty((count, self.n), dtype=torch.float64, device=kappa.device)
        _check(_lib().kitrt_vmf_moments(self.handle, _dev(centres, torch.float64), _dev(kappa, torch.float64),
                                        _dev(weight, torch.float64), int(lobes), int(count), _dev(u),
                                        _stream()), "kitrt_vmf_moments")
        return u

    def adjoint(self, u0, alpha0, sigma_a, sigma_s, q, block_of_cell, nblocks, target, dt, nsteps,
                ckpt_every=16):
        """(J, dJ/dsigma_a per block, dJ/dsigma_s per block): a float and two host FP64 arrays."""
        import torch
        J = np.zeros(1)
        gsa = np.zeros(int(nblocks))
        gss = np.zeros(int(nblocks))
        _check(_lib().kitrt_adjoint(self.handle, _dev(u0, torch.float64), _dev(alpha0, torch.float64),
                                    _dev(sigma_a, torch.float64), _dev(sigma_s, torch.float64),
                                    _dev(q, torch.float64), _dev(block_of_cell, torch.int32), int(nblocks),
                                    _dev(target, torch.uint8), float(dt), int(nsteps), int(ckpt_every),
                                    J.ctypes.data_as(C.c_void_p), gsa.ctypes.data_as(C.c_void_p),
                                    gss.ctypes.data_as(C.c_void_p), _stream()), "kitrt_adjoint")
        return float(J[0]), gsa, gss

    def set_mlp(self, params, norm, hidden: int = 64):
        import torch
        _check(_lib().kitrt_mn_set_mlp(self.handle, _dev(params, torch.float32), _dev(norm, torch.float32),
                                       int(hidden), _stream()), "kitrt_mn_set_mlp")

    def closure_noalloc(self, u, alpha, status=None, check: bool = True):
        """Closure of a batch (any number of rows up to the fixed scratch limit) through the
        allocation-free entry point."""
        import torch
        rc = _lib().kitrt_closure_noalloc(self.handle, _dev(u, torch.float64),
                                          _dev(alpha, torch.float64), _dev(status, torch.int32),
                                          int(u.shape[0]), _stream())
        if check:
            _check(rc, "kitrt_closure_noalloc")
        return rc

    def sn_step(self, psi, work, sigma_a, sigma_s, q, dt: float = 0.0, nsteps: int = 1, g=None,
                check: bool = True):
        """nsteps S_N steps of the ordinates psi [C, Q'] (float64 or float32 CUDA tensor) in
        place; work is scratch of the same shape and dtype. g: per-degree scattering coefficients
        (length N+1, g[0] = 1) or None for isotropic scattering."""
        import torch
        if psi.dtype not in (torch.float32, torch.float64) or work.dtype != psi.dtype:
            raise ValueError("psi and work must share a float32 or float64 dtype")
        if tuple(psi.shape) != (self.mesh.ncells, self.Qf) or work.shape != psi.shape:
            raise ValueError("psi and work must be [ncells, Q'] (folded quadrature points)")
        gp = None
        if g is not None:
            g = np.ascontiguousarray(g, dtype=np.float64)
            gp = _np_d(g)
        rc = _lib().kitrt_sn_step(self.handle, _dev(psi), _dev(work),
                                  int(psi.dtype == torch.float32), _dev(sigma_a, torch.float64),
                                  _dev(sigma_s, torch.float64), _dev(q, torch.float64), gp,
                                  float(dt), int(nsteps), _stream())
        if check:
            _check(rc, "kitrt_sn_step")
        return rc

    def hessian(self, alpha):
        import torch
        n = self.n
        H = torch.empty((alpha.shape[0], n, n), dtype=torch.float64, device=alpha.device)
        _check(_lib().kitrt_hessian(self.handle, _dev(alpha, torch.float64), _dev(H), _stream()),
               "kitrt_hessian")
        return H

    def ansatz(self, alpha):
        import torch
        psi = torch.empty((alpha.shape[0], self.Qf), dtype=torch.float64, device=alpha.device)
        _check(_lib().kitrt_ansatz(self.handle, _dev(alpha, torch.float64), _dev(psi), _stream()),
               "kitrt_ansatz")
        return psi

    def step(self, u, alpha, sigma_a, sigma_s, q, dt: float = 0.0, nsteps: int = 1,
             status=None, stats: bool = False, check: bool = True):
        import torch
        st = Stats()
        rc = _lib().kitrt_step(self.handle, _dev(u, torch.float64), _dev(alpha, torch.float64),
                               _dev(sigma_a, torch.float64), _dev(sigma_s, torch.float64),
                               _dev(q, torch.float64), float(dt), int(nsteps),
                               _dev(status, torch.int32), _stream(),
                               C.byref(st) if stats else None)
        if check:
            _check(rc, "kitrt_step")
        return (rc, st.as_dict()) if stats else rc

    def set_density(self, rho):
        """Density per cell of the transformed CSD equation (FP64 CUDA tensor [C]), or None to
        remove it: later first-order steps transport psi / rho."""
        import torch
        _check(_lib().kitrt_mn_set_density(self.handle, _dev(rho, torch.float64), _stream()),
               "kitrt_mn_set_density")

    def dose_accumulate(self, u, S: float, dt: float, dose):
        """dose += dt S u_0 / (m_0 rho): one pseudo-time step of the dose (FP64 CUDA tensors)."""
        import torch
        _check(_lib().kitrt_dose_accumulate(self.handle, _dev(u, torch.float64), float(S),
                                            float(dt), _dev(dose, torch.float64), _stream()),
               "kitrt_dose_accumulate")

    def reset(self):
        """Forget the closure state kept for continuation: the next step starts from its alpha."""
        _check(_lib().kitrt_mn_reset(self.handle), "kitrt_mn_reset")

    def profile(self, on: bool = True):
        _check(_lib().kitrt_profile_enable(self.handle, int(on)), "kitrt_profile_enable")

    def profile_read(self):
        arr = (ProfileEntry * 16)()
        cnt = C.c_int32()
        _check(_lib().kitrt_profile_read(self.handle, arr, 16, C.byref(cnt)), "kitrt_profile_read")
        return {arr[i].name.decode(): dict(launches=arr[i].launches, units=arr[i].units,
                                           total_ms=arr[i].total_ms) for i in range(cnt.value)}

    def close(self):
        if getattr(self, "handle", None):
            _lib().kitrt_mn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- Halo rows of a step split over ranks -----------------------------------------------------
def gather_rows(src, idx, dst):
    """dst[k] = src[idx[k]] (FP64 CUDA tensors, idx int32 CUDA)."""
    import torch
    _check(_lib().kitrt_gather_rows(_dev(src, torch.float64), _dev(idx, torch.int32), int(idx.numel()),
                                    int(src.shape[1]), _dev(dst, torch.float64), _stream()),
           "kitrt_gather_rows")


def scatter_rows(src, idx, dst):
    """dst[idx[k]] = src[k] (FP64 CUDA tensors, idx int32 CUDA)."""
    import torch
    _check(_lib().kitrt_scatter_rows(_dev(src, torch.float64), _dev(idx, torch.int32), int(idx.numel()),
                                     int(dst.shape[1]), _dev(dst, torch.float64), _stream()),
           "kitrt_scatter_rows")


def scatter_add_rows(src, idx, dst):
    """dst[idx[k]] += src[k] (FP64 CUDA tensors, idx int32 CUDA with distinct entries)."""
    import torch
    _check(_lib().kitrt_scatter_add_rows(_dev(src, torch.float64), _dev(idx, torch.int32),
                                         int(idx.numel()), int(src.shape[1]),
                                         _dev(dst, torch.float64), _stream()),
           "kitrt_scatter_add_rows")


# ---- MLP kernels of the learned closure -------------------------------------------------------
def mlp_param_count(din: int, hidden: int, dout: int) -> int:
    return int(_lib().kitrt_mlp_param_count(din, hidden, dout))


def mlp_forward(params, X, din: int, hidden: int, dout: int):
    import torch
    B = X.shape[0]
    Y = torch.empty((B, dout), dtype=torch.float32, device=X.device)
    work = torch.empty(max(1, _lib().kitrt_mlp_work_floats(B, hidden, dout)), dtype=torch.float32,
                       device=X.device)
    _check(_lib().kitrt_mlp_forward(din, hidden, dout, _dev(params, torch.float32), _dev(X, torch.float32),
                                    _dev(Y), B, _dev(work), _stream()), "kitrt_mlp_forward")
    return Y


def mlp_loss_grad(params, X, T, din: int, hidden: int, dout: int, work=None):
    import torch
    B = X.shape[0]
    grad = torch.empty_like(params)
    loss = torch.empty(1, dtype=torch.float32, device=X.device)
    if work is None:
        work = torch.empty(_lib().kitrt_mlp_work_floats(B, hidden, dout), dtype=torch.float32,
                           device=X.device)
    _check(_lib().kitrt_mlp_loss_grad(din, hidden, dout, _dev(params, torch.float32), _dev(X, torch.float32),
                                      _dev(T, torch.float32), B, _dev(grad), _dev(loss), _dev(work),
                                      _stream()), "kitrt_mlp_loss_grad")
    return loss, grad


def mlp_adam(params, grad, m, v, t: int, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    import torch
    _check(_lib().kitrt_mlp_adam(int(params.numel()), _dev(params, torch.float32), _dev(grad, torch.float32),
                                 _dev(m, torch.float32), _dev(v, torch.float32), int(t), float(lr), float(b1),
                                 float(b2), float(eps), _stream()), "kitrt_mlp_adam")
