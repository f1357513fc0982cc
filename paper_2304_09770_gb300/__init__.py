"""Python binding of libvembddc (BDDC-preconditioned CG for divergence-free
VEM Stokes on one GPU).  Argument marshalling only: every step of the
method runs inside the library's CUDA kernels.  Device vectors are torch
tensors (float64, cuda); host arrays are numpy arrays.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvembddc.so")
_lib = None

VEM_STATUS = {0: "VEM_OK", -1: "VEM_EINVAL", -2: "VEM_ENOMEM", -3: "VEM_ECUDA", -4: "VEM_ESINGULAR",
              -5: "VEM_EBREAKDOWN", -6: "VEM_ENOTCONV", -7: "VEM_ETIMEOUT"}


class VemError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{VEM_STATUS.get(status, status)}: {msg}")
        self.status = status


class _Mesh(ctypes.Structure):
    _fields_ = [("nV", ctypes.c_int32), ("xyz", ctypes.POINTER(ctypes.c_double)),
                ("nF", ctypes.c_int32), ("face_ptr", ctypes.POINTER(ctypes.c_int32)),
                ("face_vtx", ctypes.POINTER(ctypes.c_int32)), ("nE", ctypes.c_int32),
                ("elem_ptr", ctypes.POINTER(ctypes.c_int32)), ("elem_face", ctypes.POINTER(ctypes.c_int32))]


class BddcOptions(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("scaling", ctypes.c_int32), ("constraints", ctypes.c_uint32),
                ("adaptive_threshold", ctypes.c_double), ("nd_leaf", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("refine", ctypes.c_int32), ("tc_update", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 7)]


def lib():
    """Loads the in-tree library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.c_void_p
        i64p = ctypes.POINTER(ctypes.c_int64)
        L.vem_assemble.argtypes = [ctypes.POINTER(_Mesh), ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(P)]
        L.vem_assemble_reduced.argtypes = L.vem_assemble.argtypes
        L.vem_dof_layout.argtypes = [P, i64p, i64p, i64p]
        L.vem_free_dofs.argtypes = [P, i64p]
        L.vem_quad_points.argtypes = [P, ctypes.c_int, i64p, P]
        L.vem_load.argtypes = [P, ctypes.c_int, P, P]
        L.vem_load_noalloc.argtypes = [P, ctypes.c_int, P, P]
        L.vem_apply.argtypes = [P, P, P]
        L.vem_lift_dirichlet.argtypes = [P, P, P]
        L.vem_element_matrices.argtypes = [P, P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), P, P, P]
        L.vem_csr.argtypes = [P, i64p, i64p, P, P, P]
        L.vem_set_stream.argtypes = [P, P]
        L.vem_free.argtypes = [P]
        L.vem_free.restype = None
        L.vem_last_error.restype = ctypes.c_char_p
        L.vem_kernel_launches.argtypes = [i64p]
        L.vem_info.argtypes = [P, ctypes.c_char_p, ctypes.POINTER(ctypes.c_double)]
        if hasattr(L, "bddc_setup"):
            L.bddc_setup.argtypes = [P, ctypes.POINTER(ctypes.c_int32), ctypes.c_uint32, ctypes.c_int,
                                     ctypes.POINTER(BddcOptions), ctypes.POINTER(P)]
            L.bddc_apply.argtypes = [P, P, P]
            L.pcg_solve.argtypes = [P, P, P, ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double)]
            L.bddc_free.argtypes = [P]
            L.bddc_free.restype = None
        if hasattr(L, "bddc_info"):
            L.bddc_info.argtypes = [P, ctypes.c_char_p, ctypes.POINTER(ctypes.c_double)]
        if hasattr(L, "bddc_set_stream"):
            L.bddc_set_stream.argtypes = [P, P]
        if hasattr(L, "bddc_time_local_solves"):
            L.bddc_time_local_solves.argtypes = [P, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                                 ctypes.POINTER(ctypes.c_double)]
        _lib = L
    return _lib


def kernel_launches():
    """Kernels launched by the library since it was loaded."""
    c = ctypes.c_int64()
    _check(lib().vem_kernel_launches(ctypes.byref(c)))
    return c.value


def _check(status):
    if status != 0:
        raise VemError(status, lib().vem_last_error().decode())


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dptr(t):
    import torch
    assert t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
    return ctypes.c_void_p(t.data_ptr())


class VemSystem:
    """vem_assemble: VEM discretization of degree k on a polyhedral mesh
    (reduced=True: vem_assemble_reduced, the reduced scheme)."""

    def __init__(self, mesh, k, nu, reduced=False):
        L = lib()
        self._keep = dict(
            xyz=np.ascontiguousarray(mesh["xyz"], dtype=np.float64),
            fp=np.ascontiguousarray(mesh["face_ptr"], dtype=np.int32),
            fv=np.ascontiguousarray(mesh["face_vtx"], dtype=np.int32),
            ep=np.ascontiguousarray(mesh["elem_ptr"], dtype=np.int32),
            ef=np.ascontiguousarray(mesh["elem_face"], dtype=np.int32))
        kp = self._keep
        nu = np.ascontiguousarray(nu, dtype=np.float64)
        m = _Mesh(len(kp["xyz"]), kp["xyz"].ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                  len(kp["fp"]) - 1, kp["fp"].ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                  kp["fv"].ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                  len(kp["ep"]) - 1, kp["ep"].ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                  kp["ef"].ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        h = ctypes.c_void_p()
        fn = L.vem_assemble_reduced if reduced else L.vem_assemble
        _check(fn(ctypes.byref(m), int(k), nu.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(h)))
        self.h = h
        self.k = k
        self.reduced = bool(reduced)
        self.nE = len(kp["ep"]) - 1
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(L.vem_dof_layout(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        self.n_vel_free, self.n_press, self.n_vel = a.value, b.value, c.value
        self.n = self.n_vel_free + self.n_press

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.vem_free(self.h)
            self.h = None

    def free_dofs(self):
        out = np.zeros(self.n_vel_free, dtype=np.int64)
        _check(lib().vem_free_dofs(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
        return out

    def quad_points(self, degree):
        n = ctypes.c_int64()
        _check(lib().vem_quad_points(self.h, degree, ctypes.byref(n), None))
        out = np.zeros((n.value, 3))
        _check(lib().vem_quad_points(self.h, degree, ctypes.byref(n), _ptr(out)))
        return out

    def load(self, degree, f_values, out=None):
        """vem_load; f_values: numpy array (host) or float64 torch tensor
        (on the GPU: read in place; pinned host memory: copied)."""
        import torch
        if isinstance(f_values, torch.Tensor):
            assert f_values.dtype == torch.float64 and f_values.is_contiguous()
            fp = ctypes.c_void_p(f_values.data_ptr())
        else:
            f_values = np.ascontiguousarray(f_values, dtype=np.float64)
            fp = _ptr(f_values)
        if out is None:
            out = torch.empty(self.n, dtype=torch.float64, device="cuda")
        _check(lib().vem_load(self.h, degree, fp, _dptr(out)))
        return out

    def load_noalloc(self, degree, f_dev, out):
        """vem_load_noalloc: the load vector from f already on the device
        (float64 cuda tensor [n, 3] at the vem_quad_points rule), written
        into the caller's tensor `out`; the library allocates nothing."""
        _check(lib().vem_load_noalloc(self.h, int(degree), _dptr(f_dev), _dptr(out)))
        return out

    def apply(self, x, y=None):
        import torch
        if y is None:
            y = torch.empty_like(x)
        _check(lib().vem_apply(self.h, _dptr(x), _dptr(y)))
        return y

    def lift_dirichlet(self, g_values, f):
        """vem_lift_dirichlet: f -= K[:, fixed] g[fixed] in place, for
        prescribed values g (host, every velocity DOF, global numbering)."""
        g_values = np.ascontiguousarray(g_values, dtype=np.float64)
        assert g_values.shape == (self.n_vel,)
        _check(lib().vem_lift_dirichlet(self.h, _ptr(g_values), _dptr(f)))
        return f

    def element_matrices(self, elems):
        elems = np.ascontiguousarray(elems, dtype=np.int32)
        nk = ctypes.c_int32()
        # probe size with the first element
        e0 = elems[:1]
        _check(lib().vem_element_matrices(self.h, _ptr(e0), 1, ctypes.byref(nk), None, None, None))
        n, npk = nk.value, self.n_press // self.nE
        A = np.zeros((len(elems), n, n))
        B = np.zeros((len(elems), npk, n))
        D = np.zeros((len(elems), n), dtype=np.int64)
        _check(lib().vem_element_matrices(self.h, _ptr(elems), len(elems), ctypes.byref(nk), _ptr(A), _ptr(B),
                                          _ptr(D)))
        return A, B, D

    def csr(self):
        import scipy.sparse as sp
        n, nnz = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().vem_csr(self.h, ctypes.byref(n), ctypes.byref(nnz), None, None, None))
        rp = np.zeros(n.value + 1, dtype=np.int64)
        col = np.zeros(nnz.value, dtype=np.int32)
        val = np.zeros(nnz.value)
        _check(lib().vem_csr(self.h, ctypes.byref(n), ctypes.byref(nnz), _ptr(rp), _ptr(col), _ptr(val)))
        return sp.csr_matrix((val, col, rp), shape=(n.value, n.value))

    def info(self, key):
        v = ctypes.c_double()
        _check(lib().vem_info(self.h, key.encode(), ctypes.byref(v)))
        return v.value

    def set_stream(self, stream):
        _check(lib().vem_set_stream(self.h, ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)))


class Bddc:
    """bddc_setup + bddc_apply + pcg_solve over a VemSystem.

    scaling: 0 multiplicity (1/card), 1 deluxe on macro faces (1/card on
    edges), 2 deluxe on macro faces and macro edges."""

    def __init__(self, system, part, constraints=15, scaling=1, leaf=0, precision=0, refine=0, use_graph=0,
                 adaptive=0.0, tc_update=0):
        L = lib()
        self.sys = system
        part = np.ascontiguousarray(part, dtype=np.int32)
        opts = BddcOptions()
        opts.nd_leaf = int(leaf)
        opts.precision = int(precision)
        opts.refine = int(refine)
        opts.use_graph = int(use_graph)
        opts.adaptive_threshold = float(adaptive)
        opts.tc_update = int(tc_update)
        h = ctypes.c_void_p()
        _check(L.bddc_setup(system.h, part.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(constraints),
                            int(scaling), ctypes.byref(opts), ctypes.byref(h)))
        self.h = h

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.bddc_free(self.h)
            self.h = None

    def apply(self, r, z=None):
        import torch
        if z is None:
            z = torch.empty_like(r)
        _check(lib().bddc_apply(self.h, _dptr(r), _dptr(z)))
        return z

    def solve(self, f, u, rtol=1e-8, maxit=500):
        it = ctypes.c_int()
        ka, lmi, lma = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        st = lib().pcg_solve(self.h, _dptr(f), _dptr(u), float(rtol), int(maxit), ctypes.byref(it),
                             ctypes.byref(ka), ctypes.byref(lmi), ctypes.byref(lma))
        if st not in (0, -6):
            _check(st)
        return dict(status=st, iters=it.value, kappa=ka.value, lam_min=lmi.value, lam_max=lma.value)

    def info(self, key):
        v = ctypes.c_double()
        _check(lib().bddc_info(self.h, key.encode(), ctypes.byref(v)))
        return v.value

    def time_local_solves(self, nrep=5):
        ms, by = ctypes.c_double(), ctypes.c_double()
        _check(lib().bddc_time_local_solves(self.h, int(nrep), ctypes.byref(ms), ctypes.byref(by)))
        return ms.value, by.value

    def set_stream(self, stream):
        _check(lib().bddc_set_stream(self.h, ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)))
