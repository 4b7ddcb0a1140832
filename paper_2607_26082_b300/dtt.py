"""ctypes binding of libdtt (include/dtt.h): argument marshalling only.

Every method maps to one C entry point of the same name; all computation happens in the
CUDA library.  Host arrays are numpy float64/uint8/int32/int8; device arrays may be
passed as torch CUDA tensors (their data_ptr is handed over with ptr_is_device = 1).
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdtt.so")

OK, ERR_ARG, ERR_BC, ERR_OVERLAP, ERR_CUDA, ERR_OOM, ERR_NOT_CONVERGED, ERR_DIVERGED, ERR_STATE, ERR_NULLMODE = range(10)
BC_PERIODIC, BC_DIRICHLET, BC_NEUMANN = 0, 1, 2
SCHEME_TETRA2, SCHEME_HEX1 = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
INIT_ZERO, INIT_PREVIOUS, INIT_GUESS = 0, 1, 2
ACV_U, ACV_P = 0, 1
SMALL_STRAIN, FINITE_STRAIN = 0, 1
MEDIUM_PAUX, MEDIUM_ISOTROPIC = 0, 1


class DttError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("dtt status %d: %s" % (status, msg))
        self.status = status


class SolveOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int32), ("acv_mod", C.c_int32),
                ("acv_on", C.c_int32), ("init", C.c_int32), ("update_tol", C.c_double),
                ("graph_iters", C.c_int32), ("acv_pivot", C.c_double)]


class Report(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("accelerations", C.c_int32),
                ("active_set_updates", C.c_int32), ("status", C.c_int32),
                ("residual", C.c_double), ("seconds", C.c_double), ("start_from_guess", C.c_int32),
                ("start_residual", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Tuning(C.Structure):
    _fields_ = [("residual_zchunk", C.c_int32), ("fft_generic", C.c_int32), ("z_route", C.c_int32),
                ("fft_warp", C.c_int32), ("ms_per_iteration", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None

EXPORTS = ["dtt_grid_create", "dtt_grid_destroy", "dtt_grid_sizes", "dtt_set_material",
           "dtt_set_reference", "dtt_set_load", "dtt_set_constraints", "dtt_set_indenter",
           "dtt_move_indenter", "dtt_clear_indenter", "dtt_set_initial", "dtt_solve_step",
           "dtt_get_history", "dtt_get_fields", "dtt_get_reactions", "dtt_get_contact",
           "dtt_set_kinematics", "dtt_get_stress_tensor", "dtt_get_min_jacobian", "dtt_set_reference_medium",
           "dtt_apply_residual", "dtt_apply_green", "dtt_apply_green_noalloc", "dtt_transform", "dtt_set_initial_contact",
           "dtt_profile_iteration", "dtt_autotune", "dtt_set_tuning", "dtt_batch_solve",
           "dtt_last_error", "dtt_version"]
NPROF = 7
PROF_GROUPS = ["residual", "projections", "anderson", "forward_dt", "green", "inverse_dt", "increment"]


def lib():
    """Load libdtt.so (in-tree).  Raises if it is missing: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libdtt.so not built: run python -m paper_2607_26082_b300.build")
    L = C.CDLL(LIB_PATH)
    P = C.c_void_p
    i32, i64, f64 = C.c_int32, C.c_int64, C.c_double
    L.dtt_grid_create.argtypes = [C.POINTER(P), P, f64, P, i32, i32, P]
    L.dtt_grid_destroy.argtypes = [P]
    L.dtt_grid_destroy.restype = None
    L.dtt_grid_sizes.argtypes = [P, C.POINTER(i64), C.POINTER(i64), P]
    L.dtt_set_material.argtypes = [P, P, i32, P, P, i32]
    L.dtt_set_reference.argtypes = [P, f64, f64]
    L.dtt_set_load.argtypes = [P, P]
    L.dtt_set_constraints.argtypes = [P, i32, P, P, P, P, P, P]
    L.dtt_set_indenter.argtypes = [P, i32, i32, P, f64]
    L.dtt_move_indenter.argtypes = [P, P]
    L.dtt_clear_indenter.argtypes = [P]
    L.dtt_set_initial.argtypes = [P, P, i32]
    L.dtt_set_initial_contact.argtypes = [P, P, i32]
    L.dtt_solve_step.argtypes = [P, C.POINTER(SolveOpts), C.POINTER(Report)]
    L.dtt_get_history.argtypes = [P, P, C.POINTER(i32)]
    L.dtt_get_fields.argtypes = [P, P, P, i32]
    L.dtt_set_kinematics.argtypes = [P, i32]
    L.dtt_set_reference_medium.argtypes = [P, i32]
    L.dtt_get_stress_tensor.argtypes = [P, P, i32]
    L.dtt_get_min_jacobian.argtypes = [P, C.POINTER(f64)]
    L.dtt_get_reactions.argtypes = [P, P, P]
    L.dtt_get_contact.argtypes = [P, C.POINTER(i32), P, P, P, P]
    L.dtt_apply_residual.argtypes = [P, P, P, P, P, i32]
    L.dtt_apply_green.argtypes = [P, P, P, i32]
    L.dtt_apply_green_noalloc.argtypes = [P, P, P]
    L.dtt_transform.argtypes = [P, i32, i32, P, P, i32]
    L.dtt_profile_iteration.argtypes = [P, C.POINTER(SolveOpts), i32, P]
    L.dtt_autotune.argtypes = [P, C.POINTER(SolveOpts), i32, C.POINTER(Tuning)]
    L.dtt_set_tuning.argtypes = [P, C.POINTER(Tuning)]
    L.dtt_batch_solve.argtypes = [i32, P, C.POINTER(SolveOpts), P]
    L.dtt_last_error.restype = C.c_char_p
    L.dtt_version.restype = C.c_char_p
    for name in EXPORTS:
        fn = getattr(L, name)
        if fn.restype is C.c_int:   # default
            fn.restype = i32
    _lib = L
    return L


def _check(st):
    if st != OK:
        raise DttError(st, lib().dtt_last_error().decode())


def _ptr(a, dtype=None):
    """(pointer, is_device) of a numpy array or a torch tensor (None -> NULL)."""
    if a is None:
        return None, 0
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr()), 1 if a.is_cuda else 0
    arr = np.ascontiguousarray(a, dtype=dtype) if dtype is not None else a
    if not arr.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return arr.ctypes.data_as(C.c_void_p), 0


class Grid:
    """One cell (dtt_grid).  Methods mirror the C entry points."""

    def __init__(self, nvox, h, bc, scheme=SCHEME_TETRA2, precision=PREC_FP64, stream=None):
        L = lib()
        self._h = C.c_void_p()
        nv = np.ascontiguousarray(nvox, dtype=np.int32)
        b = np.ascontiguousarray(np.asarray(bc).reshape(18), dtype=np.int32)
        st = L.dtt_grid_create(C.byref(self._h), nv.ctypes.data_as(C.c_void_p), float(h),
                               b.ctypes.data_as(C.c_void_p), int(scheme), int(precision),
                               C.c_void_p(stream) if stream else None)
        _check(st)
        nn_nodes, nn_vox = C.c_int64(), C.c_int64()
        nn = np.zeros(3, dtype=np.int32)
        _check(L.dtt_grid_sizes(self._h, C.byref(nn_nodes), C.byref(nn_vox), nn.ctypes.data_as(C.c_void_p)))
        self.n_nodes, self.n_voxels = nn_nodes.value, nn_vox.value
        self.nn = tuple(int(v) for v in nn)
        self.node_shape = (self.nn[2], self.nn[1], self.nn[0])
        self.nvox = tuple(int(v) for v in nvox)
        self.scheme = int(scheme)
        self.precision = int(precision)

    def close(self):
        if self._h:
            lib().dtt_grid_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def dtt_set_material(self, phase, lam, mu):
        ph = np.ascontiguousarray(phase, dtype=np.uint8).reshape(-1)
        l = np.ascontiguousarray(lam, dtype=np.float64)
        m = np.ascontiguousarray(mu, dtype=np.float64)
        _check(lib().dtt_set_material(self._h, ph.ctypes.data_as(C.c_void_p), len(l),
                                      l.ctypes.data_as(C.c_void_p), m.ctypes.data_as(C.c_void_p), 0))

    def dtt_set_reference(self, lam0, mu0):
        _check(lib().dtt_set_reference(self._h, float(lam0), float(mu0)))

    def dtt_set_load(self, eps_star):
        e = np.ascontiguousarray(eps_star, dtype=np.float64).reshape(9)
        _check(lib().dtt_set_load(self._h, e.ctypes.data_as(C.c_void_p)))

    def dtt_set_constraints(self, row_ptr, node, comp, a, b, value):
        n_rows = len(value)
        arrs = [np.ascontiguousarray(row_ptr, dtype=np.int32), np.ascontiguousarray(node, dtype=np.int32),
                np.ascontiguousarray(comp, dtype=np.int8), np.ascontiguousarray(a, dtype=np.float64),
                None if b is None else np.ascontiguousarray(b, dtype=np.float64),
                np.ascontiguousarray(value, dtype=np.float64)]
        ptrs = [None if x is None else x.ctypes.data_as(C.c_void_p) for x in arrs]
        _check(lib().dtt_set_constraints(self._h, n_rows, *ptrs))

    def dtt_set_indenter(self, axis, face, center, radius):
        c = np.ascontiguousarray(center, dtype=np.float64)
        _check(lib().dtt_set_indenter(self._h, int(axis), int(face), c.ctypes.data_as(C.c_void_p), float(radius)))

    def dtt_move_indenter(self, center):
        c = np.ascontiguousarray(center, dtype=np.float64)
        _check(lib().dtt_move_indenter(self._h, c.ctypes.data_as(C.c_void_p)))

    def dtt_clear_indenter(self):
        _check(lib().dtt_clear_indenter(self._h))

    def dtt_set_initial(self, u):
        arr = u if hasattr(u, "data_ptr") else np.ascontiguousarray(u, dtype=np.float64)
        p, dev = _ptr(arr)
        _check(lib().dtt_set_initial(self._h, p, dev))

    def dtt_set_initial_contact(self, active):
        arr = active if hasattr(active, "data_ptr") else np.ascontiguousarray(active, dtype=np.uint8)
        p, dev = _ptr(arr)
        _check(lib().dtt_set_initial_contact(self._h, p, dev))

    def dtt_solve_step(self, tol, max_iter, acv_mod=3, acv_on=ACV_P, init=INIT_ZERO, update_tol=1e-2,
                       graph_iters=0, acv_pivot=0.0, raise_on_error=False):
        o = SolveOpts(float(tol), int(max_iter), int(acv_mod), int(acv_on), int(init), float(update_tol),
                      int(graph_iters), float(acv_pivot))
        r = Report()
        st = lib().dtt_solve_step(self._h, C.byref(o), C.byref(r))
        if st not in (OK, ERR_NOT_CONVERGED, ERR_DIVERGED) or (raise_on_error and st != OK):
            _check(st)
        return r

    def dtt_get_history(self):
        n = C.c_int32(0)
        _check(lib().dtt_get_history(self._h, None, C.byref(n)))
        out = np.zeros(max(n.value, 1))
        n2 = C.c_int32(len(out))
        _check(lib().dtt_get_history(self._h, out.ctypes.data_as(C.c_void_p), C.byref(n2)))
        return out[: n.value]

    def dtt_get_fields(self, sigma=False, u_out=None):
        u = np.zeros((3,) + self.node_shape) if u_out is None else u_out
        nip = 2 if self.scheme == SCHEME_TETRA2 else 1
        s = np.zeros((self.nvox[2], self.nvox[1], self.nvox[0], nip, 6)) if sigma else None
        pu, dev = _ptr(u)
        ps, _ = _ptr(s)
        _check(lib().dtt_get_fields(self._h, pu, ps, dev))
        return (u, s) if sigma else u

    def dtt_set_reference_medium(self, medium):
        _check(lib().dtt_set_reference_medium(self._h, int(medium)))

    def dtt_set_kinematics(self, kinematics):
        _check(lib().dtt_set_kinematics(self._h, int(kinematics)))

    def dtt_get_stress_tensor(self, out=None):
        """(nvox_z, nvox_y, nvox_x, n_ip, 3, 3): sigma, or Pi in finite strain."""
        nip = 2 if self.scheme == SCHEME_TETRA2 else 1
        t = np.zeros((self.nvox[2], self.nvox[1], self.nvox[0], nip, 3, 3)) if out is None else out
        pt, dev = _ptr(t)
        _check(lib().dtt_get_stress_tensor(self._h, pt, dev))
        return t

    def dtt_get_min_jacobian(self):
        v = C.c_double()
        _check(lib().dtt_get_min_jacobian(self._h, C.byref(v)))
        return v.value

    def dtt_get_reactions(self, n_rows):
        per = np.zeros(max(n_rows, 1))
        tot = np.zeros(3)
        _check(lib().dtt_get_reactions(self._h, per.ctypes.data_as(C.c_void_p), tot.ctypes.data_as(C.c_void_p)))
        return per[:n_rows], tot

    def dtt_get_contact(self):
        n = C.c_int32(0)
        _check(lib().dtt_get_contact(self._h, C.byref(n), None, None, None, None))
        m = n.value
        act = np.zeros(m, dtype=np.uint8)
        gap = np.zeros(m)
        fn = np.zeros(m)
        force = np.zeros(3)
        _check(lib().dtt_get_contact(self._h, C.byref(n), act.ctypes.data_as(C.c_void_p),
                                     gap.ctypes.data_as(C.c_void_p), fn.ctypes.data_as(C.c_void_p),
                                     force.ctypes.data_as(C.c_void_p)))
        return act.astype(bool), gap, fn, force

    def dtt_apply_residual(self, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        p = np.zeros_like(u)
        pt = np.zeros_like(u)
        norms = np.zeros(2)
        _check(lib().dtt_apply_residual(self._h, u.ctypes.data_as(C.c_void_p), p.ctypes.data_as(C.c_void_p),
                                        pt.ctypes.data_as(C.c_void_p), norms.ctypes.data_as(C.c_void_p), 0))
        return p, pt, norms

    def dtt_apply_green(self, ptilde):
        pt = np.ascontiguousarray(ptilde, dtype=np.float64)
        u = np.zeros_like(pt)
        _check(lib().dtt_apply_green(self._h, pt.ctypes.data_as(C.c_void_p), u.ctypes.data_as(C.c_void_p), 0))
        return u

    def dtt_apply_green_noalloc(self, ptilde_dev, u_dev):
        """Green step on caller-owned float64 device arrays (torch CUDA tensors), using the
        library's fixed scratch instead of any allocation."""
        p_in, d_in = _ptr(ptilde_dev)
        p_out, d_out = _ptr(u_dev)
        if not (d_in and d_out):
            raise ValueError("dtt_apply_green_noalloc takes device arrays")
        _check(lib().dtt_apply_green_noalloc(self._h, p_in, p_out))

    def dtt_transform(self, component, inverse, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        out = np.zeros_like(x)
        _check(lib().dtt_transform(self._h, int(component), int(inverse), x.ctypes.data_as(C.c_void_p),
                                   out.ctypes.data_as(C.c_void_p), 0))
        return out


    def dtt_autotune(self, iters=5, acv_mod=3, acv_on=ACV_P):
        o = SolveOpts(0.0, 1 << 30, int(acv_mod), int(acv_on), INIT_ZERO, 1e-2, 0, 0.0)
        t = Tuning()
        _check(lib().dtt_autotune(self._h, C.byref(o), int(iters), C.byref(t)))
        return t

    def dtt_set_tuning(self, tuning):
        t = tuning if isinstance(tuning, Tuning) else Tuning(int(tuning["residual_zchunk"]),
                                                                 int(tuning["fft_generic"]),
                                                                 int(tuning.get("z_route", 0)),
                                                                 int(tuning.get("fft_warp", 1)), 0.0)
        _check(lib().dtt_set_tuning(self._h, C.byref(t)))

    def dtt_profile_iteration(self, iters, acv_mod=3, acv_on=ACV_P):
        o = SolveOpts(0.0, 1 << 30, int(acv_mod), int(acv_on), INIT_PREVIOUS, 1e-2, 0, 0.0)
        ms = np.zeros(NPROF)
        _check(lib().dtt_profile_iteration(self._h, C.byref(o), int(iters), ms.ctypes.data_as(C.c_void_p)))
        return dict(zip(PROF_GROUPS, ms))


def version():
    return lib().dtt_version().decode()


def dtt_batch_solve(grids, tol, max_iter, acv_mod=3, acv_on=ACV_P, init=INIT_ZERO, update_tol=1e-2,
                    graph_iters=0, acv_pivot=0.0):
    """Solve independent grids together (dtt_batch_solve); returns (status, [Report])."""
    n = len(grids)
    arr = (C.c_void_p * n)(*[g._h.value for g in grids])
    o = SolveOpts(float(tol), int(max_iter), int(acv_mod), int(acv_on), int(init), float(update_tol),
                  int(graph_iters), float(acv_pivot))
    reps = (Report * n)()
    st = lib().dtt_batch_solve(n, C.cast(arr, C.c_void_p), C.byref(o), C.cast(reps, C.c_void_p))
    if st not in (OK, ERR_NOT_CONVERGED, ERR_DIVERGED):
        _check(st)
    return st, list(reps)
