"""Thin ctypes binding of the C ABI in include/pdf_canyon.h.

Argument marshalling only: every step of the method runs in the CUDA library
(_build/libpdfcanyon.so, built from csrc/ for sm_103a). There is no CPU
fallback: if the library cannot be built or loaded, the import of the
functions below raises.

The function names are those of the C ABI. ``Canyon`` is a small convenience
owner of one ``pdf_ctx`` that converts numpy arrays and torch tensors to
pointers.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

PDF_OK = 0
ERRORS = {-1: "PDF_ERR_ARG", -2: "PDF_ERR_MESH", -3: "PDF_ERR_CUDA", -4: "PDF_ERR_NONFINITE",
          -5: "PDF_ERR_LOST_PARTICLE", -6: "PDF_ERR_WALL", -7: "PDF_ERR_CG_NOCONV", -8: "PDF_ERR_DT",
          -9: "PDF_ERR_STATE", -10: "PDF_ERR_CAPACITY"}

PDF_WALL_FUNCTIONS, PDF_ELLIPTIC_RELAXATION = 0, 1
PDF_FP64, PDF_FP32, PDF_FP32_KAHAN = 0, 1, 2
PRECISION = {"fp64": PDF_FP64, "fp32": PDF_FP32, "fp32_kahan": PDF_FP32_KAHAN}

FIELD = dict(x=0, y=1, u=2, v=3, w=4, om=5, psi=6, id=7, elem=8, bin=9, elem_n=10, elem_mean=11, elem_R=12,
             elem_psivar=13, elem_cm=14, node_mean=15, node_R=16, node_ke=17, elem_der=18, node_pack=19,
             node_wp=20, node_wdist=21, node_grad=22, node_psivar=23, particle_wp=24,
             elem_omw=25, node_omw=26, node_p=27)
KERNEL = dict(particle=0, sort=1, moments=2, fields=3, elliptic=4, pressure=5, bins=6)

_DOUBLES = ("C1", "C2", "C3", "C4", "CT", "CL", "Ceta", "Cv", "gamma5", "Comega1", "Comega2", "Cs", "Ct",
            "C0", "Cmu", "kappa", "E", "nu", "fx", "fy", "yp", "wall_offset", "x0", "y0", "r0", "period",
            "k0", "ustar", "y_roof", "er_wall", "floor_k", "floor_eps", "floor_omega", "cg_tol")


class pdf_params(C.Structure):
    _fields_ = [(n, C.c_double) for n in _DOUBLES] + [
        ("cg_maxit", C.c_int32), ("nb1", C.c_int32), ("nb2", C.c_int32), ("nb3", C.c_int32),
        ("wall_model", C.c_int32), ("mix_exp", C.c_int32), ("reflect_max", C.c_int32), ("rotta", C.c_int32),
        ("seed", C.c_uint64), ("case_id", C.c_uint32), ("precision", C.c_int32), ("cg_precision", C.c_int32),
        ("omega_wall", C.c_int32), ("pressure", C.c_int32), ("reserved_", C.c_int32),
        ("pressure_tol", C.c_double)]


EXPORTS = ("pdf_default_params", "pdf_init_mesh", "pdf_seed_particles", "pdf_set_particles",
           "pdf_estimate_stats", "pdf_step", "pdf_sync", "pdf_get_fields", "pdf_num_particles",
           "pdf_num_elements", "pdf_num_nodes", "pdf_num_bins", "pdf_step_index", "pdf_cg_iterations",
           "pdf_pressure_iterations",
           "pdf_set_timing", "pdf_kernel_time", "pdf_reset_timing", "pdf_launch_count", "pdf_last_error",
           "pdf_destroy", "pdf_sort_by_element_static", "pdf_mlp_work_floats", "pdf_mlp_forward",
           "pdf_mlp_loss_grad", "pdf_mlp_loss_grad_bf16", "pdf_mlp_adam", "pdf_mlp_column_stats", "pdf_mlp_gather_rows",
           "pdf_mlp_standardize", "pdf_surrogate_rows", "pdf_surrogate_harvest", "pdf_set_surrogate",
           "pdf_surrogate_stats", "pdf_batch_create", "pdf_batch_create_out", "pdf_batch_step", "pdf_batch_sync", "pdf_batch_destroy",
           "pdf_autotune", "pdf_apply_tuning", "pdf_measure_fp64_fma_rate", "pdf_set_averaging", "pdf_averaging_count", "pdf_get_averages", "pdf_probe",
           "pdf_set_cdf_probes", "pdf_get_cdf", "pdf_set_wait_limit")

MLP_IN, MLP_HIDDEN, MLP_OUT, MLP_NPARAM, MLP_NNORM = 10, 64, 5, 9349, 30

SORT_STATIC_MAX_ELEMENTS = 131072  # PDF_SORT_STATIC_MAX_ELEMENTS


class pdf_tuning(C.Structure):
    _fields_ = [("step_blocks_per_sm", C.c_int32), ("scatter_threads", C.c_int32), ("cg_rows_per_block", C.c_int32),
                ("bins_blocks_per_sm", C.c_int32), ("ms_particle", C.c_double), ("ms_sort", C.c_double),
                ("ms_elliptic", C.c_double), ("ms_step_bins", C.c_double * 5)]


def library_path() -> str:
    return _build.LIB


def lib(allow_build: bool = True):
    """Load the CUDA library (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if allow_build else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library missing: {path}")
        L = C.CDLL(path)
        P, vp = C.POINTER, C.c_void_p
        d, i32, u32 = P(C.c_double), P(C.c_int32), P(C.c_uint32)
        L.pdf_default_params.argtypes = [P(pdf_params)]
        L.pdf_init_mesh.argtypes = [P(pdf_params), d, C.c_int32, i32, C.c_int32, i32, i32, vp, P(vp)]
        L.pdf_seed_particles.argtypes = [vp, C.c_int32]
        L.pdf_set_particles.argtypes = [vp, C.c_int32, d, d, d, d, d, d, d, u32, i32, C.c_int32]
        L.pdf_estimate_stats.argtypes = [vp]
        L.pdf_step.argtypes = [vp, C.c_double, C.c_int32]
        L.pdf_sync.argtypes = [vp]
        L.pdf_set_wait_limit.argtypes = [vp, C.c_int64]
        L.pdf_get_fields.argtypes = [vp, C.c_int32, vp, C.c_size_t, C.c_int32]
        for n in ("pdf_num_particles", "pdf_launch_count"):
            getattr(L, n).argtypes = [vp]
            getattr(L, n).restype = C.c_int64
        for n in ("pdf_num_elements", "pdf_num_nodes", "pdf_num_bins", "pdf_step_index", "pdf_cg_iterations",
                  "pdf_pressure_iterations"):
            getattr(L, n).argtypes = [vp]
            getattr(L, n).restype = C.c_int32
        L.pdf_set_timing.argtypes = [vp, C.c_int32]
        L.pdf_kernel_time.argtypes = [vp, C.c_int32, d, P(C.c_int64)]
        L.pdf_reset_timing.argtypes = [vp]
        L.pdf_last_error.argtypes = [vp]
        L.pdf_last_error.restype = C.c_char_p
        L.pdf_destroy.argtypes = [vp]
        L.pdf_destroy.restype = None
        L.pdf_sort_by_element_static.argtypes = [vp, C.c_int64, C.c_int32, vp, vp, vp]
        L.pdf_mlp_work_floats.argtypes = [C.c_int32]
        L.pdf_mlp_work_floats.restype = C.c_int64
        L.pdf_mlp_forward.argtypes = [vp, vp, C.c_int32, vp, vp, C.c_int32, vp]
        L.pdf_mlp_loss_grad.argtypes = [vp, vp, vp, C.c_int32, vp, vp, vp, vp]
        L.pdf_mlp_loss_grad_bf16.argtypes = [vp, vp, vp, C.c_int32, vp, vp, vp, vp]
        L.pdf_mlp_adam.argtypes = [vp, vp, vp, vp, C.c_int32, C.c_float, C.c_float, C.c_float, C.c_float, vp]
        L.pdf_mlp_column_stats.argtypes = [vp, C.c_int64, C.c_int32, vp, vp, vp]
        L.pdf_mlp_gather_rows.argtypes = [vp, vp, C.c_int32, C.c_int32, vp, vp]
        L.pdf_mlp_standardize.argtypes = [vp, C.c_int64, C.c_int32, vp, vp, vp]
        L.pdf_surrogate_rows.argtypes = [vp]
        L.pdf_surrogate_rows.restype = C.c_int32
        L.pdf_surrogate_harvest.argtypes = [vp, vp, vp]
        L.pdf_set_surrogate.argtypes = [vp, C.c_int32, P(C.c_float), P(C.c_float), C.c_double]
        L.pdf_surrogate_stats.argtypes = [vp, P(C.c_int64), P(C.c_int64), d]
        L.pdf_batch_create.argtypes = [P(vp), d, C.c_int32, vp, P(vp)]
        L.pdf_batch_create_out.argtypes = [P(vp), d, C.c_int32, vp, C.c_int32, P(vp), P(C.c_size_t), P(vp)]
        L.pdf_batch_step.argtypes = [vp, C.c_int32]
        L.pdf_batch_sync.argtypes = [vp, i32]
        L.pdf_batch_destroy.argtypes = [vp]
        L.pdf_batch_destroy.restype = None
        L.pdf_autotune.argtypes = [vp, C.c_double, C.c_int32, P(pdf_tuning)]
        L.pdf_apply_tuning.argtypes = [vp, P(pdf_tuning)]
        L.pdf_measure_fp64_fma_rate.argtypes = [vp, d]
        L.pdf_set_averaging.argtypes = [vp, C.c_int32, C.c_int32]
        L.pdf_averaging_count.argtypes = [vp]
        L.pdf_averaging_count.restype = C.c_int64
        L.pdf_get_averages.argtypes = [vp, C.c_int32, d]
        L.pdf_probe.argtypes = [vp, C.c_int32, C.c_int32, d, d, C.c_int32, d, i32]
        L.pdf_set_cdf_probes.argtypes = [vp, d, d, C.c_int32, C.c_int32]
        L.pdf_get_cdf.argtypes = [vp, d, i32]
        _lib = L
        return L


class PdfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def default_params(**over) -> pdf_params:
    p = pdf_params()
    lib().pdf_default_params(C.byref(p))
    for k, v in over.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISION[v]
        setattr(p, k, v)
    return p


def sort_by_element_static(elem_ptr: int, n: int, nt: int, perm_ptr: int, off_ptr: int, stream: int = 0):
    """pdf_sort_by_element_static on device pointers (int32 elem[n], perm[n],
    off[nt+1]); raises PdfError on a non-zero status."""
    L = lib()
    st = L.pdf_sort_by_element_static(C.c_void_p(elem_ptr), n, nt, C.c_void_p(perm_ptr), C.c_void_p(off_ptr),
                                      C.c_void_p(stream))
    if st != PDF_OK:
        raise PdfError(st, L.pdf_last_error(None).decode())


def _chk(st, what):
    if st != PDF_OK:
        raise PdfError(st, f"{what}: " + lib().pdf_last_error(None).decode())


def _vp(x):
    return C.c_void_p(int(x))


def mlp_work_floats(n: int) -> int:
    return int(lib().pdf_mlp_work_floats(n))


def mlp_forward(params, X, n, Y, work, bf16_weights=False, stream=0):
    """pdf_mlp_forward on device pointers."""
    _chk(lib().pdf_mlp_forward(_vp(params), _vp(X), n, _vp(Y), _vp(work), 1 if bf16_weights else 0, _vp(stream)),
         "pdf_mlp_forward")


def mlp_loss_grad(params, X, T, n, work, grad, loss, stream=0):
    _chk(lib().pdf_mlp_loss_grad(_vp(params), _vp(X), _vp(T), n, _vp(work), _vp(grad), _vp(loss), _vp(stream)),
         "pdf_mlp_loss_grad")


def measure_fp64_fma_rate(stream=0) -> float:
    """Measured FP64 FMA rate of the current device in TFLOP/s."""
    r = C.c_double()
    _chk(lib().pdf_measure_fp64_fma_rate(_vp(stream), C.byref(r)), "pdf_measure_fp64_fma_rate")
    return r.value


def mlp_loss_grad_bf16(params, X, T, n, work, grad, loss, stream=0):
    _chk(lib().pdf_mlp_loss_grad_bf16(_vp(params), _vp(X), _vp(T), n, _vp(work), _vp(grad), _vp(loss),
                                      _vp(stream)), "pdf_mlp_loss_grad_bf16")


def mlp_adam(params, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=0):
    _chk(lib().pdf_mlp_adam(_vp(params), _vp(grad), _vp(m), _vp(v), t, lr, beta1, beta2, eps, _vp(stream)),
         "pdf_mlp_adam")


def mlp_column_stats(X, n, d, mean, std, stream=0):
    _chk(lib().pdf_mlp_column_stats(_vp(X), n, d, _vp(mean), _vp(std), _vp(stream)), "pdf_mlp_column_stats")


def mlp_gather_rows(src, idx, n, d, dst, stream=0):
    _chk(lib().pdf_mlp_gather_rows(_vp(src), _vp(idx), n, d, _vp(dst), _vp(stream)), "pdf_mlp_gather_rows")


def mlp_standardize(X, n, d, mean, std, stream=0):
    _chk(lib().pdf_mlp_standardize(_vp(X), n, d, _vp(mean), _vp(std), _vp(stream)), "pdf_mlp_standardize")


def params_dict(p: pdf_params) -> dict:
    return {n: getattr(p, n) for n, _ in pdf_params._fields_}


class Canyon:
    """Owner of one pdf_ctx over one mesh (see include/pdf_canyon.h)."""

    def __init__(self, params: pdf_params, mesh: dict, stream=None):
        L = lib()
        self.params = params
        xy = np.ascontiguousarray(mesh["xy"], np.float64)
        tri = np.ascontiguousarray(mesh["tri"], np.int32)
        tag = np.ascontiguousarray(mesh["edge_tag"], np.int32)
        pair = np.ascontiguousarray(mesh["periodic_pair"], np.int32)
        self._keep = (xy, tri, tag, pair)
        h = C.c_void_p()
        st = L.pdf_init_mesh(C.byref(params), _ptr(xy, C.c_double), xy.shape[0], _ptr(tri, C.c_int32),
                             tri.shape[0], _ptr(tag, C.c_int32), _ptr(pair, C.c_int32),
                             C.c_void_p(stream or 0), C.byref(h))
        if st != PDF_OK:
            raise PdfError(st, L.pdf_last_error(None).decode())
        self._h = h
        self.nt = L.pdf_num_elements(h)
        self.nn = L.pdf_num_nodes(h)
        self.nbins = L.pdf_num_bins(h)

    def close(self):
        if getattr(self, "_h", None):
            lib().pdf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != PDF_OK:
            raise PdfError(st, lib().pdf_last_error(self._h).decode())
        return st

    @property
    def handle(self):
        return self._h

    # -- calls of the C ABI -------------------------------------------------
    def seed_particles(self, per_element: int):
        self._check(lib().pdf_seed_particles(self._h, per_element))

    def set_particles(self, st: dict, step: int = 0):
        n = int(len(st["x"]))
        arrs = [np.ascontiguousarray(st[k], np.float64) for k in ("x", "y", "u", "v", "w", "om", "psi")]
        ids = np.ascontiguousarray(st["id"], np.uint32)
        el = np.ascontiguousarray(st["elem"], np.int32)
        self._check(lib().pdf_set_particles(self._h, n, *[_ptr(a, C.c_double) for a in arrs],
                                            _ptr(ids, C.c_uint32), _ptr(el, C.c_int32), step))

    def estimate_stats(self):
        self._check(lib().pdf_estimate_stats(self._h))

    def step(self, dt: float, nsteps: int = 1):
        self._check(lib().pdf_step(self._h, dt, nsteps))

    def sync(self, check: bool = True) -> int:
        st = lib().pdf_sync(self._h)
        if check:
            self._check(st)
        return st

    def set_wait_limit(self, spins: int):
        self._check(lib().pdf_set_wait_limit(self._h, spins))

    @property
    def last_error(self) -> str:
        return lib().pdf_last_error(self._h).decode()

    @property
    def num_particles(self) -> int:
        return lib().pdf_num_particles(self._h)

    @property
    def step_index(self) -> int:
        return lib().pdf_step_index(self._h)

    @property
    def cg_iterations(self) -> int:
        return lib().pdf_cg_iterations(self._h)

    @property
    def pressure_iterations(self) -> int:
        return lib().pdf_pressure_iterations(self._h)

    def field_shape(self, name: str):
        n = self.num_particles
        w = dict(elem_mean=5, elem_R=6, elem_cm=self.nbins, node_mean=4, node_R=6, node_ke=2, elem_der=9,
                 node_pack=11, node_wp=5, node_grad=4, particle_wp=5, elem_omw=5,
                 node_omw=5).get(name, 1)
        rows = n if (FIELD[name] <= 9 or name == "particle_wp") else (self.nt if name.startswith("elem") else self.nn)
        dt = {"id": np.uint32, "elem": np.int32, "bin": np.uint8, "elem_n": np.int32,
              "particle_wp": np.float32}.get(name, np.float64)
        return (rows, w) if w > 1 else (rows,), dt

    def field(self, name: str) -> np.ndarray:
        shape, dt = self.field_shape(name)
        out = np.empty(shape, dt)
        self._check(lib().pdf_get_fields(self._h, FIELD[name], out.ctypes.data_as(C.c_void_p), out.nbytes, 0))
        return out

    def field_into(self, name: str, ptr: int, nbytes: int, device: bool, asynchronous: bool = False):
        """Copy a field to ptr; a host copy is synchronous unless asynchronous
        (then ptr should be page-locked and is valid after the next sync)."""
        mode = 1 if device else (2 if asynchronous else 0)
        self._check(lib().pdf_get_fields(self._h, FIELD[name], C.c_void_p(ptr), nbytes, mode))

    def particles(self) -> dict:
        return {k: self.field(k) for k in ("x", "y", "u", "v", "w", "om", "psi", "id", "elem", "bin")}

    # -- learned surrogate of the elliptic solve ------------------------------
    def surrogate_rows(self) -> int:
        r = lib().pdf_surrogate_rows(self._h)
        if r < 0:
            raise PdfError(-1, lib().pdf_last_error(self._h).decode())
        return r

    def surrogate_harvest(self, X_ptr: int, T_ptr: int):
        self._check(lib().pdf_surrogate_harvest(self._h, _vp(X_ptr), _vp(T_ptr)))

    def set_surrogate(self, mode: int, params=None, norm=None, residual_tol: float = 0.0):
        if mode == 0 or mode == 5:  # mode 5 (lagged FE) has no network
            self._check(lib().pdf_set_surrogate(self._h, mode, None, None, float(residual_tol)))
            return
        p = np.ascontiguousarray(params, np.float32)
        q = np.ascontiguousarray(norm, np.float32)
        assert p.size == MLP_NPARAM and q.size == MLP_NNORM
        self._check(lib().pdf_set_surrogate(self._h, mode, _ptr(p, C.c_float), _ptr(q, C.c_float),
                                            float(residual_tol)))

    def surrogate_stats(self):
        """(solves, fallbacks, (coarse residual, fine residual)) of the last check."""
        a, b, r = C.c_int64(), C.c_int64(), (C.c_double * 2)()
        self._check(lib().pdf_surrogate_stats(self._h, C.byref(a), C.byref(b), r))
        return a.value, b.value, (r[0], r[1])

    def autotune(self, dt: float, steps_per_trial: int = 3) -> dict:
        t = pdf_tuning()
        self._check(lib().pdf_autotune(self._h, dt, steps_per_trial, C.byref(t)))
        out = {n: getattr(t, n) for n, _ in pdf_tuning._fields_}
        out["ms_step_bins"] = list(out["ms_step_bins"])
        return out

    def apply_tuning(self, tuning: dict):
        """Set launch shapes (a dict as autotune returns it; missing keys keep
        the defaults of pdf_tuning's fields as autotune would report them)."""
        t = pdf_tuning()
        t.step_blocks_per_sm = int(tuning.get("step_blocks_per_sm", 4))
        t.scatter_threads = int(tuning.get("scatter_threads", 256))
        t.cg_rows_per_block = int(tuning.get("cg_rows_per_block", 0))
        t.bins_blocks_per_sm = int(tuning.get("bins_blocks_per_sm", -1))
        self._check(lib().pdf_apply_tuning(self._h, C.byref(t)))

    # -- time averaging, probes, scalar CDFs --------------------------------
    def set_averaging(self, on: bool, reset: bool = False):
        self._check(lib().pdf_set_averaging(self._h, 1 if on else 0, 1 if reset else 0))

    @property
    def averaging_count(self) -> int:
        return int(lib().pdf_averaging_count(self._h))

    def averages(self, which: str) -> np.ndarray:
        k = {"elem_mean": 0, "elem_R": 1, "elem_psivar": 2, "node_mean": 3}[which]
        rows = self.nn if k == 3 else self.nt
        out = np.empty((rows, (5, 6, 1, 4)[k]), np.float64)
        self._check(lib().pdf_get_averages(self._h, k, _ptr(out, C.c_double)))
        return out[:, 0] if k == 2 else out

    PROBE = {"node_mean": 0, "elem_mean": 1, "elem_R": 2, "avg_node_mean": 3, "avg_elem_mean": 4, "avg_elem_R": 5}

    def probe(self, which: str, comp: int, x, y):
        x = np.ascontiguousarray(x, np.float64)
        y = np.ascontiguousarray(y, np.float64)
        out = np.empty(x.size, np.float64)
        el = np.empty(x.size, np.int32)
        self._check(lib().pdf_probe(self._h, self.PROBE[which], comp, _ptr(x, C.c_double), _ptr(y, C.c_double),
                                    x.size, _ptr(out, C.c_double), _ptr(el, C.c_int32)))
        return out, el

    def set_cdf_probes(self, x, y, nbins: int):
        x = np.ascontiguousarray(x, np.float64)
        y = np.ascontiguousarray(y, np.float64)
        self._cdf = (x.size, nbins)
        self._check(lib().pdf_set_cdf_probes(self._h, _ptr(x, C.c_double), _ptr(y, C.c_double), x.size, nbins))

    def cdf(self):
        n, nb = self._cdf
        out = np.empty((n, nb), np.float64)
        el = np.empty(n, np.int32)
        self._check(lib().pdf_get_cdf(self._h, _ptr(out, C.c_double), _ptr(el, C.c_int32)))
        return out, el

    def set_timing(self, on: bool):
        self._check(lib().pdf_set_timing(self._h, 1 if on else 0))

    def kernel_time(self, kernel: str):
        ms = C.c_double()
        n = C.c_int64()
        self._check(lib().pdf_kernel_time(self._h, KERNEL[kernel], C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def reset_timing(self):
        self._check(lib().pdf_reset_timing(self._h))


class Batch:
    """One CUDA graph holding a time step of several contexts (pdf_batch_*)."""

    def __init__(self, canyons, dts, stream: int, outputs=None):
        """outputs: None, or (field name, 2n device pointers, n byte counts) for
        pdf_batch_create_out (the field after each of the two captured steps
        of every context)."""
        L = lib()
        self.canyons = list(canyons)
        n = len(self.canyons)
        hs = (C.c_void_p * n)(*[c.handle.value for c in self.canyons])
        dt = (C.c_double * n)(*[float(x) for x in dts])
        h = C.c_void_p()
        if outputs is None:
            st = L.pdf_batch_create(hs, dt, n, C.c_void_p(stream), C.byref(h))
        else:
            name, ptrs, nbytes = outputs
            if len(ptrs) != 2 * n or len(nbytes) != n:
                raise ValueError("outputs: 2 device pointers and one byte count per context")
            pv = (C.c_void_p * (2 * n))(*[int(q) for q in ptrs])
            bv = (C.c_size_t * n)(*[int(q) for q in nbytes])
            st = L.pdf_batch_create_out(hs, dt, n, C.c_void_p(stream), FIELD[name], pv, bv, C.byref(h))
        if st != PDF_OK:
            raise PdfError(st, L.pdf_last_error(None).decode())
        self._h = h

    def step(self, nsteps: int = 1):
        _chk(lib().pdf_batch_step(self._h, nsteps), "pdf_batch_step")

    def sync(self):
        f = C.c_int32(-1)
        st = lib().pdf_batch_sync(self._h, C.byref(f))
        if st != PDF_OK:
            raise PdfError(st, f"case {f.value}: " + lib().pdf_last_error(self.canyons[f.value].handle).decode())

    def close(self):
        if getattr(self, "_h", None):
            lib().pdf_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
