"""TEST INFRASTRUCTURE ONLY: ctypes wrapper of the plain FP64 CPU oracle.

The oracle (pdf_oracle.c) restates the per-particle time step of the joint
velocity-frequency-scalar PDF method (Bakosi, Franzese & Boybeyi, Section 2
and Section 3) in plain single-threaded C. Only the test-suite, the smoke
check and the benchmark's CPU-baseline leg may import this module. It shares
no code with the CUDA library.

Functions without an independent pin ("parity unpinned"): the elliptic
relaxation wall value wp_ij = -4.5 eps n_i n_j (Section 2.1 defers the wall
conditions to companion work that is not part of the paper).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pdf_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "liborc.so")

_lock = threading.Lock()
_lib = None

# Table 2 of the paper and the wall-function constants of Section 2.2
TABLE2 = dict(C1=1.85, C2=0.63, C3=5.0, C4=0.25, CT=6.0, CL=0.134, Ceta=72.0, Cv=1.4,
              gamma5=0.1, Comega1=0.5, Comega2=0.73, Cs=0.02, Ct=0.7)
WALL = dict(C0=3.5, Cmu=0.09, kappa=0.41, E=8.5)


class orc_params(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "C1", "C2", "C3", "C4", "CT", "CL", "Ceta", "Cv", "gamma5", "Comega1", "Comega2", "Cs", "Ct",
        "C0", "Cmu", "kappa", "E", "nu", "fx", "fy", "yp", "wall_offset", "x0", "y0", "r0",
        "period", "k0", "ustar", "y_roof", "er_wall", "floor_k", "floor_eps", "floor_omega",
        "cg_tol")] + [
        ("cg_maxit", C.c_int32), ("nb1", C.c_int32), ("nb2", C.c_int32), ("nb3", C.c_int32),
        ("wall_model", C.c_int32), ("mix_exp", C.c_int32), ("reflect_max", C.c_int32),
        ("rotta", C.c_int32), ("seed", C.c_uint64), ("case_id", C.c_uint32), ("omega_wall", C.c_int32),
        ("pressure", C.c_int32), ("pad_", C.c_int32)]


def build(force: bool = False) -> str:
    """Compile the oracle with plain IEEE arithmetic (no FMA contraction)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "pdf_oracle.h"))):
        compile_source(SRC, LIB)
    return LIB


def compile_source(src: str, out: str) -> str:
    """Compile one copy of the oracle's C source into a shared library (the
    mutation pins build altered copies with the same flags)."""
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-I", HERE, "-o", tmp, src, "-lm"])
    os.replace(tmp, out)
    return out


def load(path: str):
    """Open an oracle library and declare its entry points."""
    L = C.CDLL(path)
    P = C.POINTER
    d, i32, u8, u32 = P(C.c_double), P(C.c_int32), P(C.c_uint8), P(C.c_uint32)
    L.orc_create.restype = C.c_void_p
    L.orc_create.argtypes = [P(orc_params), C.c_int32, d, C.c_int32, i32, i32, i32, i32]
    L.orc_destroy.argtypes = [C.c_void_p]
    L.orc_num_particles.argtypes = [C.c_void_p]
    L.orc_step_index.argtypes = [C.c_void_p]
    L.orc_cg_iterations.argtypes = [C.c_void_p]
    L.orc_seed.argtypes = [C.c_void_p, C.c_int32]
    L.orc_set_particles.argtypes = [C.c_void_p, C.c_int32] + [d] * 7 + [u32, i32, C.c_int32]
    L.orc_get_particles.argtypes = [C.c_void_p] + [d] * 7 + [u32, i32, u8]
    L.orc_estimate_stats.argtypes = [C.c_void_p]
    L.orc_advance.argtypes = [C.c_void_p, C.c_double]
    L.orc_project.argtypes = [C.c_void_p, C.c_double]
    L.orc_step.argtypes = [C.c_void_p, C.c_double, C.c_int32]
    L.orc_advance_subset.argtypes = [C.c_void_p, C.c_double, i32, C.c_int32]
    L.orc_get_field.argtypes = [C.c_void_p, C.c_int32, d]
    L.orc_philox4x32_10.argtypes = [u32, u32, u32]
    L.orc_philox4x32_10.restype = None
    L.orc_gauss8.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, d]
    L.orc_gauss8.restype = None
    L.orc_locate.argtypes = [C.c_void_p, C.c_double, C.c_double]
    L.orc_reflect.argtypes = [C.c_void_p, C.c_int32, d, d, d, d, d, d]
    L.orc_sde.argtypes = [P(orc_params), C.c_int32, C.c_double, d, d, d, d, d, d, d]
    L.orc_sde.restype = None
    L.orc_fe_solve.argtypes = [C.c_void_p, d, d, d, u8, d, C.c_int32]
    L.orc_bins.argtypes = [P(orc_params), C.c_int32, d, d, d, u32, i32]
    L.orc_set_node_fields.argtypes = [C.c_void_p, d, d, d]
    L.orc_set_node_wp.argtypes = [C.c_void_p, d]
    L.orc_h_contract.argtypes = [P(orc_params), d, d, C.c_double, C.c_double, d]
    L.orc_set_averaging.argtypes = [C.c_void_p, C.c_int32, C.c_int32]
    L.orc_averaging_count.argtypes = [C.c_void_p]
    L.orc_get_averages.argtypes = [C.c_void_p, C.c_int32, d]
    L.orc_probe.argtypes = [C.c_void_p, C.c_int32, C.c_int32, d, d, C.c_int32, d, i32]
    L.orc_set_cdf_probes.argtypes = [C.c_void_p, d, d, C.c_int32, C.c_int32]
    L.orc_get_cdf.argtypes = [C.c_void_p, d, i32]
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load(build())
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def default_params(**over) -> dict:
    nu, ustar = 1.0 / 12000.0, 0.05
    p = dict(TABLE2)
    p.update(WALL)
    p.update(nu=nu, fx=ustar ** 2 / 1.0, fy=0.0, yp=30 * nu / ustar, wall_offset=0.0,
             x0=1.5, y0=0.0, r0=0.05, period=3.0, k0=1e-3, ustar=ustar, y_roof=1.0, er_wall=4.5,
             floor_k=1e-12, floor_eps=1e-12, floor_omega=1e-12, cg_tol=1e-12, cg_maxit=50000,
             nb1=2, nb2=2, nb3=2, wall_model=0, mix_exp=0, reflect_max=8, rotta=0, seed=0,
             case_id=0, omega_wall=0, pressure=0, pad_=0)
    p.update(over)
    return p


def make_params(d: dict) -> orc_params:
    s = orc_params()
    for name, _ in orc_params._fields_:
        setattr(s, name, d[name])
    return s


FIELDS = dict(elem_n=(0, 1), elem_mean=(1, 5), elem_R=(2, 6), elem_psivar=(3, 1), elem_cm=(4, None),
              node_mean=(5, 4), node_R=(6, 6), node_ke=(7, 2), elem_der=(8, 9), node_pack=(9, 11),
              node_wp=(10, 5), node_wdist=(11, 1), node_grad=(12, 4), node_psivar=(13, 1),
              elem_omw=(14, 5), node_omw=(15, 5), node_p=(16, 1))


class Oracle:
    """One oracle context over one mesh."""

    def __init__(self, params: dict, mesh: dict, library=None):
        L = self._L = library if library is not None else lib()
        self.params = dict(params)
        self._p = make_params(self.params)
        self.nnode = int(mesh["xy"].shape[0])
        self.ntri = int(mesh["tri"].shape[0])
        self.nbins = params["nb1"] * params["nb2"] * params["nb3"]
        xy = np.ascontiguousarray(mesh["xy"], dtype=np.float64)
        tri = np.ascontiguousarray(mesh["tri"], dtype=np.int32)
        tag = np.ascontiguousarray(mesh["edge_tag"], dtype=np.int32)
        pair = np.ascontiguousarray(mesh["periodic_pair"], dtype=np.int32)
        st = C.c_int32(0)
        self._c = L.orc_create(C.byref(self._p), self.nnode, _p(xy, C.c_double), self.ntri,
                               _p(tri, C.c_int32), _p(tag, C.c_int32), _p(pair, C.c_int32),
                               C.byref(st))
        if not self._c:
            raise RuntimeError(f"oracle rejected the mesh (status {st.value})")

    def __del__(self):
        c = getattr(self, "_c", None)
        if c:
            self._L.orc_destroy(c)
            self._c = None

    def seed(self, per_element: int):
        self._check(self._L.orc_seed(self._c, per_element))

    def set_particles(self, st: dict, step: int = 0):
        n = int(st["x"].shape[0])
        arr = {k: np.ascontiguousarray(st[k], dtype=np.float64) for k in ("x", "y", "u", "v", "w", "om", "psi")}
        ids = np.ascontiguousarray(st["id"], dtype=np.uint32)
        el = np.ascontiguousarray(st["elem"], dtype=np.int32)
        self._check(self._L.orc_set_particles(self._c, n, *[_p(arr[k], C.c_double) for k in
                                                          ("x", "y", "u", "v", "w", "om", "psi")],
                                            _p(ids, C.c_uint32), _p(el, C.c_int32), step))

    def particles(self) -> dict:
        n = self._L.orc_num_particles(self._c)
        out = {k: np.empty(n, np.float64) for k in ("x", "y", "u", "v", "w", "om", "psi")}
        out["id"] = np.empty(n, np.uint32)
        out["elem"] = np.empty(n, np.int32)
        out["bin"] = np.empty(n, np.uint8)
        self._check(self._L.orc_get_particles(self._c, *[_p(out[k], C.c_double) for k in
                                                       ("x", "y", "u", "v", "w", "om", "psi")],
                                            _p(out["id"], C.c_uint32), _p(out["elem"], C.c_int32),
                                            _p(out["bin"], C.c_uint8)))
        return out

    @property
    def step_index(self) -> int:
        return self._L.orc_step_index(self._c)

    @property
    def cg_iterations(self) -> int:
        return self._L.orc_cg_iterations(self._c)

    def estimate_stats(self, check: bool = True) -> int:
        st = self._L.orc_estimate_stats(self._c)
        if check:
            self._check(st)
        return st

    def advance(self, dt: float, check: bool = True) -> int:
        st = self._L.orc_advance(self._c, dt)
        if check:
            self._check(st)
        return st

    def project(self, dt: float, check: bool = True) -> int:
        st = self._L.orc_project(self._c, dt)
        if check:
            self._check(st)
        return st

    def advance_subset(self, dt: float, idx, check: bool = True) -> int:
        idx = np.ascontiguousarray(idx, np.int32)
        st = self._L.orc_advance_subset(self._c, dt, _p(idx, C.c_int32), idx.size)
        if check:
            self._check(st)
        return st

    def step(self, dt: float, nsteps: int = 1, check: bool = True) -> int:
        st = self._L.orc_step(self._c, dt, nsteps)
        if check:
            self._check(st)
        return st

    def field(self, name: str) -> np.ndarray:
        fid, width = FIELDS[name]
        if width is None:
            width = self.nbins
        rows = self.ntri if name.startswith("elem") else self.nnode
        out = np.empty(rows * width, np.float64)
        self._check(self._L.orc_get_field(self._c, fid, _p(out, C.c_double)))
        return out.reshape(rows, width) if width > 1 else out

    def set_node_fields(self, nmean, nR, nke):
        a = [np.ascontiguousarray(v, np.float64) for v in (nmean, nR, nke)]
        self._check(self._L.orc_set_node_fields(self._c, *[_p(v, C.c_double) for v in a]))

    def set_node_wp(self, wp):
        wp = np.ascontiguousarray(wp, np.float64)
        self._check(self._L.orc_set_node_wp(self._c, _p(wp, C.c_double)))

    # time averages, probes, scalar CDFs (Section 3, Table 1, Fig. 7)
    AVERAGES = dict(elem_mean=(0, 5), elem_R=(1, 6), elem_psivar=(2, 1), node_mean=(3, 4))
    PROBES = dict(node_mean=0, elem_mean=1, elem_R=2, avg_node_mean=3, avg_elem_mean=4, avg_elem_R=5)

    def set_averaging(self, on: bool, reset: bool = False):
        self._check(self._L.orc_set_averaging(self._c, int(on), int(reset)))

    @property
    def averaging_count(self) -> int:
        return self._L.orc_averaging_count(self._c)

    def averages(self, name: str) -> np.ndarray:
        which, width = self.AVERAGES[name]
        rows = self.nnode if name == "node_mean" else self.ntri
        out = np.empty(rows * width, np.float64)
        self._check(self._L.orc_get_averages(self._c, which, _p(out, C.c_double)))
        return out.reshape(rows, width) if width > 1 else out

    def probe(self, name: str, comp: int, x, y):
        x = np.ascontiguousarray(x, np.float64)
        y = np.ascontiguousarray(y, np.float64)
        out = np.empty(x.size, np.float64)
        el = np.empty(x.size, np.int32)
        self._check(self._L.orc_probe(self._c, self.PROBES[name], comp, _p(x, C.c_double), _p(y, C.c_double),
                                      x.size, _p(out, C.c_double), _p(el, C.c_int32)))
        return out, el

    def set_cdf_probes(self, x, y, nbins: int):
        x = np.ascontiguousarray(x, np.float64)
        y = np.ascontiguousarray(y, np.float64)
        self._cdf_shape = (x.size, nbins)
        self._check(self._L.orc_set_cdf_probes(self._c, _p(x, C.c_double), _p(y, C.c_double), x.size, nbins))

    def cdf(self):
        n, nb = self._cdf_shape
        out = np.empty(n * nb, np.float64)
        el = np.empty(n, np.int32)
        self._check(self._L.orc_get_cdf(self._c, _p(out, C.c_double), _p(el, C.c_int32)))
        return out.reshape(n, nb), el

    def locate(self, x: float, y: float) -> int:
        return self._L.orc_locate(self._c, x, y)

    def reflect(self, tag: int, n, stat, u, v, w, om):
        n = np.ascontiguousarray(n, np.float64)
        stat = np.pad(np.asarray(stat, np.float64), (0, 12 - len(stat)))
        vals = [C.c_double(u), C.c_double(v), C.c_double(w), C.c_double(om)]
        self._check(self._L.orc_reflect(self._c, tag, _p(n, C.c_double), _p(stat, C.c_double),
                                      *[C.byref(x) for x in vals]))
        return tuple(x.value for x in vals)

    def fe_solve(self, L_elem, f_node, g_node, is_dir, x0=None):
        ncomp = f_node.shape[1]
        L_elem = np.ascontiguousarray(L_elem, np.float64)
        f_node = np.ascontiguousarray(f_node, np.float64)
        g_node = np.ascontiguousarray(g_node, np.float64)
        is_dir = np.ascontiguousarray(is_dir, np.uint8)
        x = np.zeros_like(f_node) if x0 is None else np.ascontiguousarray(x0, np.float64).copy()
        st = self._L.orc_fe_solve(self._c, _p(L_elem, C.c_double), _p(f_node, C.c_double),
                                _p(g_node, C.c_double), _p(is_dir, C.c_uint8), _p(x, C.c_double), ncomp)
        self._check(st)
        return x

    @staticmethod
    def _check(st):
        if st != 0:
            raise RuntimeError(f"oracle error {st}")


def philox4x32_10(key, ctr) -> np.ndarray:
    k = np.ascontiguousarray(key, np.uint32)
    c = np.ascontiguousarray(ctr, np.uint32)
    o = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(k, C.c_uint32), _p(c, C.c_uint32), _p(o, C.c_uint32))
    return o


def gauss8(seed: int, case_id: int, pid: int, step: int) -> np.ndarray:
    z = np.zeros(8, np.float64)
    lib().orc_gauss8(seed, case_id, pid, step, _p(z, C.c_double))
    return z


def sde(params: dict, dt: float, fields: np.ndarray, z: np.ndarray, state: dict) -> dict:
    """Mixing, frequency and velocity updates of n particles with given fields
    (n x 22, layout of the oracle's per-particle field vector) and Gaussians (n x 8)."""
    p = make_params(params)
    n = fields.shape[0]
    f = np.ascontiguousarray(fields, np.float64)
    zz = np.ascontiguousarray(z, np.float64)
    out = {k: np.ascontiguousarray(state[k], np.float64).copy() for k in ("u", "v", "w", "om", "psi")}
    lib().orc_sde(C.byref(p), n, dt, _p(f, C.c_double), _p(zz, C.c_double),
                  *[_p(out[k], C.c_double) for k in ("u", "v", "w", "om", "psi")])
    return out


def bins(params: dict, u, v, w, ids) -> np.ndarray:
    p = make_params(params)
    n = len(u)
    arrs = [np.ascontiguousarray(a, np.float64) for a in (u, v, w)]
    ids = np.ascontiguousarray(ids, np.uint32)
    out = np.zeros(n, np.int32)
    st = lib().orc_bins(C.byref(p), n, *[_p(a, C.c_double) for a in arrs], _p(ids, C.c_uint32),
                        _p(out, C.c_int32))
    if st:
        raise RuntimeError(st)
    return out


def h_contract(params: dict, R, g, k, om) -> np.ndarray:
    p = make_params(params)
    R = np.ascontiguousarray(R, np.float64)
    g = np.ascontiguousarray(g, np.float64)
    f = np.zeros(5, np.float64)
    lib().orc_h_contract(C.byref(p), _p(R, C.c_double), _p(g, C.c_double), k, om, _p(f, C.c_double))
    return f
