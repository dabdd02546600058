"""Python binding of the libisc C ABI (include/isc.h): argument marshalling only.

Every computation runs in libisc's CUDA kernels. There is no CPU fallback:
loading fails loudly if the library has not been built (``build.build()``)
or no CUDA device is available when a handle is created.

Array conventions on this side: the state ``u`` is (8, N) (SoA, rows p, x_LO,
y_O2, y_N2, y_CO2, T, S_w, S_g); residuals and Newton updates are returned as
(8, N) as well (the library's block-major layout transposed); Jacobian blocks
are (nnzb, 8, 8) with val[b][r][c] = dF_r/du_c.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB

c_double_p = C.POINTER(C.c_double)
c_int32_p = C.POINTER(C.c_int32)

ISC_OK = 0
STATUS = {0: "ok", -1: "invalid argument", -2: "CUDA error", -3: "out of device memory",
          -4: "singular diagonal block", -5: "Krylov solver did not converge",
          -6: "Newton did not converge", -7: "non-finite value", -8: "coke equation did not converge",
          -9: "device wait timed out", -10: "not implemented", -11: "call order violated"}
KRYLOV = {"gmres": 0, "bicgstab": 1}
PREC = {"none": 0, "bjacobi": 1, "bilu0": 2, "ilu0": 2, "cpr": 3}
PRECISION = {"fp64": 0, "mixed": 1, "mixed_fgmres": 2}
ORTH = {"cgs2": 0, "cgs1": 1}
K_CLASSES = ("props", "flux", "norm", "gj", "ilu_factor", "spmv", "prec_apply", "blas1", "update", "adjoint",
             "cpr", "spmv32")


class isc_grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double), ("depth", c_double_p)]


class isc_rock(C.Structure):
    _fields_ = [("phi_ref", c_double_p), ("perm", c_double_p)] + [
        (k, C.c_double) for k in ("cpor", "ctpor", "cptpor", "p_ref", "T_ref", "cv1", "cv2", "K_rock")]


D6 = C.c_double * 6
D3 = C.c_double * 3


class isc_fluid(C.Structure):
    _fields_ = [("M", D6), ("pc", D6), ("Tc", D6),
                ("rho_ref", D3), ("cp", D3), ("ct1", D3), ("ct2", D3), ("cpt", D3),
                ("p_ref", C.c_double), ("T_ref", C.c_double),
                ("cpg", (C.c_double * 4) * 6), ("hvr", D3), ("ev", D3),
                ("avg", D6), ("bvg", D6), ("avisc", D3), ("bvisc", D3),
                ("kv", (C.c_double * 5) * 3), ("K_phase", D3),
                ("coke_rho", C.c_double), ("coke_cp", C.c_double), ("coke_K", C.c_double), ("coke_M", C.c_double),
                ("Swc", C.c_double), ("Sorw", C.c_double), ("Sgc", C.c_double), ("Sorg", C.c_double),
                ("per_eps", C.c_double), ("gravity", C.c_double)]


class isc_reactions(C.Structure):
    _fields_ = [("nr", C.c_int32), ("kind", C.c_int32 * 8), ("comp", C.c_int32 * 8),
                ("stoich", (C.c_double * 7) * 8), ("A", C.c_double * 8), ("Ea", C.c_double * 8),
                ("dH", C.c_double * 8), ("coke_max", C.c_double)]


class isc_well(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_perf", C.c_int32), ("cells", c_int32_p), ("WI", c_double_p),
                ("target", C.c_double), ("inj_y", C.c_double * 6), ("inj_T", C.c_double),
                ("inj_phase", C.c_int32), ("control", C.c_int32), ("ref_depth", C.c_double),
                ("bhp_init", C.c_double)]


class isc_wells(C.Structure):
    _fields_ = [("nw", C.c_int32), ("wells", C.POINTER(isc_well))]


class isc_options(C.Structure):
    _fields_ = [("krylov", C.c_int32), ("restart", C.c_int32), ("prec", C.c_int32), ("decouple", C.c_int32),
                ("tol_lin", C.c_double), ("maxit_lin", C.c_int32), ("tol_newton", C.c_double),
                ("maxit_newton", C.c_int32), ("max_dp_frac", C.c_double), ("max_dT", C.c_double),
                ("profile", C.c_int32), ("precision", C.c_int32), ("stream", C.c_void_p),
                ("inner_its", C.c_int32), ("orth", C.c_int32)]


class isc_newton_info(C.Structure):
    _fields_ = [("status", C.c_int32), ("converged", C.c_int32), ("norm", C.c_double),
                ("norm_mass", C.c_double), ("norm_energy", C.c_double), ("norm_gs", C.c_double),
                ("krylov_iterations", C.c_int32), ("krylov_rel_residual", C.c_double)]


class isc_step_info(C.Structure):
    _fields_ = [("status", C.c_int32), ("newton_iterations", C.c_int32), ("krylov_iterations", C.c_int32),
                ("final_norm", C.c_double)]


class isc_run_info(C.Structure):
    _fields_ = [("status", C.c_int32), ("steps", C.c_int32), ("cuts", C.c_int32), ("newton_iterations", C.c_int32),
                ("krylov_iterations", C.c_int64), ("t", C.c_double), ("dt_next", C.c_double)]


class isc_stats(C.Structure):
    _fields_ = [("ms", C.c_double * 12), ("launches", C.c_int64 * 12), ("calls", C.c_int64 * 12)]


class isc_adjoint_spec(C.Structure):
    _fields_ = [("n_steps", C.c_int32), ("dt", c_double_p), ("checkpoint_every", C.c_int32),
                ("tol_adjoint", C.c_double)]


class isc_adjoint_info(C.Structure):
    _fields_ = [("status", C.c_int32), ("newton_iterations", C.c_int32), ("krylov_iterations_forward", C.c_int32),
                ("krylov_iterations_adjoint", C.c_int32), ("recomputed_steps", C.c_int32), ("loss", C.c_double),
                ("adjoint_rel_residual", C.c_double)]


_lib = None

# name -> (restype, argtypes)
_SIGS = {
    "isc_create": (C.c_int, [C.POINTER(isc_grid), C.POINTER(isc_rock), C.POINTER(isc_fluid),
                             C.POINTER(isc_reactions), C.POINTER(isc_wells), C.POINTER(isc_options),
                             C.POINTER(C.c_void_p)]),
    "isc_destroy": (None, [C.c_void_p]),
    "isc_set_options": (C.c_int, [C.c_void_p, C.POINTER(isc_options)]),
    "isc_default_options": (None, [C.POINTER(isc_options)]),
    "isc_status_string": (C.c_char_p, [C.c_int]),
    "isc_last_error": (C.c_char_p, [C.c_void_p]),
    "isc_num_cells": (C.c_int32, [C.c_void_p]),
    "isc_nnzb": (C.c_int32, [C.c_void_p]),
    "isc_init_equilibrium": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                       c_double_p, C.c_int32, c_int32_p, C.c_double]),
    "isc_set_state": (C.c_int, [C.c_void_p, c_double_p, c_double_p]),
    "isc_get_state": (C.c_int, [C.c_void_p, c_double_p, c_double_p]),
    "isc_set_state_device": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "isc_get_state_device": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "isc_begin_step": (C.c_int, [C.c_void_p]),
    "isc_assemble": (C.c_int, [C.c_void_p, C.c_double]),
    "isc_decouple": (C.c_int, [C.c_void_p]),
    "isc_solve": (C.c_int, [C.c_void_p, C.POINTER(isc_newton_info)]),
    "isc_update": (C.c_int, [C.c_void_p]),
    "isc_newton_step": (C.c_int, [C.c_void_p, C.c_double, C.POINTER(isc_newton_info)]),
    "isc_timestep": (C.c_int, [C.c_void_p, C.c_double, C.POINTER(isc_step_info)]),
    "isc_run": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int32,
                          C.c_int32, c_double_p, C.POINTER(isc_run_info)]),
    "isc_get_residual": (C.c_int, [C.c_void_p, c_double_p]),
    "isc_get_jacobian_bsr": (C.c_int, [C.c_void_p, c_int32_p, c_int32_p, c_double_p]),
    "isc_get_update": (C.c_int, [C.c_void_p, c_double_p]),
    "isc_set_system": (C.c_int, [C.c_void_p, c_double_p, c_double_p, C.c_int32]),
    "isc_set_heat_loss": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int32]),
    "isc_solve_external": (C.c_int, [C.c_void_p, c_int32_p, c_int32_p, c_double_p, c_double_p, c_double_p,
                                     C.POINTER(isc_newton_info)]),
    "isc_get_coke": (C.c_int, [C.c_void_p, c_double_p]),
    "isc_spmv": (C.c_int, [C.c_void_p, c_double_p, c_double_p]),
    "isc_build_preconditioner": (C.c_int, [C.c_void_p]),
    "isc_precond_apply": (C.c_int, [C.c_void_p, c_double_p, c_double_p]),
    "isc_get_stats": (C.c_int, [C.c_void_p, C.POINTER(isc_stats)]),
    "isc_get_ilu_diag": (C.c_int, [C.c_void_p, c_double_p]),
    "isc_reset_stats": (C.c_int, [C.c_void_p]),
    "isc_get_device_bytes": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint64)]),
    "isc_bsr_spmv_device": (C.c_int, [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_int32, C.c_void_p]),
    "isc_bilu0_apply_noalloc": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_void_p, C.c_void_p]),
    "isc_set_parameters": (C.c_int, [C.c_void_p, c_double_p, c_double_p, c_double_p]),
    "isc_check_reciprocal": (C.c_int, [C.c_int32, c_double_p, c_double_p, c_double_p]),
    "isc_check_bounded_wait": (C.c_int, []),
    "isc_check_row_starts": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, c_int32_p, C.POINTER(C.c_int64),
                                       C.POINTER(C.c_int32)]),
    "isc_measure_fma_rates": (C.c_int, [c_double_p, c_double_p]),
    "isc_num_coupled_wells": (C.c_int32, [C.c_void_p]),
    "isc_set_well_bhp": (C.c_int, [C.c_void_p, c_double_p]),
    "isc_get_well_bhp": (C.c_int, [C.c_void_p, c_double_p]),
    "isc_get_well_system": (C.c_int, [C.c_void_p, c_double_p, c_double_p, c_double_p, c_double_p]),
    "isc_get_parameters": (C.c_int, [C.c_void_p, c_double_p, c_double_p, c_double_p]),
    "isc_adjoint": (C.c_int, [C.c_void_p, C.POINTER(isc_adjoint_spec), c_double_p, c_double_p, c_double_p,
                              c_double_p, C.POINTER(isc_adjoint_info)]),
    "isc_adjoint_forward": (C.c_int, [C.c_void_p, C.POINTER(isc_adjoint_spec), c_double_p,
                                      C.POINTER(isc_adjoint_info)]),
    "isc_adjoint_backward": (C.c_int, [C.c_void_p, c_double_p, c_double_p, c_double_p, C.POINTER(isc_adjoint_info)]),
}


def load_library(path: str = LIB):
    """Load libisc.so and declare every exported entry point."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libisc is not built ({path} missing): run paper_1811_11992_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class IscError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)} ({status}): {msg}")
        self.status = status


def _dp(a):
    return a.ctypes.data_as(c_double_p)


def _ip(a):
    return a.ctypes.data_as(c_int32_p)


def default_options(**kw) -> isc_options:
    lib = load_library()
    o = isc_options()
    lib.isc_default_options(C.byref(o))
    for k, v in kw.items():
        if k == "krylov":
            v = KRYLOV[v] if isinstance(v, str) else v
        if k == "prec":
            v = PREC[v] if isinstance(v, str) else v
        if k == "precision":
            v = PRECISION[v] if isinstance(v, str) else v
        if k == "orth":
            v = ORTH[v] if isinstance(v, str) else v
        setattr(o, k, v)
    return o


def _fill(arr, values):
    flat = np.asarray(values, dtype=np.float64).reshape(-1)
    C.memmove(C.addressof(arr), flat.ctypes.data, flat.nbytes)


def create_args(case, keep):
    """The isc_create arguments of a Case: (isc_grid, isc_rock, isc_fluid,
    isc_reactions, isc_wells). The numpy arrays their pointers refer to are
    appended to keep, which must outlive the isc_create call."""

    def _k(a):
        keep.append(a)
        return a

    g = isc_grid(case.nx, case.ny, case.nz, case.dx, case.dy, case.dz,
                 _dp(_k(np.ascontiguousarray(case.depth, np.float64))))
    r = case.rock
    rock = isc_rock(_dp(_k(np.ascontiguousarray(case.phi_ref, np.float64))),
                    _dp(_k(np.ascontiguousarray(case.perm, np.float64).reshape(-1))),
                    r["cpor"], r["ctpor"], r["cptpor"], r["p_ref"], r["T_ref"], r["cv1"], r["cv2"], r["K_rock"])
    fl = isc_fluid()
    f = case.fluid
    for k in ("M", "pc", "Tc", "rho_ref", "cp", "ct1", "ct2", "cpt", "cpg", "hvr", "ev", "avg", "bvg",
              "avisc", "bvisc", "kv", "K_phase"):
        _fill(getattr(fl, k), f[k])
    for k in ("p_ref", "T_ref", "coke_rho", "coke_cp", "coke_K", "coke_M", "Swc", "Sorw", "Sgc", "Sorg",
              "per_eps", "gravity"):
        setattr(fl, k, float(f[k]))
    rx = isc_reactions()
    x = case.reactions
    rx.nr = int(x["nr"])
    for i in range(rx.nr):
        rx.kind[i] = int(x["kind"][i])
        rx.comp[i] = int(x["comp"][i])
        rx.A[i] = float(x["A"][i])
        rx.Ea[i] = float(x["Ea"][i])
        rx.dH[i] = float(x["dH"][i])
        for c in range(7):
            rx.stoich[i][c] = float(x["stoich"][i][c])
    rx.coke_max = float(x["coke_max"])
    wl = (isc_well * max(1, len(case.wells)))()
    for i, w in enumerate(case.wells):
        cells = _k(np.ascontiguousarray(w.cells, np.int32))
        WI = _k(np.ascontiguousarray(w.WI, np.float64))
        wl[i].kind = int(w.kind)
        wl[i].n_perf = len(cells)
        wl[i].cells = _ip(cells)
        wl[i].WI = _dp(WI)
        wl[i].target = float(w.target)
        _fill(wl[i].inj_y, w.inj_y)
        wl[i].inj_T = float(w.inj_T)
        wl[i].inj_phase = int(getattr(w, "inj_phase", 2))
        wl[i].control = int(getattr(w, "control", 0))
        wl[i].ref_depth = float(getattr(w, "ref_depth", 0.0))
        wl[i].bhp_init = float(getattr(w, "bhp_init", 0.0))
    wells = isc_wells(len(case.wells), _k(wl))
    return g, rock, fl, rx, wells


class Simulator:
    """A libisc handle built from an ``isc_inputs.Case``."""

    def __init__(self, case, options: isc_options | None = None, **opt_kw):
        lib = load_library()
        self.lib = lib
        self.case = case
        n = case.n
        self.n = n
        self._keep = []
        g, rock, fl, rx, wells = create_args(case, self._keep)
        if options is None:
            options = default_options(**opt_kw)
        self.options = options
        h = C.c_void_p()
        st = lib.isc_create(C.byref(g), C.byref(rock), C.byref(fl), C.byref(rx), C.byref(wells),
                            C.byref(options), C.byref(h))
        self._keep = []
        if st != ISC_OK:
            raise IscError(st, "isc_create failed")
        self.h = h
        self.nnzb = lib.isc_nnzb(h)
        self.nwc = lib.isc_num_coupled_wells(h)
        hl = getattr(case, "heat_loss", None)
        if hl:
            self.set_heat_loss(**hl)

    def _k(self, a):
        self._keep.append(a)
        return a

    def _check(self, st):
        if st != ISC_OK:
            raise IscError(st, self.lib.isc_last_error(self.h).decode())
        return st

    def close(self):
        if getattr(self, "h", None):
            self.lib.isc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_heat_loss(self, K_ob, d, T_ini, rho=0.0, faces=3):
        """Heat loss to the overburden (faces bit 1) and underburden (bit 2)."""
        self._check(self.lib.isc_set_heat_loss(self.h, float(K_ob), float(d), float(T_ini), float(rho), int(faces)))

    # ------------------------------------------------------------- options
    def set_options(self, **kw):
        for k, v in kw.items():
            if k == "krylov":
                v = KRYLOV[v] if isinstance(v, str) else v
            if k == "prec":
                v = PREC[v] if isinstance(v, str) else v
            if k == "precision":
                v = PRECISION[v] if isinstance(v, str) else v
            if k == "orth":
                v = ORTH[v] if isinstance(v, str) else v
            setattr(self.options, k, v)
        self._check(self.lib.isc_set_options(self.h, C.byref(self.options)))

    # --------------------------------------------------------------- state
    def init_equilibrium(self):
        ini = self.case.init
        yr = np.ascontiguousarray(ini["y_rest"], np.float64)
        ign = np.ascontiguousarray(self.case.ignited, np.int32)
        self._check(self.lib.isc_init_equilibrium(self.h, ini["p"], ini["T"], ini["Sw"], ini["So"], ini["x_LO"],
                                                  _dp(yr), len(ign), _ip(ign), ini["T_ignite"]))

    def set_state(self, u, coke=None):
        u = np.ascontiguousarray(u, np.float64).reshape(8, self.n)
        cp = None if coke is None else _dp(np.ascontiguousarray(coke, np.float64))
        cc = None if coke is None else np.ascontiguousarray(coke, np.float64)
        self._check(self.lib.isc_set_state(self.h, _dp(u), None if cc is None else _dp(cc)))

    def get_state(self, u=None, coke=None):
        """The state as (8, N) and (N,) float64 arrays: new ones, or the caller's
        own (pinned host buffers, for one, which the copy reaches directly)."""
        u = np.empty((8, self.n)) if u is None else u
        coke = np.empty(self.n) if coke is None else coke
        for a, shape in ((u, (8, self.n)), (coke, (self.n,))):
            if a.dtype != np.float64 or a.shape != shape or not a.flags["C_CONTIGUOUS"]:
                raise ValueError(f"get_state needs a C-contiguous float64 array of shape {shape}")
        self._check(self.lib.isc_get_state(self.h, _dp(u), _dp(coke)))
        return u, coke

    def begin_step(self):
        self._check(self.lib.isc_begin_step(self.h))

    # ------------------------------------------------------------ hot path
    def assemble(self, dt):
        self._check(self.lib.isc_assemble(self.h, float(dt)))

    def decouple(self):
        self._check(self.lib.isc_decouple(self.h))

    def solve(self):
        info = isc_newton_info()
        self._check(self.lib.isc_solve(self.h, C.byref(info)))
        return info

    def update(self):
        self._check(self.lib.isc_update(self.h))

    def newton_step(self, dt, check=True):
        info = isc_newton_info()
        st = self.lib.isc_newton_step(self.h, float(dt), C.byref(info))
        if check:
            self._check(st)
        return info

    def timestep(self, dt, check=True):
        info = isc_step_info()
        st = self.lib.isc_timestep(self.h, float(dt), C.byref(info))
        if check:
            self._check(st)
        return info

    def run(self, t_end, dt0, dt_max, dT_target=20.0, dS_target=0.2, max_cuts=8, max_steps=100000, check=True):
        """Time loop with step cuts and the step controller (isc_run) from the
        accepted state over t_end seconds: (isc_run_info, accepted step lengths)."""
        hist = np.zeros(int(max_steps))
        info = isc_run_info()
        st = self.lib.isc_run(self.h, float(t_end), float(dt0), float(dt_max), float(dT_target), float(dS_target),
                              int(max_cuts), int(max_steps), _dp(hist), C.byref(info))
        if check:
            self._check(st)
        return info, hist[:info.steps].copy()

    # ------------------------------------------------------------- exports
    def residual(self):
        F = np.empty((self.n, 8))
        self._check(self.lib.isc_get_residual(self.h, _dp(F)))
        return F.T.copy()

    def jacobian(self):
        rowptr = np.empty(self.n + 1, np.int32)
        col = np.empty(self.nnzb, np.int32)
        val = np.empty((self.nnzb, 8, 8))
        self._check(self.lib.isc_get_jacobian_bsr(self.h, _ip(rowptr), _ip(col), _dp(val)))
        return rowptr, col, val

    def newton_update(self):
        du = np.empty((self.n, 8))
        self._check(self.lib.isc_get_update(self.h, _dp(du)))
        return du.T.copy()

    def set_system(self, val, F, decoupled=False):
        """Load a caller's system: val (nnzb, 8, 8) blocks on this handle's
        pattern and F (8, N) residual (the solve targets J du = -F)."""
        v = np.ascontiguousarray(val, np.float64).reshape(self.nnzb, 8, 8)
        f = np.ascontiguousarray(np.asarray(F, np.float64).reshape(8, self.n).T)
        self._check(self.lib.isc_set_system(self.h, _dp(v), _dp(f), 1 if decoupled else 0))

    def solve_external(self, rowptr, col, val, b):
        """x with A x = b for a caller's BSR matrix on this handle's pattern
        (b and x as (8, N)); returns (x, isc_newton_info)."""
        rp = np.ascontiguousarray(rowptr, np.int32)
        cl = np.ascontiguousarray(col, np.int32)
        v = np.ascontiguousarray(val, np.float64).reshape(self.nnzb, 8, 8)
        bb = np.ascontiguousarray(np.asarray(b, np.float64).reshape(8, self.n).T)
        x = np.empty((self.n, 8))
        info = isc_newton_info()
        self._check(self.lib.isc_solve_external(self.h, _ip(rp), _ip(cl), _dp(v), _dp(bb), _dp(x), C.byref(info)))
        return x.T.copy(), info

    def coke(self):
        c = np.empty(self.n)
        self._check(self.lib.isc_get_coke(self.h, _dp(c)))
        return c

    def spmv(self, x):
        """y = A x for x given as (8, N) (no coupled wells; else spmv_full)."""
        if self.nwc:
            raise ValueError("the system has coupled wells: use spmv_full")
        xb = np.ascontiguousarray(np.asarray(x, np.float64).reshape(8, self.n).T)
        y = np.empty((self.n, 8))
        self._check(self.lib.isc_spmv(self.h, _dp(xb), _dp(y)))
        return y.T.copy()

    def build_preconditioner(self):
        self._check(self.lib.isc_build_preconditioner(self.h))

    def precond_apply(self, r):
        if self.nwc:
            raise ValueError("the system has coupled wells: use precond_apply_full")
        rb = np.ascontiguousarray(np.asarray(r, np.float64).reshape(8, self.n).T)
        z = np.empty((self.n, 8))
        self._check(self.lib.isc_precond_apply(self.h, _dp(rb), _dp(z)))
        return z.T.copy()

    def ilu_diag(self):
        """(N, 8, 8) inverted diagonal blocks of the block ILU(0) factors."""
        d = np.empty((self.n, 8, 8))
        self._check(self.lib.isc_get_ilu_diag(self.h, _dp(d)))
        return d

    def stats(self):
        s = isc_stats()
        self._check(self.lib.isc_get_stats(self.h, C.byref(s)))
        return {k: dict(ms=s.ms[i], launches=s.launches[i], calls=s.calls[i]) for i, k in enumerate(K_CLASSES)}

    def reset_stats(self):
        self._check(self.lib.isc_reset_stats(self.h))

    def device_bytes(self):
        """Bytes of device memory the handle holds now (isc_get_device_bytes)."""
        b = C.c_uint64()
        self._check(self.lib.isc_get_device_bytes(self.h, C.byref(b)))
        return int(b.value)

    # -------------------------------------------------------- coupled wells
    def well_bhp(self):
        b = np.empty(max(self.nwc, 1))
        self._check(self.lib.isc_get_well_bhp(self.h, _dp(b)))
        return b[:self.nwc]

    def set_well_bhp(self, bhp):
        b = np.ascontiguousarray(bhp, np.float64).reshape(self.nwc)
        self._check(self.lib.isc_set_well_bhp(self.h, _dp(b)))

    def well_system(self):
        """(B (nperf, 8), C (nperf, 8), D (nwc,), Fw (nwc,)) after assemble."""
        nperf = sum(len(w.cells) for w in self.case.wells if w.kind in (2, 3))
        B, Cm = np.empty((max(nperf, 1), 8)), np.empty((max(nperf, 1), 8))
        D, Fw = np.empty(max(self.nwc, 1)), np.empty(max(self.nwc, 1))
        self._check(self.lib.isc_get_well_system(self.h, _dp(B), _dp(Cm), _dp(D), _dp(Fw)))
        return B[:nperf], Cm[:nperf], D[:self.nwc], Fw[:self.nwc]

    def spmv_full(self, x):
        """y = [J B; C D] x on the flat vector (8N block-major, then the wells)."""
        x = np.ascontiguousarray(x, np.float64).reshape(-1)
        y = np.empty_like(x)
        self._check(self.lib.isc_spmv(self.h, _dp(x), _dp(y)))
        return y

    def precond_apply_full(self, r):
        r = np.ascontiguousarray(r, np.float64).reshape(-1)
        z = np.empty_like(r)
        self._check(self.lib.isc_precond_apply(self.h, _dp(r), _dp(z)))
        return z

    # -------------------------------------------------------- sensitivities
    def set_parameters(self, log_k=None, Ea=None, lnA=None):
        """Per-cell ln k multipliers (N), activation energies E_a (J/mol) and
        ln A of the reactions (nr); None leaves a group unchanged."""
        nr = int(self.case.reactions["nr"])
        lk = None if log_k is None else np.ascontiguousarray(log_k, np.float64).reshape(self.n)
        ea = None if Ea is None else np.ascontiguousarray(Ea, np.float64).reshape(nr)
        la = None if lnA is None else np.ascontiguousarray(lnA, np.float64).reshape(nr)
        self._check(self.lib.isc_set_parameters(self.h, None if lk is None else _dp(lk),
                                                None if ea is None else _dp(ea), None if la is None else _dp(la)))

    def get_parameters(self):
        nr = int(self.case.reactions["nr"])
        lk, ea, la = np.empty(self.n), np.empty(max(nr, 1)), np.empty(max(nr, 1))
        self._check(self.lib.isc_get_parameters(self.h, _dp(lk), _dp(ea), _dp(la)))
        return lk, ea[:nr], la[:nr]

    def adjoint(self, dts, checkpoint_every=5, tol_adjoint=0.0, gradient=True):
        """Run the time loop with the frozen step sizes dts from the current
        accepted state; return (L, g_log_k, g_Ea, g_lnA, info) with L the
        cumulative produced oil mass (kg). With gradient=False only L is
        computed and the gradients are None."""
        nr = int(self.case.reactions["nr"])
        d = np.ascontiguousarray(dts, np.float64).reshape(-1)
        spec = isc_adjoint_spec(len(d), _dp(d), int(checkpoint_every), float(tol_adjoint))
        info = isc_adjoint_info()
        L = C.c_double(0.0)
        if gradient:
            gk, ge, ga = np.empty(self.n), np.empty(max(nr, 1)), np.empty(max(nr, 1))
            st = self.lib.isc_adjoint(self.h, C.byref(spec), C.byref(L), _dp(gk), _dp(ge), _dp(ga), C.byref(info))
        else:
            st = self.lib.isc_adjoint(self.h, C.byref(spec), C.byref(L), None, None, None, C.byref(info))
        self._check(st)
        info_d = {k: getattr(info, k) for k, _ in isc_adjoint_info._fields_}
        if not gradient:
            return L.value, None, None, None, info_d
        return L.value, gk, ge[:nr], ga[:nr], info_d

    def adjoint_forward(self, dts, checkpoint_every=5, tol_adjoint=0.0):
        """The time loop with the frozen step sizes dts from the accepted state:
        returns (L, info) and keeps the checkpoints for adjoint_backward."""
        d = np.ascontiguousarray(dts, np.float64).reshape(-1)
        spec = isc_adjoint_spec(len(d), _dp(d), int(checkpoint_every), float(tol_adjoint))
        info = isc_adjoint_info()
        L = C.c_double(0.0)
        self._check(self.lib.isc_adjoint_forward(self.h, C.byref(spec), C.byref(L), C.byref(info)))
        return L.value, {k: getattr(info, k) for k, _ in isc_adjoint_info._fields_}

    def adjoint_backward(self):
        """The reverse sweep over the last adjoint_forward: (g_log_k, g_Ea, g_lnA, info)."""
        nr = int(self.case.reactions["nr"])
        gk, ge, ga = np.empty(self.n), np.empty(max(nr, 1)), np.empty(max(nr, 1))
        info = isc_adjoint_info()
        self._check(self.lib.isc_adjoint_backward(self.h, _dp(gk), _dp(ge), _dp(ga), C.byref(info)))
        return gk, ge[:nr], ga[:nr], {k: getattr(info, k) for k, _ in isc_adjoint_info._fields_}

    def set_state_device(self, d_u, d_coke=None):
        self._check(self.lib.isc_set_state_device(self.h, C.c_void_p(d_u), C.c_void_p(d_coke) if d_coke else None))

    def get_state_device(self, d_u, d_coke=None):
        self._check(self.lib.isc_get_state_device(self.h, C.c_void_p(d_u), C.c_void_p(d_coke) if d_coke else None))


def bsr_spmv_device(nrows, d_rowptr, d_col, d_val, d_x, d_y, unit_diag=0, stream=None):
    lib = load_library()
    st = lib.isc_bsr_spmv_device(nrows, C.c_void_p(d_rowptr), C.c_void_p(d_col), C.c_void_p(d_val),
                                 C.c_void_p(d_x), C.c_void_p(d_y), unit_diag, C.c_void_p(stream) if stream else None)
    if st != ISC_OK:
        raise IscError(st, "isc_bsr_spmv_device failed")


NOALLOC_MAX_CELLS = 65536


def bilu0_apply_noalloc(nx, ny, nz, d_rowptr, d_A, d_Dinv, d_r, d_z, stream=None):
    """Allocation-free ILU(0) apply on caller-owned device buffers (pointers as
    ints). Raises IscError with the library's status on any failure (grids
    beyond NOALLOC_MAX_CELLS cells give status -1, invalid argument)."""
    lib = load_library()
    st = lib.isc_bilu0_apply_noalloc(nx, ny, nz, C.c_void_p(d_rowptr), C.c_void_p(d_A), C.c_void_p(d_Dinv),
                                     C.c_void_p(d_r), C.c_void_p(d_z), C.c_void_p(stream) if stream else None)
    if st != ISC_OK:
        raise IscError(st, "isc_bilu0_apply_noalloc failed")


def measure_fma_rates():
    """(FP64, FP32) FMA throughput of the current device in GFLOP/s."""
    lib = load_library()
    f64, f32 = C.c_double(0.0), C.c_double(0.0)
    st = lib.isc_measure_fma_rates(C.byref(f64), C.byref(f32))
    if st != ISC_OK:
        raise IscError(st, "isc_measure_fma_rates failed")
    return f64.value, f32.value


def check_reciprocal(x):
    """(device reciprocal of the pivots, device 1.0 / x) for host doubles x."""
    lib = load_library()
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    z = np.empty_like(x)
    st = lib.isc_check_reciprocal(x.size, _dp(x), _dp(y), _dp(z))
    if st:
        raise IscError(st, "isc_check_reciprocal failed")
    return y, z


def check_bounded_wait():
    """Status of the bounded-wait self-test (ISC_ERR_TIMEOUT expected)."""
    return load_library().isc_check_bounded_wait()


def check_row_starts(nx, ny, nz, rowptr):
    """(mismatching cells, first of them or -1) of the sweeps' closed-form BSR
    row starts against rowptr (isc_check_row_starts)."""
    rp = np.ascontiguousarray(rowptr, np.int32)
    cnt, first = C.c_int64(), C.c_int32()
    st = load_library().isc_check_row_starts(int(nx), int(ny), int(nz), _ip(rp), C.byref(cnt), C.byref(first))
    if st != ISC_OK:
        raise IscError(st, "isc_check_row_starts failed")
    return int(cnt.value), int(first.value)


# the binding uses the C-ABI names
def isc_create(case, **opt):
    return Simulator(case, **opt)
