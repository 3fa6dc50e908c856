"""ctypes binding of libofdft (include/ofdft.h): argument marshalling only.

Every function named ``ofdft_*`` here calls the C entry point of the same
name; :class:`Context` is a small convenience wrapper over them.  There is no
CPU fallback: if the CUDA library is missing, loading raises.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libofdft.so")

FUNCTIONALS = {"fttf": 0, "sga": 1, "vt84f": 2, "kst2": 3, "vwtf": 4, "tw": 5, "apbef": 6}
PRECISIONS = {"fp64": 0, "mixed": 1}
POINTWISE = {"f32x2": 0, "f64": 1}
LPP = {"gauss": 0, "ha": 1}
STATUS = {0: "OFDFT_OK", -1: "OFDFT_EINVAL", -2: "OFDFT_ENOMEM", -3: "OFDFT_ENOCONV",
          -4: "OFDFT_ENUMERIC", -5: "OFDFT_ETIMEOUT", -6: "OFDFT_EDEVICE", -7: "OFDFT_EBUSY",
          -8: "OFDFT_ECANCELED"}

_P = ctypes.POINTER(ctypes.c_double)

# Gradient tolerances of the batched and serving mixed-precision forms.
# Single points (the batched form) to 1e-5 stay within 1e-6 Ha/atom (free
# energy), 1e-4 Ha/bohr (forces) and 1e-3 relative (pressure) of the FP64
# path at gtol 1e-8, with margin (measured over the 64-instance batch:
# 5e-8 Ha/atom, 1.1e-6 Ha/bohr, 1.4e-5; tests/test_gpu_mixed.py checks it at
# 10 kK, 250 kK and 4 MK).  MD requests (the serving form) converge every
# step to 1e-6: their per-step force errors feed the trajectory, and at 1e-5
# five steps already moved the free energy by 4.5e-6 Ha/atom (at 1e-6:
# 1.7e-7).
MIXED_FORM_GTOL = 1e-5
MIXED_MD_GTOL = 1e-6


class Params(ctypes.Structure):
    _fields_ = [("xc", ctypes.c_int), ("rc", ctypes.c_double), ("precision", ctypes.c_int),
                ("device", ctypes.c_int), ("stream", ctypes.c_void_p), ("pointwise", ctypes.c_int),
                ("lpp", ctypes.c_int), ("lpp_A", ctypes.c_double), ("lpp_qc", ctypes.c_double)]


class Energy(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "F_tot", "F_s", "minus_TS", "E_H", "E_loc", "F_xc", "E_ion", "E_int", "mu", "E_alphaZ",
        "P", "P_s", "P_xc", "P_H", "P_loc", "P_ion")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("evaluations", ctypes.c_int),
                ("gnorm", ctypes.c_double), ("status", ctypes.c_int),
                ("evaluations_lo", ctypes.c_int)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class MDParams(ctypes.Structure):
    _fields_ = [("dt_fs", ctypes.c_double), ("T_kelvin", ctypes.c_double),
                ("tau_steps", ctypes.c_double), ("gtol", ctypes.c_double), ("maxit", ctypes.c_int)]


class ServeParams(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("max_slots", ctypes.c_int),
                ("hbm_budget_bytes", ctypes.c_double), ("dry_run", ctypes.c_int),
                ("dry_run_ms", ctypes.c_double), ("max_bypass", ctypes.c_int)]


class Request(ctypes.Structure):
    _fields_ = [("cell", ctypes.c_double * 9), ("grid", ctypes.c_int * 3), ("nat", ctypes.c_int),
                ("ions", _P), ("Z", _P), ("vel", _P), ("T_kelvin", ctypes.c_double),
                ("functional", ctypes.c_int), ("precision", ctypes.c_int), ("xc", ctypes.c_int),
                ("rc", ctypes.c_double), ("md_steps", ctypes.c_int), ("dt_fs", ctypes.c_double),
                ("gtol", ctypes.c_double), ("maxit", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_longlong), ("status", ctypes.c_int), ("E", Energy),
                ("P_mean", ctypes.c_double), ("steps_done", ctypes.c_int),
                ("evaluations", ctypes.c_longlong), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
                ("footprint_bytes", ctypes.c_double)]

    def as_dict(self):
        d = {n: getattr(self, n) for n, _ in self._fields_ if n != "E"}
        d["E"] = self.E.as_dict()
        return d


class OfdftError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


_lib = None

SIGNATURES = {
    "ofdft_default_params": (None, [ctypes.POINTER(Params)]),
    "ofdft_setup": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.c_int, _P, _P,
                                   ctypes.c_double, ctypes.c_int, ctypes.POINTER(Params),
                                   ctypes.POINTER(ctypes.c_void_p)]),
    "ofdft_set_positions": (ctypes.c_int, [ctypes.c_void_p, _P]),
    "ofdft_set_phi": (ctypes.c_int, [ctypes.c_void_p, _P]),
    "ofdft_energy_potential": (ctypes.c_int, [ctypes.c_void_p, _P, ctypes.POINTER(Energy), _P]),
    "ofdft_minimize": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int,
                                      ctypes.POINTER(Energy), ctypes.POINTER(Stats)]),
    "ofdft_minimize_tn": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double, ctypes.POINTER(Energy), ctypes.POINTER(Stats),
                                         ctypes.POINTER(ctypes.c_int)]),
    "ofdft_forces": (ctypes.c_int, [ctypes.c_void_p, _P, _P]),
    "ofdft_get_density": (ctypes.c_int, [ctypes.c_void_p, _P]),
    "ofdft_stress": (ctypes.c_int, [ctypes.c_void_p, _P, _P]),
    "ofdft_set_masses": (ctypes.c_int, [ctypes.c_void_p, _P]),
    "ofdft_md_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(MDParams), ctypes.c_int, _P, _P,
                                     _P, ctypes.POINTER(Energy), ctypes.POINTER(Stats)]),
    "ofdft_md_andersen": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, _P, _P,
                                         ctypes.POINTER(ctypes.c_int)]),
    "ofdft_md_state": (ctypes.c_int, [ctypes.c_void_p, _P, _P]),
    "ofdft_md_conserved": (ctypes.c_int, [ctypes.c_void_p, _P]),
    "ofdft_sizes": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong),
                                   ctypes.POINTER(ctypes.c_int)]),
    "ofdft_timer_select": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "ofdft_timer_read": (ctypes.c_int, [ctypes.c_void_p, _P, ctypes.POINTER(ctypes.c_longlong),
                                        ctypes.c_int]),
    "ofdft_kernel_launches": (ctypes.c_longlong, [ctypes.c_void_p]),
    "ofdft_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "ofdft_tfunc_eval": (ctypes.c_int, [ctypes.c_longlong, _P, _P]),
    "ofdft_pointwise_eval": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_longlong,
                                            _P, _P, ctypes.c_int, _P, ctypes.POINTER(ctypes.c_longlong)]),
    "ofdft_ffmath_eval": (ctypes.c_int, [ctypes.c_int, ctypes.c_longlong, _P, _P, _P]),
    "ofdft_destroy": (None, [ctypes.c_void_p]),
    "ofdft_minimize_start": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int]),
    "ofdft_minimize_query": (ctypes.c_int, [ctypes.c_void_p]),
    "ofdft_minimize_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Energy),
                                           ctypes.POINTER(Stats)]),
    "ofdft_batch_minimize": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_void_p),
                                            ctypes.c_double, ctypes.c_int, ctypes.POINTER(Energy),
                                            ctypes.POINTER(Stats)]),
    "ofdft_footprint": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int, _P]),
    "ofdft_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "ofdft_serve_start": (ctypes.c_int, [ctypes.POINTER(ServeParams), ctypes.POINTER(ctypes.c_void_p)]),
    "ofdft_serve_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Request),
                                          ctypes.POINTER(ctypes.c_longlong)]),
    "ofdft_serve_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong, ctypes.POINTER(Result)]),
    "ofdft_serve_drain": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    "ofdft_serve_cancel": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong]),
    "ofdft_serve_clock": (ctypes.c_double, [ctypes.c_void_p]),
    "ofdft_serve_peaks": (ctypes.c_int, [ctypes.c_void_p, _P, ctypes.POINTER(ctypes.c_int)]),
    "ofdft_serve_stop": (ctypes.c_int, [ctypes.c_void_p]),
    "ofdft_energy_potential_static": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                                     _P, _P, ctypes.c_double, ctypes.c_int,
                                                     ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
                                                     ctypes.c_void_p, ctypes.POINTER(Energy),
                                                     ctypes.c_void_p]),
}


def load(path=LIB_PATH):
    """Load libofdft.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError("libofdft.so not built (run __graft_entry__.build()): %s" % path)
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_P)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _check(ctx, status):
    if status != 0:
        msg = load().ofdft_last_error(ctx)
        raise OfdftError(status, msg.decode() if msg else "")


# ----------------------------------------------------- ABI-named functions
def ofdft_default_params():
    p = Params()
    load().ofdft_default_params(ctypes.byref(p))
    return p


def ofdft_setup(cell, grid, ions, Z, T_kelvin, functional, params=None):
    lib = load()
    cell = _f64(cell).reshape(-1)
    if cell.size == 3:
        cell = np.diag(cell).reshape(-1)
    grid = (ctypes.c_int * 3)(*[int(x) for x in grid])
    ions = _f64(ions, (-1, 3))
    Z = _f64(Z, (-1,))
    f = FUNCTIONALS[functional] if isinstance(functional, str) else int(functional)
    p = params if params is not None else ofdft_default_params()
    out = ctypes.c_void_p()
    st = lib.ofdft_setup(_ptr(cell), grid, ions.shape[0], _ptr(ions), _ptr(Z), float(T_kelvin), f,
                         ctypes.byref(p), ctypes.byref(out))
    _check(None, st)
    return out.value


def ofdft_set_positions(ctx, ions):
    _check(ctx, load().ofdft_set_positions(ctx, _ptr(_f64(ions, (-1, 3)))))


def ofdft_set_phi(ctx, phi=None):
    _check(ctx, load().ofdft_set_phi(ctx, None if phi is None else _ptr(_f64(phi))))


def ofdft_energy_potential(ctx, phi=None, want_v=False):
    N = ofdft_sizes(ctx)[0]
    E = Energy()
    v = np.empty(N) if want_v else None
    ph = None if phi is None else _f64(phi).reshape(-1)
    _check(ctx, load().ofdft_energy_potential(ctx, _ptr(ph), ctypes.byref(E), _ptr(v)))
    return E.as_dict(), v


def ofdft_minimize(ctx, gtol=1e-8, maxit=5000, raise_on_noconv=True):
    E, S = Energy(), Stats()
    st = load().ofdft_minimize(ctx, float(gtol), int(maxit), ctypes.byref(E), ctypes.byref(S))
    if st != -3 or raise_on_noconv:
        _check(ctx, st)
    return E.as_dict(), S.as_dict()


def ofdft_minimize_tn(ctx, gtol=1e-8, maxit=500, inner_max=20, eta=0.1, raise_on_noconv=True):
    """Truncated-Newton minimisation; returns (energy dict, stats dict, Hessian products)."""
    E, S, nh = Energy(), Stats(), ctypes.c_int()
    st = load().ofdft_minimize_tn(ctx, float(gtol), int(maxit), int(inner_max), float(eta), ctypes.byref(E),
                                  ctypes.byref(S), ctypes.byref(nh))
    if st != 0 and not (st == -3 and not raise_on_noconv):
        _check(ctx, st)
    return E.as_dict(), S.as_dict(), nh.value


def ofdft_minimize_start(ctx, gtol=1e-8, maxit=5000):
    _check(ctx, load().ofdft_minimize_start(ctx, float(gtol), int(maxit)))


def ofdft_minimize_query(ctx):
    """True once the minimisation started last has finished."""
    st = load().ofdft_minimize_query(ctx)
    if st == -7:
        return False
    _check(ctx, st)
    return True


def ofdft_minimize_wait(ctx, raise_on_noconv=True):
    E, S = Energy(), Stats()
    st = load().ofdft_minimize_wait(ctx, ctypes.byref(E), ctypes.byref(S))
    if st != -3 or raise_on_noconv:
        _check(ctx, st)
    return E.as_dict(), S.as_dict()


def ofdft_batch_minimize(ctxs, gtol=1e-8, maxit=5000):
    """Minimise every context concurrently; returns ([E], [stats], status)."""
    n = len(ctxs)
    arr = (ctypes.c_void_p * n)(*ctxs)
    E = (Energy * n)()
    S = (Stats * n)()
    st = load().ofdft_batch_minimize(n, arr, float(gtol), int(maxit), E, S)
    return [e.as_dict() for e in E], [x.as_dict() for x in S], st


def ofdft_footprint(grid, nat, precision="fp64"):
    g = (ctypes.c_int * 3)(*[int(x) for x in grid])
    b = np.zeros(1)
    _check(None, load().ofdft_footprint(g, int(nat), PRECISIONS.get(precision, precision), _ptr(b)))
    return float(b[0])


def ofdft_autotune(ctx, reps=3):
    _check(ctx, load().ofdft_autotune(ctx, int(reps)))


def ofdft_forces(ctx):
    nat = ofdft_sizes(ctx)[1]
    F = np.empty((nat, 3))
    P = np.zeros(1)
    _check(ctx, load().ofdft_forces(ctx, _ptr(F), _ptr(P)))
    return F, float(P[0])


def ofdft_get_density(ctx):
    n = np.empty(ofdft_sizes(ctx)[0])
    _check(ctx, load().ofdft_get_density(ctx, _ptr(n)))
    return n


def ofdft_set_masses(ctx, m):
    _check(ctx, load().ofdft_set_masses(ctx, _ptr(_f64(m, (-1,)))))


def ofdft_md_step(ctx, dt_fs, T_kelvin, nsteps=1, pos=None, vel=None, tau_steps=100.0,
                  gtol=1e-8, maxit=5000):
    mp = MDParams(float(dt_fs), float(T_kelvin), float(tau_steps), float(gtol), int(maxit))
    nat = ofdft_sizes(ctx)[1]
    pos = None if pos is None else _f64(pos, (-1, 3)).copy()
    vel = None if vel is None else _f64(vel, (-1, 3)).copy()
    F = np.empty((nat, 3))
    E, S = Energy(), Stats()
    _check(ctx, load().ofdft_md_step(ctx, ctypes.byref(mp), int(nsteps), _ptr(pos), _ptr(vel),
                                     _ptr(F), ctypes.byref(E), ctypes.byref(S)))
    return dict(pos=pos, vel=vel, F=F, E=E.as_dict(), stats=S.as_dict())


FFMATH_OPS = {"add": 0, "mul": 1, "div": 2, "sqrt": 3, "exp": 4, "expm1_neg": 5, "log": 6, "rcbrt": 7}


def ofdft_ffmath_eval(op, x, y=None):
    """The double-float primitive `op` on the host (binary64 in and out)."""
    x = _f64(x, (-1,))
    y = None if y is None else _f64(y, (-1,))
    if FFMATH_OPS.get(op, op) in (0, 1, 2) and (y is None or y.size != x.size):
        raise ValueError("ofdft_ffmath_eval: binary operations need y with x's length")
    out = np.empty_like(x)
    st = load().ofdft_ffmath_eval(FFMATH_OPS.get(op, op), x.size, _ptr(x), _ptr(y), _ptr(out))
    if st != 0:
        raise OfdftError(st, "ofdft_ffmath_eval")
    return out


STRESS_TERMS = ("s", "xc", "H", "loc", "ion")


def ofdft_stress(ctx):
    """Stress tensor Sigma (3x3, hartree/bohr^3) and its five terms."""
    sig = np.empty(9)
    terms = np.empty(45)
    _check(ctx, load().ofdft_stress(ctx, _ptr(sig), _ptr(terms)))
    out = {k: terms[9 * i:9 * i + 9].reshape(3, 3) for i, k in enumerate(STRESS_TERMS)}
    out["Sigma"] = sig.reshape(3, 3)
    return out


def ofdft_md_andersen(ctx, T_kelvin, prob, u, xi):
    nat = ofdft_sizes(ctx)[1]
    u = _f64(u, (nat,))
    xi = _f64(xi, (nat, 3))
    n = ctypes.c_int()
    _check(ctx, load().ofdft_md_andersen(ctx, float(T_kelvin), float(prob), _ptr(u), _ptr(xi),
                                         ctypes.byref(n)))
    return n.value


def ofdft_md_state(ctx):
    nat = ofdft_sizes(ctx)[1]
    pos = np.empty((nat, 3))
    vel = np.empty((nat, 3))
    _check(ctx, load().ofdft_md_state(ctx, _ptr(pos), _ptr(vel)))
    return pos, vel


def ofdft_md_conserved(ctx):
    H = np.zeros(1)
    _check(ctx, load().ofdft_md_conserved(ctx, _ptr(H)))
    return float(H[0])


def ofdft_sizes(ctx):
    N = ctypes.c_longlong()
    nat = ctypes.c_int()
    _check(ctx, load().ofdft_sizes(ctx, ctypes.byref(N), ctypes.byref(nat)))
    return N.value, nat.value


TIMERS = {"pw": 1, "dline": 2, "ypass": 4, "zfwd": 5, "zfinal": 6, "xhl": 7}


def ofdft_timer_select(ctx, which):
    """which: a TIMERS name or id, optionally suffixed ":f32" or ":f64" to
    time only that precision's launches; 0 or None switches timing off."""
    if not which:
        _check(ctx, load().ofdft_timer_select(ctx, 0))
        return
    name, _, prec = str(which).partition(":") if isinstance(which, str) else (which, "", "")
    tid = TIMERS.get(name, name)
    tid = int(tid) + {"": 0, "f32": 8, "f64": 16}[prec]
    _check(ctx, load().ofdft_timer_select(ctx, tid))


def ofdft_timer_read(ctx, reset=True):
    ms = np.zeros(1)
    n = ctypes.c_longlong()
    _check(ctx, load().ofdft_timer_read(ctx, _ptr(ms), ctypes.byref(n), int(reset)))
    return float(ms[0]), n.value


def ofdft_kernel_launches(ctx):
    return int(load().ofdft_kernel_launches(ctx))


def ofdft_last_error(ctx=None):
    m = load().ofdft_last_error(ctx)
    return m.decode() if m else ""


def ofdft_tfunc_eval(t):
    t = _f64(t).reshape(-1)
    out = np.empty((t.size, 8))
    st = load().ofdft_tfunc_eval(t.size, _ptr(t), _ptr(out))
    if st != 0:
        raise OfdftError(st, "bad t")
    return out


def ofdft_pointwise_eval(functional, xc, T_kelvin, n, g2, arith="f32x2"):
    """Host evaluation of the kernels' pointwise functional: returns
    (out[count, 6] = f_s, T s_s, df/dn, W, eps_xc, v_xc; points handled in
    double-float)."""
    n = _f64(n).reshape(-1)
    g2 = _f64(g2).reshape(-1)
    if g2.size != n.size:
        raise ValueError("n and g2 differ in size")
    out = np.empty((n.size, 6))
    used = ctypes.c_longlong()
    st = load().ofdft_pointwise_eval(FUNCTIONALS.get(functional, functional), int(bool(xc)), float(T_kelvin),
                                     n.size, _ptr(n), _ptr(g2), POINTWISE.get(arith, arith), _ptr(out),
                                     ctypes.byref(used))
    if st != 0:
        raise OfdftError(st, "bad argument")
    return out, used.value


def ofdft_destroy(ctx):
    if ctx:
        load().ofdft_destroy(ctx)


# ------------------------------------------------------------ convenience
class Context:
    """One OF-DFT system on one GPU (owns a libofdft context).  precision:
    "fp64" or "mixed"; pointwise: arithmetic of the FP64 field sets, "f32x2"
    (double-float on the FP32 units, the default) or "f64" (binary64);
    lpp: "gauss" (Gaussian ion of radius rc) or "ha" (Heine-Abarenkov,
    Eq. (E4A), core radius rc, depth lpp_A, cutoff lpp_qc; one species);
    cell: lattice vectors as rows (3x3) for a general cell, else diag(L)."""

    def __init__(self, L, grid, ions, Z, T_kelvin, functional="fttf", xc=True, rc=0.25,
                 precision="fp64", device=0, stream=None, pointwise="f32x2", lpp="gauss",
                 lpp_A=6.18, lpp_qc=29.97, cell=None):
        p = ofdft_default_params()
        p.xc = int(bool(xc))
        p.rc = float(rc)
        p.lpp = LPP.get(lpp, lpp)
        p.lpp_A = float(lpp_A)
        p.lpp_qc = float(lpp_qc)
        p.precision = PRECISIONS[precision]
        p.pointwise = POINTWISE[pointwise]
        p.device = int(device)
        p.stream = stream
        cm = np.diag(np.asarray(L, dtype=np.float64)) if cell is None else np.asarray(cell, dtype=np.float64)
        self.ctx = ofdft_setup(cm, grid, ions, Z, T_kelvin, functional, p)
        self.grid = tuple(int(x) for x in grid)

    def close(self):
        if self.ctx:
            ofdft_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_positions(self, ions):
        ofdft_set_positions(self.ctx, ions)

    def set_phi(self, phi=None):
        ofdft_set_phi(self.ctx, phi)

    def energy_potential(self, phi=None, want_v=True):
        E, v = ofdft_energy_potential(self.ctx, phi, want_v)
        return E, (None if v is None else v.reshape(self.grid))

    def minimize(self, gtol=1e-8, maxit=5000, raise_on_noconv=True):
        return ofdft_minimize(self.ctx, gtol, maxit, raise_on_noconv)

    def minimize_tn(self, gtol=1e-8, maxit=500, inner_max=20, eta=0.1, raise_on_noconv=True):
        return ofdft_minimize_tn(self.ctx, gtol, maxit, inner_max, eta, raise_on_noconv)

    def minimize_start(self, gtol=1e-8, maxit=5000):
        ofdft_minimize_start(self.ctx, gtol, maxit)

    def minimize_wait(self, raise_on_noconv=True):
        return ofdft_minimize_wait(self.ctx, raise_on_noconv)

    def autotune(self, reps=3):
        ofdft_autotune(self.ctx, reps)

    def forces(self):
        return ofdft_forces(self.ctx)

    def stress(self):
        return ofdft_stress(self.ctx)

    def density(self):
        return ofdft_get_density(self.ctx).reshape(self.grid)

    def md_step(self, dt_fs, T_kelvin, nsteps=1, pos=None, vel=None, **kw):
        return ofdft_md_step(self.ctx, dt_fs, T_kelvin, nsteps, pos, vel, **kw)

    def md_andersen(self, T_kelvin, prob, u, xi):
        return ofdft_md_andersen(self.ctx, T_kelvin, prob, u, xi)

    def md_state(self):
        return ofdft_md_state(self.ctx)

    def md_conserved(self):
        return ofdft_md_conserved(self.ctx)

    def kernel_launches(self):
        return ofdft_kernel_launches(self.ctx)


def ofdft_energy_potential_static(cell, grid, ions, Z, T_kelvin, functional, phi_dev, v_dev,
                                  xc=True, rc=0.25, stream=None):
    """Allocation-free evaluation for callers that cannot allocate device
    memory: phi_dev and v_dev are device addresses (ints) of N doubles the
    caller owns; the library's fixed scratch array does the rest.  Limits:
    edges <= 64, N <= 32768, nat <= 64 (larger raises OFDFT_EINVAL)."""
    lib = load()
    cell = _f64(cell).reshape(-1)
    if cell.size == 3:
        cell = np.diag(cell).reshape(-1)
    g = (ctypes.c_int * 3)(*[int(x) for x in grid])
    ions = _f64(ions, (-1, 3))
    Z = _f64(Z, (-1,))
    f = FUNCTIONALS[functional] if isinstance(functional, str) else int(functional)
    E = Energy()
    st = lib.ofdft_energy_potential_static(_ptr(cell), g, ions.shape[0], _ptr(ions), _ptr(Z),
                                           float(T_kelvin), f, int(bool(xc)), float(rc),
                                           ctypes.c_void_p(int(phi_dev)), ctypes.c_void_p(int(v_dev)),
                                           ctypes.byref(E), stream)
    if st != 0:
        raise OfdftError(st, "static path: edges even, {2,3,5}-smooth, <= 64; "
                             "nx*ny*nz <= 32768; 1 <= nat <= 64; valid cell, T, functional")
    return E.as_dict()


# ------------------------------------------------------------------ serving
class Server:
    """Request loop of the serving form (ofdft_serve_*): submit systems with
    a number of MD steps, poll or drain for results.  max_bypass: how many
    later requests may be admitted ahead of one that does not fit yet."""

    def __init__(self, max_slots=4, hbm_budget_bytes=0.0, device=0, dry_run_ms=None, max_bypass=8):
        p = ServeParams(int(device), int(max_slots), float(hbm_budget_bytes),
                        0 if dry_run_ms is None else 1, float(dry_run_ms or 0.0), int(max_bypass))
        h = ctypes.c_void_p()
        st = load().ofdft_serve_start(ctypes.byref(p), ctypes.byref(h))
        if st != 0:
            raise OfdftError(st, "ofdft_serve_start failed")
        self.h = h.value

    def submit(self, L, grid, ions, Z, T_kelvin, functional="vt84f", precision="mixed",
               md_steps=0, dt_fs=0.2, vel=None, gtol=1e-8, maxit=5000, xc=True, rc=0.25):
        ions = _f64(ions, (-1, 3))
        Z = _f64(Z, (-1,))
        vel = None if vel is None else _f64(vel, (-1, 3))
        r = Request()
        cell = np.diag(np.asarray(L, dtype=np.float64)).reshape(-1) if np.size(L) == 3 else _f64(L).reshape(-1)
        for i in range(9):
            r.cell[i] = float(cell[i])
        for i in range(3):
            r.grid[i] = int(grid[i])
        r.nat = len(Z)
        r.ions, r.Z, r.vel = _ptr(ions), _ptr(Z), _ptr(vel)
        r.T_kelvin = float(T_kelvin)
        r.functional = FUNCTIONALS[functional] if isinstance(functional, str) else int(functional)
        r.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        r.xc, r.rc = int(bool(xc)), float(rc)
        r.md_steps, r.dt_fs, r.gtol, r.maxit = int(md_steps), float(dt_fs), float(gtol), int(maxit)
        rid = ctypes.c_longlong()
        st = load().ofdft_serve_submit(self.h, ctypes.byref(r), ctypes.byref(rid))
        if st != 0:
            raise OfdftError(st, "ofdft_serve_submit failed")
        return rid.value

    def poll(self, rid):
        res = Result()
        st = load().ofdft_serve_poll(self.h, int(rid), ctypes.byref(res))
        if st == -7:
            return None
        if st != 0:
            raise OfdftError(st, "ofdft_serve_poll failed")
        return res.as_dict()

    def cancel(self, rid):
        """Cancel request rid (queued: removed; running: stops before its
        next MD step); its result then carries status OFDFT_ECANCELED."""
        st = load().ofdft_serve_cancel(self.h, int(rid))
        if st != 0:
            raise OfdftError(st, "ofdft_serve_cancel")

    def drain(self, timeout_s=0.0):
        st = load().ofdft_serve_drain(self.h, float(timeout_s))
        if st != 0:
            raise OfdftError(st, "ofdft_serve_drain")

    def clock(self):
        return load().ofdft_serve_clock(self.h)

    def peaks(self):
        b = np.zeros(1)
        n = ctypes.c_int()
        load().ofdft_serve_peaks(self.h, _ptr(b), ctypes.byref(n))
        return float(b[0]), n.value

    def stop(self):
        if self.h:
            load().ofdft_serve_stop(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.stop()
