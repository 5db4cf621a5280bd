"""Thin Python binding of the COLA C ABI (include/cola.h).

Argument marshalling only: every step of the computation runs in the CUDA library
libcola_gb300.so.  PyTorch supplies device memory (the workspace and the particle / mesh
tensors) and the current CUDA stream.  The functions named ``cola_*`` mirror the C entry
points one to one; ``Plan`` bundles a plan handle with its workspace.

If the library has not been built, importing works but the first call raises ImportError
(there is no fallback implementation).
"""
import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcola_gb300.so")

COLA_OK = 0
COLA_NCOEF = 16
ERRORS = {1: "COLA_EINVAL", 2: "COLA_ECUDA", 3: "COLA_EOVERFLOW", 4: "COLA_EUNSUPPORTED", 5: "COLA_ENOWORKSPACE",
          6: "COLA_ETIMEOUT"}


class ColaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class cola_cosmo(ctypes.Structure):
    _fields_ = [("omega_m", ctypes.c_double), ("omega_l", ctypes.c_double), ("h", ctypes.c_double),
                ("sigma8", ctypes.c_double), ("n_s", ctypes.c_double)]


class cola_config(ctypes.Structure):
    _fields_ = [("np", ctypes.c_int64), ("ng", ctypes.c_int64), ("box", ctypes.c_double),
                ("cosmo", cola_cosmo), ("n_lpt", ctypes.c_double), ("nsteps", ctypes.c_int32),
                ("a_init", ctypes.c_double), ("a_final", ctypes.c_double), ("deconv", ctypes.c_int32),
                ("fixed_bits", ctypes.c_int32), ("adjoint", ctypes.c_int32), ("scheme", ctypes.c_int32),
                ("log_a", ctypes.c_int32)]


# cola_config.scheme values (include/cola.h) and the oracle's names for them
SCHEMES = {"cola": 0, "cola_std": 1, "pm_std": 2, "cola_u1": 3}


class cola_ensemble_tuning(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("tile_shape", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("radix", ctypes.c_int32), ("launch", ctypes.c_int32), ("mesh_streams", ctypes.c_int32)]


_P = ctypes.c_void_p
_SIGNATURES = {
    "cola_config_default": [ctypes.POINTER(cola_config)],
    "cola_plan_create": [ctypes.POINTER(cola_config), ctypes.POINTER(_P)],
    "cola_plan_destroy": [_P],
    "cola_workspace_bytes": [_P, ctypes.POINTER(ctypes.c_size_t)],
    "cola_set_workspace": [_P, _P, ctypes.c_size_t, _P],
    "cola_coeffs": [_P, _P],
    "cola_noise": [_P, ctypes.c_uint64, _P, _P],
    "cola_ic_2lpt": [_P, _P, _P, _P, _P, _P, _P],
    "cola_step": [_P, ctypes.c_int32, _P, _P, _P, _P, _P],
    "cola_force": [_P, _P, _P, _P],
    "cola_density": [_P, _P, _P, _P, _P],
    "cola_power": [_P, _P, ctypes.c_int32, _P, _P, _P, _P],
    "cola_density_power": [_P, _P, ctypes.c_int32, _P, _P, _P, _P],
    "cola_fft_r2c": [_P, ctypes.c_int32, _P, _P, _P],
    "cola_cross_power": [_P, _P, _P, ctypes.c_int32, _P, _P, _P, _P, _P, _P, _P, _P],
    "cola_fof": [_P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P, _P, ctypes.c_int32, _P, _P, _P],
    "cola_set_fof_union_tries": [_P, ctypes.c_int32],
    "cola_status": [_P, _P],
    "cola_power_noalloc": [_P, ctypes.c_int32, ctypes.c_double, ctypes.c_int32, _P, _P, _P, _P],
    "cola_step_adjoint": [_P, ctypes.c_int32, _P, _P, _P, _P, _P, _P],
    "cola_density_adjoint": [_P, _P, _P, _P, _P],
    "cola_ic_2lpt_adjoint": [_P, _P, _P, _P, _P, _P, _P],
    "cola_profile": [_P, ctypes.c_int32],
    "cola_profile_read": [_P, ctypes.c_int32, _P, _P, _P, _P],
    "cola_launch_count": [_P],
    "cola_last_error": [],
    "cola_ensemble_create": [_P, ctypes.c_int32, ctypes.POINTER(_P)],
    "cola_ensemble_destroy": [_P],
    "cola_ensemble_workspace_bytes": [_P, ctypes.POINTER(ctypes.c_size_t)],
    "cola_ensemble_set_workspace": [_P, _P, ctypes.c_size_t, _P],
    "cola_ensemble_offsets": [_P, _P, _P],
    "cola_ensemble_noise": [_P, _P, _P, _P],
    "cola_ensemble_ic_2lpt": [_P, _P, _P, _P, _P, _P, _P],
    "cola_ensemble_step": [_P, ctypes.c_int32, _P, _P, _P, _P, _P],
    "cola_ensemble_density": [_P, _P, _P, _P],
    "cola_ensemble_power": [_P, _P, ctypes.c_int32, _P, _P, _P, _P],
    "cola_ensemble_tune": [_P, _P, ctypes.c_int32, _P, _P, _P],
    "cola_ensemble_get_tuning": [_P, _P],
    "cola_ensemble_set_tuning": [_P, _P, _P],
    "cola_ensemble_use_graphs": [_P, ctypes.c_int32],
    "cola_ensemble_status": [_P, _P],
    "cola_ensemble_profile": [_P, ctypes.c_int32],
    "cola_ensemble_profile_read": [_P, ctypes.c_int32, _P, _P, _P, _P],
}
COLA_ENSEMBLE_TUNE_CANDIDATES = 25
_lib = None


def load_library():
    """Load libcola_gb300.so (raises ImportError if it is missing: no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is not built; run `python -m paper_1301_0322_gb300.build`")
        lib = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_char_p if name == "cola_last_error" else ctypes.c_int
        _lib = lib
    return _lib


def _check(code):
    if code != COLA_OK:
        raise ColaError(code, load_library().cola_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if not t.is_contiguous():
            raise ValueError("tensors passed to the COLA library must be contiguous")
        return ctypes.c_void_p(t.data_ptr())
    return ctypes.c_void_p(t)


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _expect(t, dtype, numel, name):
    if not isinstance(t, torch.Tensor) or t.dtype != dtype or t.numel() != numel or not t.is_cuda:
        raise ValueError(f"{name}: expected a CUDA {dtype} tensor with {numel} elements")


# ---- one-to-one wrappers of the C entry points ---------------------------------------------
def cola_config_default():
    cfg = cola_config()
    _check(load_library().cola_config_default(ctypes.byref(cfg)))
    return cfg


def cola_plan_create(cfg):
    h = ctypes.c_void_p()
    _check(load_library().cola_plan_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def cola_plan_destroy(h):
    _check(load_library().cola_plan_destroy(h))


def cola_workspace_bytes(h):
    n = ctypes.c_size_t()
    _check(load_library().cola_workspace_bytes(h, ctypes.byref(n)))
    return n.value


def cola_set_workspace(h, ws, stream=None):
    _check(load_library().cola_set_workspace(h, _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)))


def cola_coeffs(h, nsteps):
    out = np.zeros((nsteps + 1, COLA_NCOEF), dtype=np.float64)
    _check(load_library().cola_coeffs(h, out.ctypes.data_as(ctypes.c_void_p)))
    return out


def cola_noise(h, seed, noise, stream=None):
    _check(load_library().cola_noise(h, ctypes.c_uint64(seed), _ptr(noise), _stream(stream)))


def cola_ic_2lpt(h, noise, s, v, s1, s2, stream=None):
    _check(load_library().cola_ic_2lpt(h, _ptr(noise), _ptr(s), _ptr(v), _ptr(s1), _ptr(s2), _stream(stream)))


def cola_step(h, step, s, v, s1, s2, stream=None):
    _check(load_library().cola_step(h, int(step), _ptr(s), _ptr(v), _ptr(s1), _ptr(s2), _stream(stream)))


def cola_force(h, s, g, stream=None):
    _check(load_library().cola_force(h, _ptr(s), _ptr(g), _stream(stream)))


def cola_density(h, s, rho_fix, delta, stream=None):
    _check(load_library().cola_density(h, _ptr(s), _ptr(rho_fix), _ptr(delta), _stream(stream)))


def cola_power(h, delta, nbins, k, pk, nmodes, stream=None):
    _check(load_library().cola_power(h, _ptr(delta), int(nbins), _ptr(k), _ptr(pk), _ptr(nmodes), _stream(stream)))


def cola_density_power(h, s, nbins, k, pk, nmodes, stream=None):
    _check(load_library().cola_density_power(h, _ptr(s), int(nbins), _ptr(k), _ptr(pk), _ptr(nmodes),
                                             _stream(stream)))


def cola_power_noalloc(delta, ng, box, nbins, k, pk, nmodes, stream=None):
    """P(k) of a density mesh (ng <= 128) with no plan, workspace or device allocation."""
    _check(load_library().cola_power_noalloc(_ptr(delta), int(ng), float(box), int(nbins), _ptr(k), _ptr(pk),
                                             _ptr(nmodes), _stream(stream)))


def cola_cross_power(h, delta_a, delta_b, nbins, k, pk_a, pk_b, pk_ab, rho, nmax, nmodes, stream=None):
    _check(load_library().cola_cross_power(h, _ptr(delta_a), _ptr(delta_b), int(nbins), _ptr(k), _ptr(pk_a),
                                           _ptr(pk_b), _ptr(pk_ab), _ptr(rho), _ptr(nmax), _ptr(nmodes),
                                           _stream(stream)))


def cola_fof(h, s, b_num, b_den, nmin, group, size, thresholds, n_ge, stream=None):
    thr = np.ascontiguousarray(thresholds if thresholds is not None else [], dtype=np.int32)
    _check(load_library().cola_fof(h, _ptr(s), int(b_num), int(b_den), int(nmin), _ptr(group), _ptr(size),
                                   int(thr.size), thr.ctypes.data_as(ctypes.c_void_p) if thr.size else None,
                                   _ptr(n_ge), _stream(stream)))


def cola_set_fof_union_tries(h, tries):
    _check(load_library().cola_set_fof_union_tries(h, int(tries)))


def cola_fft_r2c(h, which, x, out, stream=None):
    _check(load_library().cola_fft_r2c(h, int(which), _ptr(x), _ptr(out), _stream(stream)))


def cola_step_adjoint(h, step, s_ckpt, lam_s, lam_v, lam_s1, lam_s2, stream=None):
    _check(load_library().cola_step_adjoint(h, int(step), _ptr(s_ckpt), _ptr(lam_s), _ptr(lam_v), _ptr(lam_s1),
                                            _ptr(lam_s2), _stream(stream)))


def cola_density_adjoint(h, s, delta_bar, lam_s, stream=None):
    _check(load_library().cola_density_adjoint(h, _ptr(s), _ptr(delta_bar), _ptr(lam_s), _stream(stream)))


def cola_ic_2lpt_adjoint(h, noise, lam_s, lam_s1, lam_s2, grad_noise, stream=None):
    _check(load_library().cola_ic_2lpt_adjoint(h, _ptr(noise), _ptr(lam_s), _ptr(lam_s1), _ptr(lam_s2),
                                               _ptr(grad_noise), _stream(stream)))


def cola_status(h, stream=None):
    _check(load_library().cola_status(h, _stream(stream)))


def cola_ensemble_create(cfgs):
    arr = (cola_config * len(cfgs))(*cfgs)
    h = ctypes.c_void_p()
    _check(load_library().cola_ensemble_create(arr, len(cfgs), ctypes.byref(h)))
    return h


def cola_ensemble_destroy(h):
    _check(load_library().cola_ensemble_destroy(h))


def cola_ensemble_workspace_bytes(h):
    n = ctypes.c_size_t()
    _check(load_library().cola_ensemble_workspace_bytes(h, ctypes.byref(n)))
    return n.value


def cola_ensemble_set_workspace(h, ws, stream=None):
    _check(load_library().cola_ensemble_set_workspace(h, _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)))


def cola_ensemble_offsets(h, nbox):
    poff = np.zeros(nbox + 1, dtype=np.int64)
    moff = np.zeros(nbox + 1, dtype=np.int64)
    _check(load_library().cola_ensemble_offsets(h, poff.ctypes.data_as(ctypes.c_void_p),
                                                moff.ctypes.data_as(ctypes.c_void_p)))
    return poff, moff


def cola_ensemble_noise(h, seeds, noise, stream=None):
    sd = np.ascontiguousarray(seeds, dtype=np.uint64)
    _check(load_library().cola_ensemble_noise(h, sd.ctypes.data_as(ctypes.c_void_p), _ptr(noise), _stream(stream)))


def cola_ensemble_ic_2lpt(h, noise, s, v, s1, s2, stream=None):
    _check(load_library().cola_ensemble_ic_2lpt(h, _ptr(noise), _ptr(s), _ptr(v), _ptr(s1), _ptr(s2),
                                                _stream(stream)))


def cola_ensemble_step(h, step, s, v, s1, s2, stream=None):
    _check(load_library().cola_ensemble_step(h, int(step), _ptr(s), _ptr(v), _ptr(s1), _ptr(s2), _stream(stream)))


def cola_ensemble_density(h, s, delta, stream=None):
    _check(load_library().cola_ensemble_density(h, _ptr(s), _ptr(delta), _stream(stream)))


def cola_ensemble_power(h, delta, nbins, k, pk, nmodes, stream=None):
    _check(load_library().cola_ensemble_power(h, _ptr(delta), int(nbins), _ptr(k), _ptr(pk), _ptr(nmodes),
                                              _stream(stream)))


def cola_ensemble_tune(h, s, reps=3, stream=None):
    best = cola_ensemble_tuning()
    ms = np.zeros(COLA_ENSEMBLE_TUNE_CANDIDATES, dtype=np.float64)
    _check(load_library().cola_ensemble_tune(h, _ptr(s), int(reps), ctypes.byref(best),
                                             ms.ctypes.data_as(ctypes.c_void_p), _stream(stream)))
    return best, ms


def cola_ensemble_get_tuning(h):
    t = cola_ensemble_tuning()
    _check(load_library().cola_ensemble_get_tuning(h, ctypes.byref(t)))
    return t


def cola_ensemble_set_tuning(h, tuning, stream=None):
    _check(load_library().cola_ensemble_set_tuning(h, ctypes.byref(tuning), _stream(stream)))


def cola_ensemble_use_graphs(h, enable):
    _check(load_library().cola_ensemble_use_graphs(h, int(bool(enable))))


def cola_ensemble_status(h, stream=None):
    _check(load_library().cola_ensemble_status(h, _stream(stream)))


# ---- convenience wrapper ----------------------------------------------------------------------
class Plan:
    """A COLA plan plus its device workspace (allocated with torch on ``device``)."""

    def __init__(self, np_side=32, ng=64, box=100.0, omega_m=0.27, omega_l=0.73, h=0.7, sigma8=0.8, n_s=0.96,
                 n_lpt=-2.5, nsteps=10, a_init=0.1, a_final=1.0, deconv=1, fixed_bits=16, adjoint=False,
                 scheme="cola", log_a=False, device="cuda"):
        cfg = _make_config(np_side, ng, box, omega_m, omega_l, h, sigma8, n_s, n_lpt, nsteps, a_init, a_final, deconv,
                           fixed_bits, adjoint, scheme, log_a)
        self.cfg = cfg
        self.np, self.ng, self.nsteps = int(np_side), int(ng), int(nsteps)
        self.n3 = self.np**3
        self.device = torch.device(device)
        self.handle = cola_plan_create(cfg)
        nbytes = cola_workspace_bytes(self.handle)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        off = (-self.workspace.data_ptr()) % 256
        self._ws_view = self.workspace[off:off + nbytes]
        cola_set_workspace(self.handle, self._ws_view)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.cola_plan_destroy(h)
            self.handle = None

    def _empty(self, shape, dtype=torch.float32):
        return torch.empty(shape, dtype=dtype, device=self.device)

    def coeffs(self):
        return cola_coeffs(self.handle, self.nsteps)

    def noise(self, seed, out=None):
        out = self._empty(self.n3) if out is None else out
        _expect(out, torch.float32, self.n3, "noise")
        cola_noise(self.handle, seed, out)
        return out

    def ic_2lpt(self, noise):
        _expect(noise, torch.float32, self.n3, "noise")
        s, v, s1, s2 = (self._empty((3, self.n3)) for _ in range(4))
        cola_ic_2lpt(self.handle, noise, s, v, s1, s2)
        return s, v, s1, s2

    def step(self, i, s, v, s1, s2):
        for t, n in ((s, "s"), (v, "v"), (s1, "s1"), (s2, "s2")):
            _expect(t, torch.float32, 3 * self.n3, n)
        cola_step(self.handle, i, s, v, s1, s2)

    def run(self, noise):
        """2LPT initial conditions, then the nsteps+1 force evaluations of eq. ALCtimestep."""
        s, v, s1, s2 = self.ic_2lpt(noise)
        for i in range(self.nsteps + 1):
            self.step(i, s, v, s1, s2)
        return s, v, s1, s2

    def force(self, s):
        _expect(s, torch.float32, 3 * self.n3, "s")
        g = self._empty((3, self.n3))
        cola_force(self.handle, s, g)
        return g

    def density(self, s, rho=True, delta=True):
        _expect(s, torch.float32, 3 * self.n3, "s")
        ng3 = self.ng**3
        r = self._empty(ng3, torch.int64) if rho else None
        d = self._empty(ng3) if delta else None
        cola_density(self.handle, s, r, d)
        return r, d

    def power(self, delta, nbins):
        _expect(delta, torch.float32, self.ng**3, "delta")
        k = self._empty(nbins, torch.float64)
        pk = self._empty(nbins, torch.float64)
        nm = self._empty(nbins, torch.int64)
        cola_power(self.handle, delta, nbins, k, pk, nm)
        return k, pk, nm

    def density_power(self, s, nbins):
        """(k, P, nmodes) of the CIC density at displacements s, with no density mesh of the
        caller's (the plan's force meshes serve as scratch); equal to power(density(s)[1])."""
        _expect(s, torch.float32, 3 * self.n3, "s")
        k = self._empty(nbins, torch.float64)
        pk = self._empty(nbins, torch.float64)
        nm = self._empty(nbins, torch.int64)
        cola_density_power(self.handle, s, nbins, k, pk, nm)
        return k, pk, nm

    def cross_power(self, delta_a, delta_b, nbins):
        """(k, P_a, P_b, P_ab, rho, n_max, nmodes) per shell (Sec. 3.1, eq. nmax)."""
        _expect(delta_a, torch.float32, self.ng**3, "delta_a")
        _expect(delta_b, torch.float32, self.ng**3, "delta_b")
        out = [self._empty(nbins, torch.float64) for _ in range(6)] + [self._empty(nbins, torch.int64)]
        cola_cross_power(self.handle, delta_a, delta_b, nbins, *out)
        return tuple(out)

    def fof(self, s, nmin=25, b=(1, 5), thresholds=None):
        """Friends-of-friends groups (Sec. 3.2): (group label per particle, group size per
        particle, number of halos with at least thresholds[k] particles)."""
        _expect(s, torch.float32, 3 * self.n3, "s")
        group = self._empty(self.n3, torch.int32)
        size = self._empty(self.n3, torch.int32)
        thr = [] if thresholds is None else list(thresholds)
        n_ge = self._empty(max(1, len(thr)), torch.int64)
        cola_fof(self.handle, s, b[0], b[1], nmin, group, size, thr, n_ge if thr else None)
        return group, size, n_ge[:len(thr)]

    def fft_r2c(self, x, which=0):
        n = self.ng if which == 0 else self.np
        _expect(x, torch.float32, n**3, "x")
        out = self._empty((n, n, n // 2 + 1), torch.complex64)
        cola_fft_r2c(self.handle, which, x, out)
        return out

    def status(self):
        cola_status(self.handle)

    # ---- reverse mode ----
    def step_adjoint(self, i, s_ckpt, lam_s, lam_v, lam_s1, lam_s2):
        cola_step_adjoint(self.handle, i, s_ckpt, lam_s, lam_v, lam_s1, lam_s2)

    def density_adjoint(self, s, delta_bar):
        _expect(delta_bar, torch.float32, self.ng**3, "delta_bar")
        lam_s = self._empty((3, self.n3))
        cola_density_adjoint(self.handle, s, delta_bar, lam_s)
        return lam_s

    def ic_adjoint(self, noise, lam_s, lam_s1, lam_s2):
        grad = self._empty(self.n3)
        cola_ic_2lpt_adjoint(self.handle, noise, lam_s, lam_s1, lam_s2, grad)
        return grad


def _make_config(np_side, ng, box, omega_m=0.27, omega_l=0.73, h=0.7, sigma8=0.8, n_s=0.96, n_lpt=-2.5, nsteps=10,
                 a_init=0.1, a_final=1.0, deconv=1, fixed_bits=16, adjoint=False, scheme="cola", log_a=False):
    cfg = cola_config_default()
    cfg.np, cfg.ng, cfg.box = int(np_side), int(ng), float(box)
    cfg.cosmo = cola_cosmo(omega_m, omega_l, h, sigma8, n_s)
    cfg.n_lpt, cfg.nsteps, cfg.a_init, cfg.a_final = float(n_lpt), int(nsteps), float(a_init), float(a_final)
    cfg.deconv, cfg.fixed_bits, cfg.adjoint = int(deconv), int(fixed_bits), int(bool(adjoint))
    cfg.scheme = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
    cfg.log_a = int(bool(log_a))
    return cfg


class Ensemble:
    """Independent COLA boxes of different sizes evolved together, each step replayed from a
    CUDA graph: either one multi-box launch per kernel class and force evaluation, or every
    box's own single-box launches dealt over 1, 2 or 4 forked streams (``tuning``; ``tune``
    times all candidates and keeps the fastest).

    ``boxes``: sequence of (np_side, ng, box) tuples or dicts of Plan keyword arguments.
    Particle arrays are concatenated over boxes: a [3, n_total] tensor holds box b's SoA block
    in its flat elements [3 poff[b], 3 poff[b+1]); ``split`` returns the per-box [3, np^3] views."""

    def __init__(self, boxes, device="cuda", **common):
        cfgs = []
        for b in boxes:
            kw = dict(common)
            if isinstance(b, dict):
                kw.update(b)
            else:
                kw.update(np_side=b[0], ng=b[1], box=b[2])
            cfgs.append(_make_config(**kw))
        self.cfgs = cfgs
        self.nbox = len(cfgs)
        self.nps = [int(c.np) for c in cfgs]
        self.ngs = [int(c.ng) for c in cfgs]
        self.nsteps = int(cfgs[0].nsteps)
        self.device = torch.device(device)
        self.handle = cola_ensemble_create(cfgs)
        nbytes = cola_ensemble_workspace_bytes(self.handle)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        off = (-self.workspace.data_ptr()) % 256
        self._ws_view = self.workspace[off:off + nbytes]
        cola_ensemble_set_workspace(self.handle, self._ws_view)
        self.poff, self.moff = cola_ensemble_offsets(self.handle, self.nbox)
        self.n_total = int(self.poff[-1])
        self.cells_total = int(self.moff[-1])

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.cola_ensemble_destroy(h)
            self.handle = None

    def _empty(self, shape, dtype=torch.float32):
        return torch.empty(shape, dtype=dtype, device=self.device)

    def split(self, x):
        """Per-box [3, np^3] views of a concatenated particle array."""
        flat = x.reshape(-1)
        return [flat[3 * self.poff[b]:3 * self.poff[b + 1]].view(3, -1) for b in range(self.nbox)]

    def split_mesh(self, m):
        return [m[self.moff[b]:self.moff[b + 1]] for b in range(self.nbox)]

    def noise(self, seeds):
        out = self._empty(self.n_total)
        cola_ensemble_noise(self.handle, seeds, out)
        return out

    def ic_2lpt(self, noise):
        _expect(noise, torch.float32, self.n_total, "noise")
        s, v, s1, s2 = (self._empty(3 * self.n_total) for _ in range(4))
        cola_ensemble_ic_2lpt(self.handle, noise, s, v, s1, s2)
        return s, v, s1, s2

    def step(self, i, s, v, s1, s2):
        for t, n in ((s, "s"), (v, "v"), (s1, "s1"), (s2, "s2")):
            _expect(t, torch.float32, 3 * self.n_total, n)
        cola_ensemble_step(self.handle, i, s, v, s1, s2)

    def run(self, noise):
        s, v, s1, s2 = self.ic_2lpt(noise)
        for i in range(self.nsteps + 1):
            self.step(i, s, v, s1, s2)
        return s, v, s1, s2

    def density(self, s):
        _expect(s, torch.float32, 3 * self.n_total, "s")
        d = self._empty(self.cells_total)
        cola_ensemble_density(self.handle, s, d)
        return d

    def power(self, delta, nbins):
        _expect(delta, torch.float32, self.cells_total, "delta")
        k = self._empty((self.nbox, nbins), torch.float64)
        pk = self._empty((self.nbox, nbins), torch.float64)
        nm = self._empty((self.nbox, nbins), torch.int64)
        cola_ensemble_power(self.handle, delta, nbins, k, pk, nm)
        return k, pk, nm

    def tune(self, s, reps=3):
        """Times the COLA_ENSEMBLE_TUNE_CANDIDATES launch shapes at displacements s (read only),
        keeps the fastest; returns (best tuning struct, per-candidate milliseconds)."""
        _expect(s, torch.float32, 3 * self.n_total, "s")
        return cola_ensemble_tune(self.handle, s, reps)

    @property
    def tuning(self):
        """(threads, tile_shape, blocks_per_sm, radix, launch, mesh_streams); a shorter tuple given
        to the setter is padded with zeros (launch 0 = the multi-box kernels, mesh_streams 0 = the
        mesh passes multi-box too)."""
        t = cola_ensemble_get_tuning(self.handle)
        return (t.threads, t.tile_shape, t.blocks_per_sm, t.radix, t.launch, t.mesh_streams)

    @tuning.setter
    def tuning(self, value):
        value = tuple(value) + (0,) * (6 - len(value))
        cola_ensemble_set_tuning(self.handle, cola_ensemble_tuning(*value))

    def use_graphs(self, enable):
        cola_ensemble_use_graphs(self.handle, enable)

    def status(self):
        cola_ensemble_status(self.handle)


class ColaDensity(torch.autograd.Function):
    """delta_final(noise): 2LPT initial conditions, all force evaluations and the final CIC
    density, differentiable with respect to the white noise.  The forward pass keeps the
    displacement of every force evaluation (nsteps+1 checkpoints); the backward pass runs the
    library's adjoint calls in reverse order.  The plan must have been built with adjoint=True."""

    @staticmethod
    def forward(ctx, noise, plan):
        s, v, s1, s2 = plan.ic_2lpt(noise)
        ckpts = torch.empty((plan.nsteps + 1, 3, plan.n3), dtype=torch.float32, device=noise.device)
        for i in range(plan.nsteps + 1):
            ckpts[i].copy_(s)
            plan.step(i, s, v, s1, s2)
        _, delta = plan.density(s, rho=False, delta=True)
        ctx.plan = plan
        ctx.save_for_backward(noise, s, ckpts)
        return delta

    @staticmethod
    def backward(ctx, delta_bar):
        noise, s, ckpts = ctx.saved_tensors
        plan = ctx.plan
        lam_s = plan.density_adjoint(s, delta_bar.contiguous().float())
        lam_v = torch.zeros_like(lam_s)
        lam_s1 = torch.zeros_like(lam_s)
        lam_s2 = torch.zeros_like(lam_s)
        for i in reversed(range(plan.nsteps + 1)):
            plan.step_adjoint(i, ckpts[i], lam_s, lam_v, lam_s1, lam_s2)
        return plan.ic_adjoint(noise, lam_s, lam_s1, lam_s2), None


def cola_density_from_noise(noise, plan):
    """Differentiable final CIC overdensity of a COLA run started from ``noise`` (see ColaDensity)."""
    return ColaDensity.apply(noise, plan)
