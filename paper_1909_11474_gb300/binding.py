"""Thin Python binding of the C ABI in include/tersoff.h (argument marshalling only).

Every method of `Context` wraps the C function of the same name with the `tersoff_` prefix dropped;
all arithmetic runs in the CUDA library. PyTorch provides device memory and streams. There is no CPU
fallback: a missing or unloadable library raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# TSF_DEBUG_BOUNDS=1 selects the bounds-checked debug build of the library
LIB_PATH = os.path.join(_HERE, "libtersoff_gb300_debug.so" if os.environ.get("TSF_DEBUG_BOUNDS") == "1"
                        else "libtersoff_gb300.so")

OK, E_ARG, E_NBR_OVERFLOW, E_CUDA, E_NONFINITE, E_TIMEOUT, E_STATE, E_UNSUPPORTED = range(8)
STATUS_NBR_OVERFLOW, STATUS_MANY_NBRS, STATUS_NONFINITE, STATUS_TIMEOUT = 1, 2, 4, 8
LOSS_SQ, LOSS_Z = 0, 1

LAUNCH_GRAPHS = 1
LAUNCH_PDL = 2
FORM_MINIMAL, FORM_TERSOFF = 0, 1

EXPORTED = (
    "tersoff_create", "tersoff_destroy", "tersoff_last_error", "tersoff_get_status",
    "tersoff_build_neighbors", "tersoff_export_neighbors", "tersoff_build_info", "tersoff_eval",
    "tersoff_fitness", "tersoff_param_grad", "tersoff_eval_plain", "tersoff_md_force",
    "tersoff_md_export_neighbors", "tersoff_fitness_static", "tersoff_kernel_launches",
    "tersoff_profile", "tersoff_profile_read", "tersoff_set_launch_mode", "tersoff_autotune",
    "tersoff_set_schedule", "tersoff_schedule_info", "tersoff_ga_step", "tersoff_md_nve", "tersoff_set_form",
    "tersoff_set_wait_limit", "tersoff_measure_peaks",
)

_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_f64 = ctypes.c_double


class _Configs(ctypes.Structure):
    _fields_ = [("C", _i32), ("atom_off", _vp), ("pos", _vp), ("box", _vp)]


class _Targets(ctypes.Structure):
    _fields_ = [("E", _vp), ("W", _vp), ("F", _vp), ("mask", _vp)]


_lib = None


def load():
    """Open the shared library (built in-tree by paper_1909_11474_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_1909_11474_gb300.build`")
    lib = ctypes.CDLL(LIB_PATH)
    sig = {
        "tersoff_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int]),
        "tersoff_destroy": (None, [_vp]),
        "tersoff_last_error": (ctypes.c_char_p, [_vp]),
        "tersoff_get_status": (ctypes.c_int, [_vp, _vp]),
        "tersoff_build_neighbors": (ctypes.c_int, [_vp, ctypes.POINTER(_Configs), _f64, _f64, _i32, _vp]),
        "tersoff_export_neighbors": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
        "tersoff_build_info": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int64),
                                              ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(_i32)]),
        "tersoff_eval": (ctypes.c_int, [_vp, _vp, _i32, _i32, _vp, _vp, _vp, _vp]),
        "tersoff_fitness": (ctypes.c_int, [_vp, _vp, _i32, ctypes.POINTER(_Targets), _vp, _i32,
                                           _vp, _vp, _vp, _vp]),
        "tersoff_param_grad": (ctypes.c_int, [_vp, _vp, _i32, ctypes.POINTER(_Targets), _vp, _i32,
                                              _vp, _vp, _vp]),
        "tersoff_eval_plain": (ctypes.c_int, [_vp, _vp, _i32, _vp, _vp, _vp, _vp]),
        "tersoff_md_force": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp, _f64, _f64, _i32, _i32,
                                            _vp, _vp, _vp, _vp]),
        "tersoff_md_export_neighbors": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
        "tersoff_set_form": (ctypes.c_int, [_vp, _i32]),
        "tersoff_md_nve": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _f64, _f64, _i32, _i32, _f64, _i32,
                                          _vp, _vp, _vp, _vp, _vp]),
        "tersoff_fitness_static": (ctypes.c_int, [_vp, _vp, _i32, ctypes.POINTER(_Targets), _vp, _i32,
                                                  _vp, _vp, _vp, _vp]),
        "tersoff_kernel_launches": (ctypes.c_int64, []),
        "tersoff_profile": (ctypes.c_int, [_vp, _i32]),
        "tersoff_set_launch_mode": (ctypes.c_int, [_vp, _i32]),
        "tersoff_set_wait_limit": (ctypes.c_int, [_vp, ctypes.c_int64]),
        "tersoff_measure_peaks": (ctypes.c_int, [_i32, _vp]),
        "tersoff_set_schedule": (ctypes.c_int, [_vp, _i32, _i32, _i32, _i32, _i32, _i32]),
        "tersoff_schedule_info": (ctypes.c_int, [_vp, _i32, _i32, _vp]),
        "tersoff_ga_step": (ctypes.c_int, [_i32, _i32, _i32, _f64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
        "tersoff_autotune": (ctypes.c_int, [_vp, _vp, _i32, ctypes.POINTER(_Targets), _i32, _i32,
                                            ctypes.POINTER(_f64), ctypes.POINTER(_i32), _vp]),
        "tersoff_profile_read": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(_f64)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    lib.tersoff_debug_bounds.restype = ctypes.c_int
    lib.tersoff_debug_bounds.argtypes = [_vp]
    _lib = lib
    return lib


def ga_step(Z: torch.Tensor, genes_in: torch.Tensor, uniforms: torch.Tensor, lo: torch.Tensor, hi: torch.Tensor,
            n_par: int, rate: float, genes_out: torch.Tensor, params_out: torch.Tensor, order=None, stream=None):
    """One GA generation on the device (tersoff_ga_step); all tensors CUDA float64 (order int32);
    genes [P][G] with G = len(lo)."""
    P = genes_in.shape[0]
    G = lo.shape[0]
    _cuda(Z, torch.float64, (P,), "Z")
    _cuda(genes_in, torch.float64, (P, G), "genes_in")
    _cuda(genes_out, torch.float64, (P, G), "genes_out")
    _cuda(params_out, torch.float64, (P, G), "params_out")
    _cuda(lo, torch.float64, (G,), "lo")
    _cuda(hi, torch.float64, (G,), "hi")
    _cuda(uniforms, torch.float64, None, "uniforms")
    if uniforms.numel() < (G + 2) * (P - n_par) + 2 * G * (P - 1):
        raise ValueError("too few uniform random numbers for one generation")
    if order is not None:
        _cuda(order, torch.int32, (P,), "order")
    rc = load().tersoff_ga_step(P, G, n_par, float(rate), Z.data_ptr(), genes_in.data_ptr(), uniforms.data_ptr(),
                                lo.data_ptr(), hi.data_ptr(), genes_out.data_ptr(), params_out.data_ptr(),
                                _ptr(order), _stream(stream))
    if rc != OK:
        raise TersoffError(rc, "tersoff_ga_step: bad arguments or CUDA error")


def measure_peaks(device: int = 0) -> dict:
    """Measured arithmetic throughput of the device (tersoff_measure_peaks), in operations per second."""
    out = np.zeros(6, np.float64)
    rc = load().tersoff_measure_peaks(int(device), out.ctypes.data)
    if rc != OK:
        raise TersoffError(rc, "tersoff_measure_peaks failed")
    keys = ("fp32_fma_flops", "fp32x2_fma_flops", "fp64_fma_flops", "fp64_add_ops", "xu_ex2_ops", "cvt_f32_f64_ops")
    return dict(zip(keys, (float(v) for v in out)))


class TersoffError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"tersoff error {code}: {msg}")
        self.code = code


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _cuda(t: torch.Tensor, dtype, shape=None, name="tensor") -> torch.Tensor:
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous CUDA {dtype} tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


class Context:
    """One tersoff_ctx on one CUDA device."""

    def __init__(self, device: int = 0):
        self.lib = load()
        self.device = device
        h = _vp()
        rc = self.lib.tersoff_create(ctypes.byref(h), device)
        if rc != OK:
            raise TersoffError(rc, "tersoff_create failed")
        self.h = h
        self.C = 0
        self.Ntot = 0
        self.form = FORM_MINIMAL
        self.atom_off = None
        self.max_nbr = 0

    def close(self):
        if getattr(self, "h", None):
            self.lib.tersoff_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int):
        if rc != OK:
            raise TersoffError(rc, self.lib.tersoff_last_error(self.h).decode())

    # ---- calls ---------------------------------------------------------------------------------
    def get_status(self, stream=None) -> int:
        return int(self.lib.tersoff_get_status(self.h, _stream(stream)))

    def kernel_launches(self) -> int:
        """Kernels launched by the library in this process so far (all contexts)."""
        return int(self.lib.tersoff_kernel_launches())

    def set_form(self, form: int):
        """FORM_MINIMAL (parameter vectors of 6, Eq. 16) or FORM_TERSOFF (9: D0, alpha, r0, S, n, h,
        gamma, c, d; Eq. 8 angular function, free S) for later eval and fitness calls."""
        self._check(self.lib.tersoff_set_form(self.h, int(form)))
        self.form = int(form)

    @property
    def n_params(self) -> int:
        return 9 if self.form == FORM_TERSOFF else 6

    def set_launch_mode(self, graphs: bool = True, pdl: bool = True):
        """Replay the fitness call's launch sequence from a cached CUDA graph (graphs) and/or launch its
        kernels with programmatic dependent launch (pdl); both on by default."""
        self._check(self.lib.tersoff_set_launch_mode(self.h, (LAUNCH_GRAPHS if graphs else 0) | (LAUNCH_PDL if pdl else 0)))

    def set_wait_limit(self, spins: int = -1):
        """Bound (polls) of the device-side wait of later calls, the batched kernel's wait for its staged
        geometry (tersoff_set_wait_limit); negative restores the built-in bound. A wait that gives up
        sets STATUS_TIMEOUT and its kernel stops early."""
        self._check(self.lib.tersoff_set_wait_limit(self.h, int(spins)))

    def profile(self, enable: bool = True):
        """Start or stop CUDA-event timing of the batched E/F/W kernel (clears earlier records)."""
        self._check(self.lib.tersoff_profile(self.h, 1 if enable else 0))

    def profile_read(self):
        """(timed launch sequences, summed milliseconds) since the last read; clears the records."""
        n = ctypes.c_int64()
        ms = _f64()
        self._check(self.lib.tersoff_profile_read(self.h, ctypes.byref(n), ctypes.byref(ms)))
        return int(n.value), float(ms.value)

    def debug_bounds(self):
        """First shared-memory bounds violation recorded by a TSF_DEBUG_BOUNDS build (zeros if none)."""
        out = np.zeros(4, np.uint32)
        self.lib.tersoff_debug_bounds(out.ctypes.data)
        return out

    def build_neighbors(self, atom_off, pos: torch.Tensor, box: torch.Tensor, R1: float = 2.8,
                        R2: float = 3.2, max_nbr: int = 16, stream=None):
        """atom_off: host int32 [C+1]; pos: CUDA float64 [Ntot][3]; box: CUDA float64 [C][3][3]."""
        off = np.ascontiguousarray(np.asarray(atom_off, dtype=np.int32))
        C = len(off) - 1
        N = int(off[-1]) if C >= 0 else 0
        _cuda(pos, torch.float64, (N, 3), "pos")
        _cuda(box, torch.float64, (C, 3, 3), "box")
        cfg = _Configs(C, off.ctypes.data, pos.data_ptr(), box.data_ptr())
        self._check(self.lib.tersoff_build_neighbors(self.h, ctypes.byref(cfg), R1, R2, max_nbr,
                                                     _stream(stream)))
        self.C, self.Ntot, self.atom_off, self.max_nbr = C, N, off, max_nbr

    def build_info(self):
        n, b, m = ctypes.c_int64(), ctypes.c_int64(), _i32()
        self._check(self.lib.tersoff_build_info(self.h, ctypes.byref(n), ctypes.byref(b), ctypes.byref(m)))
        return n.value, b.value, m.value

    def export_neighbors(self):
        N, M = self.Ntot, self.max_nbr
        cnt = np.zeros(N, np.int32)
        nbr = np.zeros((N, M), np.int32)
        shift = np.zeros((N, M, 3), np.int8)
        self._check(self.lib.tersoff_export_neighbors(self.h, _ptr(cnt), _ptr(nbr), _ptr(shift)))
        return cnt, nbr, shift

    def eval(self, params: torch.Tensor, precision: int = 32, want_F: bool = True, stream=None):
        """E [P][C], F [P][Ntot][3] (float32 or float64), W [P][C][6] on the params' device."""
        P = params.shape[0]
        _cuda(params, torch.float64, (P, self.n_params), "params")
        dev = params.device
        E = torch.empty((P, self.C), dtype=torch.float64, device=dev)
        W = torch.empty((P, self.C, 6), dtype=torch.float64, device=dev)
        F = None
        if want_F:
            F = torch.empty((P, self.Ntot, 3), dtype=torch.float32 if precision == 32 else torch.float64,
                            device=dev)
        self._check(self.lib.tersoff_eval(self.h, params.data_ptr(), P, precision, E.data_ptr(),
                                          _ptr(F), W.data_ptr(), _stream(stream)))
        return E, F, W

    def _targets(self, targets):
        tE = _cuda(targets["E"], torch.float64, (self.C,), "targets E")
        tW = _cuda(targets["W"], torch.float64, (self.C, 6), "targets W")
        tF = _cuda(targets["F"], torch.float64, (self.Ntot, 3), "targets F")
        tm = _cuda(targets["mask"], torch.uint8, (self.C,), "targets mask")
        return _Targets(tE.data_ptr(), tW.data_ptr(), tF.data_ptr(), tm.data_ptr())

    def fitness(self, params: torch.Tensor, targets: dict, w=(1.0, 1.0, 1.0), precision: int = 32,
                stream=None, out=None):
        """Z [P], Zq [P][3], S [P][3] (FP64) of Eq. 15, 17-19."""
        P = params.shape[0]
        _cuda(params, torch.float64, (P, self.n_params), "params")
        dev = params.device
        if out is None:
            out = (torch.empty(P, dtype=torch.float64, device=dev),
                   torch.empty((P, 3), dtype=torch.float64, device=dev),
                   torch.empty((P, 3), dtype=torch.float64, device=dev))
        Z, Zq, S = out
        t = self._targets(targets)
        wv = (ctypes.c_double * 3)(*[float(x) for x in w])
        self._check(self.lib.tersoff_fitness(self.h, params.data_ptr(), P, ctypes.byref(t), ctypes.addressof(wv),
                                             precision, Z.data_ptr(), _ptr(Zq), _ptr(S), _stream(stream)))
        return Z, Zq, S

    def fitness_static(self, params: torch.Tensor, targets: dict, w=(1.0, 1.0, 1.0), precision: int = 32,
                       stream=None, out=None):
        """tersoff_fitness_static: the fitness of `fitness` without any device allocation in the call.

        For callers that cannot have the library call cudaMalloc (it stalls the device; or their
        memory is already reserved by another allocator). The output tensors here come from the
        caller (`out`) or from PyTorch's allocator in this wrapper, never from the library; the
        library's per-call scratch is a fixed 8 MiB device array shared by all calls, so calls that
        overlap on the GPU race. Every other buffer the call uses is allocated by build_neighbors, and
        creating the context looks up the array's device address.
        """
        P = params.shape[0]
        _cuda(params, torch.float64, (P, 6), "params")
        dev = params.device
        if out is None:
            out = (torch.empty(P, dtype=torch.float64, device=dev),
                   torch.empty((P, 3), dtype=torch.float64, device=dev),
                   torch.empty((P, 3), dtype=torch.float64, device=dev))
        Z, Zq, S = out
        t = self._targets(targets)
        wv = (ctypes.c_double * 3)(*[float(x) for x in w])
        self._check(self.lib.tersoff_fitness_static(self.h, params.data_ptr(), P, ctypes.byref(t),
                                                    ctypes.addressof(wv), precision, Z.data_ptr(), _ptr(Zq),
                                                    _ptr(S), _stream(stream)))
        return Z, Zq, S

    def autotune(self, params: torch.Tensor, targets: dict, precision: int = 32, reps: int = 3, stream=None):
        """Time the candidate schedules of the batched fitness launch for this P and keep the fastest
        (tersoff_autotune). Returns (tuned launch time in ms, candidates timed)."""
        P = params.shape[0]
        _cuda(params, torch.float64, (P, 6), "params")
        t = self._targets(targets)
        ms, n = _f64(), _i32()
        self._check(self.lib.tersoff_autotune(self.h, params.data_ptr(), P, ctypes.byref(t), precision, reps,
                                              ctypes.byref(ms), ctypes.byref(n), _stream(stream)))
        return float(ms.value), int(n.value)

    def set_schedule(self, P: int, tile: int = 32, items_per_config: int = 1, narrow: bool = True,
                     precision: int = 32, warps: int = 8):
        """Fix the batched fitness schedule for this P (tersoff_set_schedule)."""
        self._check(self.lib.tersoff_set_schedule(self.h, precision, P, tile, warps, items_per_config,
                                                  1 if narrow else 0))

    def schedule_info(self, precision: int = 32):
        """Per launch bucket: dict of mmax, cluster, configs, tuned_P, tile, items_per_config, narrow."""
        n = np.zeros(8, np.int32)
        self._check(self.lib.tersoff_schedule_info(self.h, precision, -1, n.ctypes.data))
        out = []
        for b in range(int(n[0])):
            v = np.zeros(8, np.int32)
            self._check(self.lib.tersoff_schedule_info(self.h, precision, b, v.ctypes.data))
            out.append(dict(zip(("mmax", "cluster", "configs", "tuned_P", "tile", "items_per_config", "narrow",
                                 "warps"),
                                (int(x) for x in v))))
        return out

    def param_grad(self, params: torch.Tensor, targets: dict, w=(1.0, 1.0, 1.0), loss: int = LOSS_SQ,
                   stream=None):
        """L [P] and dL/dx [P][6] ([P][9] in the Tersoff form) (FP64)."""
        P = params.shape[0]
        _cuda(params, torch.float64, (P, self.n_params), "params")
        dev = params.device
        L = torch.empty(P, dtype=torch.float64, device=dev)
        dL = torch.empty((P, self.n_params), dtype=torch.float64, device=dev)
        t = self._targets(targets)
        wv = (ctypes.c_double * 3)(*[float(x) for x in w])
        self._check(self.lib.tersoff_param_grad(self.h, params.data_ptr(), P, ctypes.byref(t), ctypes.addressof(wv),
                                                loss, L.data_ptr(), dL.data_ptr(), _stream(stream)))
        return L, dL

    def eval_plain(self, params: torch.Tensor, stream=None):
        """Plain FP64 path, one launch per (p, c): E [P][C], F [P][Ntot][3] float64, W [P][C][6]."""
        P = params.shape[0]
        _cuda(params, torch.float64, (P, 6), "params")
        dev = params.device
        E = torch.empty((P, self.C), dtype=torch.float64, device=dev)
        F = torch.empty((P, self.Ntot, 3), dtype=torch.float64, device=dev)
        W = torch.empty((P, self.C, 6), dtype=torch.float64, device=dev)
        self._check(self.lib.tersoff_eval_plain(self.h, params.data_ptr(), P, E.data_ptr(), F.data_ptr(),
                                                W.data_ptr(), _stream(stream)))
        return E, F, W

    def md_force(self, pos: torch.Tensor, box, params, R1: float = 2.8, R2: float = 3.2,
                 max_nbr: int = 16, precision: int = 32, stream=None, out=None):
        """One large cell: neighbour rebuild + E [1], F [N][3], W [6]."""
        N = pos.shape[0]
        _cuda(pos, torch.float64, (N, 3), "pos")
        boxh = np.ascontiguousarray(np.asarray(box, dtype=np.float64).reshape(3, 3))
        ph = np.ascontiguousarray(np.asarray(params, dtype=np.float64).reshape(6))
        dev = pos.device
        if out is None:
            out = (torch.empty(1, dtype=torch.float64, device=dev),
                   torch.empty((N, 3), dtype=torch.float32 if precision == 32 else torch.float64, device=dev),
                   torch.empty(6, dtype=torch.float64, device=dev))
        E, F, W = out
        self._check(self.lib.tersoff_md_force(self.h, N, pos.data_ptr(), boxh.ctypes.data, ph.ctypes.data,
                                              R1, R2, max_nbr, precision, E.data_ptr(), F.data_ptr(),
                                              W.data_ptr(), _stream(stream)))
        self.md_N, self.md_M = N, max_nbr
        return E, F, W

    def md_nve(self, pos: torch.Tensor, vel: torch.Tensor, mass: torch.Tensor, box, params, dt: float,
               nsteps: int, R1: float = 2.8, R2: float = 3.2, max_nbr: int = 16, precision: int = 64,
               stream=None, out=None):
        """Velocity-Verlet NVE (tersoff_md_nve): pos, vel [N][3] float64 CUDA, updated in place; mass [N]
        (amu); dt (fs). Returns Epot, Ekin [nsteps + 1] (eV), F [N][3] and W [6] at the end."""
        N = pos.shape[0]
        _cuda(pos, torch.float64, (N, 3), "pos")
        _cuda(vel, torch.float64, (N, 3), "vel")
        _cuda(mass, torch.float64, (N,), "mass")
        boxh = np.ascontiguousarray(np.asarray(box, dtype=np.float64).reshape(3, 3))
        ph = np.ascontiguousarray(np.asarray(params, dtype=np.float64).reshape(6))
        dev = pos.device
        if out is None:
            out = (torch.empty(nsteps + 1, dtype=torch.float64, device=dev),
                   torch.empty(nsteps + 1, dtype=torch.float64, device=dev),
                   torch.empty((N, 3), dtype=torch.float32 if precision == 32 else torch.float64, device=dev),
                   torch.empty(6, dtype=torch.float64, device=dev))
        Ep, Ek, F, W = out
        self._check(self.lib.tersoff_md_nve(self.h, N, pos.data_ptr(), vel.data_ptr(), mass.data_ptr(),
                                            boxh.ctypes.data, ph.ctypes.data, R1, R2, max_nbr, precision, float(dt),
                                            int(nsteps), Ep.data_ptr(), Ek.data_ptr(), F.data_ptr(), W.data_ptr(),
                                            _stream(stream)))
        self.md_N, self.md_M = N, max_nbr
        return Ep, Ek, F, W

    def md_export_neighbors(self):
        N, M = self.md_N, self.md_M
        cnt = np.zeros(N, np.int32)
        nbr = np.zeros((N, M), np.int32)
        shift = np.zeros((N, M, 3), np.int8)
        self._check(self.lib.tersoff_md_export_neighbors(self.h, _ptr(cnt), _ptr(nbr), _ptr(shift)))
        return cnt, nbr, shift
