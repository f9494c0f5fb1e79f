"""Python binding of the C-ABI in ``include/lbm.h`` (ctypes; argument marshalling only).

Every step of the lattice Boltzmann path runs in the CUDA library ``_build/liblbm_gb300.so``;
this module only converts arguments.  There is no CPU fallback: if the library is missing or
no GPU is present, the calls raise.  PyTorch supplies device memory (the library allocates
through callbacks backed by the caching allocator) and the CUDA stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# LBM_GB300_LIBRARY selects another build of the library (e.g. the bounds-checked LBM_DEBUG
# variant, _build_debug/liblbm_gb300_debug.so); it must exist like the default one
LIB_PATH = os.environ.get("LBM_GB300_LIBRARY") or os.path.join(HERE, "_build", "liblbm_gb300.so")

STORE = {"fp32": 0, "fp16": 1, "bf16": 2}
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "UNSTABLE", 5: "TIMEOUT", 6: "STATE", 7: "IO"}

# every entry point declared in include/lbm.h
EXPORTS = ["lbm_default_params", "lbm_create_domain", "lbm_set_inlet_waveform", "lbm_init_equilibrium",
           "lbm_step", "lbm_get_macroscopic", "lbm_get_diagnostics", "lbm_get_info", "lbm_sync",
           "lbm_save_state", "lbm_load_state", "lbm_destroy", "lbm_last_error", "lbm_set_launch_config",
           "lbm_autotune", "lbm_get_diagnostics_noalloc", "lbm_batch_create", "lbm_batch_step",
           "lbm_batch_set_launch_config", "lbm_batch_autotune", "lbm_batch_destroy", "lbm_corrector_num_params",
           "lbm_corrector_create", "lbm_corrector_get_params", "lbm_corrector_set_params", "lbm_corrector_forward",
           "lbm_corrector_gradients", "lbm_corrector_train_step", "lbm_corrector_apply", "lbm_corrector_destroy",
           "lbm_apply_velocity_correction", "lbm_restrict", "lbm_mean_reset", "lbm_mean_sample", "lbm_mean_get",
           "lbm_probe", "lbm_similarity_index", "lbm_halo_size", "lbm_halo_pack", "lbm_halo_unpack",
           "lbm_batch_set_persistent", "lbm_batch_sync"]
N_LAUNCH_CONFIGS = 8
LAUNCH_CONFIG_NAMES = ["256x3", "128x7", "128x6", "128x8", "128x10", "pipe128x6", "2c128x4", "2c128x3"]
SCHEME = {"ab": 0, "esoteric": 1}
COLLISION = {"chm": 0, "srt2": 1, "trt2": 2}


class LbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("omega_hi", ctypes.c_double * 4),
                ("force", ctypes.c_double * 3), ("force_amp", ctypes.c_double * 3),
                ("force_omega", ctypes.c_double), ("rho_out", ctypes.c_double),
                ("periodic", ctypes.c_int32 * 3), ("storage", ctypes.c_int32), ("scheme", ctypes.c_int32),
                ("collision", ctypes.c_int32), ("trt_magic", ctypes.c_double)]


class Info(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("n_fluid", ctypes.c_int64), ("n_bricks", ctypes.c_int64), ("n_slots", ctypes.c_int64),
                ("n_wall_cells", ctypes.c_int64), ("n_bouzidi_cells", ctypes.c_int64),
                ("n_open_cells", ctypes.c_int64), ("time", ctypes.c_int64), ("storage", ctypes.c_int32),
                ("bytes_per_value", ctypes.c_int32), ("device_bytes", ctypes.c_int64),
                ("launch_config", ctypes.c_int32), ("scheme", ctypes.c_int32),
                ("n_store_bricks", ctypes.c_int64), ("n_halo", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Diagnostics(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("flux_in", ctypes.c_double), ("flux_out", ctypes.c_double),
                ("max_u", ctypes.c_double), ("n_nonfinite", ctypes.c_int64), ("time", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_lib = None


def load_library(path: str = LIB_PATH):
    """Loads the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    L = ctypes.CDLL(path)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    L.lbm_default_params.argtypes = [ctypes.POINTER(Params)]
    L.lbm_default_params.restype = None
    L.lbm_create_domain.argtypes = [vp, i32, i32, i32, vp, vp, vp, i64, vp, dbl, vp, ctypes.POINTER(Params),
                                    ALLOC_FN, FREE_FN, vp, vp, ctypes.POINTER(vp)]
    L.lbm_set_inlet_waveform.argtypes = [vp, vp, vp, i32, dbl, dbl]
    L.lbm_init_equilibrium.argtypes = [vp, vp, vp, i32]
    L.lbm_step.argtypes = [vp, i64]
    L.lbm_get_macroscopic.argtypes = [vp, vp, vp, i32, i32]
    L.lbm_get_diagnostics.argtypes = [vp, ctypes.POINTER(Diagnostics)]
    L.lbm_get_diagnostics_noalloc.argtypes = [vp, ctypes.POINTER(Diagnostics)]
    L.lbm_get_info.argtypes = [vp, ctypes.POINTER(Info)]
    L.lbm_sync.argtypes = [vp]
    L.lbm_save_state.argtypes = [vp, ctypes.c_char_p]
    L.lbm_load_state.argtypes = [vp, ctypes.c_char_p]
    L.lbm_set_launch_config.argtypes = [vp, i32]
    L.lbm_autotune.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_float)]
    L.lbm_destroy.argtypes = [vp]
    L.lbm_destroy.restype = None
    L.lbm_batch_create.argtypes = [ctypes.POINTER(vp), i32, i32, vp, ctypes.POINTER(vp)]
    L.lbm_batch_step.argtypes = [vp, i64]
    L.lbm_batch_set_launch_config.argtypes = [vp, i32]
    L.lbm_batch_autotune.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_float)]
    L.lbm_batch_set_persistent.argtypes = [vp, i32, dbl]
    L.lbm_batch_sync.argtypes = [vp]
    L.lbm_batch_destroy.argtypes = [vp]
    L.lbm_batch_destroy.restype = None
    L.lbm_corrector_num_params.argtypes = []
    L.lbm_corrector_num_params.restype = i64
    L.lbm_corrector_create.argtypes = [vp, i32, i32, i32, dbl, dbl, dbl, vp, ALLOC_FN, FREE_FN, vp, vp,
                                       ctypes.POINTER(vp)]
    L.lbm_corrector_get_params.argtypes = [vp, vp]
    L.lbm_corrector_set_params.argtypes = [vp, vp]
    L.lbm_corrector_forward.argtypes = [vp, vp, vp, vp, vp, vp]
    L.lbm_corrector_gradients.argtypes = [vp, vp, vp, vp, vp, vp, vp, ctypes.POINTER(dbl)]
    L.lbm_corrector_train_step.argtypes = [vp, vp, vp, vp, vp, vp, dbl, ctypes.POINTER(dbl)]
    L.lbm_corrector_apply.argtypes = [vp, vp, vp, vp, dbl]
    L.lbm_corrector_destroy.argtypes = [vp]
    L.lbm_corrector_destroy.restype = None
    L.lbm_apply_velocity_correction.argtypes = [vp, vp, i32]
    L.lbm_restrict.argtypes = [vp, vp, vp, i32, i32, i32, vp, vp, vp]
    L.lbm_mean_reset.argtypes = [vp]
    L.lbm_mean_sample.argtypes = [vp]
    L.lbm_mean_get.argtypes = [vp, vp, vp, i32, i32, ctypes.POINTER(i64)]
    L.lbm_probe.argtypes = [vp, vp, i32, vp, i32]
    L.lbm_similarity_index.argtypes = [vp, vp, vp, i64, ctypes.POINTER(dbl), vp]
    L.lbm_halo_size.argtypes = [vp, i32, ctypes.POINTER(i64)]
    L.lbm_halo_pack.argtypes = [vp, i32, vp]
    L.lbm_halo_unpack.argtypes = [vp, i32, vp]
    L.lbm_last_error.argtypes = []
    L.lbm_last_error.restype = ctypes.c_char_p
    for name in ["lbm_create_domain", "lbm_set_inlet_waveform", "lbm_init_equilibrium", "lbm_step",
                 "lbm_get_macroscopic", "lbm_get_diagnostics", "lbm_get_info", "lbm_sync",
                 "lbm_save_state", "lbm_load_state", "lbm_set_launch_config", "lbm_autotune",
                 "lbm_get_diagnostics_noalloc", "lbm_batch_create", "lbm_batch_step",
                 "lbm_batch_set_launch_config", "lbm_batch_autotune", "lbm_mean_reset", "lbm_mean_sample",
                 "lbm_mean_get", "lbm_probe", "lbm_similarity_index", "lbm_halo_size", "lbm_halo_pack",
                 "lbm_halo_unpack", "lbm_batch_set_persistent", "lbm_batch_sync"]:
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(status):
    if status != 0:
        raise LbmError(status, load_library().lbm_last_error().decode())


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


class TorchAllocator:
    """Device allocator callbacks backed by the PyTorch caching allocator."""

    def __init__(self, device):
        import torch
        self._torch = torch
        self._device = device
        self._live = {}
        self.alloc_fn = ALLOC_FN(self._alloc)
        self.free_fn = FREE_FN(self._free)

    def _alloc(self, nbytes, ctx):
        try:
            t = self._torch.empty(int(nbytes), dtype=self._torch.uint8, device=self._device)
        except Exception:  # out of memory: report NULL to the library
            return None
        p = t.data_ptr()
        self._live[p] = t
        return p

    def _free(self, ptr, ctx):
        self._live.pop(ptr, None)


class Domain:
    """A voxel domain on the GPU (see include/lbm.h for the semantics of each call)."""

    def __init__(self, mask, periodic=(0, 0, 0), links=None, inlet_center=None, inlet_radius=0.0,
                 tau=0.6, omega_hi=(1.0, 1.0, 1.0, 1.0), force=(0.0, 0.0, 0.0), force_amp=(0.0, 0.0, 0.0),
                 force_omega=0.0, rho_out=1.0, storage="fp32", scheme="esoteric", tau_cell=None, device=None,
                 stream=None, collision="chm", trt_magic=3.0 / 16.0):
        import torch
        L = load_library()
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
        if mask.ndim != 3:
            raise ValueError("mask must have shape (nz, ny, nx)")
        self.shape = mask.shape
        self._mask = mask
        nz, ny, nx = mask.shape
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.stream = torch.cuda.current_stream(self.device) if stream is None else stream
        p = Params()
        L.lbm_default_params(ctypes.byref(p))
        p.tau = tau
        for k in range(4):
            p.omega_hi[k] = omega_hi[k]
        for d in range(3):
            p.force[d] = force[d]
            p.force_amp[d] = force_amp[d]
            p.periodic[d] = int(bool(periodic[d]))
        p.force_omega = force_omega
        p.rho_out = rho_out
        p.storage = STORE[storage] if isinstance(storage, str) else int(storage)
        p.scheme = SCHEME[scheme] if isinstance(scheme, str) else int(scheme)
        p.collision = COLLISION[collision] if isinstance(collision, str) else int(collision)
        p.trt_magic = trt_magic
        self.storage = storage
        self.collision = collision
        self.omega_hi = tuple(float(w) for w in omega_hi)
        if links is None or len(links[0]) == 0:
            lc = ld = lq = None
            n_links = 0
        else:
            lc = np.ascontiguousarray(links[0], dtype=np.int64)
            ld = np.ascontiguousarray(links[1], dtype=np.uint8)
            lq = np.ascontiguousarray(links[2], dtype=np.float64)
            n_links = len(lc)
        ic = None if inlet_center is None else np.ascontiguousarray(inlet_center, dtype=np.float64)
        tc = None if tau_cell is None else np.ascontiguousarray(tau_cell, dtype=np.float64)
        self._alloc = TorchAllocator(self.device)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(L.lbm_create_domain(_ptr(mask), nx, ny, nz, _ptr(lc), _ptr(ld), _ptr(lq), n_links, _ptr(ic),
                                       float(inlet_radius), _ptr(tc), ctypes.byref(p), self._alloc.alloc_fn,
                                       self._alloc.free_fn, None, ctypes.c_void_p(self.stream.cuda_stream),
                                       ctypes.byref(h)))
        self._h = h

    @classmethod
    def from_geometry(cls, g, storage="fp32", scheme="esoteric", **kw):
        dom = cls(g.mask, periodic=g.periodic, links=g.links, inlet_center=g.inlet_center,
                  inlet_radius=g.inlet_radius, tau=g.tau, force=g.g0, force_amp=g.gamp,
                  force_omega=g.gomega, storage=storage, scheme=scheme, tau_cell=g.tau_cell, **kw)
        if g.wave is not None:
            a, b, P, up = g.wave
            dom.set_inlet_waveform(a, b, P, up)
        return dom

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load_library().lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_inlet_waveform(self, a, b, period, u_peak):
        a = np.ascontiguousarray(a, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        _check(load_library().lbm_set_inlet_waveform(self._h, _ptr(a), _ptr(b) if b.size else None, len(a) - 1,
                                                      float(period), float(u_peak)))

    def init_equilibrium(self, rho, u):
        """rho (nz,ny,nx) and u (3,nz,ny,nx): numpy arrays or CUDA tensors."""
        import torch
        L = load_library()
        if isinstance(rho, torch.Tensor):
            rho_t = rho.to(torch.float32).contiguous()
            u_t = u.to(torch.float32).contiguous()
            _check(L.lbm_init_equilibrium(self._h, ctypes.c_void_p(rho_t.data_ptr()),
                                          ctypes.c_void_p(u_t.data_ptr()), 1))
        else:
            r = np.ascontiguousarray(rho, dtype=np.float32)
            uu = np.ascontiguousarray(u, dtype=np.float32)
            _check(L.lbm_init_equilibrium(self._h, _ptr(r), _ptr(uu), 0))

    def step(self, n=1):
        _check(load_library().lbm_step(self._h, int(n)))

    def sync(self):
        _check(load_library().lbm_sync(self._h))

    def info(self) -> dict:
        i = Info()
        _check(load_library().lbm_get_info(self._h, ctypes.byref(i)))
        return i.as_dict()

    @property
    def time(self):
        return self.info()["time"]

    def macroscopic(self, dense=True):
        """(rho, u) as numpy float32 arrays: dense (nz,ny,nx)/(3,nz,ny,nx), or compact
        (n_fluid,)/(3,n_fluid) in increasing box order."""
        nz, ny, nx = self.shape
        n = nx * ny * nz if dense else self.info()["n_fluid"]
        rho = np.empty(n, np.float32)
        u = np.empty(3 * n, np.float32)
        _check(load_library().lbm_get_macroscopic(self._h, _ptr(rho), _ptr(u), int(dense), 0))
        if dense:
            return rho.reshape(nz, ny, nx), u.reshape(3, nz, ny, nx)
        return rho, u.reshape(3, n)

    def macroscopic_device(self, rho, u, dense=True):
        """Writes into CUDA float32 tensors on the domain's stream (no host round trip)."""
        _check(load_library().lbm_get_macroscopic(self._h, ctypes.c_void_p(rho.data_ptr()),
                                                  ctypes.c_void_p(u.data_ptr()), int(dense), 1))

    # ---------------------------------------------------------------- flow metrics
    def mean_reset(self):
        _check(load_library().lbm_mean_reset(self._h))

    def mean_sample(self):
        _check(load_library().lbm_mean_sample(self._h))

    def mean(self, dense=True):
        """(rho_mean, u_mean, n_samples) as numpy float32 arrays, shaped as macroscopic()."""
        nz, ny, nx = self.shape
        n = nx * ny * nz if dense else self.info()["n_fluid"]
        rho = np.empty(n, np.float32)
        u = np.empty(3 * n, np.float32)
        ns = ctypes.c_int64()
        _check(load_library().lbm_mean_get(self._h, _ptr(rho), _ptr(u), int(dense), 0, ctypes.byref(ns)))
        if dense:
            return rho.reshape(nz, ny, nx), u.reshape(3, nz, ny, nx), ns.value
        return rho, u.reshape(3, n), ns.value

    def fluid_index(self, points):
        """Positions in the compact fluid list of box cells given as (z, y, x) triples."""
        if not hasattr(self, "_fluid_rank"):
            fl = self._mask.reshape(-1) != 0
            rank = np.cumsum(fl) - 1
            self._fluid_rank = np.where(fl, rank, -1)
        nz, ny, nx = self.shape
        pts = np.asarray(points, dtype=np.int64).reshape(-1, 3)
        idx = self._fluid_rank[(pts[:, 0] * ny + pts[:, 1]) * nx + pts[:, 2]]
        if np.any(idx < 0):
            raise ValueError("probe point is not a fluid cell")
        return idx.astype(np.int64)

    def probe(self, points):
        """(n, 4) float32 array of (rho, ux, uy, uz) at box cells given as (z, y, x) triples."""
        idx = np.ascontiguousarray(self.fluid_index(points))
        out = np.empty((len(idx), 4), np.float32)
        _check(load_library().lbm_probe(self._h, _ptr(idx), len(idx), _ptr(out), 0))
        return out

    def diagnostics(self, raise_unstable=True) -> dict:
        dg = Diagnostics()
        st = load_library().lbm_get_diagnostics(self._h, ctypes.byref(dg))
        if st != 0 and (raise_unstable or st != 4):
            _check(st)
        return dg.as_dict()

    def set_launch_config(self, config):
        _check(load_library().lbm_set_launch_config(self._h, int(config)))

    def autotune(self, trial_steps=20, cache=None):
        """Times every launch configuration on this domain and keeps the fastest; returns
        (best, {name: ms_per_step}).  cache: path of a JSON file of earlier choices keyed by GPU
        and domain configuration (autotune_cache_key); a hit selects the stored configuration
        without timing (self.autotuned_from_cache tells which happened), a miss times and adds
        the result."""
        key = autotune_cache_key(self) if cache else None
        if key is not None:
            hit = autotune_cache_get(cache, key)
            if hit is not None:
                self.set_launch_config(LAUNCH_CONFIG_NAMES.index(hit["best"]))
                self.autotuned_from_cache = True
                return LAUNCH_CONFIG_NAMES.index(hit["best"]), dict(hit["ms"])
        best = ctypes.c_int32()
        ms = (ctypes.c_float * N_LAUNCH_CONFIGS)()
        _check(load_library().lbm_autotune(self._h, int(trial_steps), ctypes.byref(best), ms))
        out = dict(zip(LAUNCH_CONFIG_NAMES, [float(v) for v in ms]))
        self.autotuned_from_cache = False
        if key is not None:
            autotune_cache_put(cache, key, {"best": LAUNCH_CONFIG_NAMES[best.value], "ms": out,
                                            "trial_steps": int(trial_steps)})
        return best.value, out

    def diagnostics_noalloc(self, raise_unstable=True) -> dict:
        """lbm_get_diagnostics_noalloc: the same reduction with the library's fixed scratch
        array, for callers that cannot allocate device memory at that point."""
        dg = Diagnostics()
        st = load_library().lbm_get_diagnostics_noalloc(self._h, ctypes.byref(dg))
        if st != 0 and (raise_unstable or st != 4):
            _check(st)
        return dg.as_dict()

    def macroscopic_tensors(self):
        """(rho, u) of the current level as dense CUDA float32 tensors (nz,ny,nx), (3,nz,ny,nx)."""
        import torch
        nz, ny, nx = self.shape
        rho = torch.empty((nz, ny, nx), dtype=torch.float32, device=self.device)
        u = torch.empty((3, nz, ny, nx), dtype=torch.float32, device=self.device)
        self.macroscopic_device(rho, u, dense=True)
        return rho, u

    def apply_velocity_correction(self, du):
        """Post-collision populations of the previous level += f_eq(rho, u + du) - f_eq(rho, u);
        du: (3, nz, ny, nx) numpy array (the call waits) or CUDA tensor (enqueued on the domain's
        stream)."""
        import torch
        L = load_library()
        if isinstance(du, torch.Tensor):
            t = du.to(torch.float32).contiguous()
            _check(L.lbm_apply_velocity_correction(self._h, ctypes.c_void_p(t.data_ptr()), 1))
            t.record_stream(self.stream)  # keep t's memory until the domain's stream has read it
        else:
            a = np.ascontiguousarray(du, dtype=np.float32)
            _check(L.lbm_apply_velocity_correction(self._h, _ptr(a), 0))

    # ---------------------------------------------------------------- slab decomposition
    def halo_size(self, face):
        """Values per exchange buffer of `face` (0 if it has no halo layer)."""
        n = ctypes.c_int64()
        _check(load_library().lbm_halo_size(self._h, int(face), ctypes.byref(n)))
        return n.value

    def halo_pack(self, face, buf):
        """Post-collision populations leaving through `face` into the CUDA tensor buf (storage
        precision: int32 for FP32, int16 for 16-bit storage, raw bits)."""
        _check(load_library().lbm_halo_pack(self._h, int(face), ctypes.c_void_p(buf.data_ptr())))

    def halo_unpack(self, face, buf):
        _check(load_library().lbm_halo_unpack(self._h, int(face), ctypes.c_void_p(buf.data_ptr())))

    def save_state(self, path):
        _check(load_library().lbm_save_state(self._h, os.fsencode(path)))

    def load_state(self, path):
        _check(load_library().lbm_load_state(self._h, os.fsencode(path)))


def autotune_cache_key(dom) -> str:
    """Key of a domain's autotuning result: the GPU (name, SM count, compute capability), the
    library file (size and modification time: a rebuilt library is tuned again), and what the
    step kernel's speed depends on -- storage, scheme, collision operator and whether the
    higher-order rates are all 1 (the second-order-only collision), box extents, fluid cells,
    bricks and wall / Bouzidi / open cells."""
    import json

    import torch
    pr = torch.cuda.get_device_properties(dom.device)
    st = os.stat(LIB_PATH)
    i = dom.info()
    return json.dumps({"gpu": pr.name, "sms": pr.multi_processor_count, "cc": [pr.major, pr.minor],
                       "lib": [st.st_size, int(st.st_mtime)], "storage": i["storage"], "scheme": i["scheme"],
                       "collision": str(dom.collision), "unit_rates": all(w == 1.0 for w in dom.omega_hi),
                       "box": [i["nx"], i["ny"], i["nz"]], "fluid": i["n_fluid"], "bricks": i["n_bricks"],
                       "wall": i["n_wall_cells"], "bouzidi": i["n_bouzidi_cells"], "open": i["n_open_cells"]},
                      sort_keys=True)


def autotune_cache_get(path, key):
    """The stored entry for key in the JSON cache file at path, or None (no file, no entry, or an
    unreadable file)."""
    import json

    try:
        with open(path) as f:
            return json.load(f).get(key)
    except (OSError, ValueError):
        return None


def autotune_cache_put(path, key, value):
    """Adds or replaces key in the JSON cache file (written to a temporary file and renamed, so
    that a reader never sees a partial file)."""
    import json

    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        data = {}
    data[key] = value
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def similarity_index(u_a, u_b, mask=None, stream=None) -> float:
    """lbm_similarity_index on CUDA tensors u_a, u_b of shape (3, ...) (float32) and an optional
    uint8 mask of shape (...): the similarity index of Sec. 3.4 (factor 1/2, bounded by 1)."""
    import torch
    ua = u_a.to(torch.float32).contiguous()
    ub = u_b.to(torch.float32).contiguous()
    n = ua[0].numel()
    if ub[0].numel() != n or ua.shape[0] != 3 or ub.shape[0] != 3:
        raise ValueError("u_a and u_b must have shape (3, ...) with the same number of points")
    m = None if mask is None else mask.to(torch.uint8).contiguous()
    if m is not None and m.numel() != n:
        raise ValueError("mask must have one entry per point")
    st = torch.cuda.current_stream(ua.device) if stream is None else stream
    out = ctypes.c_double()
    _check(load_library().lbm_similarity_index(ctypes.c_void_p(ua.data_ptr()), ctypes.c_void_p(ub.data_ptr()),
                                                None if m is None else ctypes.c_void_p(m.data_ptr()), n,
                                                ctypes.byref(out), ctypes.c_void_p(st.cuda_stream)))
    return out.value


def flatten_params(params):
    """[W1, b1, W2, b2, W3, b3] -> one FP32 vector in the C-ABI's order."""
    return np.concatenate([np.asarray(p, dtype=np.float32).reshape(-1) for p in params])


def unflatten_params(vec):
    out, k = [], 0
    for _ in range(3):
        out.append(np.asarray(vec[k:k + 27 * 256], dtype=np.float64).reshape(27, 16, 16))
        k += 27 * 256
        out.append(np.asarray(vec[k:k + 16], dtype=np.float64))
        k += 16
    return out


class Corrector:
    """The learned coarse-grid corrector (lbm_corrector_* in include/lbm.h).  Fields are dense
    CUDA float32 tensors on the coarse box: rho (nz,ny,nx), u (3,nz,ny,nx)."""

    def __init__(self, mask, params, u_scale=0.05, rho_scale=0.01, du_scale=0.005, device=None, stream=None):
        import torch
        L = load_library()
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
        self.shape = mask.shape
        nz, ny, nx = mask.shape
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.stream = torch.cuda.current_stream(self.device) if stream is None else stream
        self.n_params = int(L.lbm_corrector_num_params())
        vec = flatten_params(params) if isinstance(params, (list, tuple)) else np.asarray(params, np.float32)
        assert vec.size == self.n_params
        self._alloc = TorchAllocator(self.device)
        h = ctypes.c_void_p()
        _check(L.lbm_corrector_create(_ptr(mask), nx, ny, nz, float(u_scale), float(rho_scale), float(du_scale),
                                      _ptr(vec), self._alloc.alloc_fn, self._alloc.free_fn, None,
                                      ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self._h = h

    @staticmethod
    def _p(t):
        return ctypes.c_void_p(t.data_ptr()) if t is not None else None

    def forward(self, rho, u, mask=None, out_mask=None):
        """du (3,nz,ny,nx) CUDA tensor; mask / out_mask: optional dense uint8 CUDA tensors of the
        feature cells and of the cells the correction acts on."""
        import torch
        du = torch.empty_like(u, dtype=torch.float32)
        _check(load_library().lbm_corrector_forward(self._h, self._p(mask), self._p(out_mask), self._p(rho.contiguous()),
                                                    self._p(u.contiguous()), self._p(du)))
        return du

    def gradients(self, rho, u, u_target, mask=None, out_mask=None):
        g = np.zeros(self.n_params, np.float32)
        loss = ctypes.c_double()
        _check(load_library().lbm_corrector_gradients(self._h, self._p(mask), self._p(out_mask),
                                                      self._p(rho.contiguous()), self._p(u.contiguous()),
                                                      self._p(u_target.contiguous()), _ptr(g), ctypes.byref(loss)))
        return loss.value, unflatten_params(g)

    def train_step(self, rho, u, u_target, lr, mask=None, out_mask=None):
        loss = ctypes.c_double()
        _check(load_library().lbm_corrector_train_step(self._h, self._p(mask), self._p(out_mask),
                                                       self._p(rho.contiguous()), self._p(u.contiguous()),
                                                       self._p(u_target.contiguous()), float(lr), ctypes.byref(loss)))
        return loss.value

    def apply(self, domain, mask=None, out_mask=None, gain=1.0):
        _check(load_library().lbm_corrector_apply(self._h, domain._h, self._p(mask), self._p(out_mask), float(gain)))

    def params(self):
        vec = np.zeros(self.n_params, np.float32)
        _check(load_library().lbm_corrector_get_params(self._h, _ptr(vec)))
        return vec

    def set_params(self, vec):
        vec = np.ascontiguousarray(vec, dtype=np.float32)
        _check(load_library().lbm_corrector_set_params(self._h, _ptr(vec)))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load_library().lbm_corrector_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def restrict(fine_rho, fine_u, fine_mask):
    """Coarse (rho, u) = mean over the fluid children of each coarse cell (CUDA tensors)."""
    import torch
    nz, ny, nx = fine_rho.shape
    crho = torch.empty((nz // 2, ny // 2, nx // 2), dtype=torch.float32, device=fine_rho.device)
    cu = torch.empty((3, nz // 2, ny // 2, nx // 2), dtype=torch.float32, device=fine_rho.device)
    m = fine_mask.to(torch.uint8).contiguous()
    _check(load_library().lbm_restrict(ctypes.c_void_p(fine_rho.contiguous().data_ptr()),
                                       ctypes.c_void_p(fine_u.contiguous().data_ptr()), ctypes.c_void_p(m.data_ptr()),
                                       nx, ny, nz, ctypes.c_void_p(crho.data_ptr()), ctypes.c_void_p(cu.data_ptr()),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return crho, cu


class Batch:
    """Several domains advanced together (one launch per step over all of them, chunks of
    graph_steps steps replayed as a CUDA graph); see lbm_batch_* in include/lbm.h."""

    def __init__(self, domains, graph_steps=50, stream=None):
        import torch
        L = load_library()
        self.domains = list(domains)
        self.stream = torch.cuda.current_stream() if stream is None else stream
        arr = (ctypes.c_void_p * len(self.domains))(*[d._h.value for d in self.domains])
        h = ctypes.c_void_p()
        _check(L.lbm_batch_create(arr, len(self.domains), int(graph_steps),
                                  ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self._h = h

    def step(self, n=1):
        _check(load_library().lbm_batch_step(self._h, int(n)))

    def set_launch_config(self, config):
        _check(load_library().lbm_batch_set_launch_config(self._h, int(config)))

    def autotune(self, trial_steps=20):
        best = ctypes.c_int32()
        ms = (ctypes.c_float * N_LAUNCH_CONFIGS)()
        _check(load_library().lbm_batch_autotune(self._h, int(trial_steps), ctypes.byref(best), ms))
        return best.value, dict(zip(LAUNCH_CONFIG_NAMES, list(ms)))

    def set_persistent(self, enable=True, barrier_timeout_s=1.0):
        """One cooperative launch per graph chunk with a bounded grid barrier between steps
        (lbm_batch_set_persistent)."""
        _check(load_library().lbm_batch_set_persistent(self._h, int(bool(enable)), float(barrier_timeout_s)))

    def sync(self):
        """Waits for the batch; raises LbmError (TIMEOUT) if a persistent chunk gave up."""
        _check(load_library().lbm_batch_sync(self._h))

    @property
    def n_fluid(self):
        return sum(d.info()["n_fluid"] for d in self.domains)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load_library().lbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
