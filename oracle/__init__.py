"""FP64 CPU oracle of the D3Q27 CHM-MRT lattice Boltzmann method (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``; never by the library.  It shares
no code with the CUDA path.  The arithmetic lives in ``lbm_oracle.c``; each C function cites
the section of the paper it restates.  Pins (tests/test_oracle_*.py) tie it to closed forms,
invariants and special cases.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        L.oracle_create.restype = ctypes.c_void_p
        L.oracle_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ip,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                    dp, ctypes.c_double, ctypes.c_double, dp, dp, dp, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_void_p, ctypes.c_char_p, ctypes.c_int]
        L.oracle_destroy.argtypes = [ctypes.c_void_p]
        L.oracle_step.argtypes = [ctypes.c_void_p, ctypes.c_int64]
        L.oracle_macroscopic.argtypes = [ctypes.c_void_p, dp, dp]
        L.oracle_nfluid.restype = ctypes.c_int64
        L.oracle_nfluid.argtypes = [ctypes.c_void_p]
        L.oracle_time.restype = ctypes.c_int64
        L.oracle_time.argtypes = [ctypes.c_void_p]
        L.oracle_get_f.argtypes = [ctypes.c_void_p, dp]
        L.oracle_set_f.argtypes = [ctypes.c_void_p, dp]
        L.oracle_set_waveform.restype = ctypes.c_int
        L.oracle_set_waveform.argtypes = [ctypes.c_void_p, dp, dp, ctypes.c_int, ctypes.c_double,
                                          ctypes.c_double]
        L.oracle_waveform.restype = ctypes.c_double
        L.oracle_waveform.argtypes = [dp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double]
        L.oracle_init_equilibrium.argtypes = [ctypes.c_void_p, dp, dp]
        L.oracle_apply_velocity_correction.argtypes = [ctypes.c_void_p, dp]
        L.oracle_set_threads.argtypes = [ctypes.c_int]
        L.oracle_get_threads.restype = ctypes.c_int
        L.oracle_stencil.argtypes = [ip, dp]
        L.oracle_feq_product.argtypes = [ctypes.c_double, dp, dp]
        L.oracle_feq_hermite.argtypes = [ctypes.c_double, dp, dp]
        L.oracle_hermite_tensor.argtypes = [ctypes.c_int, ip, dp, dp]
        L.oracle_chm_matrix.argtypes = [dp, dp]
        L.oracle_chm_inverse_matrix.argtypes = [dp, dp]
        L.oracle_rates.argtypes = [ctypes.c_double, dp, dp]
        L.oracle_collide.argtypes = [dp, dp, dp, dp]
        L.oracle_bgk.argtypes = [dp, ctypes.c_double, dp]
        L.oracle_zouhe.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ctypes.c_double]
        L.oracle_feq2.argtypes = [ctypes.c_double, dp, dp]
        L.oracle_collide_srt2.argtypes = [dp, dp, ctypes.c_double, dp]
        L.oracle_collide_trt2.argtypes = [dp, dp, ctypes.c_double, ctypes.c_double, dp]
        L.oracle_trt_minus_rate.restype = ctypes.c_double
        L.oracle_trt_minus_rate.argtypes = [ctypes.c_double, ctypes.c_double]
        L.oracle_set_collision.restype = ctypes.c_int
        L.oracle_set_collision.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double]
        _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


# ---------------------------------------------------------------- single-node functions
def stencil():
    c = np.zeros((27, 3), np.int32)
    w = np.zeros(27)
    lib().oracle_stencil(c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                         w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return c, w


def feq_product(rho, u):
    out = np.zeros(27)
    u, up = _d(u)
    lib().oracle_feq_product(float(rho), up, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def feq_hermite(rho, u):
    out = np.zeros(27)
    u, up = _d(u)
    lib().oracle_feq_hermite(float(rho), up, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def hermite_tensor(idx, x):
    idx, ip = _i(idx)
    x, xp = _d(x)
    out = np.zeros(1)
    lib().oracle_hermite_tensor(len(idx), ip, xp, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return float(out[0])


def chm_matrix(u):
    T = np.zeros((27, 27))
    u, up = _d(u)
    lib().oracle_chm_matrix(up, T.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return T


def chm_inverse_matrix(u):
    T = np.zeros((27, 27))
    u, up = _d(u)
    lib().oracle_chm_inverse_matrix(up, T.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return T


def rates(tau, omega_hi=(1.0, 1.0, 1.0, 1.0)):
    s = np.zeros(27)
    oh, ohp = _d(omega_hi)
    lib().oracle_rates(float(tau), ohp, s.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return s


def collide(f, g, s):
    f, fp = _d(f)
    g, gp = _d(g)
    s, sp = _d(s)
    out = np.zeros(27)
    lib().oracle_collide(fp, gp, sp, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def bgk(f, tau):
    f, fp = _d(f)
    out = np.zeros(27)
    lib().oracle_bgk(fp, float(tau), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def feq2(rho, u):
    out = np.zeros(27)
    u, up = _d(u)
    lib().oracle_feq2(float(rho), up, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def collide_srt2(f, g, tau):
    f, fp = _d(f)
    g, gp = _d(g)
    out = np.zeros(27)
    lib().oracle_collide_srt2(fp, gp, float(tau), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def collide_trt2(f, g, tau, magic):
    f, fp = _d(f)
    g, gp = _d(g)
    out = np.zeros(27)
    lib().oracle_collide_trt2(fp, gp, float(tau), float(magic), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def trt_minus_rate(tau, magic):
    return float(lib().oracle_trt_minus_rate(float(tau), float(magic)))


COLLISIONS = {"chm": 0, "srt2": 1, "trt2": 2}


def zouhe(f, axis, sign, is_inlet, u_in=(0.0, 0.0, 0.0), rho_out=1.0):
    f = np.array(f, dtype=np.float64, copy=True)
    u_in, up = _d(u_in)
    lib().oracle_zouhe(f.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(axis), int(sign),
                       int(bool(is_inlet)), up, float(rho_out))
    return f


def waveform(a, b, period, u_peak, t):
    a, ap = _d(a)
    b_arr = np.asarray(b, dtype=np.float64)
    b_arr, bp = _d(b_arr if b_arr.size else np.zeros(1))
    return lib().oracle_waveform(ap, bp, len(a) - 1, float(period), float(u_peak), float(t))


def set_threads(n):
    lib().oracle_set_threads(int(n))


def get_threads():
    return int(lib().oracle_get_threads())


# ---------------------------------------------------------------- whole case
class Case:
    """A voxel-box case advanced by the oracle.

    mask: uint8 array of shape (nz, ny, nx) (x fastest in memory): 0 solid, 1 fluid,
    2 inlet, 3 outlet.  links: (cell, beta, q) arrays -- box linear index of the fluid cell,
    the direction pointing into the wall, and the wall fraction q in (0, 1].
    """

    def __init__(self, mask, periodic=(0, 0, 0), links=None, inlet_center=(0.0, 0.0, 0.0),
                 inlet_radius=1.0, tau=0.6, omega_hi=(1.0, 1.0, 1.0, 1.0), g0=(0.0, 0.0, 0.0),
                 gamp=(0.0, 0.0, 0.0), gomega=0.0, rho_out=1.0, tau_cell=None, collision="chm",
                 trt_magic=3.0 / 16.0):
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
        assert mask.ndim == 3
        self.shape = mask.shape
        nz, ny, nx = mask.shape
        self._mask = mask
        per, perp = _i(periodic)
        if links is None:
            lc = np.zeros(0, np.int64)
            ld = np.zeros(0, np.uint8)
            lq = np.zeros(0, np.float64)
        else:
            lc = np.ascontiguousarray(links[0], dtype=np.int64)
            ld = np.ascontiguousarray(links[1], dtype=np.uint8)
            lq = np.ascontiguousarray(links[2], dtype=np.float64)
        self._keep = (lc, ld, lq)
        ic, icp = _d(inlet_center)
        oh, ohp = _d(omega_hi)
        g0a, g0p = _d(g0)
        ga, gap = _d(gamp)
        err = ctypes.create_string_buffer(256)
        tc = None if tau_cell is None else np.ascontiguousarray(tau_cell, dtype=np.float64).reshape(-1)
        self._tc = tc
        h = lib().oracle_create(nx, ny, nz, mask.ctypes.data, perp, lc.ctypes.data, ld.ctypes.data,
                                lq.ctypes.data, len(lc), icp, float(inlet_radius), float(tau), ohp,
                                g0p, gap, float(gomega), float(rho_out),
                                None if tc is None else tc.ctypes.data, err, 256)
        if not h:
            raise ValueError("oracle_create: " + err.value.decode())
        self._h = h
        if lib().oracle_set_collision(h, COLLISIONS[collision], float(trt_magic)) != 0:
            raise ValueError("bad collision model or magic parameter")

    def __del__(self):
        if getattr(self, "_h", None):
            lib().oracle_destroy(self._h)
            self._h = None

    @property
    def nfluid(self):
        return int(lib().oracle_nfluid(self._h))

    @property
    def time(self):
        return int(lib().oracle_time(self._h))

    def set_waveform(self, a, b, period, u_peak):
        a, ap = _d(a)
        b_arr = np.asarray(b, dtype=np.float64)
        b_arr, bp = _d(b_arr if b_arr.size else np.zeros(1))
        rc = lib().oracle_set_waveform(self._h, ap, bp, len(a) - 1, float(period), float(u_peak))
        if rc != 0:
            raise ValueError("oracle_set_waveform: bad arguments")

    def step(self, n=1):
        lib().oracle_step(self._h, int(n))

    def macroscopic(self):
        nz, ny, nx = self.shape
        rho = np.zeros(nx * ny * nz)
        u = np.zeros(3 * nx * ny * nz)
        lib().oracle_macroscopic(self._h, rho.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                 u.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return rho.reshape(nz, ny, nx), u.reshape(3, nz, ny, nx)

    def init_equilibrium(self, rho, u):
        """Post-collision populations of the previous time level := f_eq(rho, u) on every
        fluid cell, then streamed and closed (rho: (nz,ny,nx), u: (3,nz,ny,nx))."""
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
        lib().oracle_init_equilibrium(self._h, rho.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      u.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))

    def apply_velocity_correction(self, du):
        """Post-collision populations of the previous level += f_eq(rho, u + du) - f_eq(rho, u)
        at every fluid cell (rho, u of the current level), then re-streamed and re-closed;
        du: (3, nz, ny, nx)."""
        du = np.ascontiguousarray(du, dtype=np.float64).reshape(-1)
        lib().oracle_apply_velocity_correction(self._h, du.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))

    def get_f(self):
        out = np.zeros((self.nfluid, 27))
        lib().oracle_get_f(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return out

    def set_f(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.shape == (self.nfluid, 27)
        lib().oracle_set_f(self._h, f.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
