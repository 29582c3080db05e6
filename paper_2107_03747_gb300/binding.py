"""Thin ctypes binding of libtgf (include/tgf.h): the same entry points, argument marshalling only.

Device buffers are torch tensors (the caller owns them); streams are torch streams.  Every
call raises ``TgfError`` with the library's message when the status is not TGF_OK.  The
library must be built first (``paper_2107_03747_gb300.build.build()``); importing this
module without it raises, there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
# TGF_LIB_PATH selects another build of the same library (kernel-variant sweeps of the tuner)
LIB_PATH = os.environ.get("TGF_LIB_PATH", os.path.join(PKG, "libtgf.so"))

TGF_OK, TGF_EINVAL, TGF_ENOMEM, TGF_ECUDA, TGF_EKERNEL, TGF_ESTATE, TGF_EIO = 0, 1, 2, 3, 4, 6, 7
TGF_FP64, TGF_FP32, TGF_FP32_R12 = 0, 1, 2
TGF_CLOVER_TRACELESS = 1
TGF_NO_GRAPH = 2
TGF_SYNC = 4
TGF_ANY_EXTENTS = 1
TGF_MAX_CFG = 256
TGF_FMA_PEAK_FP32X2, TGF_FMA_PEAK_FP32_MIXED = 3, 4
PRECISIONS = {"fp64": TGF_FP64, "fp32": TGF_FP32, "fp32_r12": TGF_FP32_R12}


class TgfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"tgf status {status}: {msg}")
        self.status = status


class tgf_lattice(C.Structure):
    _fields_ = [("L", C.c_int * 4), ("twist", C.c_int * 6), ("flags", C.c_uint)]


class tgf_obs(C.Structure):
    _fields_ = [("t", C.c_double), ("E", C.c_double), ("Q", C.c_double), ("P", C.c_double), ("S", C.c_double)]


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with paper_2107_03747_gb300.build.build()")
_lib = C.CDLL(LIB_PATH)

_P = C.c_void_p
_SZ = C.c_size_t
_LATP = C.POINTER(tgf_lattice)
_SIGS = {
    "tgf_links_bytes": [C.c_int, _LATP, C.c_int, C.POINTER(_SZ)],
    "tgf_accum_bytes": [C.c_int, _LATP, C.c_int, C.POINTER(_SZ)],
    "tgf_scratch_bytes": [C.c_int, _LATP, C.c_int, C.POINTER(_SZ)],
    "tgf_canonical_bytes": [_LATP, C.POINTER(_SZ)],
    "tgf_pack": [C.c_int, _LATP, C.c_int, _P, _P, _P],
    "tgf_unpack": [C.c_int, _LATP, C.c_int, _P, _P, _P],
    "tgf_upload": [C.c_int, _LATP, C.c_int, _P, _P, _SZ, _P, _P],
    "tgf_download": [C.c_int, _LATP, C.c_int, _P, _P, _SZ, _P, _P],
    "tgf_stage": [C.c_int, _LATP, C.c_int, _P, _P, _P, C.c_int, C.c_double, C.c_int, C.c_uint, _P],
    "tgf_measure": [C.c_int, _LATP, C.c_int, _P, _P, _SZ, _P, _SZ, C.c_int, C.c_double, C.c_uint, _P],
    "tgf_flow": [C.c_int, _LATP, C.c_int, _P, _P, _P, _P, _SZ, C.c_double, C.POINTER(C.c_double), C.c_int,
                 C.c_int, C.c_uint, _P, _SZ, C.POINTER(C.c_int), _P],
    "tgf_flow_records": [C.c_double, C.c_double, C.c_int, C.POINTER(C.c_int)],
    "tgf_measure_slices": [C.c_int, _LATP, C.c_int, _P, _P, _SZ, C.c_int, _P, _SZ, C.c_uint, _P],
    "tgf_slice_correlator": [C.POINTER(C.c_double), _SZ, C.POINTER(C.c_double), C.c_int, C.c_int,
                             C.POINTER(C.c_double), C.POINTER(C.c_int)],
    "tgf_measure_noalloc": [C.c_int, _LATP, C.c_int, _P, _P, _SZ, C.c_int, C.c_double, C.c_uint, _P],
    "tgf_sun_links_bytes": [C.c_int, _LATP, C.c_int, C.POINTER(_SZ)],
    "tgf_sun_accum_bytes": [C.c_int, _LATP, C.c_int, C.POINTER(_SZ)],
    "tgf_sun_scratch_bytes": [C.c_int, _LATP, C.c_int, C.POINTER(_SZ)],
    "tgf_sun_pack": [C.c_int, _LATP, C.c_int, _P, _P, _P],
    "tgf_sun_unpack": [C.c_int, _LATP, C.c_int, _P, _P, _P],
    "tgf_sun_stage": [C.c_int, _LATP, C.c_int, _P, _P, _P, C.c_int, C.c_double, _P],
    "tgf_sun_measure": [C.c_int, _LATP, C.c_int, _P, _P, _SZ, _P, _SZ, C.c_int, C.c_double, C.c_uint, _P],
    "tgf_mc_sweeps": [C.c_int, _LATP, C.c_int, _P, C.c_double, C.c_int, C.c_int, C.c_ulonglong, C.c_ulonglong, _P],
    "tgf_save": [C.c_char_p, C.c_int, _LATP, C.c_int, _P, _P, _SZ, C.c_double, C.c_longlong, C.c_ulonglong, _P],
    "tgf_load": [C.c_char_p, C.c_int, _LATP, C.c_int, _P, _P, _SZ, C.POINTER(C.c_double), C.POINTER(C.c_longlong),
                 C.POINTER(C.c_ulonglong), _P],
    "tgf_check_errors": [C.POINTER(C.c_uint)],
    "tgf_kernel_status": [_P],
    "tgf_create": [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_int, _LATP, C.c_int, C.c_uint],
    "tgf_set_links": [C.c_void_p, C.c_int, _P, _SZ],
    "tgf_set_links_device": [C.c_void_p, C.c_int, _P, _SZ, _P],
    "tgf_get_links": [C.c_void_p, C.c_int, _P, _SZ],
    "tgf_ctx_measure": [C.c_void_p, C.c_double, _P, _P],
    "tgf_ctx_flow": [C.c_void_p, C.c_double, C.POINTER(C.c_double), C.c_int, _P, _SZ, C.POINTER(C.c_int), _P],
    "tgf_ctx_save": [C.c_void_p, C.c_char_p, C.c_double, C.c_longlong, C.c_ulonglong],
    "tgf_ctx_load": [C.c_void_p, C.c_char_p, C.POINTER(C.c_double), C.POINTER(C.c_longlong), C.POINTER(C.c_ulonglong)],
    "tgf_norm": [C.c_double, C.c_int, C.c_int, C.POINTER(C.c_double)],
    "tgf_fma_peak": [C.c_int, _P, C.c_int, C.c_int, C.POINTER(C.c_double), _P],
    "tgf_lambda": [C.c_double, C.c_int, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int,
                   C.POINTER(C.c_double), C.POINTER(C.c_int)],
}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = C.c_int
_lib.tgf_crc32.restype = C.c_uint
_lib.tgf_crc32.argtypes = [C.c_void_p, C.c_size_t]
_lib.tgf_last_error.restype = C.c_char_p
_lib.tgf_last_error.argtypes = []
_lib.tgf_status_string.restype = C.c_char_p
_lib.tgf_status_string.argtypes = [C.c_int]
_lib.tgf_version.restype = C.c_char_p
_lib.tgf_version.argtypes = []
_lib.tgf_destroy.restype = None
_lib.tgf_destroy.argtypes = [C.c_void_p]

EXPORTED = sorted(list(_SIGS) + ["tgf_last_error", "tgf_status_string", "tgf_version", "tgf_crc32", "tgf_destroy"])


def _check(status: int):
    if status != TGF_OK:
        raise TgfError(status, _lib.tgf_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def lattices(Ls, twists=None, any_extents=False):
    """ctypes array of tgf_lattice from extents (L0, L1, L2, L3) and twist 6-tuples (default n_01 = 1).

    The library accepts only the paper's box (l, l, 3l, 3l) (SU(N): (l, l, Nl, Nl)) unless
    `any_extents` sets TGF_ANY_EXTENTS."""
    n = len(Ls)
    arr = (tgf_lattice * n)()
    for i, L in enumerate(Ls):
        arr[i].L[:] = [int(x) for x in L]
        tw = (1, 0, 0, 0, 0, 0) if twists is None else twists[i]
        arr[i].twist[:] = [int(x) for x in tw]
        arr[i].flags = TGF_ANY_EXTENTS if any_extents else 0
    return arr


def twist6(n):
    """Six upper entries (01, 02, 03, 12, 13, 23) of a 4x4 antisymmetric twist tensor."""
    return tuple(int(n[a][b]) for a, b in ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)))


def version() -> str:
    return _lib.tgf_version().decode()


def status_string(s: int) -> str:
    return _lib.tgf_status_string(s).decode()


def tgf_links_bytes(prec, lat) -> int:
    out = _SZ()
    _check(_lib.tgf_links_bytes(prec, lat, len(lat), C.byref(out)))
    return out.value


def tgf_accum_bytes(prec, lat) -> int:
    out = _SZ()
    _check(_lib.tgf_accum_bytes(prec, lat, len(lat), C.byref(out)))
    return out.value


def tgf_scratch_bytes(prec, lat) -> int:
    out = _SZ()
    _check(_lib.tgf_scratch_bytes(prec, lat, len(lat), C.byref(out)))
    return out.value


def tgf_canonical_bytes(lat1) -> int:
    out = _SZ()
    _check(_lib.tgf_canonical_bytes(lat1, C.byref(out)))
    return out.value


def tgf_pack(prec, lat, canon_dev, links, stream=None):
    _check(_lib.tgf_pack(prec, lat, len(lat), _ptr(canon_dev), _ptr(links), _stream(stream)))


def tgf_unpack(prec, lat, links, canon_dev, stream=None):
    _check(_lib.tgf_unpack(prec, lat, len(lat), _ptr(links), _ptr(canon_dev), _stream(stream)))


def tgf_upload(prec, lat, canon_host, staging, links, stream=None):
    """canon_host: a (pinned) CPU tensor or numpy complex128 array in canonical layout."""
    p = canon_host.ctypes.data if isinstance(canon_host, np.ndarray) else canon_host.data_ptr()
    _check(_lib.tgf_upload(prec, lat, len(lat), p, _ptr(staging), staging.numel() * staging.element_size(),
                           _ptr(links), _stream(stream)))


def tgf_download(prec, lat, links, staging, canon_host, stream=None):
    p = canon_host.ctypes.data if isinstance(canon_host, np.ndarray) else canon_host.data_ptr()
    _check(_lib.tgf_download(prec, lat, len(lat), _ptr(links), _ptr(staging),
                             staging.numel() * staging.element_size(), p, _stream(stream)))


def tgf_stage(prec, lat, w_in, w_out, accum, stage, eps, reunit=0, flags=0, stream=None):
    _check(_lib.tgf_stage(prec, lat, len(lat), _ptr(w_in), _ptr(w_out), _ptr(accum), stage, eps, reunit, flags,
                          _stream(stream)))


def tgf_measure(prec, lat, links, scratch, obs_dev, obs_stride, rec, t, flags=0, stream=None):
    _check(_lib.tgf_measure(prec, lat, len(lat), _ptr(links), _ptr(scratch),
                            scratch.numel() * scratch.element_size(), _ptr(obs_dev), obs_stride, rec, t, flags,
                            _stream(stream)))


def tgf_measure_noalloc(prec, lat, links, obs_dev, obs_stride, rec, t, flags=0, stream=None):
    """tgf_measure with the library's fixed device scratch (no caller scratch, no allocation)."""
    _check(_lib.tgf_measure_noalloc(prec, lat, len(lat), _ptr(links), _ptr(obs_dev), obs_stride, rec, t, flags,
                                    _stream(stream)))


def tgf_measure_slices(prec, lat, links, scratch, dir, q_dev, q_stride, flags=0, stream=None):
    _check(_lib.tgf_measure_slices(prec, lat, len(lat), _ptr(links), _ptr(scratch),
                                   scratch.numel() * scratch.element_size(), dir, _ptr(q_dev), q_stride, flags,
                                   _stream(stream)))


def tgf_slice_correlator(q, Q):
    """q: (ncfg, T) array of slice charges, Q: (ncfg,) charges -> (C over d = 0..T-1, kept) or (None, 0)."""
    q = np.ascontiguousarray(np.asarray(q, dtype=np.float64))
    Qa = np.ascontiguousarray(np.asarray(Q, dtype=np.float64))
    n, T = q.shape
    out = np.zeros(T)
    kept = C.c_int()
    s = _lib.tgf_slice_correlator(q.ctypes.data_as(C.POINTER(C.c_double)), T, Qa.ctypes.data_as(C.POINTER(C.c_double)),
                                  n, T, out.ctypes.data_as(C.POINTER(C.c_double)), C.byref(kept))
    if s == TGF_ESTATE:
        return None, 0
    _check(s)
    return out, kept.value


def tgf_flow_records(eps, t_end, measure_every=1) -> int:
    out = C.c_int()
    _check(_lib.tgf_flow_records(eps, t_end, measure_every, C.byref(out)))
    return out.value


def tgf_flow(prec, lat, w, w_tmp, accum, scratch, eps, t_end, obs_dev, obs_cap, measure_every=1,
             reunit_every=0, flags=0, stream=None):
    """Returns the number of records written per configuration (list)."""
    n = len(lat)
    te = (C.c_double * n)(*[float(x) for x in t_end])
    nrec = (C.c_int * n)()
    _check(_lib.tgf_flow(prec, lat, n, _ptr(w), _ptr(w_tmp), _ptr(accum), _ptr(scratch),
                         scratch.numel() * scratch.element_size(), eps, te, measure_every, reunit_every, flags,
                         _ptr(obs_dev), obs_cap, nrec, _stream(stream)))
    return list(nrec)


def tgf_fma_peak(prec, blocks_per_sm=8, iters=4096, stream=None) -> float:
    """Measured FMA-pipe peak (TFLOP/s) of the current device for TGF_FP32 or TGF_FP64."""
    import torch

    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    sink = torch.empty(nsm * blocks_per_sm, dtype=torch.float64, device="cuda")
    out = C.c_double()
    _check(_lib.tgf_fma_peak(prec, _ptr(sink), blocks_per_sm, iters, C.byref(out), _stream(stream)))
    return out.value


def tgf_mc_sweeps(prec, lat, links, beta, n_hybrid, n_or, seed, first_sweep, stream=None):
    """n_hybrid hybrid sweeps (1 heat-bath + n_or over-relaxation each) of FP64 `links`, in place."""
    _check(_lib.tgf_mc_sweeps(prec, lat, len(lat), _ptr(links), float(beta), int(n_hybrid), int(n_or),
                              int(seed) & 0xFFFFFFFFFFFFFFFF, int(first_sweep), _stream(stream)))


def _sun_size(fn, N, lat) -> int:
    n = _SZ()
    _check(fn(N, lat, len(lat), C.byref(n)))
    return n.value


class SunBatch:
    """SU(N) configurations (FP64) with their device buffers: links, the ping-pong buffer, X, scratch."""

    def __init__(self, N, Ls, twists=None, device="cuda", any_extents=False):
        import torch

        self.N, self.Ls, self.device = N, [tuple(L) for L in Ls], device
        self.lat = lattices(self.Ls, twists, any_extents)
        nb = _sun_size(_lib.tgf_sun_links_bytes, N, self.lat)
        self.links = torch.empty(nb, dtype=torch.uint8, device=device)
        self.links_tmp = torch.empty(nb, dtype=torch.uint8, device=device)
        self.accum = torch.empty(_sun_size(_lib.tgf_sun_accum_bytes, N, self.lat), dtype=torch.uint8, device=device)
        self.scratch = torch.empty(_sun_size(_lib.tgf_sun_scratch_bytes, N, self.lat), dtype=torch.uint8, device=device)

    def set_links(self, fields, stream=None):
        import torch

        flat = np.concatenate([np.ascontiguousarray(f).view(np.float64).reshape(-1) for f in fields])
        canon = torch.from_numpy(flat).to(self.device)
        _check(_lib.tgf_sun_pack(self.N, self.lat, len(self.lat), _ptr(canon), _ptr(self.links), _stream(stream)))
        return canon

    def get_links(self, stream=None):
        import torch

        N = self.N
        n = sum(L[0] * L[1] * L[2] * L[3] * 4 * N * N * 2 for L in self.Ls)
        canon = torch.empty(n, dtype=torch.float64, device=self.device)
        _check(_lib.tgf_sun_unpack(N, self.lat, len(self.lat), _ptr(self.links), _ptr(canon), _stream(stream)))
        flat = canon.cpu().numpy()
        out, off = [], 0
        for L in self.Ls:
            m = L[0] * L[1] * L[2] * L[3] * 4 * N * N * 2
            out.append(flat[off:off + m].view(np.complex128).reshape(L[3], L[2], L[1], L[0], 4, N, N))
            off += m
        return out

    def stage(self, stage, eps, stream=None):
        _check(_lib.tgf_sun_stage(self.N, self.lat, len(self.lat), _ptr(self.links), _ptr(self.links_tmp),
                                  _ptr(self.accum), stage, eps, _stream(stream)))
        self.links, self.links_tmp = self.links_tmp, self.links

    def step(self, eps, stream=None):
        for s in (1, 2, 3):
            self.stage(s, eps, stream)

    def measure(self, t=0.0, flags=0, stream=None):
        """{t, E, Q, P, S} per configuration as an (ncfg, 5) numpy array."""
        import torch

        n = len(self.lat)
        obs = torch.zeros(n * 5, dtype=torch.float64, device=self.device)
        _check(_lib.tgf_sun_measure(self.N, self.lat, n, _ptr(self.links), _ptr(self.scratch),
                                    self.scratch.numel(), _ptr(obs), 1, 0, t, flags, _stream(stream)))
        return obs.cpu().numpy().reshape(n, 5)


def tgf_kernel_status(stream=None):
    """Synchronise `stream`; raises TgfError(TGF_EKERNEL) if a record came out non-finite since the last check."""
    _check(_lib.tgf_kernel_status(_stream(stream)))


def tgf_check_errors() -> int:
    """Bits of the kernel files that recorded an out-of-range site index (self-checking builds)."""
    b = C.c_uint()
    _check(_lib.tgf_check_errors(C.byref(b)))
    return b.value


def tgf_crc32(data: bytes) -> int:
    return int(_lib.tgf_crc32(data, len(data)))


def tgf_save(path, prec, lat, links, staging, t, step, seed, stream=None):
    """Checkpoint `links` (canonical FP64 + t, step, seed, CRC-32) to `path`; synchronises `stream`."""
    _check(_lib.tgf_save(str(path).encode(), prec, lat, len(lat), _ptr(links), _ptr(staging),
                         staging.numel() * staging.element_size(), float(t), int(step),
                         int(seed) & 0xFFFFFFFFFFFFFFFF, _stream(stream)))


def tgf_load(path, prec, lat, links, staging, stream=None):
    """Load a checkpoint into `links`; returns (t, step, seed)."""
    t, step, seed = C.c_double(), C.c_longlong(), C.c_ulonglong()
    _check(_lib.tgf_load(str(path).encode(), prec, lat, len(lat), _ptr(links), _ptr(staging),
                         staging.numel() * staging.element_size(), C.byref(t), C.byref(step), C.byref(seed),
                         _stream(stream)))
    return t.value, step.value, seed.value


def tgf_norm(c, Lt, N=3) -> float:
    out = C.c_double()
    _check(_lib.tgf_norm(c, Lt, N, C.byref(out)))
    return out.value


def tgf_lambda(c, Lt, t, E, Q):
    """(lambda, n_kept); lambda is None when no configuration has |Q| < 1/2."""
    n = len(E)
    Ea = (C.c_double * n)(*[float(x) for x in E])
    Qa = (C.c_double * n)(*[float(x) for x in Q])
    lam = C.c_double()
    kept = C.c_int()
    s = _lib.tgf_lambda(c, Lt, t, Ea, Qa, n, C.byref(lam), C.byref(kept))
    if s == TGF_ESTATE:
        return None, 0
    _check(s)
    return lam.value, kept.value


# ---------------------------------------------------------------------------------------------
# convenience: a batch of configurations with its device buffers (torch tensors)
# ---------------------------------------------------------------------------------------------

class FlowBatch:
    """Device buffers for flowing a batch of configurations in one precision.

    ``links`` holds the current field; ``links_tmp`` and ``accum`` are the RK3 work buffers;
    ``scratch`` the measurement partials.  All are torch uint8 tensors on ``device``.
    """

    def __init__(self, Ls, prec="fp64", twists=None, device="cuda", any_extents=False):
        import torch

        self.prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
        self.lat = lattices(Ls, twists, any_extents)
        self.Ls = [tuple(int(x) for x in L) for L in Ls]
        self.device = torch.device(device)
        nb = tgf_links_bytes(self.prec, self.lat)
        self.links = torch.empty(nb, dtype=torch.uint8, device=self.device)
        self.links_tmp = torch.empty(nb, dtype=torch.uint8, device=self.device)
        self.accum = torch.empty(tgf_accum_bytes(self.prec, self.lat), dtype=torch.uint8, device=self.device)
        self.scratch = torch.empty(tgf_scratch_bytes(self.prec, self.lat), dtype=torch.uint8,
                                   device=self.device)

    @property
    def ncfg(self):
        return len(self.Ls)

    def canonical_numel(self):
        return sum(L[0] * L[1] * L[2] * L[3] * 72 for L in self.Ls)

    def set_links(self, fields, stream=None):
        """fields: list of complex128 numpy arrays in canonical layout, one per configuration."""
        import torch

        flat = np.concatenate([np.ascontiguousarray(f).view(np.float64).reshape(-1) for f in fields])
        canon = torch.from_numpy(flat).to(self.device)
        tgf_pack(self.prec, self.lat, canon, self.links, stream)
        return canon

    def set_links_device(self, canon_dev, stream=None):
        tgf_pack(self.prec, self.lat, canon_dev, self.links, stream)

    def get_links(self, stream=None):
        """Current fields as complex128 numpy arrays in canonical layout."""
        import torch

        canon = torch.empty(self.canonical_numel(), dtype=torch.float64, device=self.device)
        tgf_unpack(self.prec, self.lat, self.links, canon, stream)
        flat = canon.cpu().numpy()
        out, off = [], 0
        for L in self.Ls:
            n = L[0] * L[1] * L[2] * L[3] * 72
            out.append(flat[off:off + n].view(np.complex128).reshape(L[3], L[2], L[1], L[0], 4, 3, 3))
            off += n
        return out

    def measure(self, t=0.0, flags=0, stream=None):
        """{t, E, Q, P, S} per configuration as an (ncfg, 5) numpy array."""
        import torch

        obs = torch.zeros(self.ncfg * 5, dtype=torch.float64, device=self.device)
        tgf_measure(self.prec, self.lat, self.links, self.scratch, obs, 1, 0, t, flags, stream)
        return obs.cpu().numpy().reshape(self.ncfg, 5)

    def slices(self, direction=3, flags=0, stream=None):
        """q(x, t) per configuration along `direction` as a list of numpy arrays."""
        import torch

        T = max(L[direction] for L in self.Ls)
        q = torch.zeros(self.ncfg * T, dtype=torch.float64, device=self.device)
        tgf_measure_slices(self.prec, self.lat, self.links, self.scratch, direction, q, T, flags, stream)
        qn = q.cpu().numpy().reshape(self.ncfg, T)
        return [qn[c, : L[direction]].copy() for c, L in enumerate(self.Ls)]

    def stage(self, stage, eps, reunit=0, stream=None):
        """One RK3 stage from ``links`` into ``links_tmp``; then the two are swapped."""
        tgf_stage(self.prec, self.lat, self.links, self.links_tmp, self.accum, stage, eps, reunit, 0, stream)
        self.links, self.links_tmp = self.links_tmp, self.links

    def flow(self, eps, t_end, measure_every=1, reunit_every=0, flags=0, stream=None, obs=None):
        """Flow every configuration to t_end (scalar or per-configuration list).

        Returns (obs tensor of shape (ncfg, cap, 5) on the device, records per configuration).
        """
        import torch

        te = [float(t_end)] * self.ncfg if np.isscalar(t_end) else [float(x) for x in t_end]
        cap = max(tgf_flow_records(eps, t, measure_every) for t in te)
        if obs is None or obs.numel() < self.ncfg * cap * 5:
            obs = torch.zeros(self.ncfg * cap * 5, dtype=torch.float64, device=self.device)
        nrec = tgf_flow(self.prec, self.lat, self.links, self.links_tmp, self.accum, self.scratch, eps, te, obs,
                        cap, measure_every, reunit_every, flags, stream)
        return obs[: self.ncfg * cap * 5].view(self.ncfg, cap, 5), nrec


class Context:
    """The library-owned context (tgf_create ... tgf_destroy): the library allocates and owns the
    batch's device memory; fields go in and out as canonical complex128 numpy arrays."""

    def __init__(self, Ls, prec="fp64", twists=None, device=0, reunit_every=0, flags=0, any_extents=False):
        self.prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
        self.Ls = [tuple(int(x) for x in L) for L in Ls]
        self.lat = lattices(self.Ls, twists, any_extents)
        self._h = C.c_void_p()
        _check(_lib.tgf_create(C.byref(self._h), int(device), self.prec, len(self.Ls), self.lat, int(reunit_every),
                               int(flags)))

    def close(self):
        if self._h:
            _lib.tgf_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_links(self, cfg, field):
        f = np.ascontiguousarray(field, dtype=np.complex128)
        _check(_lib.tgf_set_links(self._h, int(cfg), f.ctypes.data, f.size * 2))

    def get_links(self, cfg):
        L = self.Ls[cfg]
        out = np.empty((L[3], L[2], L[1], L[0], 4, 3, 3), dtype=np.complex128)
        _check(_lib.tgf_get_links(self._h, int(cfg), out.ctypes.data, out.size * 2))
        return out

    def measure(self, t=0.0, stream=None):
        out = (tgf_obs * len(self.Ls))()
        _check(_lib.tgf_ctx_measure(self._h, float(t), C.addressof(out), _stream(stream)))
        return np.array([[o.t, o.E, o.Q, o.P, o.S] for o in out])

    def flow(self, eps, t_end, measure_every=1, stream=None):
        """Records as an (ncfg, cap, 5) numpy array and the count per configuration."""
        n = len(self.Ls)
        te = [float(t_end)] * n if np.isscalar(t_end) else [float(x) for x in t_end]
        cap = max(tgf_flow_records(eps, t, measure_every) for t in te)
        out = (tgf_obs * (n * cap))()
        nw = (C.c_int * n)()
        _check(_lib.tgf_ctx_flow(self._h, float(eps), (C.c_double * n)(*te), int(measure_every), C.addressof(out), cap,
                                 nw, _stream(stream)))
        rec = np.array([[o.t, o.E, o.Q, o.P, o.S] for o in out]).reshape(n, cap, 5)
        return rec, list(nw)

    def save(self, path, t, step, seed):
        _check(_lib.tgf_ctx_save(self._h, str(path).encode(), float(t), int(step), int(seed) & 0xFFFFFFFFFFFFFFFF))

    def load(self, path):
        t, step, seed = C.c_double(), C.c_longlong(), C.c_ulonglong()
        _check(_lib.tgf_ctx_load(self._h, str(path).encode(), C.byref(t), C.byref(step), C.byref(seed)))
        return t.value, step.value, seed.value
