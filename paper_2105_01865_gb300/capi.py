"""Thin ctypes binding of libch.so (include/ch.h).

Every function here has the name of the C entry point it wraps and only
marshals arguments: torch tensors are passed as raw device pointers, the
stream as the raw cudaStream_t.  All arithmetic of the step runs in the CUDA
kernels of libch.so; there is no CPU fallback, and loading fails loudly when
the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libch.so")

CH_OK, CH_EINVAL, CH_ECUDA, CH_ENONFINITE, CH_ETIMEOUT, CH_ENOMEM = range(6)
CH_PERIODIC, CH_NOFLUX, CH_DIRICHLET = 0, 1, 2
CH_F32, CH_F64 = 0, 1
CH_SCHEME_SPLIT, CH_SCHEME_STANDARD = 0, 1


class CHError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class ch_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64),
        ("h", ctypes.c_double),
        ("bc", ctypes.c_int32 * 3),
        ("precision", ctypes.c_int32),
        ("cn", ctypes.c_double), ("pe", ctypes.c_double), ("dt", ctypes.c_double),
        ("w", ctypes.c_double), ("weno_eps", ctypes.c_double),
        ("advect", ctypes.c_int32), ("scheme", ctypes.c_int32),
        ("ncx", ctypes.c_int64), ("ncy", ctypes.c_int64), ("ncz", ctypes.c_int64),
        ("xf_coarse", ctypes.POINTER(ctypes.c_double)),
        ("yf_coarse", ctypes.POINTER(ctypes.c_double)),
        ("zf_coarse", ctypes.POINTER(ctypes.c_double)),
    ]


_lib = None

# (name, restype, argtypes) of every entry point declared in include/ch.h
_P = ctypes.c_void_p
SIGNATURES = [
    ("ch_workspace_bytes", ctypes.c_size_t, [ctypes.POINTER(ch_params)]),
    ("ch_create", ctypes.c_int, [ctypes.POINTER(ch_params), _P, _P, ctypes.c_size_t, _P, ctypes.POINTER(_P)]),
    ("ch_free", ctypes.c_int, [_P]),
    ("ch_set_velocity_fine", ctypes.c_int, [_P, _P, _P, _P]),
    ("ch_set_velocity_coarse", ctypes.c_int, [_P, _P, _P, _P]),
    ("ch_interp_to_fine", ctypes.c_int, [_P]),
    ("ch_get_velocity_fine", ctypes.c_int, [_P, _P, _P, _P]),
    ("ch_get_interp_tables", ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    ("ch_profile_interp", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    ("ch_restrict_workspace_bytes", ctypes.c_size_t, [_P]),
    ("ch_restrict_to_coarse", ctypes.c_int, [_P, ctypes.c_double, ctypes.c_double, _P, _P, _P, _P, _P, _P, _P,
                                             ctypes.c_size_t]),
    ("ch_step", ctypes.c_int, [_P, ctypes.c_int64]),
    ("ch_mass", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    ("ch_free_energy", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    ("ch_diagnostics", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    ("ch_sync", ctypes.c_int, [_P]),
    ("ch_launches_per_step", ctypes.c_int, [_P]),
    ("ch_profile_step", ctypes.c_int, [_P, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)]),
    ("ch_mass_noalloc", ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                        ctypes.c_int, _P, _P]),
    ("ch_adjoint_workspace_bytes", ctypes.c_size_t, [_P, ctypes.c_int64, ctypes.c_int64]),
    ("ch_step_adjoint", ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_int64, _P, _P, ctypes.POINTER(ctypes.c_double),
                                       _P, ctypes.c_size_t]),
    ("ch_batch_workspace_bytes", ctypes.c_size_t, [ctypes.POINTER(ch_params), ctypes.c_int]),
    ("ch_batch_create", ctypes.c_int, [ctypes.POINTER(ch_params), ctypes.c_int, ctypes.POINTER(_P), _P, ctypes.c_size_t,
                                       _P, ctypes.POINTER(_P)]),
    ("ch_batch_step", ctypes.c_int, [_P, ctypes.c_int64]),
    ("ch_batch_mass", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    ("ch_batch_sync", ctypes.c_int, [_P]),
    ("ch_batch_set_schedule", ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    ("ch_batch_get_schedule", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    ("ch_batch_autotune", ctypes.c_int, [_P, ctypes.c_int, ctypes.c_char_p, ctypes.c_size_t]),
    ("ch_batch_set_barrier_limit", ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int]),
    ("ch_batch_launches_per_step", ctypes.c_int, [_P]),
    ("ch_batch_free", ctypes.c_int, [_P]),
    ("ch_batch_last_error", ctypes.c_char_p, [_P]),
    ("ch_error_string", ctypes.c_char_p, [ctypes.c_int]),
    ("ch_last_error", ctypes.c_char_p, [_P]),
]


def load():
    """Load libch.so (built by paper_2105_01865_gb300.build).  Raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                              "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(status, handle=None, what=""):
    if status != CH_OK:
        lib = load()
        msg = lib.ch_last_error(handle).decode() if handle else ""
        raise CHError(status, f"{what}: {lib.ch_error_string(status).decode()} {msg}".strip())


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def make_params(shape, h, bc, cn, pe, dt, precision=CH_F32, w=4.0, weno_eps=1e-6, advect=False, coarse_faces=None,
                scheme=0):
    """Fill a ch_params.  shape = (nz, ny, nx); coarse_faces = (xf, yf, zf) numpy arrays or None;
    scheme = CH_SCHEME_SPLIT (0) or CH_SCHEME_STANDARD (1).
    The returned object keeps the coarse arrays alive as attribute ``_keep``."""
    nz, ny, nx = shape
    p = ch_params()
    p.nx, p.ny, p.nz = nx, ny, nz
    p.h = h
    p.bc[0], p.bc[1], p.bc[2] = bc
    p.precision = precision
    p.cn, p.pe, p.dt, p.w, p.weno_eps = cn, pe, dt, w, weno_eps
    p.advect = 1 if advect else 0
    p.scheme = scheme
    keep = []
    if coarse_faces is not None:
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in coarse_faces]
        keep = arrs
        p.ncx, p.ncy, p.ncz = (len(a) - 1 for a in arrs)
        p.xf_coarse, p.yf_coarse, p.zf_coarse = (a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for a in arrs)
    p._keep = keep
    return p


def ch_workspace_bytes(params):
    return int(load().ch_workspace_bytes(ctypes.byref(params)))


def ch_create(params, C, work, stream):
    """C, work: torch CUDA tensors; stream: torch.cuda.Stream.  Returns the handle."""
    lib = load()
    out = ctypes.c_void_p()
    st = lib.ch_create(ctypes.byref(params), _ptr(C), _ptr(work), work.numel() * work.element_size(),
                       ctypes.c_void_p(stream.cuda_stream), ctypes.byref(out))
    _check(st, None, "ch_create")
    return out


def ch_free(handle):
    _check(load().ch_free(handle), None, "ch_free")


def ch_set_velocity_fine(handle, u, v, w):
    _check(load().ch_set_velocity_fine(handle, _ptr(u), _ptr(v), _ptr(w)), handle, "ch_set_velocity_fine")


def ch_set_velocity_coarse(handle, uc, vc, wc):
    _check(load().ch_set_velocity_coarse(handle, _ptr(uc), _ptr(vc), _ptr(wc)), handle, "ch_set_velocity_coarse")


def ch_interp_to_fine(handle):
    _check(load().ch_interp_to_fine(handle), handle, "ch_interp_to_fine")


def ch_get_velocity_fine(handle, u, v, w):
    _check(load().ch_get_velocity_fine(handle, _ptr(u), _ptr(v), _ptr(w)), handle, "ch_get_velocity_fine")


def ch_profile_interp(handle):
    """ms of [coarse gradients, x, y, z integration] of one ch_interp_to_fine."""
    out = (ctypes.c_double * 4)()
    _check(load().ch_profile_interp(handle, out), handle, "ch_profile_interp")
    return list(out)


def ch_get_interp_tables(handle, direction, n):
    start = np.zeros(n, dtype=np.int32)
    wts = np.zeros((n, 4), dtype=np.float64)
    _check(load().ch_get_interp_tables(handle, direction, start.ctypes.data_as(ctypes.c_void_p),
                                       wts.ctypes.data_as(ctypes.c_void_p)), handle, "ch_get_interp_tables")
    return start, wts


def ch_restrict_workspace_bytes(handle):
    return int(load().ch_restrict_workspace_bytes(handle))


def ch_restrict_to_coarse(handle, lam_rho, lam_mu, outs, work):
    """outs: six device tensors (C_c, rho_c, mu_c, Fx_c, Fy_c, Fz_c); work: a uint8 device tensor."""
    _check(load().ch_restrict_to_coarse(handle, lam_rho, lam_mu, *[_ptr(t) for t in outs], _ptr(work),
                                        work.numel()), handle, "ch_restrict_to_coarse")


def ch_step(handle, nsteps):
    _check(load().ch_step(handle, nsteps), handle, "ch_step")


def ch_mass(handle):
    out = ctypes.c_double()
    _check(load().ch_mass(handle, ctypes.byref(out)), handle, "ch_mass")
    return out.value


def ch_free_energy(handle):
    out = ctypes.c_double()
    _check(load().ch_free_energy(handle, ctypes.byref(out)), handle, "ch_free_energy")
    return out.value


def ch_diagnostics(handle):
    """(mass, free energy) from one pass over C."""
    m, e = ctypes.c_double(), ctypes.c_double()
    _check(load().ch_diagnostics(handle, ctypes.byref(m), ctypes.byref(e)), handle, "ch_diagnostics")
    return m.value, e.value


def ch_sync(handle):
    _check(load().ch_sync(handle), handle, "ch_sync")


def ch_launches_per_step(handle):
    return int(load().ch_launches_per_step(handle))


def ch_profile_step(handle, nsteps):
    """Mean ms per launch of [explicit, x-solve, y-solve, z-solve+update]."""
    out = (ctypes.c_double * 4)()
    _check(load().ch_profile_step(handle, nsteps, out), handle, "ch_profile_step")
    return list(out)


def ch_mass_noalloc(C, h, out, stream):
    """h^3 sum(C) into the one-element FP64 device tensor ``out`` on ``stream``,
    with no device allocation by the library (scratch is a fixed device array)."""
    import torch
    if not (torch.is_tensor(C) and C.is_cuda and C.dim() == 3 and C.is_contiguous()):
        raise ValueError("ch_mass_noalloc: C must be a contiguous 3D CUDA tensor [nz][ny][nx]")
    if C.dtype not in (torch.float32, torch.float64):
        raise ValueError(f"ch_mass_noalloc: C must be float32 or float64, not {C.dtype}")
    if not (torch.is_tensor(out) and out.is_cuda and out.dtype == torch.float64 and out.numel() >= 1
            and out.device == C.device):
        raise ValueError("ch_mass_noalloc: out must be a float64 CUDA tensor of >= 1 element on C's device")
    nz, ny, nx = C.shape
    prec = CH_F64 if C.dtype == torch.float64 else CH_F32
    st = load().ch_mass_noalloc(_ptr(C), nx, ny, nz, h, prec, _ptr(out), ctypes.c_void_p(stream.cuda_stream))
    if st != CH_OK:
        raise CHError(st, f"ch_mass_noalloc: {ch_error_string(st)} (grid limit 268435456 cells)")


def ch_adjoint_workspace_bytes(handle, nsteps, ckpt_every):
    return int(load().ch_adjoint_workspace_bytes(handle, nsteps, ckpt_every))


def ch_step_adjoint(handle, C0, nsteps, ckpt_every, lam_T, lam_0, work):
    """C0, lam_T, lam_0, work: torch CUDA tensors.  Returns dL/dM."""
    out = ctypes.c_double()
    _check(load().ch_step_adjoint(handle, _ptr(C0), nsteps, ckpt_every, _ptr(lam_T), _ptr(lam_0), ctypes.byref(out),
                                  _ptr(work), work.numel() * work.element_size()), handle, "ch_step_adjoint")
    return out.value


def _bcheck(status, batch, what):
    if status != CH_OK:
        lib = load()
        msg = lib.ch_batch_last_error(batch).decode() if batch else ""
        raise CHError(status, f"{what}: {lib.ch_error_string(status).decode()} {msg}".strip())


def ch_batch_workspace_bytes(params_list):
    arr = (ch_params * len(params_list))(*params_list)
    return int(load().ch_batch_workspace_bytes(arr, len(params_list)))


def ch_batch_create(params_list, C_list, work, stream):
    lib = load()
    arr = (ch_params * len(params_list))(*params_list)
    ptrs = (_P * len(C_list))(*[t.data_ptr() for t in C_list])
    out = ctypes.c_void_p()
    st = lib.ch_batch_create(arr, len(params_list), ptrs, _ptr(work), work.numel() * work.element_size(),
                             ctypes.c_void_p(stream.cuda_stream), ctypes.byref(out))
    _bcheck(st, None, "ch_batch_create")
    return out


def ch_batch_step(batch, nsteps):
    _bcheck(load().ch_batch_step(batch, nsteps), batch, "ch_batch_step")


def ch_batch_mass(batch, nbox):
    out = (ctypes.c_double * nbox)()
    _bcheck(load().ch_batch_mass(batch, out), batch, "ch_batch_mass")
    return list(out)


def ch_batch_sync(batch):
    _bcheck(load().ch_batch_sync(batch), batch, "ch_batch_sync")


def ch_batch_set_schedule(batch, mode, blocks_per_sm, zchunk, lpt):
    _bcheck(load().ch_batch_set_schedule(batch, mode, blocks_per_sm, zchunk, lpt), batch, "ch_batch_set_schedule")


def ch_batch_get_schedule(batch):
    out = (ctypes.c_int * 4)()
    _bcheck(load().ch_batch_get_schedule(batch, out), batch, "ch_batch_get_schedule")
    return tuple(out)


def ch_batch_autotune(batch, steps_per_trial):
    buf = ctypes.create_string_buffer(8192)
    _bcheck(load().ch_batch_autotune(batch, steps_per_trial, buf, len(buf)), batch, "ch_batch_autotune")
    return buf.value.decode()


def ch_batch_set_barrier_limit(batch, limit_ns, poison):
    _bcheck(load().ch_batch_set_barrier_limit(batch, limit_ns, poison), batch, "ch_batch_set_barrier_limit")


def ch_batch_launches_per_step(batch):
    return int(load().ch_batch_launches_per_step(batch))


def ch_batch_free(batch):
    _bcheck(load().ch_batch_free(batch), None, "ch_batch_free")


def ch_batch_last_error(batch):
    return load().ch_batch_last_error(batch).decode()


def ch_error_string(status):
    return load().ch_error_string(status).decode()


def ch_last_error(handle):
    return load().ch_last_error(handle).decode()
