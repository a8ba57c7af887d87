"""Python-side owner of one Cahn-Hilliard solver handle.

Holds the torch tensors the C ABI borrows (C and the workspace) and the
stream; every operation is one call into libch.so through ``capi``.
"""
from __future__ import annotations

import numpy as np
import torch

from . import capi


class Solver:
    """Fine-mesh Cahn-Hilliard solver on one GPU.

    shape = (nz, ny, nx); bc = (bc_x, bc_y, bc_z) with capi.CH_PERIODIC /
    capi.CH_NOFLUX (bc_z may also be capi.CH_DIRICHLET); precision "f32" or "f64".  C0 is a numpy or torch array of
    the initial volume fraction.  coarse_faces = (xf, yf, zf) enables the
    velocity transfer from a stretched coarse mesh.  scheme "split" is the
    paper's factorised implicit biharmonic; "standard" the explicit 25-point
    comparison scheme (Eq. eq-disbi).
    """

    def __init__(self, shape, h, bc, cn, pe, dt, C0, precision="f32", w=4.0, weno_eps=1e-6,
                 advect=False, coarse_faces=None, device="cuda:0", stream=None, scheme="split"):
        self.shape = tuple(int(s) for s in shape)
        self.bc = tuple(bc)
        self.dtype = torch.float64 if precision == "f64" else torch.float32
        self.device = torch.device(device)
        # a dedicated stream by default, so ch_step runs as a captured CUDA graph
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        prec = capi.CH_F64 if precision == "f64" else capi.CH_F32
        if scheme not in ("split", "standard"):
            raise ValueError("scheme must be 'split' or 'standard'")
        self.params = capi.make_params(self.shape, h, bc, cn, pe, dt, prec, w, weno_eps,
                                       advect or coarse_faces is not None, coarse_faces,
                                       capi.CH_SCHEME_STANDARD if scheme == "standard" else capi.CH_SCHEME_SPLIT)
        nbytes = capi.ch_workspace_bytes(self.params)
        if nbytes == 0:
            raise capi.CHError(capi.CH_EINVAL, "invalid parameters")
        self.C = torch.as_tensor(np.asarray(C0) if not torch.is_tensor(C0) else C0).to(
            device=self.device, dtype=self.dtype).contiguous().clone()
        self.work = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self._order()
        with torch.cuda.device(self.device):
            self.handle = capi.ch_create(self.params, self.C, self.work, self.stream)
        nz, ny, nx = self.shape
        nf = [n + (1 if b != capi.CH_PERIODIC else 0) for n, b in zip((nx, ny, nz), self.bc)]
        self.vel_shapes = ((nz, ny, nf[0]), (nz, nf[1], nx), (nf[2], ny, nx))
        if coarse_faces is not None:
            nc = [len(f) - 1 for f in coarse_faces]
            ncf = [n + (1 if b != capi.CH_PERIODIC else 0) for n, b in zip(nc, self.bc)]
            self.coarse_shapes = ((nc[2], nc[1], ncf[0]), (nc[2], ncf[1], nc[0]), (ncf[2], nc[1], nc[0]))

    def _order(self):
        """Make the library's stream wait for tensors prepared on torch's current stream."""
        self.stream.wait_stream(torch.cuda.current_stream(self.device))

    def _dev(self, a):
        t = a if torch.is_tensor(a) else torch.as_tensor(np.asarray(a))
        return t.to(device=self.device, dtype=self.dtype).contiguous()

    def set_velocity_fine(self, u, v, w):
        self._vel_keep = [self._dev(a) for a in (u, v, w)]
        self._order()
        capi.ch_set_velocity_fine(self.handle, *self._vel_keep)

    def set_velocity_coarse(self, uc, vc, wc):
        self._velc_keep = [self._dev(a) for a in (uc, vc, wc)]
        self._order()
        capi.ch_set_velocity_coarse(self.handle, *self._velc_keep)

    def interp_to_fine(self):
        capi.ch_interp_to_fine(self.handle)

    def velocity_fine(self):
        out = [torch.empty(s, dtype=self.dtype, device=self.device) for s in self.vel_shapes]
        self._order()
        capi.ch_get_velocity_fine(self.handle, *out)
        self.stream.synchronize()
        return out

    def restrict_to_coarse(self, lam_rho, lam_mu):
        """Down-sampling of C (Sec. 3.4) and the coarse rho, mu and surface
        tension (Eqs. eq-rho, eq-mu, eq-fst).  Returns a dict of device
        tensors [ncz][ncy][ncx]: C, rho, mu, Fx, Fy, Fz.  Asynchronous: the
        work runs on the solver's stream and torch's current stream is made
        to wait for it."""
        if not hasattr(self, "coarse_shapes"):
            raise ValueError("restrict_to_coarse needs a coarse mesh")
        ncz, ncy = self.coarse_shapes[0][0], self.coarse_shapes[0][1]
        ncx = self.coarse_shapes[1][2]
        names = ("C", "rho", "mu", "Fx", "Fy", "Fz")
        outs = [torch.empty((ncz, ncy, ncx), dtype=self.dtype, device=self.device) for _ in names]
        if getattr(self, "_rs_work", None) is None:
            self._rs_work = torch.empty(capi.ch_restrict_workspace_bytes(self.handle), dtype=torch.uint8,
                                        device=self.device)
        self._order()
        capi.ch_restrict_to_coarse(self.handle, lam_rho, lam_mu, outs, self._rs_work)
        # torch work on the returned tensors (on the current stream) waits for the library's
        torch.cuda.current_stream(self.device).wait_stream(self.stream)
        return dict(zip(names, outs))

    def interp_tables(self, direction):
        n = (self.shape[2], self.shape[1], self.shape[0])[direction]
        return capi.ch_get_interp_tables(self.handle, direction, n)

    def step(self, nsteps=1):
        capi.ch_step(self.handle, nsteps)

    def mass(self):
        return capi.ch_mass(self.handle)

    def free_energy(self):
        return capi.ch_free_energy(self.handle)

    def diagnostics(self):
        """(mass, free energy) in one pass over C."""
        return capi.ch_diagnostics(self.handle)

    def sync(self):
        capi.ch_sync(self.handle)

    def field(self):
        self.stream.synchronize()
        return self.C.detach().cpu().numpy().astype(np.float64)

    def launches_per_step(self):
        return capi.ch_launches_per_step(self.handle)

    def explicit_terms(self):
        """(H^2, H^3): the explicit terms of the second and third RK3 substeps of
        the last step (split scheme, after at least one step), read from the
        workspace at the offsets include/ch.h states, as float64 numpy arrays."""
        self.stream.synchronize()
        nbytes = self.C.numel() * self.C.element_size()
        B = (nbytes + 255) // 256 * 256
        H3 = self.work[:nbytes].view(self.dtype).reshape(self.shape)
        H2 = self.work[B:B + nbytes].view(self.dtype).reshape(self.shape)
        return tuple(t.cpu().numpy().astype(np.float64) for t in (H2, H3))

    def adjoint(self, C0, nsteps, lam_T, ckpt_every=10):
        """dL/dC0 and dL/dM of nsteps steps from C0, given lam_T = dL/dC_T.
        C0 and lam_T are numpy arrays or CUDA tensors; returns (tensor, float)."""
        C0d, lamd = self._dev(C0), self._dev(lam_T)
        lam0 = torch.empty_like(C0d)
        nbytes = capi.ch_adjoint_workspace_bytes(self.handle, nsteps, ckpt_every)
        if nbytes == 0:
            raise capi.CHError(capi.CH_EINVAL, "adjoint unsupported for these parameters (u must be 0)")
        work = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self._order()
        dM = capi.ch_step_adjoint(self.handle, C0d, nsteps, ckpt_every, lamd, lam0, work)
        return lam0, dM

    def close(self):
        if getattr(self, "handle", None) is not None:
            self.stream.synchronize()
            capi.ch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many independent FP32 boxes (u = 0) advanced together by libch.so's
    batched form.  boxes: list of dicts with shape, h, bc, cn, pe, dt, C."""

    def __init__(self, boxes, w=4.0, weno_eps=1e-6, device="cuda:0", stream=None):
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        self.params = [capi.make_params(b["shape"], b["h"], b["bc"], b["cn"], b["pe"], b["dt"], capi.CH_F32, w,
                                        weno_eps, False) for b in boxes]
        nbytes = capi.ch_batch_workspace_bytes(self.params)
        if nbytes == 0:
            raise capi.CHError(capi.CH_EINVAL, "invalid batch parameters")
        self.C = [torch.as_tensor(np.asarray(b["C"]), dtype=torch.float32).to(self.device).contiguous()
                  for b in boxes]
        self.work = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.device(self.device):
            self.handle = capi.ch_batch_create(self.params, self.C, self.work, self.stream)

    def step(self, nsteps=1):
        capi.ch_batch_step(self.handle, nsteps)

    def mass(self):
        return capi.ch_batch_mass(self.handle, len(self.C))

    def sync(self):
        capi.ch_batch_sync(self.handle)

    def set_schedule(self, mode, blocks_per_sm, zchunk, lpt):
        capi.ch_batch_set_schedule(self.handle, mode, blocks_per_sm, zchunk, lpt)

    def schedule(self):
        return capi.ch_batch_get_schedule(self.handle)

    def autotune(self, steps_per_trial=3):
        return capi.ch_batch_autotune(self.handle, steps_per_trial)

    def fields(self):
        self.stream.synchronize()
        return [c.cpu().numpy().astype(np.float64) for c in self.C]

    def set_fields(self, arrays):
        for c, a in zip(self.C, arrays):
            c.copy_(torch.as_tensor(np.asarray(a), dtype=torch.float32))
        self.stream.wait_stream(torch.cuda.current_stream(self.device))

    def launches_per_step(self):
        return capi.ch_batch_launches_per_step(self.handle)

    def close(self):
        if getattr(self, "handle", None) is not None:
            self.stream.synchronize()
            capi.ch_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
