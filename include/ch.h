/*
 * ch.h -- C ABI of the GB300 Cahn-Hilliard fine-grid step library (libch.so).
 *
 * The library advances the volume fraction C of the phase-field method of
 * "An efficient phase-field method for turbulent multiphase flows"
 * (Liu, Ng, Chong, Lohse, Verzicco, arXiv 2105.01865) on a uniform fine mesh:
 *
 *   dC/dt + div(u C) = (1/Pe) [ -Cn^2 lap^2 C + lap(C^3 - 1.5 C^2 + 0.5 C) ]   (Sec. 2.1, Eq. eq-ch)
 *
 * with WENO5 advection and central lap(psi') treated explicitly by a
 * low-storage RK3, and the biharmonic term replaced by A_x + A_y + A_z
 * (Sec. 3.1, Eq. eq-a3d) treated by Crank-Nicolson in delta form with
 * approximate factorisation into three pentadiagonal line solves
 * (Eqs. eq-re, eq-fac, eq-fac-1..3).  It also transfers a face velocity from
 * a stretched coarse mesh to the fine mesh (Sec. 3.4).
 *
 * Conventions shared by every entry point:
 *  - Every call returns an int status (CH_OK = 0 or a CH_E* code below);
 *    ch_error_string() names a code, ch_last_error() gives the handle's last
 *    message.  On error nothing is enqueued after the failing launch.
 *  - Fields are 3D arrays indexed [z][y][x], x fastest, contiguous, in the
 *    handle's precision (float for CH_F32, double for CH_F64).  Face
 *    velocities live on the staggered mesh: u on x-faces with nfx = nx
 *    (periodic x) or nx + 1 (walls at x = 0 and x = nx h) planes, shape
 *    [nz][ny][nfx]; v shape [nz][nfy][nx]; w shape [nfz][ny][nx].  Face f
 *    lies between cells f - 1 and f.
 *  - Device pointers passed in are BORROWED: the caller allocates them, keeps
 *    them alive and unmodified by other work until the handle is freed (C and
 *    the workspace) or until the call's work on the stream has completed (the
 *    velocity inputs and outputs).  The library allocates only small tables
 *    (LU factors, Hermite tables, reduction partials, a status word), freed
 *    by ch_free().
 *  - All work is enqueued on the stream given to ch_create (a cudaStream_t,
 *    NULL = legacy default stream).  Only ch_mass, ch_free_energy,
 *    ch_diagnostics, ch_sync and ch_get_interp_tables wait for the stream.
 */
#ifndef CH_GB300_H
#define CH_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define CH_OK 0
#define CH_EINVAL 1      /* invalid argument or size (nothing was enqueued) */
#define CH_ECUDA 2       /* a CUDA runtime call failed; see ch_last_error() */
#define CH_ENONFINITE 3  /* a NaN/Inf appeared in C since the last check */
#define CH_ETIMEOUT 4    /* a bounded device-side wait gave up */
#define CH_ENOMEM 5      /* workspace too small or a table allocation failed */

/* boundary condition per direction (Sec. 3.1: "first and last rows are
 * determined by boundary conditions") */
#define CH_PERIODIC 0    /* wrap: cyclic pentadiagonal line solves */
#define CH_NOFLUX 1      /* walls: mirror ghosts C_{-1-m} = C_m, zero wall flux */
#define CH_DIRICHLET 2   /* z only: C = 0 on the wall faces (antisymmetric ghosts); a wall for the flow */

/* arithmetic precision of fields and kernels */
#define CH_F32 0         /* float fields, float arithmetic; FP64 reductions */
#define CH_F64 1         /* double everywhere (the plain method) */

/* time-stepping scheme (ch_params.scheme) */
#define CH_SCHEME_SPLIT 0
#define CH_SCHEME_STANDARD 1

typedef struct ch_params {
    int64_t nx, ny, nz;   /* fine cells per direction, each >= 5 */
    double h;             /* uniform fine spacing (Sec. 3: same h in all directions) */
    int32_t bc[3];        /* CH_PERIODIC / CH_NOFLUX for x, y, z; z may also be CH_DIRICHLET */
    int32_t precision;    /* CH_F32 or CH_F64 */
    double cn;            /* Cahn number Cn (> 0) */
    double pe;            /* Peclet number Pe (> 0); mobility M = 1/Pe */
    double dt;            /* full RK3 step (> 0) */
    double w;             /* biharmonic weight: A_d = (w Cn^2/h^4)[1,-4,6,-4,1]; 4 = Eq. eq-a3d as printed */
    double weno_eps;      /* WENO5 regulariser (1e-6) */
    int32_t advect;       /* 0: u = 0, no advection term; 1: advect with the fine face velocity */
    int32_t scheme;       /* CH_SCHEME_SPLIT (0): the paper's A_x + A_y + A_z Crank-Nicolson step,
                             approximately factorised (Sec. 3.1); CH_SCHEME_STANDARD (1): the standard
                             25-point biharmonic of Eq. eq-disbi (lap_h applied twice), all terms
                             explicit in the same RK3 -- the comparison scheme of Sec. 4.1 */
    /* optional coarse (Navier-Stokes) mesh for the velocity transfer; all 0/NULL if unused.
     * Host arrays of face coordinates, read during ch_create only: xf has ncx+1 entries,
     * starting at 0 and ending at nx*h (likewise y, z).  Any (stretched) spacing;
     * 4 to 2048 coarse cells per direction and fewer than 2^31 in all. */
    int64_t ncx, ncy, ncz;
    const double* xf_coarse;
    const double* yf_coarse;
    const double* zf_coarse;
} ch_params;

typedef struct ch_handle ch_handle;

/* Bytes of device workspace ch_create needs for these parameters (the
 * explicit terms H of two RK3 substeps, the right-hand side / increment of
 * the factorised solve, the fine face velocity and, with a coarse mesh, the
 * coarse face velocity).  Returns 0 for invalid parameters.  For inspection
 * only, the first two regions are, with B = nx ny nz times the element size
 * rounded up to a multiple of 256: bytes [0, B) hold H of the third substep of
 * the last split-scheme step, bytes [B, 2B) H of its second substep. */
size_t ch_workspace_bytes(const ch_params* p);

/* Create a solver for the fine mesh of p (Sec. 3).  C: device array
 * [nz][ny][nx] holding the volume fraction, advanced in place by ch_step.
 * work: device workspace of >= ch_workspace_bytes(p) bytes, 256-byte aligned.
 * stream: cudaStream_t for all work.  Builds the LU factors of the line
 * operators (I + (alpha_l dt M / 2) A_d) for the three RK3 substeps, and with
 * a coarse mesh the Hermite index/weight tables (Sec. 3.4: the tables are built
 * once per mesh pair).  nz = 1 with a periodic z is a single plane: the 2D
 * scheme of Sec. 3.1 (A_x + A_y; Eq. eq-a2d is w = 2), with no z-solve.
 * Errors: CH_EINVAL (nx or ny < 5, nz < 5 other than that single plane,
 * non-positive h/cn/pe/dt/w, bad bc, coarse faces not spanning the fine box, a
 * coarse mesh with nz < 5, misaligned pointers), CH_ENOMEM, CH_ECUDA.  On
 * success *out owns the tables until ch_free. */
int ch_create(const ch_params* p, void* C, void* work, size_t work_bytes, void* stream, ch_handle** out);

/* Release the library-owned tables and the handle (not C or the workspace). */
int ch_free(ch_handle* h);

/* Copy a fine face velocity (device arrays, shapes in the header comment)
 * into the workspace, for cases that prescribe u on the fine mesh
 * (e.g. an imposed shear).  Requires advect = 1.  Asynchronous. */
int ch_set_velocity_fine(ch_handle* h, const void* u, const void* v, const void* w);

/* Copy the coarse staggered face velocity into the workspace (Sec. 3.4: the
 * "base mesh" velocity).  Shapes: uc [ncz][ncy][ncfx], vc [ncz][ncfy][ncx],
 * wc [ncfz][ncy][ncx] with ncf = nc (periodic) or nc + 1 (walls).  For an
 * exactly solenoidal fine field it must be discretely divergence-free.
 * Requires a coarse mesh at create.  Asynchronous. */
int ch_set_velocity_coarse(ch_handle* h, const void* uc, const void* vc, const void* wc);

/* Sec. 3.4: coarse normal gradients du/dx, dv/dy, dw/dz at coarse cell
 * centres -> tri-cubic Hermite (4 points per direction) to fine cell centres
 * -> integration along x, y, z from the reference planes x = 0, y = 0, z = 0
 * (2D Hermite of the coarse face plane there; zero at a wall) -> fine face
 * velocity in the workspace.  Requires a coarse mesh.  Asynchronous. */
int ch_interp_to_fine(ch_handle* h);

/* Measurement aid: run ch_interp_to_fine once with CUDA events recorded on
 * the handle's stream around each of its launches, wait, and write their
 * durations in milliseconds to ms_out[4]: [0] coarse normal gradients,
 * [1] x integration (u), [2] y integration (v), [3] z integration (w).
 * Errors: CH_EINVAL (no coarse mesh, NULL), CH_ECUDA. */
int ch_profile_interp(ch_handle* h, double* ms_out);

/* Copy the workspace's fine face velocity out to device arrays (shapes as
 * for ch_set_velocity_fine).  Asynchronous. */
int ch_get_velocity_fine(ch_handle* h, void* u, void* v, void* w);

/* Copy the Hermite table of direction dir (0 = x, 1 = y, 2 = z) to HOST
 * arrays: start[n_fine_dir] (first of the 4 coarse nodes; wrapped index for
 * periodic directions) and weights[n_fine_dir][4] (double).  Synchronous. */
int ch_get_interp_tables(ch_handle* h, int dir, int32_t* start, double* weights);

/* Bytes of device workspace ch_restrict_to_coarse needs for this handle (0
 * without a coarse mesh): 4 nz ny ncx + 4 nz ncy ncx elements of the
 * handle's precision for the two intermediate passes. */
size_t ch_restrict_workspace_bytes(const ch_handle* h);

/* Down-sampling back-coupling (Sec. 3.4: the fine C projected directly to the
 * stretched mesh, used for the coarse density, viscosity and surface tension;
 * Sec. 2.2, Eqs. eq-rho, eq-mu, eq-fst).  The projection is the 4-point-per-
 * direction Hermite stencil of the transfer with nodes at the fine cell
 * centres and queries at the coarse cell centres, applied to C and to the
 * fine F_st = 6 sqrt(2) phi grad C / Cn (phi = psi'(C) - Cn^2 lap_h C, central
 * differences, the step's ghost cells).  Outputs (DEVICE, caller-owned,
 * [ncz][ncy][ncx], the handle's precision): C_c, rho_c = C_c + lambda_rho
 * (1 - C_c), mu_c = C_c + lambda_mu (1 - C_c), and the three F_st components
 * at the coarse cell centres.  work: >= ch_restrict_workspace_bytes(h) bytes,
 * 256-byte aligned.  Requires a coarse mesh.  Asynchronous.  Errors:
 * CH_EINVAL (no coarse mesh, NULL/misaligned pointers, non-finite ratios),
 * CH_ENOMEM (workspace too small), CH_ECUDA. */
int ch_restrict_to_coarse(ch_handle* h, double lambda_rho, double lambda_mu, void* C_c, void* rho_c, void* mu_c,
                          void* fx_c, void* fy_c, void* fz_c, void* work, size_t work_bytes);

/* Advance C by nsteps full RK3 steps (three substeps each; Sec. 3 and
 * Eqs. eq-re .. eq-fac-3).  Asynchronous; a non-finite C sets a device flag
 * reported by the next ch_sync / ch_mass / ch_free_energy.  nsteps >= 0. */
int ch_step(ch_handle* h, int64_t nsteps);

/* Drop mass m = h^3 sum C in FP64 (Sec. 4.3: l_loss = (m_t - m_0)/m_0).
 * Waits for the stream; *out is a host double.  CH_ENONFINITE if C holds a
 * NaN/Inf. */
int ch_mass(ch_handle* h, double* out);

/* Free energy F = h^3 sum [psi(C) + (Cn^2/2) sum_d ((C_{+e_d} - C)/h)^2],
 * psi = C^2 (C-1)^2 / 4 (Sec. 1; forward differences, zero across a wall),
 * accumulated in FP64.  Waits for the stream; *out is a host double. */
int ch_free_energy(ch_handle* h, double* out);

/* Both diagnostics of Sec. 4.3 / Sec. 1 in one pass over C: *mass as ch_mass and
 * *free_energy as ch_free_energy (host doubles; the same FP64 results up to the
 * order of the additions).  Waits for the stream.  Errors: CH_EINVAL (NULL),
 * CH_ENONFINITE (a NaN/Inf in C), CH_ECUDA. */
int ch_diagnostics(ch_handle* h, double* mass, double* free_energy);

/* Wait for the handle's stream and report (then clear) the non-finite flag
 * (CH_ENONFINITE).  A library built with the explicit kernel's tensor-map
 * staging (CH_EXPLICIT_TMA, off by default) also reports CH_ETIMEOUT when a
 * tile load did not complete within 2 s; the step's results are then void. */
int ch_sync(ch_handle* h);

/* Number of kernel launches one ch_step(h, 1) enqueues. */
int ch_launches_per_step(const ch_handle* h);

/* Measurement aid: run nsteps full steps (the same kernels as ch_step, but
 * launched directly instead of as a graph) with CUDA events recorded on the
 * handle's stream around every launch, wait for the stream, and write the mean
 * duration in milliseconds of one launch of each kernel class to ms_out[4]:
 * [0] explicit right-hand side, [1] x-line solve, [2] y-line solve,
 * [3] z-line solve + update (averaged over the three substeps).  nsteps >= 1.
 * Errors: CH_EINVAL, CH_ECUDA. */
int ch_profile_step(ch_handle* h, int64_t nsteps, double* ms_out);

/* ---------------------------------------------------------------------------
 * Differentiation form (u = 0): the adjoint of nsteps steps.  The paper has
 * no derivative; this is the exact transpose of the discrete step of Sec. 3
 * (line solves, A_d, lap psi', the RK3 history term and the M-dependence of
 * the factorised operator), evaluated in the handle's precision with FP64
 * dot products for dL/dM.
 * ------------------------------------------------------------------------- */

/* Device workspace bytes for ch_step_adjoint (checkpoints every ckpt_every
 * steps, one recomputed segment, 15 scratch fields); 0 if unsupported
 * (advect = 1) or invalid. */
size_t ch_adjoint_workspace_bytes(const ch_handle* h, int64_t nsteps, int64_t ckpt_every);

/* Reverse nsteps steps of the handle's problem started from C0 (device field,
 * not modified): given lam_T = dL/dC_T (device field), write lam_0 = dL/dC_0
 * (device field) and *dL_dM = dL/dM through every occurrence of M = 1/Pe
 * (host double).  The forward trajectory is recomputed from checkpoints
 * stored every ckpt_every steps (memory ~ (nsteps/ckpt_every + ckpt_every)
 * fields, work ~ 2 forward passes + the reverse).  Does not touch the handle's
 * C.  Waits for the stream.  Errors: CH_EINVAL (advect = 1, bad args),
 * CH_ENOMEM (workspace too small), CH_ECUDA. */
int ch_step_adjoint(ch_handle* h, const void* C0, int64_t nsteps, int64_t ckpt_every, const void* lam_T, void* lam_0,
                    double* dL_dM, void* work, size_t work_bytes);

/* ---------------------------------------------------------------------------
 * Batched form: many independent boxes of uneven sizes and parameters
 * (each box is the Sec. 3 step of its own ch_params) advanced together.  The
 * paper advances one box; batching is this library's addition.
 * Restrictions: precision CH_F32, advect = 0, no coarse mesh, nx even,
 * 6 <= nx and 5 <= ny, nz, every size <= 256.  Same conventions as above.
 * ------------------------------------------------------------------------- */
typedef struct ch_batch ch_batch;

/* Workspace bytes for the boxes (3 fields per box, 256-byte aligned); 0 if
 * any box violates the restrictions. */
size_t ch_batch_workspace_bytes(const ch_params* boxes, int nbox);

/* Create a batch.  C[i]: device array [nz][ny][nx] of box i (16-byte
 * aligned), advanced in place.  work: >= ch_batch_workspace_bytes bytes,
 * 256-byte aligned.  Builds every box's line-solve tables.  Default schedule:
 * one persistent cooperative launch per step (if the device supports it).
 * Errors: CH_EINVAL, CH_ENOMEM, CH_ECUDA. */
int ch_batch_create(const ch_params* boxes, int nbox, void* const* C, void* work, size_t work_bytes, void* stream,
                    ch_batch** out);

/* nsteps full RK3 steps of every box.  Persistent schedule: one cooperative
 * launch per step, 12 phases separated by grid barriers whose wait is
 * bounded in time; an expired wait makes the kernel return early and the
 * next ch_batch_sync / ch_batch_mass report CH_ETIMEOUT.  After a timeout the
 * boxes' fields are undefined, and later persistent launches return at once
 * without work until ch_batch_sync has reported and cleared it.  Phased schedule:
 * 12 launches per step.  Both are captured once in a CUDA graph on a user
 * stream.  Asynchronous. */
int ch_batch_step(ch_batch* b, int64_t nsteps);

/* FP64 mass h^3 sum C of every box into the host array out[nbox]; waits. */
int ch_batch_mass(ch_batch* b, double* out);

/* Wait for the stream; report (then clear) a barrier timeout (CH_ETIMEOUT)
 * or a non-finite value (CH_ENONFINITE). */
int ch_batch_sync(ch_batch* b);

/* Schedule: mode 0 = persistent, 1 = phased; CTAs per SM (capped by
 * occupancy); z extent of the explicit tiles; lpt = 1 orders each phase's
 * work items by decreasing cost. */
int ch_batch_set_schedule(ch_batch* b, int mode, int blocks_per_sm, int zchunk, int lpt);

/* Current schedule as {mode, blocks_per_sm, zchunk, lpt}. */
int ch_batch_get_schedule(const ch_batch* b, int* out4);

/* Autotuner: time every schedule candidate over steps_per_trial steps (the
 * boxes' fields are saved and restored), keep the fastest, and write one
 * line per candidate plus the choice into report (if not NULL). */
int ch_batch_autotune(ch_batch* b, int steps_per_trial, char* report, size_t report_len);

/* Failure-detection hook: the barrier wait limit in nanoseconds (>= 1000)
 * and, with poison = 1, a barrier that expects one CTA more than launched, so
 * that every wait expires (used to test the timeout path). */
int ch_batch_set_barrier_limit(ch_batch* b, int64_t limit_ns, int poison);

/* Kernel launches one ch_batch_step(b, 1) enqueues. */
int ch_batch_launches_per_step(const ch_batch* b);

/* Release the batch's tables (not the fields or the workspace). */
int ch_batch_free(ch_batch* b);

/* Message of the last error on this batch ("" if none). */
const char* ch_batch_last_error(const ch_batch* b);

/* Mass h^3 * sum(C) without any device allocation; the paper has no
 * counterpart (it is an interface for callers that cannot call cudaMalloc,
 * e.g. an application that owns the device memory budget through its own
 * pool, or a plug-in handed only pointers).  C: device array of nx*ny*nz
 * values, float (CH_F32) or double (CH_F64).  out: DEVICE pointer to one
 * double, written asynchronously on `stream` (a cudaStream_t, NULL = legacy
 * stream).  Scratch: a fixed 512 KB file-scope device array of 65536 FP64
 * partial sums of 4096 cells each, so at most 268435456 cells; larger grids
 * return CH_EINVAL with a message on stderr.  The array is held by every GPU
 * that loads the library until exit and is shared by all calls: calls that
 * overlap on the GPU race.  Every partial a call reads is written by that
 * call first, so nothing needs clearing.  Every call on a stream that is not
 * capturing looks up the array's address with the current device (so a device
 * reset is picked up); a call on a capturing stream reuses the address of the
 * last such call on that device, so make one call before any stream capture
 * (else CH_ECUDA).  Errors: CH_EINVAL, CH_ECUDA. */
int ch_mass_noalloc(const void* C, int64_t nx, int64_t ny, int64_t nz, double h, int precision, double* out,
                    void* stream);

/* Static description of a status code. */
const char* ch_error_string(int status);

/* Message of the last error on this handle ("" if none; never NULL). */
const char* ch_last_error(const ch_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* CH_GB300_H */
