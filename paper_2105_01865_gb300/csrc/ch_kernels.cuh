// Device kernels of the Cahn-Hilliard fine-grid step (arXiv 2105.01865, Sec. 3).
//
//  ch_explicit_rhs   explicit terms of one RK3 substep + right-hand side of
//                    the delta-form Crank-Nicolson system (Eq. eq-re):
//                    H^l = -div(u C) + M lap(psi'(C)),
//                    r   = dt (gamma_l H^l + rho_l H^{l-1}) - alpha_l dt M sum_d A_d C
//  ch_solve_x        (I + (alpha_l dt M / 2) A_x) dq*  = r     (Eq. eq-fac-1)
//  ch_solve_yz       (I + (alpha_l dt M / 2) A_y) dq** = dq*   (Eq. eq-fac-2)
//                    (I + (alpha_l dt M / 2) A_z) dq   = dq**, C += dq (Eq. eq-fac-3)
//  ch_reduce_*       FP64 mass and free-energy sums
//
// None of this is a dense contraction, so no tensor cores: the kernels are
// built around coalesced HBM access, shared-memory halo staging and
// shared-memory line buffers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ch.h"

namespace chg {

constexpr int kTX = 32;   // explicit-kernel tile, x (one warp)
constexpr int kTY = 8;    // explicit-kernel tile, y (warps per CTA)
constexpr int kTZ = 16;   // z-planes marched per CTA
constexpr int kHalo = 3;  // WENO5 needs three cells on each side

template <typename T>
struct RhsArgs {
    int nx, ny, nz;
    int bcx, bcy, bcz;
    int nfx, nfy, nfz;
    T inv_h, inv_h2;
    T mob;        // M = 1/Pe
    T dtg;        // dt * gamma_l
    T dtr;        // dt * rho_l
    T impl;       // alpha_l dt M kappa (multiplies the raw [1,-4,6,-4,1] sums)
    T eps;        // WENO regulariser
    int has_prev; // rho_l != 0
};

// Neighbour index with the boundary rule of Sec. 3.1: periodic wrap, or the
// mirror about a wall face (ghost C_{-1-m} = C_m).  Clamped so that cells
// outside the domain in a ragged tile still read valid memory.  Uses integer
// division, so it is only called once per CTA to build index tables.
__device__ __forceinline__ int bc_index(int i, int n, int bc) {
    if (bc == CH_PERIODIC) {
        i %= n;
        if (i < 0) i += n;
        return i;
    }
    if (i < 0) i = -1 - i;
    if (i >= n) i = 2 * n - 1 - i;
    return min(max(i, 0), n - 1);
}

// The same rule for indices at most one period outside [0, n) (n >= 5 and
// offsets of at most 4), without division.
// Sign of the ghost value at index i: -1 beyond a Dirichlet wall (C = 0 on
// the wall face, so the ghost is the negated mirror), else +1.
__device__ __forceinline__ bool bc_negate(int i, int n, int bc) { return bc == CH_DIRICHLET && (i < 0 || i >= n); }

__device__ __forceinline__ int bc_near(int i, int n, int bc) {
    if (n == 1) return 0;  // a single periodic plane: every neighbour is the plane itself
    if (i < 0) return bc == CH_PERIODIC ? i + n : -1 - i;
    if (i >= n) return bc == CH_PERIODIC ? i - n : 2 * n - 1 - i;
    return i;
}

template <typename T>
__device__ __forceinline__ T psi_p(T c) {  // psi'(C) = C^3 - 1.5 C^2 + 0.5 C (Eq. eq-ch)
    return c * (c * (c - T(1.5)) + T(0.5));
}

__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }

// Fifth-order WENO (Jiang-Shu) value at the face between v3 and v4 from the
// upwind-biased stencil v1..v5 (Sec. 3: "fifth-order WENO").  The nonlinear
// weights alpha_k = d_k / (eps + beta_k)^2, normalised, are formed over a
// common denominator so that one division serves all three.
template <typename T>
__device__ __forceinline__ T weno5(T v1, T v2, T v3, T v4, T v5, T eps) {
    const T q0 = T(2) * v1 - T(7) * v2 + T(11) * v3;   // 6 x candidate values
    const T q1 = -v2 + T(5) * v3 + T(2) * v4;
    const T q2 = T(2) * v3 + T(5) * v4 - v5;
    const T d0 = v1 - T(2) * v2 + v3, e0 = v1 - T(4) * v2 + T(3) * v3;
    const T d1 = v2 - T(2) * v3 + v4, e1 = v2 - v4;
    const T d2 = v3 - T(2) * v4 + v5, e2 = T(3) * v3 - T(4) * v4 + v5;
    const T s0 = eps + (T(13.0 / 12.0) * d0 * d0 + T(0.25) * e0 * e0);
    const T s1 = eps + (T(13.0 / 12.0) * d1 * d1 + T(0.25) * e1 * e1);
    const T s2 = eps + (T(13.0 / 12.0) * d2 * d2 + T(0.25) * e2 * e2);
    const T t0 = s0 * s0, t1 = s1 * s1, t2 = s2 * s2;
    const T w0 = T(0.1) * (t1 * t2), w1 = T(0.6) * (t0 * t2), w2 = T(0.3) * (t0 * t1);
    return fdiv(w0 * q0 + w1 * q1 + w2 * q2, T(6) * (w0 + w1 + w2));
}

// Flux u_f C_f through a face, C_f from the upwind WENO5 stencil.  m3..p2 are
// the cells f-3 .. f+2 around the face f (between cells f-1 and f).
template <typename T>
__device__ __forceinline__ T face_flux(T vel, T m3, T m2, T m1, T p0, T p1, T p2, T eps) {
    const bool up = vel >= T(0);
    const T a1 = up ? m3 : p2, a2 = up ? m2 : p1, a3 = up ? m1 : p0, a4 = up ? p0 : m1, a5 = up ? p1 : m2;
    return vel * weno5(a1, a2, a3, a4, a5, eps);
}

// Programmatic dependent launch.  A kernel launched with programmatic stream
// serialisation may be scheduled while its predecessor drains; pdl_wait()
// blocks until the predecessor grid has completed and its writes are
// visible, so every such kernel calls it before touching global memory.
// pdl_launch_dependents() lets the next kernel be scheduled once every CTA of
// this grid has started.  Both are no-ops for an ordinary launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Asynchronous global -> shared copies (cp.async): one element, 4 or 8 bytes.
__device__ __forceinline__ void cp_async_elem(float* smem, const float* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_elem(double* smem, const double* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
// two adjacent floats (8 bytes; both addresses 8-byte aligned)
__device__ __forceinline__ void cp_async_pair(float* smem, const float* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
// 16 bytes (both addresses 16-byte aligned)
__device__ __forceinline__ void cp_async_16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

// Tensor-memory-accelerator (TMA) tile loads completed on a shared-memory
// mbarrier (transaction count in bytes).
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// make barrier initialisation visible to the async proxy (the TMA unit)
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}
// Wait for phase `parity` of the barrier, giving up after `limit_ns`.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity, unsigned long long limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}
// 3D tile (x innermost) of a tensor map into shared memory; x must be a
// multiple of 16 bytes of elements, the destination 128-byte aligned.
__device__ __forceinline__ void tma_load_3d(void* dst, const void* tmap, int x, int y, int z, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(smem_u32(dst)),
        "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------------------
// Explicit right-hand side.  A CTA owns a 32 x 8 column of cells and marches
// kTZ planes in z.  Each plane (with a 3-cell halo in x and y) is staged in
// shared memory through per-CTA index tables (no division in the loop); the
// cell's own z-column lives in a 6-register queue.  Every face flux is
// computed exactly once (lower faces by their cell, the extra upper faces of
// the tile by dedicated lanes, z-faces carried between planes), so the
// fluxes telescope bit-exactly and mass is conserved to rounding.
// ---------------------------------------------------------------------------
template <typename T, bool ADV>
__global__ void __launch_bounds__(kTX * kTY)
ch_explicit_rhs(const T* __restrict__ C, const T* __restrict__ u, const T* __restrict__ v,
                const T* __restrict__ w, const T* __restrict__ Hprev, T* __restrict__ Hout,
                T* __restrict__ r, RhsArgs<T> a) {
    pdl_wait();
    pdl_launch_dependents();
    constexpr int PX = kTX + 2 * kHalo, PY = kTY + 2 * kHalo;
    __shared__ __align__(16) T Cs[3][PY][PX];
    __shared__ T Fx[ADV ? kTY : 1][kTX + 1];
    __shared__ T Fy[ADV ? kTY + 1 : 1][kTX];
    __shared__ int gi_tab[PX], gj_tab[PY];

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kTX + tx;
    const int i0 = blockIdx.x * kTX, j0 = blockIdx.y * kTY, k0 = blockIdx.z * kTZ;
    const int i = i0 + tx, j = j0 + ty;
    const bool in_xy = (i < a.nx) && (j < a.ny);
    const int ic = min(i, a.nx - 1), jc = min(j, a.ny - 1);
    const int64_t plane = (int64_t)a.nx * a.ny;
    const int64_t col = (int64_t)jc * a.nx + ic;
    const T eps = a.eps;
    const int kend = min(k0 + kTZ, a.nz);

    if (tid < PX) gi_tab[tid] = bc_index(i0 + tid - kHalo, a.nx, a.bcx);
    else if (tid < PX + PY) gj_tab[tid - PX] = bc_index(j0 + (tid - PX) - kHalo, a.ny, a.bcy);

    // face indices and wall flags of this thread's faces (fixed over the march)
    const bool wall_x = (a.bcx == CH_NOFLUX) && (i <= 0 || i >= a.nx);
    const int fi = (a.bcx == CH_PERIODIC) ? bc_index(i, a.nx, CH_PERIODIC) : min(i, a.nx);
    const bool wall_y = (a.bcy == CH_NOFLUX) && (j <= 0 || j >= a.ny);
    const int fj = (a.bcy == CH_PERIODIC) ? bc_index(j, a.ny, CH_PERIODIC) : min(j, a.ny);
    // extra faces: x-face i0+32 of row (j0 + tx) for warp 0 lanes < 8, y-face j0+8 for warp 1
    const int ie = i0 + kTX, je_row = min(j0 + tx, a.ny - 1);
    const bool wall_xe = (a.bcx == CH_NOFLUX) && (ie >= a.nx);
    const int fie = (a.bcx == CH_PERIODIC) ? bc_index(ie, a.nx, CH_PERIODIC) : min(ie, a.nx);
    const int je = j0 + kTY;
    const bool wall_ye = (a.bcy == CH_NOFLUX) && (je >= a.ny);
    const int fje = (a.bcy == CH_PERIODIC) ? bc_index(je, a.ny, CH_PERIODIC) : min(je, a.ny);

    // z-column queue: q[m] = C(ic, jc, k - 2 + m), m = 0..5
    T q[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) {
        q[m] = C[(int64_t)bc_near(k0 - 2 + m, a.nz, a.bcz) * plane + col];
        if (bc_negate(k0 - 2 + m, a.nz, a.bcz)) q[m] = -q[m];
    }

    T fz_lo = T(0);
    if (ADV) {
        // flux through the lower z-face of plane k0
        const bool wall = (a.bcz != CH_PERIODIC) && (k0 == 0);
        if (!wall) {
            T cm3 = C[(int64_t)bc_near(k0 - 3, a.nz, a.bcz) * plane + col];
            if (bc_negate(k0 - 3, a.nz, a.bcz)) cm3 = -cm3;
            const T wv = w[(int64_t)k0 * plane + col];
            fz_lo = face_flux(wv, cm3, q[0], q[1], q[2], q[3], q[4], eps);
        }
    }
    __syncthreads();  // index tables ready

    // Planes are staged with asynchronous 4/8-byte copies into a ring of three
    // buffers: plane k+1 is in flight while plane k is computed, and the
    // buffer being refilled was last read two planes ago (behind a barrier).
    auto stage = [&](int kk, int b) {
        const T* Ck = C + (int64_t)kk * plane;
        for (int e = tid; e < PX * PY; e += kTX * kTY) {
            const int row = e / PX, cc = e - row * PX;
            cp_async_elem(&Cs[b][row][cc], Ck + (int64_t)gj_tab[row] * a.nx + gi_tab[cc]);
        }
        cp_async_commit();
    };
    stage(k0, 0);
    for (int k = k0, buf = 0; k < kend; ++k, buf = (buf == 2 ? 0 : buf + 1)) {
        if (k + 1 < kend) {
            stage(k + 1, buf == 2 ? 0 : buf + 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        // prefetch the next queue entry C(k + 4)
        T qnext = C[(int64_t)bc_near(k + 4, a.nz, a.bcz) * plane + col];
        if (bc_negate(k + 4, a.nz, a.bcz)) qnext = -qnext;
        __syncthreads();

        const int cy = ty + kHalo, cx = tx + kHalo;
        T fz_up = T(0);
        if (ADV) {
            const int64_t kp = (int64_t)k * a.ny;
            // x: flux through this cell's lower face (face i)
            {
                T f = T(0);
                if (!wall_x) {
                    const T uv = u[(kp + jc) * a.nfx + fi];
                    f = face_flux(uv, Cs[buf][cy][cx - 3], Cs[buf][cy][cx - 2], Cs[buf][cy][cx - 1],
                                  Cs[buf][cy][cx], Cs[buf][cy][cx + 1], Cs[buf][cy][cx + 2], eps);
                }
                Fx[ty][tx] = f;
            }
            // y: flux through this cell's lower face (face j)
            {
                T f = T(0);
                if (!wall_y) {
                    const T vv = v[((int64_t)k * a.nfy + fj) * a.nx + ic];
                    f = face_flux(vv, Cs[buf][cy - 3][cx], Cs[buf][cy - 2][cx], Cs[buf][cy - 1][cx],
                                  Cs[buf][cy][cx], Cs[buf][cy + 1][cx], Cs[buf][cy + 2][cx], eps);
                }
                Fy[ty][tx] = f;
            }
            // the tile's extra upper faces
            if (ty == 0 && tx < kTY) {
                T f = T(0);
                if (!wall_xe) {
                    const T uv = u[(kp + je_row) * a.nfx + fie];
                    const int yy = tx + kHalo, xx = kTX + kHalo;
                    f = face_flux(uv, Cs[buf][yy][xx - 3], Cs[buf][yy][xx - 2], Cs[buf][yy][xx - 1],
                                  Cs[buf][yy][xx], Cs[buf][yy][xx + 1], Cs[buf][yy][xx + 2], eps);
                }
                Fx[tx][kTX] = f;
            }
            if (ty == 1) {
                T f = T(0);
                if (!wall_ye) {
                    const T vv = v[((int64_t)k * a.nfy + fje) * a.nx + ic];
                    const int yy = kTY + kHalo, xx = cx;
                    f = face_flux(vv, Cs[buf][yy - 3][xx], Cs[buf][yy - 2][xx], Cs[buf][yy - 1][xx],
                                  Cs[buf][yy][xx], Cs[buf][yy + 1][xx], Cs[buf][yy + 2][xx], eps);
                }
                Fy[kTY][tx] = f;
            }
            // z: flux through the upper face k+1 of this cell
            {
                const bool wall = (a.bcz != CH_PERIODIC) && (k + 1 >= a.nz);
                if (!wall) {
                    const int f = (k + 1 < a.nz) ? k + 1 : 0;
                    const T wv = w[(int64_t)f * plane + col];
                    fz_up = face_flux(wv, q[0], q[1], q[2], q[3], q[4], q[5], eps);
                }
            }
            __syncthreads();
        }

        // M lap(psi'(C)), 7-point central (Sec. 3); neighbour differences are
        // formed first, so FP32 keeps the accuracy of the small differences
        const T c0 = Cs[buf][cy][cx];
        const T pc = psi_p(c0);
        T pzm = psi_p(q[1]), pzp = psi_p(q[3]);
        if (a.bcz == CH_DIRICHLET) {  // the ghost of psi' is its own negated mirror (psi' = 0 on the wall)
            if (k == 0) pzm = -psi_p(-q[1]);
            if (k + 1 == a.nz) pzp = -psi_p(-q[3]);
        }
        const T lap = (((psi_p(Cs[buf][cy][cx - 1]) - pc) + (psi_p(Cs[buf][cy][cx + 1]) - pc)) +
                       ((psi_p(Cs[buf][cy - 1][cx]) - pc) + (psi_p(Cs[buf][cy + 1][cx]) - pc)) +
                       ((pzm - pc) + (pzp - pc))) *
                      a.inv_h2;
        // [1,-4,6,-4,1] sums of A_x + A_y + A_z (Eq. eq-a3d) as differences of
        // second differences: D2(i-1) - 2 D2(i) + D2(i+1)
        auto fourth = [&](T m2, T m1, T p1, T p2) {
            const T da = m1 - c0, db = p1 - c0;
            return ((m2 - m1) - da) + ((p2 - p1) - db) - T(2) * (da + db);
        };
        const T astar = fourth(Cs[buf][cy][cx - 2], Cs[buf][cy][cx - 1], Cs[buf][cy][cx + 1], Cs[buf][cy][cx + 2]) +
                        fourth(Cs[buf][cy - 2][cx], Cs[buf][cy - 1][cx], Cs[buf][cy + 1][cx], Cs[buf][cy + 2][cx]) +
                        fourth(q[0], q[1], q[3], q[4]);

        T H = a.mob * lap;
        if (ADV) {
            const T div = (Fx[ty][tx + 1] - Fx[ty][tx]) + (Fy[ty + 1][tx] - Fy[ty][tx]) + (fz_up - fz_lo);
            H -= div * a.inv_h;
        }
        if (in_xy) {
            const int64_t idx = (int64_t)k * plane + (int64_t)j * a.nx + i;
            T rhs = a.dtg * H - a.impl * astar;
            if (a.has_prev) rhs += a.dtr * Hprev[idx];
            Hout[idx] = H;
            if (r) r[idx] = rhs;
        }
        // advance the z queue
#pragma unroll
        for (int m = 0; m < 5; ++m) q[m] = q[m + 1];
        q[5] = qnext;
        fz_lo = fz_up;
    }
}

// ---------------------------------------------------------------------------
// Line solves.  The matrix (I + c A_d) is the same for every line of a
// direction, so its banded LU factors (and, for periodic directions, the
// rank-4 Woodbury correction of the corner entries) are computed once on the
// host in FP64:
//   forward  y_j = r_j - l1_j y_{j-1} - l2_j y_{j-2},   z_j = y_j / u0_j
//   backward x_j = z_j - (u1_j/u0_j) x_{j+1} - (u2_j/u0_j) x_{j+2}
//   periodic out_j = x_j - Z_j . s,  s = S (W^T r)   (Woodbury)
// One warp solves one line.  Lane l owns the M consecutive rows
// [l M, l M + M) in registers.  Both order-2 recurrences are affine maps of
// the state (y_j, y_{j-1}) (resp. (x_j, x_{j+1})); each lane first runs its
// chunk from a zero state, a 5-step warp-shuffle scan composes the chunks
// (the 2x2 transfer matrices of every lane span are coefficient-only and
// precomputed on the host), and each lane then reruns its chunk from the
// correct incoming state.  Rows past n are padding with zero coefficients.
// ---------------------------------------------------------------------------
template <typename T>
struct WCoef {
    const T* __restrict__ fwd;  // [M][32][4]: l1, l2, 1/u0, 0      (row j = lane*M + i at [i][lane])
    const T* __restrict__ bwd;  // [M][32][2]: u1/u0, u2/u0
    const T* __restrict__ W;    // [M][32][4]  periodic only
    const T* __restrict__ Z;    // [M][32][4]  periodic only
    const T* __restrict__ Pf;   // [5][32][4]  forward span matrices, row-major 2x2
    const T* __restrict__ Pb;   // [5][32][4]  backward span matrices
    const T* __restrict__ S;    // [4][4]      periodic only
    int n;
    int periodic;
    int r0 = 0, r1 = 0;         // interior rows: constant factors, negligible W, Z (warp_line_solve_sm)
    T k[5] = {T(0), T(0), T(0), T(0), T(0)};  // their l1, l2, 1/u0, u1/u0, u2/u0
};

template <typename T>
struct V4 {
    T x, y, z, w;
};

__device__ __forceinline__ V4<float> ld4(const float* p) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ V4<double> ld4(const double* p) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    return {a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ void ld2(const float* p, float& a, float& b) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    a = v.x;
    b = v.y;
}
__device__ __forceinline__ void ld2(const double* p, double& a, double& b) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    a = v.x;
    b = v.y;
}

constexpr unsigned kFull = 0xffffffffu;

// Explicitly rounded multiply-adds: the solver's arithmetic is fixed in the
// source, so every kernel that inlines it (standalone, batched persistent,
// batched per phase) rounds identically and the results agree bit for bit.
__device__ __forceinline__ float fmadd(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double fmul(double a, double b) { return __dmul_rn(a, b); }

// r . a for a 4-vector row r, as an explicit multiply-add chain
template <typename T>
__device__ __forceinline__ T dot4(const V4<T>& r, const T (&a)[4]) {
    return fmadd(r.x, a[0], fmadd(r.y, a[1], fmadd(r.z, a[2], fmul(r.w, a[3]))));
}

// Solve L lines of the same operator together; line q's rows lane*M ..
// lane*M+M-1 are in v[q][] (rhs in, solution out).  Every coefficient load
// serves the L lines, and their L recurrences are independent chains.
template <typename T, int M, int L>
__device__ __forceinline__ void warp_lines_solve(T (&v)[L][M], const WCoef<T>& cf, int lane) {
    const bool per = cf.periodic;
    // ---- forward elimination: zero-start pass over the chunk
    T y1[L], y2[L], acc[L][4];
#pragma unroll
    for (int q = 0; q < L; ++q) {
        y1[q] = y2[q] = T(0);
        acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = T(0);
    }
#pragma unroll
    for (int i = 0; i < M; ++i) {
        const V4<T> c = ld4(cf.fwd + (i * 32 + lane) * 4);
#pragma unroll
        for (int q = 0; q < L; ++q) {
            const T y = fmadd(-c.x, y1[q], fmadd(-c.y, y2[q], v[q][i]));
            y2[q] = y1[q];
            y1[q] = y;
        }
        if (per) {
            const V4<T> w = ld4(cf.W + (i * 32 + lane) * 4);
#pragma unroll
            for (int q = 0; q < L; ++q) {
                acc[q][0] = fmadd(w.x, v[q][i], acc[q][0]);
                acc[q][1] = fmadd(w.y, v[q][i], acc[q][1]);
                acc[q][2] = fmadd(w.z, v[q][i], acc[q][2]);
                acc[q][3] = fmadd(w.w, v[q][i], acc[q][3]);
            }
        }
    }
    // inclusive scan of the chunk end states over lanes 0..lane
    T q0[L], q1[L];
#pragma unroll
    for (int q = 0; q < L; ++q) {
        q0[q] = y1[q];
        q1[q] = y2[q];
    }
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int d = 1 << s;
        T o0[L], o1[L];
#pragma unroll
        for (int q = 0; q < L; ++q) {
            o0[q] = __shfl_up_sync(kFull, q0[q], d);
            o1[q] = __shfl_up_sync(kFull, q1[q], d);
        }
        if (lane >= d) {
            const V4<T> P = ld4(cf.Pf + (s * 32 + lane) * 4);
#pragma unroll
            for (int q = 0; q < L; ++q) {
                q0[q] = fmadd(P.x, o0[q], fmadd(P.y, o1[q], q0[q]));
                q1[q] = fmadd(P.z, o0[q], fmadd(P.w, o1[q], q1[q]));
            }
        }
    }
#pragma unroll
    for (int q = 0; q < L; ++q) {
        y1[q] = __shfl_up_sync(kFull, q0[q], 1);
        y2[q] = __shfl_up_sync(kFull, q1[q], 1);
        if (lane == 0) y1[q] = y2[q] = T(0);
    }
#pragma unroll
    for (int i = 0; i < M; ++i) {
        const V4<T> c = ld4(cf.fwd + (i * 32 + lane) * 4);
#pragma unroll
        for (int q = 0; q < L; ++q) {
            const T y = fmadd(-c.x, y1[q], fmadd(-c.y, y2[q], v[q][i]));
            y2[q] = y1[q];
            y1[q] = y;
            v[q][i] = fmul(y, c.z);
        }
    }
    // ---- Woodbury right-hand side s = S W^T r (warp reduction)
    T sv[L][4];
#pragma unroll
    for (int q = 0; q < L; ++q) sv[q][0] = sv[q][1] = sv[q][2] = sv[q][3] = T(0);
    if (per) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int q = 0; q < L; ++q)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[q][e] += __shfl_xor_sync(kFull, acc[q][e], o);
        const V4<T> r0 = ld4(cf.S), r1 = ld4(cf.S + 4), r2 = ld4(cf.S + 8), r3 = ld4(cf.S + 12);
#pragma unroll
        for (int q = 0; q < L; ++q) {
            sv[q][0] = dot4(r0, acc[q]);
            sv[q][1] = dot4(r1, acc[q]);
            sv[q][2] = dot4(r2, acc[q]);
            sv[q][3] = dot4(r3, acc[q]);
        }
    }
    // ---- back substitution: zero-start pass over the chunk (bottom row first)
    T x1[L], x2[L];
#pragma unroll
    for (int q = 0; q < L; ++q) x1[q] = x2[q] = T(0);
#pragma unroll
    for (int i = M - 1; i >= 0; --i) {
        T u1, u2;
        ld2(cf.bwd + (i * 32 + lane) * 2, u1, u2);
#pragma unroll
        for (int q = 0; q < L; ++q) {
            const T x = fmadd(-u1, x1[q], fmadd(-u2, x2[q], v[q][i]));
            x2[q] = x1[q];
            x1[q] = x;
        }
    }
    // inclusive scan from the last lane down
#pragma unroll
    for (int q = 0; q < L; ++q) {
        q0[q] = x1[q];
        q1[q] = x2[q];
    }
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int d = 1 << s;
        T o0[L], o1[L];
#pragma unroll
        for (int q = 0; q < L; ++q) {
            o0[q] = __shfl_down_sync(kFull, q0[q], d);
            o1[q] = __shfl_down_sync(kFull, q1[q], d);
        }
        if (lane + d < 32) {
            const V4<T> P = ld4(cf.Pb + (s * 32 + lane) * 4);
#pragma unroll
            for (int q = 0; q < L; ++q) {
                q0[q] = fmadd(P.x, o0[q], fmadd(P.y, o1[q], q0[q]));
                q1[q] = fmadd(P.z, o0[q], fmadd(P.w, o1[q], q1[q]));
            }
        }
    }
#pragma unroll
    for (int q = 0; q < L; ++q) {
        x1[q] = __shfl_down_sync(kFull, q0[q], 1);
        x2[q] = __shfl_down_sync(kFull, q1[q], 1);
        if (lane == 31) x1[q] = x2[q] = T(0);
    }
#pragma unroll
    for (int i = M - 1; i >= 0; --i) {
        T u1, u2;
        ld2(cf.bwd + (i * 32 + lane) * 2, u1, u2);
        V4<T> z = {T(0), T(0), T(0), T(0)};
        if (per) z = ld4(cf.Z + (i * 32 + lane) * 4);
#pragma unroll
        for (int q = 0; q < L; ++q) {
            const T x = fmadd(-u1, x1[q], fmadd(-u2, x2[q], v[q][i]));
            x2[q] = x1[q];
            x1[q] = x;
            T o = x;
            if (per) o = fmadd(-z.x, sv[q][0], fmadd(-z.y, sv[q][1], fmadd(-z.z, sv[q][2], fmadd(-z.w, sv[q][3], o))));
            v[q][i] = o;
        }
    }
}

// One line: rows lane*M .. lane*M+M-1 in v[].
template <typename T, int M>
__device__ __forceinline__ void warp_line_solve(T (&v)[M], const WCoef<T>& cf, int lane) {
    warp_lines_solve<T, M, 1>(*reinterpret_cast<T(*)[1][M]>(&v), cf, lane);
}


// The same solve of one line with its rows in shared memory: v(i) is a
// reference to row lane*M + i.  The arithmetic and its order are those of
// warp_lines_solve with L = 1; the rows are not held in registers, which
// keeps lines of 257..1024 cells at a few dozen registers per thread (the
// register form needs 150 or more), so several CTAs share an SM and hide each
// other's latency.  Interior rows (WCoef r0, r1; see interior_rows) take
// constant factors from registers, so only the rows near the line's ends load
// table entries: those loads were the kernel's bottleneck (L1 throughput).
template <typename T, int M, typename V>
__device__ __forceinline__ void warp_line_solve_sm(V&& v, const WCoef<T>& cf, int lane) {
    const bool per = cf.periodic;
    // rows [r0, r1) take the interior constants instead of their table rows
    // (the tables hold the same values there; W and Z are negligible)
    auto inner = [&](int i) {
        const int row = lane * M + i;
        return row >= cf.r0 && row < cf.r1;
    };
    auto fwd = [&](int i) {
        V4<T> c = {cf.k[0], cf.k[1], cf.k[2], T(0)};
        if (!inner(i)) c = ld4(cf.fwd + (i * 32 + lane) * 4);
        return c;
    };
    auto bwd = [&](int i, T& u1, T& u2) {
        u1 = cf.k[3];
        u2 = cf.k[4];
        if (!inner(i)) ld2(cf.bwd + (i * 32 + lane) * 2, u1, u2);
    };
    // ---- forward elimination: zero-start pass over the chunk
    T y1 = T(0), y2 = T(0), acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll 8
    for (int i = 0; i < M; ++i) {
        const V4<T> c = fwd(i);
        const T vi = v(i);
        const T y = fmadd(-c.x, y1, fmadd(-c.y, y2, vi));
        y2 = y1;
        y1 = y;
        if (per && !inner(i)) {
            const V4<T> w = ld4(cf.W + (i * 32 + lane) * 4);
            acc[0] = fmadd(w.x, vi, acc[0]);
            acc[1] = fmadd(w.y, vi, acc[1]);
            acc[2] = fmadd(w.z, vi, acc[2]);
            acc[3] = fmadd(w.w, vi, acc[3]);
        }
    }
    // inclusive scan of the chunk end states over lanes 0..lane
    T q0 = y1, q1 = y2;
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int d = 1 << s;
        const T o0 = __shfl_up_sync(kFull, q0, d);
        const T o1 = __shfl_up_sync(kFull, q1, d);
        if (lane >= d) {
            const V4<T> P = ld4(cf.Pf + (s * 32 + lane) * 4);
            q0 = fmadd(P.x, o0, fmadd(P.y, o1, q0));
            q1 = fmadd(P.z, o0, fmadd(P.w, o1, q1));
        }
    }
    y1 = __shfl_up_sync(kFull, q0, 1);
    y2 = __shfl_up_sync(kFull, q1, 1);
    if (lane == 0) y1 = y2 = T(0);
#pragma unroll 8
    for (int i = 0; i < M; ++i) {
        const V4<T> c = fwd(i);
        const T y = fmadd(-c.x, y1, fmadd(-c.y, y2, v(i)));
        y2 = y1;
        y1 = y;
        v(i) = fmul(y, c.z);
    }
    // ---- Woodbury right-hand side s = S W^T r (warp reduction)
    T sv[4] = {T(0), T(0), T(0), T(0)};
    if (per) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[e] += __shfl_xor_sync(kFull, acc[e], o);
        const V4<T> r0 = ld4(cf.S), r1 = ld4(cf.S + 4), r2 = ld4(cf.S + 8), r3 = ld4(cf.S + 12);
        sv[0] = dot4(r0, acc);
        sv[1] = dot4(r1, acc);
        sv[2] = dot4(r2, acc);
        sv[3] = dot4(r3, acc);
    }
    // ---- back substitution: zero-start pass over the chunk (bottom row first)
    T x1 = T(0), x2 = T(0);
#pragma unroll 8
    for (int i = M - 1; i >= 0; --i) {
        T u1, u2;
        bwd(i, u1, u2);
        const T x = fmadd(-u1, x1, fmadd(-u2, x2, v(i)));
        x2 = x1;
        x1 = x;
    }
    // inclusive scan from the last lane down
    q0 = x1;
    q1 = x2;
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int d = 1 << s;
        const T o0 = __shfl_down_sync(kFull, q0, d);
        const T o1 = __shfl_down_sync(kFull, q1, d);
        if (lane + d < 32) {
            const V4<T> P = ld4(cf.Pb + (s * 32 + lane) * 4);
            q0 = fmadd(P.x, o0, fmadd(P.y, o1, q0));
            q1 = fmadd(P.z, o0, fmadd(P.w, o1, q1));
        }
    }
    x1 = __shfl_down_sync(kFull, q0, 1);
    x2 = __shfl_down_sync(kFull, q1, 1);
    if (lane == 31) x1 = x2 = T(0);
#pragma unroll 8
    for (int i = M - 1; i >= 0; --i) {
        T u1, u2;
        bwd(i, u1, u2);
        const T x = fmadd(-u1, x1, fmadd(-u2, x2, v(i)));
        x2 = x1;
        x1 = x;
        T o = x;
        if (per && !inner(i)) {
            const V4<T> z = ld4(cf.Z + (i * 32 + lane) * 4);
            o = fmadd(-z.x, sv[0], fmadd(-z.y, sv[1], fmadd(-z.z, sv[2], fmadd(-z.w, sv[3], o))));
        }
        v(i) = o;
    }
}

// Lines solved together per warp: CH_SOLVE_LINES (default 2) while a lane
// holds at most 32 bytes of rows, else one.
#ifndef CH_SOLVE_LINES
#define CH_SOLVE_LINES 2
#endif
template <typename T, int M>
struct LinesPerWarp {
    static constexpr int value = M * sizeof(T) <= 32 ? CH_SOLVE_LINES : 1;
};

// x-lines (contiguous): one warp per L consecutive lines, lane chunks read
// and written directly (16-byte vectors when the line and chunk are aligned).
// Lines at or past nlines are solved on zeros and not stored.
template <typename T, int M, int L>
__device__ __forceinline__ void solve_x_lines(T* a, int64_t line0, int64_t nlines, int nx, const WCoef<T>& cf) {
    const int lane = threadIdx.x & 31;
    const int j0 = lane * M;
    T v[L][M];
    constexpr int VEC = 16 / sizeof(T);
    const bool vec = (M % VEC == 0) && (nx % VEC == 0) && (j0 + M <= nx);
#pragma unroll
    for (int q = 0; q < L; ++q) {
        const bool live = line0 + q < nlines;
        const T* p = a + (line0 + q) * nx;
        if (vec && live) {
#pragma unroll
            for (int i = 0; i < M; i += VEC) {
                if (sizeof(T) == 4) {
                    const float4 t = *reinterpret_cast<const float4*>(p + j0 + i);
                    v[q][i] = (T)t.x; v[q][i + 1] = (T)t.y; v[q][i + 2] = (T)t.z; v[q][i + 3] = (T)t.w;
                } else {
                    const double2 t = *reinterpret_cast<const double2*>(p + j0 + i);
                    v[q][i] = (T)t.x; v[q][i + 1] = (T)t.y;
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < M; ++i) v[q][i] = (live && j0 + i < nx) ? p[j0 + i] : T(0);
        }
    }
    warp_lines_solve<T, M, L>(v, cf, lane);
#pragma unroll
    for (int q = 0; q < L; ++q) {
        if (line0 + q >= nlines) continue;
        T* p = a + (line0 + q) * nx;
        if (vec) {
#pragma unroll
            for (int i = 0; i < M; i += VEC) {
                if (sizeof(T) == 4) {
                    float4 t;
                    t.x = (float)v[q][i]; t.y = (float)v[q][i + 1]; t.z = (float)v[q][i + 2]; t.w = (float)v[q][i + 3];
                    *reinterpret_cast<float4*>(p + j0 + i) = t;
                } else {
                    double2 t;
                    t.x = (double)v[q][i]; t.y = (double)v[q][i + 1];
                    *reinterpret_cast<double2*>(p + j0 + i) = t;
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < M; ++i)
                if (j0 + i < nx) p[j0 + i] = v[q][i];
        }
    }
}

template <typename T, int M>
__device__ __forceinline__ void solve_x_line(T* a, int64_t line, int nx, const WCoef<T>& cf) {
    solve_x_lines<T, M, 1>(a, line, line + 1, nx, cf);
}

template <typename T, int M>
__global__ void __launch_bounds__(256)
ch_solve_x(T* __restrict__ a, int64_t nlines, int nx, WCoef<T> cf) {
    pdl_wait();
    pdl_launch_dependents();
    constexpr int L = LinesPerWarp<T, M>::value;
    const int64_t line0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * L;
    if (line0 >= nlines) return;  // whole warp
    solve_x_lines<T, M, L>(a, line0, nlines, nx, cf);
}

// x-lines of 257..1024 cells (M = 16, 32): one warp per line, the line staged
// in shared memory with one pad element after every chunk of M rows (lane l's
// row i at l (M + 1) + i, so the lanes' chunk accesses and the row-wise
// staging are both free of bank conflicts), and solved there by
// warp_line_solve_sm.  Rows past nx are zero padding.
#ifndef CH_XSM_MAX_BLOCKS
#define CH_XSM_MAX_BLOCKS 4
#endif
template <typename T, int M>
struct XSmShape {
    static constexpr int kStride = M + 1;
    static constexpr size_t kWarpBytes = (size_t)32 * kStride * sizeof(T);
    static constexpr int kFit = (int)((200 * 1024) / (8 * kWarpBytes));  // CTAs whose buffers fit an SM
    static constexpr int kMinBlocks = kFit < 1 ? 1 : (kFit > CH_XSM_MAX_BLOCKS ? CH_XSM_MAX_BLOCKS : kFit);
};

template <typename T, int M>
__global__ void __launch_bounds__(256, XSmShape<T, M>::kMinBlocks)
ch_solve_x_sm(T* __restrict__ a, int64_t nlines, int nx, WCoef<T> cf) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_wait();
    pdl_launch_dependents();
    constexpr int S = XSmShape<T, M>::kStride;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t line = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (line >= nlines) return;  // whole warp
    T* sv = reinterpret_cast<T*>(smem_raw) + (size_t)warp * 32 * S;
    T* p = a + line * nx;
    constexpr int VEC = 16 / sizeof(T);
    if (nx % VEC == 0) {  // 16-byte vectors (the field is 256-byte aligned, rows are multiples of 16 bytes)
        for (int e = lane * VEC; e < 32 * M; e += 32 * VEC) {
            T t[VEC];
            if (e < nx) {
                if constexpr (sizeof(T) == 4) {
                    const float4 g = *reinterpret_cast<const float4*>(p + e);
                    t[0] = g.x; t[1] = g.y; t[2] = g.z; t[3] = g.w;
                } else {
                    const double2 g = *reinterpret_cast<const double2*>(p + e);
                    t[0] = g.x; t[1] = g.y;
                }
            } else {
#pragma unroll
                for (int k = 0; k < VEC; ++k) t[k] = T(0);
            }
#pragma unroll
            for (int k = 0; k < VEC; ++k) sv[((e + k) / M) * S + (e + k) % M] = t[k];
        }
    } else {
        for (int e = lane; e < 32 * M; e += 32) sv[(e / M) * S + e % M] = e < nx ? p[e] : T(0);
    }
    __syncwarp();
    T* mine = sv + lane * S;
    warp_line_solve_sm<T, M>([&](int i) -> T& { return mine[i]; }, cf, lane);
    __syncwarp();
    if (nx % VEC == 0) {
        for (int e = lane * VEC; e < nx; e += 32 * VEC) {
            if constexpr (sizeof(T) == 4) {
                float4 g;
                g.x = sv[(e / M) * S + e % M];
                g.y = sv[((e + 1) / M) * S + (e + 1) % M];
                g.z = sv[((e + 2) / M) * S + (e + 2) % M];
                g.w = sv[((e + 3) / M) * S + (e + 3) % M];
                *reinterpret_cast<float4*>(p + e) = g;
            } else {
                double2 g;
                g.x = sv[(e / M) * S + e % M];
                g.y = sv[((e + 1) / M) * S + (e + 1) % M];
                *reinterpret_cast<double2*>(p + e) = g;
            }
        }
    } else {
        for (int e = lane; e < nx; e += 32) p[e] = sv[(e / M) * S + e % M];
    }
}

// y- or z-lines (strided).  A CTA of 16 warps owns NC = 32 (or 16)
// consecutive x of one outer position: the [n][NC] tile is staged through
// shared memory with coalesced NC-wide rows; element (row j, column c) sits at
// j*NC + (c ^ (j/M) mod NC), so both the row-wise staging and the per-lane
// chunk reads of one column are bank-conflict free.  Warp w solves columns
// w, w + W, ... (W warps per CTA: 16 for short lines, 8 for long ones, which
// need more registers per lane).  With UPDATE the solved increment is added to
// C (Eq. eq-fac-3: q^{l+1} = q^l + dq) and non-finite results raise a flag.
// FP64 lines of 1024 cells use 16-column tiles, so the tile (128 KB) fits the
// shared memory of a CTA.
#ifndef CH_YZ_COLS_F32_1024
#define CH_YZ_COLS_F32_1024 16
#endif
#ifndef CH_YZ_COLS_F32_512
#define CH_YZ_COLS_F32_512 32
#endif
#ifndef CH_YZ_MAX_BLOCKS
#define CH_YZ_MAX_BLOCKS 3
#endif
template <typename T, int M>
struct YZShape {
    static constexpr bool kLong = M * sizeof(T) >= 64;
    static constexpr int kWarps = kLong ? 8 : 16;
    // lines of 257..1024 cells are solved in the tile itself (warp_line_solve_sm)
    static constexpr bool kSm = M >= 16;
    static constexpr int kCols = (sizeof(T) == 4 && M == 32)   ? CH_YZ_COLS_F32_1024
                                 : (sizeof(T) == 4 && M == 16) ? CH_YZ_COLS_F32_512
                                 : ((size_t)32 * M * 32 * sizeof(T) > 227 * 1024 ? 16 : 32);
    // tiles solved in place carry one pad element after every lane chunk of M rows
    static constexpr size_t kTileBytes = ((size_t)32 * M * kCols + (kSm ? 32 : 0)) * sizeof(T);
    static constexpr int kSmBlocks = (int)((227 * 1024) / kTileBytes) > CH_YZ_MAX_BLOCKS
                                         ? CH_YZ_MAX_BLOCKS
                                         : (int)((227 * 1024) / kTileBytes);
    static constexpr int kMinBlocks = kSm ? (kSmBlocks < 1 ? 1 : kSmBlocks) : (kLong ? 1 : 2);
};

// One [n][NC] tile (tile index = x-block + xblocks * outer) solved by the
// kYZWarps warps of a CTA; s is the CTA's shared tile of 32 M x NC values.
template <typename T, int M, bool UPDATE, int kYZWarps, int NC = 32>
__device__ __forceinline__ void solve_yz_tile(T* a, T* Cf, int nx, int64_t outer_stride,
                                              int64_t line_stride, const WCoef<T>& cf, unsigned int* status,
                                              int64_t tile, T* s) {
    static_assert(NC == 16 || NC == 32, "tile width");
    constexpr int kRowsPerPass = kYZWarps * 32 / NC;
    const int n = cf.n;
    const int xblocks = (nx + NC - 1) / NC;
    const int xb = (int)(tile % xblocks);
    const int64_t outer = tile / xblocks;
    const int i0 = xb * NC;
    const int nl = min(NC, nx - i0);
    const int64_t base = outer * outer_stride + i0;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x, c = tid % NC, r0 = tid / NC;
    // Layout: long lines (M >= 16, solved in place) put lane chunk l (rows
    // l M .. l M + M - 1) at l (M NC + 1), rows of NC contiguous: lane l's row i
    // of any column is then in bank (l + i NC + col) mod 32, distinct over the
    // warp, and the row-wise staging is contiguous.  Short lines (copied to
    // registers) swizzle the column by the chunk index instead.
    auto slot = [&](int j, int col) {
        if constexpr (M >= 16)
            return j * NC + j / M + col;
        else
            return j * NC + (col ^ ((j / M) & (NC - 1)));
    };
    __syncthreads();  // the tile may still be read by a previous item of this CTA
    // stage rows asynchronously (zero padding past n and past the ragged x edge)
#pragma unroll
    for (int j = r0; j < 32 * M; j += kRowsPerPass) {
        if (j < n && c < nl)
            cp_async_elem(&s[slot(j, c)], a + base + (int64_t)j * line_stride + c);
        else
            s[slot(j, c)] = T(0);
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31;
    constexpr int L = LinesPerWarp<T, M>::value;
    if constexpr (M >= 16) {
        // solved in place in the tile: lane l's row i of column col is at
        // (l M + i) NC + (col ^ (l mod NC))
#pragma unroll 1
        for (int col = warp; col < NC; col += kYZWarps) {
            T* base = s + (size_t)lane * (M * NC + 1) + col;
            warp_line_solve_sm<T, M>([&](int i) -> T& { return base[i * NC]; }, cf, lane);
        }
    } else
#pragma unroll 1
    for (int col = warp * L; col < NC; col += kYZWarps * L) {
        T v[L][M];
#pragma unroll
        for (int q = 0; q < L; ++q)
#pragma unroll
            for (int i = 0; i < M; ++i) v[q][i] = s[slot(lane * M + i, col + q)];
        warp_lines_solve<T, M, L>(v, cf, lane);
#pragma unroll
        for (int q = 0; q < L; ++q)
#pragma unroll
            for (int i = 0; i < M; ++i) s[slot(lane * M + i, col + q)] = v[q][i];
    }
    __syncthreads();
    bool bad = false;
#pragma unroll
    for (int j = r0; j < 32 * M; j += kRowsPerPass) {
        if (j < n && c < nl) {
            const int64_t idx = base + (int64_t)j * line_stride + c;
            const T d = s[slot(j, c)];
            if (UPDATE) {
                const T cnew = Cf[idx] + d;
                bad |= !isfinite(cnew);
                Cf[idx] = cnew;
            } else {
                a[idx] = d;
            }
        }
    }
    if (UPDATE && bad) atomicOr(status, 1u);
}

template <typename T, int M, bool UPDATE>
__global__ void __launch_bounds__(YZShape<T, M>::kWarps * 32, YZShape<T, M>::kMinBlocks)
ch_solve_yz(T* __restrict__ a, T* __restrict__ Cf, int nx, int64_t outer_stride, int64_t line_stride,
            WCoef<T> cf, unsigned int* status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_wait();
    pdl_launch_dependents();
    solve_yz_tile<T, M, UPDATE, YZShape<T, M>::kWarps, YZShape<T, M>::kCols>(a, Cf, nx, outer_stride, line_stride, cf,
                                                                             status, blockIdx.x,
                                                                             reinterpret_cast<T*>(smem_raw));
}

// L adjacent values of one row as one shared- or global-memory vector access
// (L = 1, 2 or 4 floats, 1 or 2 doubles; the address is L-element aligned).
template <typename T, int L>
__device__ __forceinline__ void vld(const T* p, T (&v)[L]) {
    if constexpr (L == 1) {
        v[0] = *p;
    } else if constexpr (L == 2 && sizeof(T) == 4) {
        const float2 t = *reinterpret_cast<const float2*>(p);
        v[0] = t.x; v[1] = t.y;
    } else if constexpr (L == 2) {
        const double2 t = *reinterpret_cast<const double2*>(p);
        v[0] = t.x; v[1] = t.y;
    } else {
        static_assert(L == 4 && sizeof(T) == 4, "vector width");
        const float4 t = *reinterpret_cast<const float4*>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
}
template <typename T, int L>
__device__ __forceinline__ void vst(T* p, const T (&v)[L]) {
    if constexpr (L == 1) {
        *p = v[0];
    } else if constexpr (L == 2 && sizeof(T) == 4) {
        *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
    } else if constexpr (L == 2) {
        *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    } else {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
}
// cp.async of L adjacent elements (4 L or 8 L bytes, both addresses aligned to that size)
template <typename T, int L>
__device__ __forceinline__ void cp_async_vec(T* smem, const T* gmem) {
    constexpr int kBytes = L * (int)sizeof(T);
    if constexpr (kBytes == 16) {
        cp_async_16(smem, gmem);
    } else {
        const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gmem), "n"(kBytes) : "memory");
    }
}

// warp_line_solve_sm for L lines of the same operator at once: row i of the
// lane's chunk holds the L lines' values side by side at p + i * stride, so
// one L-wide shared-memory access serves every line and the L recurrences are
// independent chains; the interior test, the table loads of the end rows and
// the scans' span matrices are shared by the L lines.  Each line's arithmetic
// is that of warp_line_solve_sm, in the same order, so the results agree with
// it bit for bit.
// CH_SMV_TABLE = 1: the LU factors of every row come from the tables (one
// L1-resident load per row, shared by the L lines) instead of register
// constants on the interior rows; the periodic correction still skips the
// interior rows.
#ifndef CH_SMV_TABLE
#define CH_SMV_TABLE 0
#endif
// rows per unrolled step of the solver's passes
#ifndef CH_SMV_UNROLL
#define CH_SMV_UNROLL 8
#endif
constexpr int kSmvUnroll = CH_SMV_UNROLL;
template <typename T, int M, int L>
__device__ __forceinline__ void warp_lines_solve_smv(T* p, int stride, const WCoef<T>& cf, int lane) {
    const bool per = cf.periodic;
    const int lo = cf.r0 - lane * M, hi = cf.r1 - lane * M;  // this chunk's interior rows: [lo, hi)
    auto inner = [&](int i) { return i >= lo && i < hi; };
    auto fwd = [&](int i) {
        if constexpr (CH_SMV_TABLE) {
            return ld4(cf.fwd + (i * 32 + lane) * 4);
        } else {
            V4<T> c = {cf.k[0], cf.k[1], cf.k[2], T(0)};
            if (!inner(i)) c = ld4(cf.fwd + (i * 32 + lane) * 4);
            return c;
        }
    };
    auto bwd = [&](int i, T& u1, T& u2) {
        if constexpr (CH_SMV_TABLE) {
            ld2(cf.bwd + (i * 32 + lane) * 2, u1, u2);
        } else {
            u1 = cf.k[3];
            u2 = cf.k[4];
            if (!inner(i)) ld2(cf.bwd + (i * 32 + lane) * 2, u1, u2);
        }
    };
    // ---- forward elimination: zero-start pass over the chunk
    T y1[L], y2[L], acc[L][4];
#pragma unroll
    for (int q = 0; q < L; ++q) {
        y1[q] = y2[q] = T(0);
        acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = T(0);
    }
#pragma unroll kSmvUnroll
    for (int i = 0; i < M; ++i) {
        const V4<T> c = fwd(i);
        T vi[L];
        vld<T, L>(p + i * stride, vi);
#pragma unroll
        for (int q = 0; q < L; ++q) {
            const T y = fmadd(-c.x, y1[q], fmadd(-c.y, y2[q], vi[q]));
            y2[q] = y1[q];
            y1[q] = y;
        }
        if (per && !inner(i)) {
            const V4<T> w = ld4(cf.W + (i * 32 + lane) * 4);
#pragma unroll
            for (int q = 0; q < L; ++q) {
                acc[q][0] = fmadd(w.x, vi[q], acc[q][0]);
                acc[q][1] = fmadd(w.y, vi[q], acc[q][1]);
                acc[q][2] = fmadd(w.z, vi[q], acc[q][2]);
                acc[q][3] = fmadd(w.w, vi[q], acc[q][3]);
            }
        }
    }
    // inclusive scan of the chunk end states over lanes 0..lane
    T q0[L], q1[L];
#pragma unroll
    for (int q = 0; q < L; ++q) {
        q0[q] = y1[q];
        q1[q] = y2[q];
    }
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int d = 1 << s;
        T o0[L], o1[L];
#pragma unroll
        for (int q = 0; q < L; ++q) {
            o0[q] = __shfl_up_sync(kFull, q0[q], d);
            o1[q] = __shfl_up_sync(kFull, q1[q], d);
        }
        if (lane >= d) {
            const V4<T> P = ld4(cf.Pf + (s * 32 + lane) * 4);
#pragma unroll
            for (int q = 0; q < L; ++q) {
                q0[q] = fmadd(P.x, o0[q], fmadd(P.y, o1[q], q0[q]));
                q1[q] = fmadd(P.z, o0[q], fmadd(P.w, o1[q], q1[q]));
            }
        }
    }
#pragma unroll
    for (int q = 0; q < L; ++q) {
        y1[q] = __shfl_up_sync(kFull, q0[q], 1);
        y2[q] = __shfl_up_sync(kFull, q1[q], 1);
        if (lane == 0) y1[q] = y2[q] = T(0);
    }
#pragma unroll kSmvUnroll
    for (int i = 0; i < M; ++i) {
        const V4<T> c = fwd(i);
        T vi[L];
        vld<T, L>(p + i * stride, vi);
#pragma unroll
        for (int q = 0; q < L; ++q) {
            const T y = fmadd(-c.x, y1[q], fmadd(-c.y, y2[q], vi[q]));
            y2[q] = y1[q];
            y1[q] = y;
            vi[q] = fmul(y, c.z);
        }
        vst<T, L>(p + i * stride, vi);
    }
    // ---- Woodbury right-hand side s = S W^T r (warp reduction)
    T sv[L][4];
#pragma unroll
    for (int q = 0; q < L; ++q) sv[q][0] = sv[q][1] = sv[q][2] = sv[q][3] = T(0);
    if (per) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int q = 0; q < L; ++q)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[q][e] += __shfl_xor_sync(kFull, acc[q][e], o);
        const V4<T> r0 = ld4(cf.S), r1 = ld4(cf.S + 4), r2 = ld4(cf.S + 8), r3 = ld4(cf.S + 12);
#pragma unroll
        for (int q = 0; q < L; ++q) {
            sv[q][0] = dot4(r0, acc[q]);
            sv[q][1] = dot4(r1, acc[q]);
            sv[q][2] = dot4(r2, acc[q]);
            sv[q][3] = dot4(r3, acc[q]);
        }
    }
    // ---- back substitution: zero-start pass over the chunk (bottom row first)
    T x1[L], x2[L];
#pragma unroll
    for (int q = 0; q < L; ++q) x1[q] = x2[q] = T(0);
#pragma unroll kSmvUnroll
    for (int i = M - 1; i >= 0; --i) {
        T u1, u2;
        bwd(i, u1, u2);
        T vi[L];
        vld<T, L>(p + i * stride, vi);
#pragma unroll
        for (int q = 0; q < L; ++q) {
            const T x = fmadd(-u1, x1[q], fmadd(-u2, x2[q], vi[q]));
            x2[q] = x1[q];
            x1[q] = x;
        }
    }
    // inclusive scan from the last lane down
#pragma unroll
    for (int q = 0; q < L; ++q) {
        q0[q] = x1[q];
        q1[q] = x2[q];
    }
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int d = 1 << s;
        T o0[L], o1[L];
#pragma unroll
        for (int q = 0; q < L; ++q) {
            o0[q] = __shfl_down_sync(kFull, q0[q], d);
            o1[q] = __shfl_down_sync(kFull, q1[q], d);
        }
        if (lane + d < 32) {
            const V4<T> P = ld4(cf.Pb + (s * 32 + lane) * 4);
#pragma unroll
            for (int q = 0; q < L; ++q) {
                q0[q] = fmadd(P.x, o0[q], fmadd(P.y, o1[q], q0[q]));
                q1[q] = fmadd(P.z, o0[q], fmadd(P.w, o1[q], q1[q]));
            }
        }
    }
#pragma unroll
    for (int q = 0; q < L; ++q) {
        x1[q] = __shfl_down_sync(kFull, q0[q], 1);
        x2[q] = __shfl_down_sync(kFull, q1[q], 1);
        if (lane == 31) x1[q] = x2[q] = T(0);
    }
#pragma unroll kSmvUnroll
    for (int i = M - 1; i >= 0; --i) {
        T u1, u2;
        bwd(i, u1, u2);
        T vi[L];
        vld<T, L>(p + i * stride, vi);
        const bool edge = per && !inner(i);
        V4<T> z = {T(0), T(0), T(0), T(0)};
        if (edge) z = ld4(cf.Z + (i * 32 + lane) * 4);
#pragma unroll
        for (int q = 0; q < L; ++q) {
            const T x = fmadd(-u1, x1[q], fmadd(-u2, x2[q], vi[q]));
            x2[q] = x1[q];
            x1[q] = x;
            T o = x;
            if (edge) o = fmadd(-z.x, sv[q][0], fmadd(-z.y, sv[q][1], fmadd(-z.z, sv[q][2], fmadd(-z.w, sv[q][3], o))));
            vi[q] = o;
        }
        vst<T, L>(p + i * stride, vi);
    }
}

// y- or z-lines of 257..1024 cells, L adjacent lines per warp.  A CTA of
// NC / L warps owns NC consecutive x of one outer position; the [n][NC] tile
// sits in shared memory with lane chunk l (rows l M .. l M + M - 1) at
// l (M NC + L), rows of NC contiguous, and every L-column group of a row
// L-element aligned.  Staging and write-back move L adjacent columns per
// access (cp.async of 4 L bytes, vector stores), and warp w solves columns
// w L .. w L + L - 1 in the tile (warp_lines_solve_smv).  Lane l's L-wide
// access to row i lands in words (l L + 16 i + w L) mod 32 + 0..L-1: within
// each group of 32 / L lanes that the hardware serves together those are
// distinct, so the solve passes are free of bank conflicts.  Needs nx a
// multiple of L.  With UPDATE the increment is added to C and non-finite
// results raise the status flag.
// At most MAXB CTAs per SM (fewer where the tiles do not fit).
template <typename T, int M, int L, int NC, int MAXB>
struct YZVShape {
    static constexpr int kWarps = NC / L;
    static constexpr size_t kTileBytes = ((size_t)32 * M * NC + (size_t)32 * L) * sizeof(T);
    static constexpr int kFit = (int)((227 * 1024) / kTileBytes);
    static constexpr int kMinBlocks = kFit < 1 ? 1 : (kFit > MAXB ? MAXB : kFit);
};

template <typename T, int M, bool UPDATE, int L, int NC, int MAXB>
__global__ void __launch_bounds__(NC / L * 32, (YZVShape<T, M, L, NC, MAXB>::kMinBlocks))
ch_solve_yz_v(T* __restrict__ a, T* __restrict__ Cf, int nx, int64_t outer_stride, int64_t line_stride,
              WCoef<T> cf, unsigned int* status, int64_t ntiles) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_wait();
    pdl_launch_dependents();
    static_assert(NC % L == 0 && M * NC % 32 == 0, "tile shape");
    constexpr int G = NC / L;           // column groups of a row = warps of the CTA
    constexpr int kChunk = M * NC + L;  // elements of one lane chunk with its pad
    T* s = reinterpret_cast<T*>(smem_raw);
    const int n = cf.n;
    const int xblocks = (nx + NC - 1) / NC;
    const int tid = threadIdx.x, g = tid % G, rr = tid / G;  // column group g, rows rr, rr + 32, ...
    const int c = g * L;
    auto slot = [&](int j) { return (j / M) * kChunk + (j % M) * NC + c; };
    // tile t: NC consecutive x (nl of them inside the mesh, a multiple of L) of one outer position
    auto tile_base = [&](int64_t t, int& nl) {
        const int i0 = (int)(t % xblocks) * NC;
        nl = min(NC, nx - i0);
        return (t / xblocks) * outer_stride + i0;
    };
    // this thread's piece of row j of a tile, or zeros past the line or the ragged x edge
    auto stage_row = [&](int j, int64_t base, int nl) {
        if (j < n && c < nl) {
            cp_async_vec<T, L>(s + slot(j), a + base + (int64_t)j * line_stride + c);
        } else {
            T z[L];
#pragma unroll
            for (int q = 0; q < L; ++q) z[q] = T(0);
            vst<T, L>(s + slot(j), z);
        }
    };
    // A CTA takes tiles blockIdx.x, blockIdx.x + gridDim.x, ...  The write-back
    // of a tile is fused with the staging of the next: each thread re-fills the
    // slots it has just written out, so the next tile's loads run while the
    // other threads still store.
    int64_t t = blockIdx.x;
    if (t >= ntiles) return;
    int nl;
    int64_t base = tile_base(t, nl);
#pragma unroll 4
    for (int j = rr; j < 32 * M; j += 32) stage_row(j, base, nl);
    cp_async_commit();
    const int warp = tid >> 5, lane = tid & 31;
    bool bad = false;
    for (;;) {
        cp_async_wait<0>();
        __syncthreads();
        warp_lines_solve_smv<T, M, L>(s + (size_t)lane * kChunk + warp * L, NC, cf, lane);
        __syncthreads();
        const int64_t tn = t + gridDim.x;
        const bool more = tn < ntiles;
        int nln = 0;
        const int64_t basen = more ? tile_base(tn, nln) : 0;
        if constexpr (UPDATE) {
            // rows rr + 32 u (u < M) in batches of 8: the batch's C loads are
            // all issued before its first store (a store to C would otherwise
            // hold back the next row's load)
            constexpr int kB = M < 8 ? M : 8;
#pragma unroll 1
            for (int u0 = 0; u0 < M; u0 += kB) {
                T cv[kB][L];
#pragma unroll
                for (int u = 0; u < kB; ++u) {
                    const int j = rr + 32 * (u0 + u);
                    if (j < n && c < nl) vld<T, L>(Cf + base + (int64_t)j * line_stride + c, cv[u]);
                }
#pragma unroll
                for (int u = 0; u < kB; ++u) {
                    const int j = rr + 32 * (u0 + u);
                    if (j < n && c < nl) {
                        T d[L];
                        vld<T, L>(s + slot(j), d);
#pragma unroll
                        for (int q = 0; q < L; ++q) {
                            cv[u][q] += d[q];
                            bad |= !isfinite(cv[u][q]);
                        }
                        vst<T, L>(Cf + base + (int64_t)j * line_stride + c, cv[u]);
                    }
                    if (more) stage_row(j, basen, nln);
                }
            }
        } else {
#pragma unroll 4
            for (int j = rr; j < 32 * M; j += 32) {
                if (j < n && c < nl) {
                    T d[L];
                    vld<T, L>(s + slot(j), d);
                    vst<T, L>(a + base + (int64_t)j * line_stride + c, d);
                }
                if (more) stage_row(j, basen, nln);
            }
        }
        if (!more) break;
        cp_async_commit();
        t = tn;
        base = basen;
        nl = nln;
    }
    if (UPDATE && bad) atomicOr(status, 1u);
}

// x-lines of 257..1024 cells, L lines per warp (FP32, nx a multiple of 4): the
// warp's L lines sit in its shared buffer side by side, row i of lane chunk l
// at l (M L + L) + i L, so one L-wide access serves all L lines in
// warp_lines_solve_smv (lane l's access to row i lands in words
// L (l (M + 1) + i) mod 32 + 0..L-1, distinct within each group of 32 / L
// lanes served together).  Staging reads 16-byte vectors of each line and
// writes L-wide rows (at most 2-way bank conflicts); the write-back is the
// reverse.  Lines at or past nlines are solved on zeros and not stored.
#ifndef CH_XSMV_MAX_BLOCKS
#define CH_XSMV_MAX_BLOCKS 12
#endif
template <typename T, int M, int L, int W>
struct XSmvShape {
    static constexpr int kChunk = M * L + L;
    static constexpr size_t kWarpBytes = (size_t)32 * kChunk * sizeof(T);
    static constexpr int kFit = (int)((200 * 1024) / (W * kWarpBytes));
    // and whose registers fit: about 80 a thread for L = 2, 120 for L = 4
    static constexpr int kRegFit = 65536 / (W * 32 * (L <= 2 ? 80 : 120));
    static constexpr int kCap = kRegFit < CH_XSMV_MAX_BLOCKS ? kRegFit : CH_XSMV_MAX_BLOCKS;
    static constexpr int kMinBlocks = kFit < 1 ? 1 : (kFit > kCap ? kCap : kFit);
};

template <typename T, int M, int L, int W>
__global__ void __launch_bounds__(W * 32, (XSmvShape<T, M, L, W>::kMinBlocks))
ch_solve_x_smv(T* __restrict__ a, int64_t nlines, int nx, WCoef<T> cf) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_wait();
    pdl_launch_dependents();
    static_assert(sizeof(T) == 4 && M % 4 == 0, "FP32 rows in 16-byte vectors");
    constexpr int kChunk = XSmvShape<T, M, L, W>::kChunk;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t line0 = ((int64_t)blockIdx.x * W + warp) * L;
    if (line0 >= nlines) return;  // whole warp
    T* sv = reinterpret_cast<T*>(smem_raw) + (size_t)warp * 32 * kChunk;
    auto slot = [&](int e) { return (e / M) * kChunk + (e % M) * L; };
    // the lane's M / 4 vectors of each line, all loads issued before the
    // first shared store (batches of 4 vectors per line)
    constexpr int kNV = M / 4, kB = kNV < 4 ? kNV : 4;
#pragma unroll
    for (int v0 = 0; v0 < kNV; v0 += kB) {
        T t[kB][L][4];
#pragma unroll
        for (int b = 0; b < kB; ++b) {
            const int e = lane * 4 + 128 * (v0 + b);
#pragma unroll
            for (int q = 0; q < L; ++q) {
                if (e < nx && line0 + q < nlines) {
                    const float4 g = *reinterpret_cast<const float4*>(a + (line0 + q) * nx + e);
                    t[b][q][0] = g.x; t[b][q][1] = g.y; t[b][q][2] = g.z; t[b][q][3] = g.w;
                } else {
                    t[b][q][0] = t[b][q][1] = t[b][q][2] = t[b][q][3] = T(0);
                }
            }
        }
#pragma unroll
        for (int b = 0; b < kB; ++b) {
            const int e = lane * 4 + 128 * (v0 + b);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                T v[L];
#pragma unroll
                for (int q = 0; q < L; ++q) v[q] = t[b][q][k];
                vst<T, L>(sv + slot(e + k), v);
            }
        }
    }
    __syncwarp();
    warp_lines_solve_smv<T, M, L>(sv + (size_t)lane * kChunk, L, cf, lane);
    __syncwarp();
    for (int e = lane * 4; e < nx; e += 128) {
        T t[L][4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            T v[L];
            vld<T, L>(sv + slot(e + k), v);
#pragma unroll
            for (int q = 0; q < L; ++q) t[q][k] = v[q];
        }
#pragma unroll
        for (int q = 0; q < L; ++q)
            if (line0 + q < nlines)
                *reinterpret_cast<float4*>(a + (line0 + q) * nx + e) = make_float4(t[q][0], t[q][1], t[q][2], t[q][3]);
    }
}

// ---------------------------------------------------------------------------
// Column solver for y- and z-lines: the 32 lanes of a warp own 32 adjacent
// lines (consecutive x, so every row access is one coalesced 128-byte line),
// and warp w of the CTA owns rows [w R, w R + R) of all 32 lines in
// registers.  Each warp runs its row chunk from a zero state; the chunk end
// states are composed across warps through shared memory with the chunks'
// 2x2 transfer matrices (host-precomputed), then each warp reruns its chunk.
// Rows stream straight between HBM and registers: no staging tile.
// ---------------------------------------------------------------------------
template <typename T>
struct CCoef {
    const T* __restrict__ fwd;  // [rows][4]: l1, l2, 1/u0, 0
    const T* __restrict__ bwd;  // [rows][2]: u1/u0, u2/u0
    const T* __restrict__ W;    // [rows][4]  periodic only
    const T* __restrict__ Z;    // [rows][4]  periodic only
    const T* __restrict__ P;    // [NW][4]    forward chunk transfer matrices
    const T* __restrict__ Q;    // [NW][4]    backward chunk transfer matrices
    const T* __restrict__ S;    // [4][4]
    // two-column form: duplicated pairs
    const T* __restrict__ fwdp;   // [rows][4]: -l1, -l1, -l2, -l2
    const T* __restrict__ dinvp;  // [rows][2]: 1/u0, 1/u0
    const T* __restrict__ bwdp;   // [rows][4]: -u1/u0 (x2), -u2/u0 (x2)
    const T* __restrict__ Wp;     // [rows][8]: W_m (x2), periodic only
    const T* __restrict__ Zp;     // [rows][8]: -Z_m (x2), periodic only
    const T* __restrict__ K;      // [4][4] corner-form correction, periodic only
    int n;
    int periodic;
};

// Coefficient loads of the column solver.  They are volatile so that the
// compiler reloads a row's coefficients in each pass (they are L1-resident)
// instead of keeping R rows of them live in registers between passes.
__device__ __forceinline__ V4<float> ldv4(const float* p) {
    V4<float> r;
    asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
                 : "l"(p));
    return r;
}
__device__ __forceinline__ V4<double> ldv4(const double* p) {
    V4<double> r;
    asm volatile("ld.global.nc.v2.f64 {%0, %1}, [%2];" : "=d"(r.x), "=d"(r.y) : "l"(p));
    asm volatile("ld.global.nc.v2.f64 {%0, %1}, [%2];" : "=d"(r.z), "=d"(r.w) : "l"(p + 2));
    return r;
}
__device__ __forceinline__ void ldv2(const float* p, float& a, float& b) {
    asm volatile("ld.global.nc.v2.f32 {%0, %1}, [%2];" : "=f"(a), "=f"(b) : "l"(p));
}
__device__ __forceinline__ void ldv2(const double* p, double& a, double& b) {
    asm volatile("ld.global.nc.v2.f64 {%0, %1}, [%2];" : "=d"(a), "=d"(b) : "l"(p));
}

template <typename T, int R, int NW, bool UPDATE>
__global__ void __launch_bounds__(NW * 32, 1024 / (NW * 32))
ch_solve_cols(T* __restrict__ a, T* __restrict__ Cf, int nx, int64_t outer_stride, int64_t line_stride, CCoef<T> cf,
              unsigned int* status) {
    pdl_wait();
    pdl_launch_dependents();
    __shared__ T fq[NW][2][32];
    __shared__ T bq[NW][2][32];
    __shared__ T wacc[NW][4][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int xblocks = (nx + 31) >> 5;
    const int xb = blockIdx.x % xblocks;
    const int64_t outer = blockIdx.x / xblocks;
    const int i0 = xb * 32;
    const bool valid = i0 + lane < nx;
    const int64_t base = outer * outer_stride + i0 + lane;
    const int n = cf.n;
    const int j0 = w * R;
    const bool per = cf.periodic;
    T v[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int j = j0 + i;
        v[i] = (valid && j < n) ? a[base + (int64_t)j * line_stride] : T(0);
    }
    // forward elimination from a zero state over this warp's rows
    T y1 = T(0), y2 = T(0), acc0 = T(0), acc1 = T(0), acc2 = T(0), acc3 = T(0);
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const V4<T> c = ldv4(cf.fwd + 4 * (j0 + i));
        const T y = (v[i] - c.y * y2) - c.x * y1;
        y2 = y1;
        y1 = y;
        if (per) {
            const V4<T> ww = ldv4(cf.W + 4 * (j0 + i));
            acc0 += ww.x * v[i];
            acc1 += ww.y * v[i];
            acc2 += ww.z * v[i];
            acc3 += ww.w * v[i];
        }
    }
    fq[w][0][lane] = y1;
    fq[w][1][lane] = y2;
    if (per) {
        wacc[w][0][lane] = acc0;
        wacc[w][1][lane] = acc1;
        wacc[w][2][lane] = acc2;
        wacc[w][3][lane] = acc3;
    }
    __syncthreads();
    // incoming state: compose the chunks of warps 0 .. w-1
    T s0 = T(0), s1 = T(0);
    for (int u = 0; u < w; ++u) {
        const V4<T> Pm = ld4(cf.P + 4 * u);
        const T n0 = Pm.x * s0 + Pm.y * s1 + fq[u][0][lane];
        const T n1 = Pm.z * s0 + Pm.w * s1 + fq[u][1][lane];
        s0 = n0;
        s1 = n1;
    }
    T sv0 = T(0), sv1 = T(0), sv2 = T(0), sv3 = T(0);
    if (per) {
        T t0 = T(0), t1 = T(0), t2 = T(0), t3 = T(0);
#pragma unroll
        for (int u = 0; u < NW; ++u) {
            t0 += wacc[u][0][lane];
            t1 += wacc[u][1][lane];
            t2 += wacc[u][2][lane];
            t3 += wacc[u][3][lane];
        }
        const V4<T> r0 = ld4(cf.S), r1 = ld4(cf.S + 4), r2 = ld4(cf.S + 8), r3 = ld4(cf.S + 12);
        sv0 = r0.x * t0 + r0.y * t1 + r0.z * t2 + r0.w * t3;
        sv1 = r1.x * t0 + r1.y * t1 + r1.z * t2 + r1.w * t3;
        sv2 = r2.x * t0 + r2.y * t1 + r2.z * t2 + r2.w * t3;
        sv3 = r3.x * t0 + r3.y * t1 + r3.z * t2 + r3.w * t3;
    }
    y1 = s0;
    y2 = s1;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const V4<T> c = ldv4(cf.fwd + 4 * (j0 + i));
        const T y = (v[i] - c.y * y2) - c.x * y1;
        y2 = y1;
        y1 = y;
        v[i] = y * c.z;
    }
    // back substitution from a zero state over this warp's rows
    T x1 = T(0), x2 = T(0);
#pragma unroll
    for (int i = R - 1; i >= 0; --i) {
        T u1, u2;
        ldv2(cf.bwd + 2 * (j0 + i), u1, u2);
        const T x = (v[i] - u2 * x2) - u1 * x1;
        x2 = x1;
        x1 = x;
    }
    bq[w][0][lane] = x1;
    bq[w][1][lane] = x2;
    __syncthreads();
    s0 = T(0);
    s1 = T(0);
    for (int u = NW - 1; u > w; --u) {
        const V4<T> Qm = ld4(cf.Q + 4 * u);
        const T n0 = Qm.x * s0 + Qm.y * s1 + bq[u][0][lane];
        const T n1 = Qm.z * s0 + Qm.w * s1 + bq[u][1][lane];
        s0 = n0;
        s1 = n1;
    }
    x1 = s0;
    x2 = s1;
    bool bad = false;
#pragma unroll
    for (int i = R - 1; i >= 0; --i) {
        T u1, u2;
        ldv2(cf.bwd + 2 * (j0 + i), u1, u2);
        const T x = (v[i] - u2 * x2) - u1 * x1;
        x2 = x1;
        x1 = x;
        T o = x;
        if (per) {
            const V4<T> z = ldv4(cf.Z + 4 * (j0 + i));
            o -= z.x * sv0 + z.y * sv1 + z.z * sv2 + z.w * sv3;
        }
        const int j = j0 + i;
        if (valid && j < n) {
            const int64_t idx = base + (int64_t)j * line_stride;
            if (UPDATE) {
                const T cnew = Cf[idx] + o;
                bad |= !isfinite(cnew);
                Cf[idx] = cnew;
            } else {
                a[idx] = o;
            }
        }
    }
    if (UPDATE && bad) atomicOr(status, 1u);
}

// C += dq for a single-plane (2D) box, which has no z-solve to fuse it into;
// non-finite results raise the status flag.
template <typename T>
__global__ void __launch_bounds__(256) ch_add_increment(T* __restrict__ C, const T* __restrict__ dq, int64_t N,
                                                        unsigned int* status) {
    bool bad = false;
    for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < N; e += (int64_t)gridDim.x * 256) {
        const T c = C[e] + dq[e];
        bad |= !isfinite(c);
        C[e] = c;
    }
    if (bad) atomicOr(status, 1u);
}

// ---------------------------------------------------------------------------
// FP64 reductions: block partial sums (warp shuffles + shared memory), then a
// single-block pass in fixed order, so results are deterministic.
// ---------------------------------------------------------------------------
constexpr int kRedThreads = 256;
// 128-cell chunks of a row in flight per warp in the free-energy pass
#ifndef CH_RED_UNROLL
#define CH_RED_UNROLL 2
#endif
constexpr int kRedUnroll = CH_RED_UNROLL;

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double ws[kRedThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) ws[w] = v;
    __syncthreads();
    v = (threadIdx.x < kRedThreads / 32) ? ws[threadIdx.x] : 0.0;
    if (w == 0)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Per-lane accumulator of the reductions.  FP64 fields add in FP64.  FP32
// fields (where FP64 arithmetic, at a small fraction of the FP32 rate on this
// GPU, would bound the kernel) form every term in FP32 and add it to a
// double-float pair (s, c): s the rounded FP32 sum, c the exact rounding
// error of every addition (Knuth's TwoSum, six FP32 operations) summed in
// FP32.  The pair is flushed to an FP64 total after at most one row segment
// of 32 terms per lane, so the flushed sums are accurate to about 32^2 u^2
// (u = 2^-24) of their size and the FP64 total carries the rest.
template <typename T>
struct RedAcc {
    double tot = 0.0;
    __device__ __forceinline__ void add(double x) { tot += x; }
    __device__ __forceinline__ void flush() {}
    __device__ __forceinline__ double total() const { return tot; }
};
template <>
struct RedAcc<float> {
    double tot = 0.0;
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float t = __fadd_rn(s, x);
        const float bp = __fsub_rn(t, s);
        const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
        s = t;
        c = __fadd_rn(c, e);
    }
    __device__ __forceinline__ void flush() {
        tot += (double)s + (double)c;
        s = c = 0.f;
    }
    __device__ __forceinline__ double total() const { return tot + ((double)s + (double)c); }
};

// Mass h^3 sum C: one warp per x-row (rows split over the grid's warps), lanes
// stride along the row; each lane flushes its pair after every row.
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
ch_reduce_mass(const T* __restrict__ C, int nx, int64_t nrows, double* partials, unsigned int* status) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * kRedThreads + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kRedThreads) >> 5;
    RedAcc<T> acc;
    bool bad = false;
    for (int64_t row = warp0; row < nrows; row += nwarps) {
        const T* p = C + row * nx;
        for (int i = lane; i < nx; i += 32) {
            const T c = p[i];
            bad |= !isfinite(c);
            acc.add(c);
        }
        acc.flush();
    }
    if (bad) atomicOr(status, 1u);
    const double v = block_sum(acc.total());
    if (threadIdx.x == 0) partials[blockIdx.x] = v;
}

// Free energy sum [psi(C) + (Cn^2/2) sum_d ((C_{+e_d} - C)/h)^2] (Sec. 1), every
// term in the field precision: one warp per x-row (k, j), lanes along x; the
// forward neighbour wraps (periodic), is the cell itself (mirror ghost, zero
// gradient at a no-flux wall) or its negation (Dirichlet ghost at the top
// z-wall).  With MASS the same pass also sums C (block partials after the
// energy partials), so both diagnostics cost one read of C.
template <typename T, bool MASS = false>
__global__ void __launch_bounds__(kRedThreads)
ch_reduce_energy(const T* __restrict__ C, int nx, int ny, int nz, int bcx, int bcy, int bcz, T inv_h,
                 T half_cn2, double* partials, unsigned int* status) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * kRedThreads + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kRedThreads) >> 5;
    const int64_t nrows = (int64_t)ny * nz;
    const int64_t plane = (int64_t)nx * ny;
    RedAcc<T> acc, macc;
    bool bad = false;
    for (int64_t row = warp0; row < nrows; row += nwarps) {
        const int j = (int)(row % ny), k = (int)(row / ny);
        const int jp = (j + 1 < ny) ? j + 1 : (bcy == CH_PERIODIC ? 0 : j);
        const int kp = (k + 1 < nz) ? k + 1 : (bcz == CH_PERIODIC ? 0 : k);
        const T zsign = (k + 1 >= nz && bcz == CH_DIRICHLET) ? T(-1) : T(1);
        const T* p = C + row * nx;
        const T* py = C + ((int64_t)k * ny + jp) * nx;
        const T* pz = C + (int64_t)kp * plane + (int64_t)j * nx;
        if constexpr (sizeof(T) == 4) {
            if (nx % 128 == 0) {  // 4 consecutive cells per lane, 16-byte loads (rows are 512-byte multiples)
                // the lane's 4 energy terms are summed plainly (no
                // cancellation: every term is non-negative; 3 roundings of
                // relative size 2^-24) and the sum enters the compensated
                // accumulator once; the mass adds every C compensated, as
                // ch_reduce_mass does
#pragma unroll kRedUnroll
                for (int i0 = 4 * lane; i0 < nx; i0 += 128) {
                    const float4 c4 = *reinterpret_cast<const float4*>(p + i0);
                    const float4 y4 = *reinterpret_cast<const float4*>(py + i0);
                    const float4 z4 = *reinterpret_cast<const float4*>(pz + i0);
                    // the +x neighbour of the lane's last cell: the next lane's first, or past the chunk
                    float xn = __shfl_down_sync(0xffffffffu, c4.x, 1);
                    if (lane == 31) {
                        const int ie = i0 + 4;
                        xn = ie < nx ? p[ie] : (bcx == CH_PERIODIC ? p[0] : c4.w);
                    }
                    const float cv[4] = {c4.x, c4.y, c4.z, c4.w}, xv[4] = {c4.y, c4.z, c4.w, xn};
                    const float yv[4] = {y4.x, y4.y, y4.z, y4.w}, zv[4] = {z4.x, z4.y, z4.z, z4.w};
                    float e4 = 0.f;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const T c = cv[q];
                        bad |= !isfinite(c);
                        const T gx = (xv[q] - c) * inv_h;
                        const T gy = (yv[q] - c) * inv_h;
                        const T gz = (zsign * zv[q] - c) * inv_h;
                        const T cc = c * (c - T(1));
                        e4 += T(0.25) * cc * cc + half_cn2 * (gx * gx + gy * gy + gz * gz);
                        if (MASS) macc.add(c);
                    }
                    acc.add(e4);
                }
                acc.flush();
                macc.flush();
                continue;
            }
        }
        for (int i = lane; i < nx; i += 32) {
            const int ip = (i + 1 < nx) ? i + 1 : (bcx == CH_PERIODIC ? 0 : i);
            const T c = p[i];
            bad |= !isfinite(c);
            const T gx = (p[ip] - c) * inv_h;
            const T gy = (py[i] - c) * inv_h;
            const T gz = (zsign * pz[i] - c) * inv_h;
            const T cc = c * (c - T(1));
            acc.add(T(0.25) * cc * cc + half_cn2 * (gx * gx + gy * gy + gz * gz));
            if (MASS) macc.add(c);
        }
        acc.flush();
        macc.flush();
    }
    if (bad) atomicOr(status, 1u);
    const double v = block_sum(acc.total());
    if (threadIdx.x == 0) partials[blockIdx.x] = v;
    if (MASS) {
        __syncthreads();  // block_sum's shared slots are reused
        const double m = block_sum(macc.total());
        if (threadIdx.x == 0) partials[gridDim.x + blockIdx.x] = m;
    }
}

static __global__ void __launch_bounds__(kRedThreads)
ch_reduce_finish(const double* __restrict__ partials, int nb, double scale, double* out) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += kRedThreads) acc += partials[b];
    acc = block_sum(acc);
    if (threadIdx.x == 0) *out = acc * scale;
}

}  // namespace chg
