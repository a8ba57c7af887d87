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

namespace chg {

constexpr int kTX = 32;   // explicit-kernel tile, x (one warp)
constexpr int kTY = 8;    // explicit-kernel tile, y (warps per CTA)
constexpr int kTZ = 16;   // z-planes marched per CTA
constexpr int kHalo = 3;  // WENO5 needs three cells on each side

struct RhsArgs {
    int nx, ny, nz;
    int bcx, bcy, bcz;
    int nfx, nfy, nfz;
    double inv_h, inv_h2;
    double mob;        // M = 1/Pe
    double dtg;        // dt * gamma_l
    double dtr;        // dt * rho_l
    double impl;       // alpha_l dt M kappa (multiplies the raw [1,-4,6,-4,1] sums)
    double eps;        // WENO regulariser
    int has_prev;      // rho_l != 0
};

// Neighbour index with the boundary rule of Sec. 3.1: periodic wrap, or the
// mirror about a wall face (ghost C_{-1-m} = C_m).  Clamped so that cells
// outside the domain in a ragged tile still read valid memory.
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

template <typename T>
__device__ __forceinline__ T psi_p(T c) {  // psi'(C) = C^3 - 1.5 C^2 + 0.5 C (Eq. eq-ch)
    return c * (c * (c - T(1.5)) + T(0.5));
}

// Fifth-order WENO (Jiang-Shu) value at the face between v3 and v4 from the
// upwind-biased stencil v1..v5 (Sec. 3: "fifth-order WENO").
template <typename T>
__device__ __forceinline__ T weno5(T v1, T v2, T v3, T v4, T v5, T eps) {
    const T q0 = (T(2) * v1 - T(7) * v2 + T(11) * v3) * T(1.0 / 6.0);
    const T q1 = (-v2 + T(5) * v3 + T(2) * v4) * T(1.0 / 6.0);
    const T q2 = (T(2) * v3 + T(5) * v4 - v5) * T(1.0 / 6.0);
    const T d0 = v1 - T(2) * v2 + v3, e0 = v1 - T(4) * v2 + T(3) * v3;
    const T d1 = v2 - T(2) * v3 + v4, e1 = v2 - v4;
    const T d2 = v3 - T(2) * v4 + v5, e2 = T(3) * v3 - T(4) * v4 + v5;
    const T b0 = T(13.0 / 12.0) * d0 * d0 + T(0.25) * e0 * e0;
    const T b1 = T(13.0 / 12.0) * d1 * d1 + T(0.25) * e1 * e1;
    const T b2 = T(13.0 / 12.0) * d2 * d2 + T(0.25) * e2 * e2;
    const T s0 = eps + b0, s1 = eps + b1, s2 = eps + b2;
    const T a0 = T(0.1) / (s0 * s0);
    const T a1 = T(0.6) / (s1 * s1);
    const T a2 = T(0.3) / (s2 * s2);
    return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
}

// Flux u_f C_f through a face, C_f from the upwind WENO5 stencil.  m3..p2 are
// the cells f-3 .. f+2 around the face f (between cells f-1 and f).
template <typename T>
__device__ __forceinline__ T face_flux(T vel, T m3, T m2, T m1, T p0, T p1, T p2, T eps) {
    const T cf = vel >= T(0) ? weno5(m3, m2, m1, p0, p1, eps) : weno5(p2, p1, p0, m1, m2, eps);
    return vel * cf;
}

// ---------------------------------------------------------------------------
// Explicit right-hand side.  A CTA owns a 32 x 8 column of cells and marches
// kTZ planes in z.  Each plane (with a 3-cell halo in x and y) is staged in
// shared memory; the cell's own z-column lives in a 6-register queue.  Every
// face flux is computed exactly once (lower faces by their cell, the extra
// upper faces of the tile by dedicated lanes, z-faces carried between planes),
// so the fluxes telescope bit-exactly and mass is conserved to rounding.
// ---------------------------------------------------------------------------
template <typename T, bool ADV>
__global__ void __launch_bounds__(kTX * kTY)
ch_explicit_rhs(const T* __restrict__ C, const T* __restrict__ u, const T* __restrict__ v,
                const T* __restrict__ w, const T* __restrict__ Hprev, T* __restrict__ Hout,
                T* __restrict__ r, RhsArgs a) {
    constexpr int PX = kTX + 2 * kHalo, PY = kTY + 2 * kHalo;
    __shared__ T Cs[2][PY][PX];
    __shared__ T Fx[ADV ? kTY : 1][kTX + 1];
    __shared__ T Fy[ADV ? kTY + 1 : 1][kTX];

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kTX + tx;
    const int i0 = blockIdx.x * kTX, j0 = blockIdx.y * kTY, k0 = blockIdx.z * kTZ;
    const int i = i0 + tx, j = j0 + ty;
    const bool in_xy = (i < a.nx) && (j < a.ny);
    const int ic = min(i, a.nx - 1), jc = min(j, a.ny - 1);
    const int64_t plane = (int64_t)a.nx * a.ny;
    const T eps = T(a.eps);
    const int kend = min(k0 + kTZ, a.nz);

    // z-column queue: q[m] = C(ic, jc, k - 2 + m), m = 0..5
    T q[6];
#pragma unroll
    for (int m = 0; m < 6; ++m)
        q[m] = C[(int64_t)bc_index(k0 - 2 + m, a.nz, a.bcz) * plane + (int64_t)jc * a.nx + ic];

    T fz_lo = T(0);
    if (ADV) {
        // flux through the lower z-face of plane k0
        const bool wall = (a.bcz == CH_NOFLUX) && (k0 == 0);
        if (!wall) {
            const T cm3 = C[(int64_t)bc_index(k0 - 3, a.nz, a.bcz) * plane + (int64_t)jc * a.nx + ic];
            const int f = (a.bcz == CH_PERIODIC) ? k0 % a.nz : k0;
            const T wv = w[((int64_t)f * a.ny + jc) * a.nx + ic];
            fz_lo = face_flux(wv, cm3, q[0], q[1], q[2], q[3], q[4], eps);
        }
    }

    for (int k = k0, buf = 0; k < kend; ++k, buf ^= 1) {
        // stage plane k with its x/y halo
        const T* Ck = C + (int64_t)k * plane;
        for (int e = tid; e < PX * PY; e += kTX * kTY) {
            const int row = e / PX, col = e - row * PX;
            const int gi = bc_index(i0 + col - kHalo, a.nx, a.bcx);
            const int gj = bc_index(j0 + row - kHalo, a.ny, a.bcy);
            Cs[buf][row][col] = Ck[(int64_t)gj * a.nx + gi];
        }
        // prefetch the next queue entry C(k + 4)
        const T qnext = C[(int64_t)bc_index(k + 4, a.nz, a.bcz) * plane + (int64_t)jc * a.nx + ic];
        __syncthreads();

        const int cy = ty + kHalo, cx = tx + kHalo;
        T fz_up = T(0);
        if (ADV) {
            // x: flux through this cell's lower face (face i)
            {
                const bool wall = (a.bcx == CH_NOFLUX) && (i <= 0 || i >= a.nx);
                T f = T(0);
                if (!wall) {
                    const int fi = (a.bcx == CH_PERIODIC) ? bc_index(i, a.nx, CH_PERIODIC) : i;
                    const T uv = u[((int64_t)k * a.ny + jc) * a.nfx + fi];
                    f = face_flux(uv, Cs[buf][cy][cx - 3], Cs[buf][cy][cx - 2], Cs[buf][cy][cx - 1],
                                  Cs[buf][cy][cx], Cs[buf][cy][cx + 1], Cs[buf][cy][cx + 2], eps);
                }
                Fx[ty][tx] = f;
            }
            // y: flux through this cell's lower face (face j)
            {
                const bool wall = (a.bcy == CH_NOFLUX) && (j <= 0 || j >= a.ny);
                T f = T(0);
                if (!wall) {
                    const int fj = (a.bcy == CH_PERIODIC) ? bc_index(j, a.ny, CH_PERIODIC) : j;
                    const T vv = v[((int64_t)k * a.nfy + fj) * a.nx + ic];
                    f = face_flux(vv, Cs[buf][cy - 3][cx], Cs[buf][cy - 2][cx], Cs[buf][cy - 1][cx],
                                  Cs[buf][cy][cx], Cs[buf][cy + 1][cx], Cs[buf][cy + 2][cx], eps);
                }
                Fy[ty][tx] = f;
            }
            // the tile's extra upper faces: x-face i0+32 of each row (warp 0,
            // lanes 0..7) and y-face j0+8 of each column (warp 1)
            if (ty == 0 && tx < kTY) {
                const int row = tx, ie = i0 + kTX, je = min(j0 + row, a.ny - 1);
                const bool wall = (a.bcx == CH_NOFLUX) && (ie >= a.nx);
                T f = T(0);
                if (!wall) {
                    const int fi = (a.bcx == CH_PERIODIC) ? bc_index(ie, a.nx, CH_PERIODIC) : ie;
                    const T uv = u[((int64_t)k * a.ny + je) * a.nfx + fi];
                    const int yy = row + kHalo, xx = kTX + kHalo;
                    f = face_flux(uv, Cs[buf][yy][xx - 3], Cs[buf][yy][xx - 2], Cs[buf][yy][xx - 1],
                                  Cs[buf][yy][xx], Cs[buf][yy][xx + 1], Cs[buf][yy][xx + 2], eps);
                }
                Fx[row][kTX] = f;
            }
            if (ty == 1) {
                const int je = j0 + kTY;
                const bool wall = (a.bcy == CH_NOFLUX) && (je >= a.ny);
                T f = T(0);
                if (!wall) {
                    const int fj = (a.bcy == CH_PERIODIC) ? bc_index(je, a.ny, CH_PERIODIC) : je;
                    const T vv = v[((int64_t)k * a.nfy + fj) * a.nx + ic];
                    const int yy = kTY + kHalo, xx = cx;
                    f = face_flux(vv, Cs[buf][yy - 3][xx], Cs[buf][yy - 2][xx], Cs[buf][yy - 1][xx],
                                  Cs[buf][yy][xx], Cs[buf][yy + 1][xx], Cs[buf][yy + 2][xx], eps);
                }
                Fy[kTY][tx] = f;
            }
            // z: flux through the upper face k+1 of this cell
            {
                const bool wall = (a.bcz == CH_NOFLUX) && (k + 1 >= a.nz);
                if (!wall) {
                    const int f = (a.bcz == CH_PERIODIC) ? (k + 1) % a.nz : k + 1;
                    const T wv = w[((int64_t)f * a.ny + jc) * a.nx + ic];
                    fz_up = face_flux(wv, q[0], q[1], q[2], q[3], q[4], q[5], eps);
                }
            }
            __syncthreads();
        }

        // M lap(psi'(C)), 7-point central (Sec. 3)
        const T c0 = Cs[buf][cy][cx];
        const T p0 = psi_p(c0);
        const T lap = (psi_p(Cs[buf][cy][cx - 1]) + psi_p(Cs[buf][cy][cx + 1]) + psi_p(Cs[buf][cy - 1][cx]) +
                       psi_p(Cs[buf][cy + 1][cx]) + psi_p(q[1]) + psi_p(q[3]) - T(6) * p0) *
                      T(a.inv_h2);
        // raw [1,-4,6,-4,1] sums of A_x + A_y + A_z (Eq. eq-a3d)
        const T ax = Cs[buf][cy][cx - 2] + Cs[buf][cy][cx + 2] - T(4) * (Cs[buf][cy][cx - 1] + Cs[buf][cy][cx + 1]);
        const T ay = Cs[buf][cy - 2][cx] + Cs[buf][cy + 2][cx] - T(4) * (Cs[buf][cy - 1][cx] + Cs[buf][cy + 1][cx]);
        const T az = q[0] + q[4] - T(4) * (q[1] + q[3]);
        const T astar = ax + ay + az + T(18) * c0;

        T H = T(a.mob) * lap;
        if (ADV) {
            const T div = (Fx[ty][tx + 1] - Fx[ty][tx]) + (Fy[ty + 1][tx] - Fy[ty][tx]) + (fz_up - fz_lo);
            H -= div * T(a.inv_h);
        }
        if (in_xy) {
            const int64_t idx = (int64_t)k * plane + (int64_t)j * a.nx + i;
            T rhs = T(a.dtg) * H - T(a.impl) * astar;
            if (a.has_prev) rhs += T(a.dtr) * Hprev[idx];
            Hout[idx] = H;
            r[idx] = rhs;
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
// host in FP64.  Per line: forward sweep (also accumulating the Woodbury dot
// products W^T r), then backward sweep emitting x_band - Z s.
// ---------------------------------------------------------------------------
template <typename T>
struct Coef {
    const T* __restrict__ l1;
    const T* __restrict__ l2;
    const T* __restrict__ u1;
    const T* __restrict__ u2;
    const T* __restrict__ dinv;
    const T* __restrict__ W;
    const T* __restrict__ Z;
    const T* __restrict__ S;
    int n;
    int periodic;
};

// Solve one line held in shared memory at s[j * stride], in place.
template <typename T>
__device__ __forceinline__ void sweep_line(T* s, int stride, const Coef<T>& cf) {
    const int n = cf.n;
    T y1 = T(0), y2 = T(0);
    T acc0 = T(0), acc1 = T(0), acc2 = T(0), acc3 = T(0);
    if (cf.periodic) {
        for (int jj = 0; jj < n; ++jj) {
            const T rj = s[jj * stride];
            const T yj = rj - __ldg(cf.l1 + jj) * y1 - __ldg(cf.l2 + jj) * y2;
            const T* Wj = cf.W + 4 * jj;
            acc0 += __ldg(Wj + 0) * rj;
            acc1 += __ldg(Wj + 1) * rj;
            acc2 += __ldg(Wj + 2) * rj;
            acc3 += __ldg(Wj + 3) * rj;
            s[jj * stride] = yj;
            y2 = y1;
            y1 = yj;
        }
    } else {
        for (int jj = 0; jj < n; ++jj) {
            const T yj = s[jj * stride] - __ldg(cf.l1 + jj) * y1 - __ldg(cf.l2 + jj) * y2;
            s[jj * stride] = yj;
            y2 = y1;
            y1 = yj;
        }
    }
    T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
    if (cf.periodic) {
        const T* S = cf.S;
        s0 = __ldg(S + 0) * acc0 + __ldg(S + 1) * acc1 + __ldg(S + 2) * acc2 + __ldg(S + 3) * acc3;
        s1 = __ldg(S + 4) * acc0 + __ldg(S + 5) * acc1 + __ldg(S + 6) * acc2 + __ldg(S + 7) * acc3;
        s2 = __ldg(S + 8) * acc0 + __ldg(S + 9) * acc1 + __ldg(S + 10) * acc2 + __ldg(S + 11) * acc3;
        s3 = __ldg(S + 12) * acc0 + __ldg(S + 13) * acc1 + __ldg(S + 14) * acc2 + __ldg(S + 15) * acc3;
    }
    T x1 = T(0), x2 = T(0);
    for (int jj = n - 1; jj >= 0; --jj) {
        const T xj = (s[jj * stride] - __ldg(cf.u1 + jj) * x1 - __ldg(cf.u2 + jj) * x2) * __ldg(cf.dinv + jj);
        T out = xj;
        if (cf.periodic) {
            const T* Zj = cf.Z + 4 * jj;
            out -= __ldg(Zj + 0) * s0 + __ldg(Zj + 1) * s1 + __ldg(Zj + 2) * s2 + __ldg(Zj + 3) * s3;
        }
        s[jj * stride] = out;
        x2 = x1;
        x1 = xj;
    }
}

constexpr int kSolveThreads = 128;

// x-lines (contiguous).  A CTA stages `lines` rows of length nx in shared
// memory (row stride nx+1 to spread banks), warp 0 sweeps one line per lane.
template <typename T>
__global__ void __launch_bounds__(kSolveThreads)
ch_solve_x(T* __restrict__ a, int64_t nlines, int nx, int lines, Coef<T> cf) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* s = reinterpret_cast<T*>(smem_raw);
    const int stride = nx + 1;
    const int64_t line0 = (int64_t)blockIdx.x * lines;
    const int nl = (int)min((int64_t)lines, nlines - line0);
    for (int l = 0; l < nl; ++l) {
        const T* src = a + (line0 + l) * nx;
        for (int x = threadIdx.x; x < nx; x += kSolveThreads) s[l * stride + x] = src[x];
    }
    __syncthreads();
    if (threadIdx.x < nl) sweep_line(s + threadIdx.x * stride, 1, cf);
    __syncthreads();
    for (int l = 0; l < nl; ++l) {
        T* dst = a + (line0 + l) * nx;
        for (int x = threadIdx.x; x < nx; x += kSolveThreads) dst[x] = s[l * stride + x];
    }
}

// y- or z-lines (strided).  A CTA owns `lanes` consecutive x of one (z) or
// (y) position; row jj of its tile is `lanes` contiguous values, so loads
// and stores are coalesced.  With UPDATE, the solved increment is added to C
// (Eq. eq-fac-3: q^{l+1} = q^l + dq) and non-finite values raise a flag.
template <typename T, bool UPDATE>
__global__ void __launch_bounds__(kSolveThreads)
ch_solve_yz(T* __restrict__ a, T* __restrict__ Cf, int nx, int64_t outer_stride, int64_t line_stride,
            int lanes, Coef<T> cf, unsigned int* status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* s = reinterpret_cast<T*>(smem_raw);
    const int n = cf.n;
    const int xblocks = (nx + lanes - 1) / lanes;
    const int xb = blockIdx.x % xblocks;
    const int64_t outer = blockIdx.x / xblocks;
    const int i0 = xb * lanes;
    const int nl = min(lanes, nx - i0);
    const int64_t base = outer * outer_stride + i0;
    const int rows_per_pass = kSolveThreads / lanes;
    const int lane = threadIdx.x % lanes, rsub = threadIdx.x / lanes;
    for (int jj = rsub; jj < n; jj += rows_per_pass)
        if (lane < nl) s[jj * lanes + lane] = a[base + (int64_t)jj * line_stride + lane];
    __syncthreads();
    if (threadIdx.x < nl) sweep_line(s + threadIdx.x, lanes, cf);
    __syncthreads();
    bool bad = false;
    for (int jj = rsub; jj < n; jj += rows_per_pass) {
        if (lane < nl) {
            const int64_t idx = base + (int64_t)jj * line_stride + lane;
            if (UPDATE) {
                const T cnew = Cf[idx] + s[jj * lanes + lane];
                bad |= !isfinite(cnew);
                Cf[idx] = cnew;
            } else {
                a[idx] = s[jj * lanes + lane];
            }
        }
    }
    if (UPDATE && bad) atomicOr(status, 1u);
}

// ---------------------------------------------------------------------------
// FP64 reductions: block partial sums (warp shuffles + shared memory), then a
// single-block pass in fixed order, so results are deterministic.
// ---------------------------------------------------------------------------
constexpr int kRedThreads = 256;

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

template <typename T>
__global__ void __launch_bounds__(kRedThreads)
ch_reduce_mass(const T* __restrict__ C, int64_t N, double* partials, unsigned int* status) {
    double acc = 0.0;
    bool bad = false;
    for (int64_t e = (int64_t)blockIdx.x * kRedThreads + threadIdx.x; e < N; e += (int64_t)gridDim.x * kRedThreads) {
        const double c = (double)C[e];
        bad |= !isfinite(c);
        acc += c;
    }
    if (bad) atomicOr(status, 1u);
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

template <typename T>
__global__ void __launch_bounds__(kRedThreads)
ch_reduce_energy(const T* __restrict__ C, int nx, int ny, int nz, int bcx, int bcy, int bcz, double inv_h,
                 double half_cn2, double* partials, unsigned int* status) {
    const int64_t N = (int64_t)nx * ny * nz;
    double acc = 0.0;
    bool bad = false;
    for (int64_t e = (int64_t)blockIdx.x * kRedThreads + threadIdx.x; e < N; e += (int64_t)gridDim.x * kRedThreads) {
        const int i = (int)(e % nx);
        const int64_t t = e / nx;
        const int j = (int)(t % ny), k = (int)(t / ny);
        const double c = (double)C[e];
        bad |= !isfinite(c);
        // forward neighbours: wrap, or the mirror ghost (zero gradient) at a wall
        const int ip = (i + 1 < nx) ? i + 1 : (bcx == CH_PERIODIC ? 0 : i);
        const int jp = (j + 1 < ny) ? j + 1 : (bcy == CH_PERIODIC ? 0 : j);
        const int kp = (k + 1 < nz) ? k + 1 : (bcz == CH_PERIODIC ? 0 : k);
        const double gx = ((double)C[e - i + ip] - c) * inv_h;
        const double gy = ((double)C[e + (int64_t)(jp - j) * nx] - c) * inv_h;
        const double gz = ((double)C[e + (int64_t)(kp - k) * nx * ny] - c) * inv_h;
        const double cc = c * (c - 1.0);
        acc += 0.25 * cc * cc + half_cn2 * (gx * gx + gy * gy + gz * gz);
    }
    if (bad) atomicOr(status, 1u);
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kRedThreads)
ch_reduce_finish(const double* __restrict__ partials, int nb, double scale, double* out) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += kRedThreads) acc += partials[b];
    acc = block_sum(acc);
    if (threadIdx.x == 0) *out = acc * scale;
}

}  // namespace chg
