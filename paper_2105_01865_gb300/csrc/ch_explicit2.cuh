// Explicit right-hand side, two x-adjacent cells per thread (even nx).
//
// Same arithmetic as ch_explicit_rhs (arXiv 2105.01865, Sec. 3 and Eq. eq-re:
// H^l = -div(uC)_WENO5 + M lap(psi'(C)), r = dt(gamma H^l + rho H^{l-1})
// - alpha dt M sum_d A_d C), but every value is a pair belonging to the cells
// (i, i+1) of one thread.  For float the pairs live in one 64-bit register and
// map onto Blackwell's paired FP32 instructions (FADD2/FMUL2/FFMA2), so one
// instruction advances the x-, y- or z-face reconstruction of both cells; the
// global accesses become 8-byte (float2) or 16-byte (double2) vectors.
#pragma once

#include <cuda.h>

#include "ch_kernels.cuh"

namespace chg {

template <typename T>
struct Pr;

template <>
struct Pr<float> {
    float2 v;
    __device__ __forceinline__ float x() const { return v.x; }
    __device__ __forceinline__ float y() const { return v.y; }
};

template <>
struct Pr<double> {
    double2 v;
    __device__ __forceinline__ double x() const { return v.x; }
    __device__ __forceinline__ double y() const { return v.y; }
};

__device__ __forceinline__ Pr<float> mk(float a, float b) { return {make_float2(a, b)}; }
__device__ __forceinline__ Pr<double> mk(double a, double b) { return {make_double2(a, b)}; }
template <typename T>
__device__ __forceinline__ Pr<T> sp(T a) { return mk(a, a); }

__device__ __forceinline__ Pr<float> add(Pr<float> a, Pr<float> b) { return {__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ Pr<float> mul(Pr<float> a, Pr<float> b) { return {__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ Pr<float> fma2(Pr<float> a, Pr<float> b, Pr<float> c) { return {__ffma2_rn(a.v, b.v, c.v)}; }
#ifndef CH_SUB_PTX
#define CH_SUB_PTX 1
#endif
__device__ __forceinline__ Pr<float> sub(Pr<float> a, Pr<float> b) {
#if CH_SUB_PTX
    // a - b with one rounding (the paired subtraction; no constant operand)
    unsigned long long ra, rb, rd;
    memcpy(&ra, &a.v, 8);
    memcpy(&rb, &b.v, 8);
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    Pr<float> d;
    memcpy(&d.v, &rd, 8);
    return d;
#else
    return {__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v)};  // a - b, one rounding
#endif
}
__device__ __forceinline__ Pr<float> divp(Pr<float> a, Pr<float> b) {
    return mk(__fdividef(a.v.x, b.v.x), __fdividef(a.v.y, b.v.y));
}

__device__ __forceinline__ Pr<double> add(Pr<double> a, Pr<double> b) { return mk(a.v.x + b.v.x, a.v.y + b.v.y); }
__device__ __forceinline__ Pr<double> mul(Pr<double> a, Pr<double> b) { return mk(a.v.x * b.v.x, a.v.y * b.v.y); }
__device__ __forceinline__ Pr<double> fma2(Pr<double> a, Pr<double> b, Pr<double> c) {
    return mk(fma(a.v.x, b.v.x, c.v.x), fma(a.v.y, b.v.y, c.v.y));
}
__device__ __forceinline__ Pr<double> sub(Pr<double> a, Pr<double> b) { return mk(a.v.x - b.v.x, a.v.y - b.v.y); }
__device__ __forceinline__ Pr<double> divp(Pr<double> a, Pr<double> b) { return mk(a.v.x / b.v.x, a.v.y / b.v.y); }

// aligned pair load/store (address of the first element of the pair)
__device__ __forceinline__ Pr<float> ldp(const float* p) { return {*reinterpret_cast<const float2*>(p)}; }
__device__ __forceinline__ Pr<double> ldp(const double* p) { return {*reinterpret_cast<const double2*>(p)}; }
__device__ __forceinline__ void stp(float* p, Pr<float> a) { *reinterpret_cast<float2*>(p) = a.v; }
__device__ __forceinline__ void stp(double* p, Pr<double> a) { *reinterpret_cast<double2*>(p) = a.v; }

template <typename T>
__device__ __forceinline__ Pr<T> psi_pp(Pr<T> c) {  // psi'(C) = C (C (C - 1.5) + 0.5)
    return mul(c, fma2(c, sub(c, sp<T>(T(1.5))), sp<T>(T(0.5))));
}

// WENO5 form of the paired kernel: the stencil values as in weno5 (0) or
// first differences (1, the measured faster one with paired subtraction: 637
// against 674 million instructions and 5.79 against 6.22 ms per launch on the
// 1024 x 1024 x 512 mesh).  The regulariser passed in is kWenoEpsScale eps.
#ifndef CH_WENO_DIFF
#define CH_WENO_DIFF 1
#endif
constexpr double kWenoEpsScale = CH_WENO_DIFF ? 4.0 : 1.0;
#if CH_WENO_DIFF
// WENO5 (Jiang-Shu) face values of two faces at once, written in first
// differences of the stencil (a' = v1 - v2, b = v3 - v2, c = v4 - v3,
// d = v5 - v4), the same function as weno5 with fewer operations and smaller
// cancellations:
//   candidates  q_k = v3 + p_k / 6,  p0 = 5b + 2a', p1 = b + 2c, p2 = 4c - d;
//   4 beta_k    = (13/3) D_k^2 + E_k^2 with D0 = b + a', D1 = c - b, D2 = d - c,
//                 E0 = 3b + a', E1 = b + c, E2 = d - 3c;
//   weights     alpha_k = d_k / (eps + beta_k)^2 with d = (0.1, 0.6, 0.3): over
//               the common denominator and with the factor 4 (and 10) that
//               cancels in the normalisation, w0 = t1 t2, w1 = 6 t0 t2,
//               w2 = 3 t0 t1 with t_k = (4 eps + 4 beta_k)^2.
// eps4 is 4 eps.
template <typename T>
__device__ __forceinline__ Pr<T> weno5p(Pr<T> v1, Pr<T> v2, Pr<T> v3, Pr<T> v4, Pr<T> v5, Pr<T> eps4) {
    const Pr<T> am = sub(v1, v2), b = sub(v3, v2), c = sub(v4, v3), d = sub(v5, v4);
    const Pr<T> D0 = add(b, am), D1 = sub(c, b), D2 = sub(d, c);
    const Pr<T> E0 = fma2(sp<T>(T(3)), b, am), E1 = add(b, c), E2 = fma2(sp<T>(T(-3)), c, d);
    const Pr<T> c133 = sp<T>(T(13.0 / 3.0));
    const Pr<T> s0 = fma2(mul(c133, D0), D0, fma2(E0, E0, eps4));
    const Pr<T> s1 = fma2(mul(c133, D1), D1, fma2(E1, E1, eps4));
    const Pr<T> s2 = fma2(mul(c133, D2), D2, fma2(E2, E2, eps4));
    const Pr<T> t0 = mul(s0, s0), t1 = mul(s1, s1), t2 = mul(s2, s2);
    const Pr<T> w0 = mul(t1, t2);
    const Pr<T> w1 = mul(sp<T>(T(6)), mul(t0, t2));
    const Pr<T> w2 = mul(sp<T>(T(3)), mul(t0, t1));
    const Pr<T> p0 = fma2(sp<T>(T(5)), b, add(am, am));
    const Pr<T> p1 = fma2(sp<T>(T(2)), c, b);
    const Pr<T> p2 = fma2(sp<T>(T(4)), c, sub(sp<T>(T(0)), d));
    const Pr<T> num = fma2(w2, p2, fma2(w1, p1, mul(w0, p0)));
    const Pr<T> den = mul(sp<T>(T(6)), add(add(w0, w1), w2));
    return add(v3, divp(num, den));
}

#else
// WENO5 (Jiang-Shu) face values of two faces at once; see weno5.
template <typename T>
__device__ __forceinline__ Pr<T> weno5p(Pr<T> v1, Pr<T> v2, Pr<T> v3, Pr<T> v4, Pr<T> v5, Pr<T> eps) {
    const Pr<T> q0 = fma2(sp<T>(T(2)), v1, fma2(sp<T>(T(-7)), v2, mul(sp<T>(T(11)), v3)));
    const Pr<T> q1 = fma2(sp<T>(T(2)), v4, fma2(sp<T>(T(5)), v3, mul(sp<T>(T(-1)), v2)));
    const Pr<T> q2 = fma2(sp<T>(T(-1)), v5, fma2(sp<T>(T(5)), v4, mul(sp<T>(T(2)), v3)));
    const Pr<T> d0 = fma2(sp<T>(T(-2)), v2, add(v1, v3));
    const Pr<T> e0 = fma2(sp<T>(T(-4)), v2, fma2(sp<T>(T(3)), v3, v1));
    const Pr<T> d1 = fma2(sp<T>(T(-2)), v3, add(v2, v4));
    const Pr<T> e1 = sub(v2, v4);
    const Pr<T> d2 = fma2(sp<T>(T(-2)), v4, add(v3, v5));
    const Pr<T> e2 = fma2(sp<T>(T(-4)), v4, fma2(sp<T>(T(3)), v3, v5));
    const Pr<T> c13 = sp<T>(T(13.0 / 12.0)), c14 = sp<T>(T(0.25));
    const Pr<T> s0 = fma2(mul(c13, d0), d0, fma2(mul(c14, e0), e0, eps));
    const Pr<T> s1 = fma2(mul(c13, d1), d1, fma2(mul(c14, e1), e1, eps));
    const Pr<T> s2 = fma2(mul(c13, d2), d2, fma2(mul(c14, e2), e2, eps));
    const Pr<T> t0 = mul(s0, s0), t1 = mul(s1, s1), t2 = mul(s2, s2);
    const Pr<T> w0 = mul(sp<T>(T(0.1)), mul(t1, t2));
    const Pr<T> w1 = mul(sp<T>(T(0.6)), mul(t0, t2));
    const Pr<T> w2 = mul(sp<T>(T(0.3)), mul(t0, t1));
    const Pr<T> num = fma2(w2, q2, fma2(w1, q1, mul(w0, q0)));
    const Pr<T> den = mul(sp<T>(T(6)), add(add(w0, w1), w2));
    return divp(num, den);
}
#endif

// Flux pair through two faces; m3..p2 are the cell pairs f-3 .. f+2.
template <typename T>
__device__ __forceinline__ Pr<T> face_flux_p(Pr<T> vel, Pr<T> m3, Pr<T> m2, Pr<T> m1, Pr<T> p0, Pr<T> p1, Pr<T> p2,
                                             Pr<T> eps) {
    const bool ux = vel.x() >= T(0), uy = vel.y() >= T(0);
    const Pr<T> a1 = mk(ux ? m3.x() : p2.x(), uy ? m3.y() : p2.y());
    const Pr<T> a2 = mk(ux ? m2.x() : p1.x(), uy ? m2.y() : p1.y());
    const Pr<T> a3 = mk(ux ? m1.x() : p0.x(), uy ? m1.y() : p0.y());
    const Pr<T> a4 = mk(ux ? p0.x() : m1.x(), uy ? p0.y() : m1.y());
    const Pr<T> a5 = mk(ux ? p1.x() : m2.x(), uy ? p1.y() : m2.y());
    return mul(vel, weno5p(a1, a2, a3, a4, a5, eps));
}

// Tuning knobs (compile-time; the defaults are the measured best on GB300)
#ifndef CH_EXPLICIT_MIN_BLOCKS
#define CH_EXPLICIT_MIN_BLOCKS 3
#endif
#ifndef CH_EXPLICIT_TZ
#define CH_EXPLICIT_TZ 10
#endif
#ifndef CH_EXPLICIT_TZ_DEEP
#define CH_EXPLICIT_TZ_DEEP 64
#endif
#ifndef CH_EXPLICIT_STAGE_OFFSETS
#define CH_EXPLICIT_STAGE_OFFSETS 1
#endif
#ifndef CH_EXPLICIT_TMA_RECOMPUTE
#define CH_EXPLICIT_TMA_RECOMPUTE 1
#endif
#ifndef CH_EXPLICIT_PREFETCH
#define CH_EXPLICIT_PREFETCH 1
#endif
constexpr int kTX2 = 64;               // cells in x per CTA (two per thread)
constexpr int kTZ2 = CH_EXPLICIT_TZ;   // z-planes marched per CTA
constexpr int kTZ2Deep = CH_EXPLICIT_TZ_DEEP;
constexpr int kHL2 = 4;   // left halo columns (even, so thread pairs stay 8/16-byte aligned)

// z-planes marched per CTA for an nx x ny x nz field.  A tile reads 4 halo
// planes besides its own, so a deep tile re-reads less of C; a shallow one
// gives more CTAs.  The FP32 path takes the deep tile when that still leaves
// at least 8 full waves of 3 CTAs on each of the 152 SMs (on large meshes,
// where the re-read dominates); the results do not depend on the depth (every
// face flux is formed by the same arithmetic in whichever tile forms it).
inline int explicit_zchunk(int nx, int ny, int nz, bool fp32) {
    const int64_t xy = (int64_t)((nx + kTX2 - 1) / kTX2) * ((ny + kTY - 1) / kTY);
    const int64_t deep = xy * ((nz + kTZ2Deep - 1) / kTZ2Deep);
    return (fp32 && deep >= 8 * 3 * 152) ? kTZ2Deep : kTZ2;
}

// One 64 x 8 x zchunk tile (tile coordinates bx, by, bz) computed by the 256
// threads of a CTA; called by the standalone kernel below and by the batched
// persistent kernel.
template <typename T, bool ADV, bool DIRI = false, bool TMA = false>
// DIRI: compiled for Dirichlet z-walls (negated ghost planes); false for every
// other wall type, which then carries no extra code.
// TMA (FP32): tiles whose 72 x 14 staged plane needs no wrapped or mirrored
// index are staged by one tensor-map tile load per plane (tmap: a 3D map of C
// with a 72 x 14 x 1 box), completed on a shared-memory mbarrier; the others
// stage element by element.  A wait that gives up sets bit 4 of *status
// (the launch's results are then void).
// Data pointers carry no __restrict__ here: the batched persistent kernel
// writes these arrays in one phase and reads them in the next, so their loads
// must not go through the non-coherent read-only path.
__device__ __forceinline__ void explicit_tile2(const T* C, const T* u, const T* v, const T* w, const T* Hprev,
                                               T* Hout, T* r, const RhsArgs<T>& a, int bx, int by, int bz,
                                               int zchunk, const void* tmap = nullptr,
                                               unsigned int* status = nullptr) {
    constexpr int PX = kTX2 + 2 * kHL2, PY = kTY + 2 * kHalo;  // 72 x 14
    // with TMA every buffer starts on a 128-byte boundary (16 rows of 288 B)
    constexpr int PYB = TMA ? 16 : PY;
    // ring of staged planes: 3 (one plane ahead), 4 with TMA (tile loads two
    // planes ahead; element staging stays one ahead)
    constexpr int NB = TMA ? 4 : 3;
    __shared__ __align__(128) T Cs[NB][PYB][PX];
    __shared__ __align__(8) unsigned long long mbar[TMA ? NB : 1];
    __shared__ __align__(16) T Fx[ADV ? kTY : 1][kTX2 + 2];
    __shared__ __align__(16) T Fy[ADV ? kTY + 1 : 1][kTX2];
    __shared__ int gi_tab[PX], gj_tab[PY];
    // FP32 with advection: the face velocities and H^{l-1} a thread uses on a
    // plane are copied by cp.async into its own shared slots one plane ahead,
    // in the commit group of that plane's C, so no global load latency is
    // exposed after the plane barrier.  Slot s of thread t holds a pair at
    // [s][2t]: 0 (u_a, u_b), 1 v, 2 w, 3 H^{l-1}, 4 the extra face's velocity.
    // Two buffers suffice: a thread consumes every slot it reads before it
    // issues the next plane's copies.
    constexpr bool kSlots = CH_EXPLICIT_PREFETCH && ADV && sizeof(T) == 4;
    constexpr int kNT = 32 * kTY;
    __shared__ __align__(16) T Ps[kSlots ? 2 : 1][kSlots ? 5 : 1][kSlots ? 2 * kNT : 2];

    const int tid = threadIdx.x + threadIdx.y * 32, tx = tid & 31, ty = tid >> 5;
    const int i0 = bx * kTX2, j0 = by * kTY, k0 = bz * zchunk;
    const int ia = i0 + 2 * tx, j = j0 + ty;   // this thread's cells: (ia, j) and (ia + 1, j)
    const bool in_xy = (ia < a.nx) && (j < a.ny);
    const int ic = min(ia, a.nx - 2), jc = min(j, a.ny - 1);
    // element indices fit in 32 bits (every extent <= 1024, so fields hold < 2^31 elements)
    const int plane = a.nx * a.ny;
    const int col = jc * a.nx + ic;
    const Pr<T> eps = sp<T>(T(kWenoEpsScale * (double)a.eps));  // the regulariser weno5p takes
    const int kend = min(k0 + zchunk, a.nz);

    __syncthreads();  // the tables and buffers may still be read by a previous tile of this CTA
    bool use_tma = false;
    if constexpr (TMA) {
        static_assert(sizeof(T) == 4, "tensor-map staging is FP32");
        use_tma = tmap != nullptr && i0 >= kHL2 && i0 + kTX2 + kHL2 <= a.nx && j0 >= kHalo &&
                  j0 + kTY + kHalo <= a.ny;
        if (use_tma && tid == 0) {
#pragma unroll
            for (int b = 0; b < NB; ++b) mbar_init(&mbar[b], 1);
            mbar_init_fence();
        }
    }
    if (tid < PX) gi_tab[tid] = bc_index(i0 + tid - kHL2, a.nx, a.bcx);
    else if (tid < PX + PY) gj_tab[tid - PX] = bc_index(j0 + (tid - PX) - kHalo, a.ny, a.bcy);

    // x-faces ia and ia+1 (lower faces of the two cells)
    const bool wxa = (a.bcx == CH_NOFLUX) && (ia <= 0 || ia >= a.nx);
    const bool wxb = (a.bcx == CH_NOFLUX) && (ia + 1 >= a.nx);
    const int fxa = (a.bcx == CH_PERIODIC) ? bc_index(ia, a.nx, CH_PERIODIC) : min(ia, a.nx);
    const int fxb = (a.bcx == CH_PERIODIC) ? bc_index(ia + 1, a.nx, CH_PERIODIC) : min(ia + 1, a.nx);
    // y-face j (lower face of both cells)
    const bool wy = (a.bcy == CH_NOFLUX) && (j <= 0 || j >= a.ny);
    const int fy = (a.bcy == CH_PERIODIC) ? bc_index(j, a.ny, CH_PERIODIC) : min(j, a.ny);
    // extra faces: y-face j0+8 for this thread's two columns (warp 0) and the
    // x-face i0+64 of rows (2 tx, 2 tx + 1) (warp 1, lanes 0..3)
    const int je = j0 + kTY;
    const bool wye = (a.bcy == CH_NOFLUX) && (je >= a.ny);
    const int fye = (a.bcy == CH_PERIODIC) ? bc_index(je, a.ny, CH_PERIODIC) : min(je, a.ny);
    const int ie = i0 + kTX2;
    const bool wxe = (a.bcx == CH_NOFLUX) && (ie >= a.nx);
    const int fxe = (a.bcx == CH_PERIODIC) ? bc_index(ie, a.nx, CH_PERIODIC) : min(ie, a.nx);
    const int jea = min(j0 + 2 * (tx & 3), a.ny - 1), jeb = min(j0 + 2 * (tx & 3) + 1, a.ny - 1);

    // z-column queue of pairs: q[m] = C(ia..ia+1, jc, k - 2 + m)
    Pr<T> q[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) {
        q[m] = ldp(C + (bc_near(k0 - 2 + m, a.nz, a.bcz) * plane + col));
        if (DIRI && bc_negate(k0 - 2 + m, a.nz, a.bcz)) q[m] = sub(sp<T>(T(0)), q[m]);
    }

    Pr<T> fz_lo = sp<T>(T(0));
    if (ADV) {
        const bool wall = (a.bcz != CH_PERIODIC) && (k0 == 0);
        if (!wall) {
            Pr<T> cm3 = ldp(C + (bc_near(k0 - 3, a.nz, a.bcz) * plane + col));
            if (DIRI && bc_negate(k0 - 3, a.nz, a.bcz)) cm3 = sub(sp<T>(T(0)), cm3);
            const Pr<T> wv = ldp(w + (k0 * plane + col));
            fz_lo = face_flux_p(wv, cm3, q[0], q[1], q[2], q[3], q[4], eps);
        }
    }
    __syncthreads();  // index tables ready

    auto prefetch = [&](int kk) {
        if constexpr (kSlots) {
            float* S = reinterpret_cast<float*>(&Ps[(kk - k0) & 1][0][2 * tid]);
            const float* uf = reinterpret_cast<const float*>(u);
            const float* vf = reinterpret_cast<const float*>(v);
            const float* wf = reinterpret_cast<const float*>(w);
            const int kp = kk * a.ny;
            if (!wxa) cp_async_elem(S, uf + ((kp + jc) * a.nfx + fxa));
            if (!wxb) cp_async_elem(S + 1, uf + ((kp + jc) * a.nfx + fxb));
            if (!wy) cp_async_pair(S + 2 * kNT, vf + ((kk * a.nfy + fy) * a.nx + ic));
            if (a.bcz == CH_PERIODIC || kk + 1 < a.nz)
                cp_async_pair(S + 4 * kNT, wf + (((kk + 1 < a.nz) ? kk + 1 : 0) * plane + col));
            if (a.has_prev && in_xy)
                cp_async_pair(S + 6 * kNT, reinterpret_cast<const float*>(Hprev) + (kk * plane + j * a.nx + ia));
            if (ty == 0 && !wye) cp_async_pair(S + 8 * kNT, vf + ((kk * a.nfy + fye) * a.nx + ic));
            if (ty == 1 && tx < 4 && !wxe) {
                cp_async_elem(S + 8 * kNT, uf + ((kp + jea) * a.nfx + fxe));
                cp_async_elem(S + 8 * kNT + 1, uf + ((kp + jeb) * a.nfx + fxe));
            }
        }
    };

#if CH_EXPLICIT_STAGE_OFFSETS
    // in-plane source offsets of this thread's staged elements e = tid + 256 m,
    // the same for every plane of the tile
    constexpr int kStageN = (PX * PY + 32 * kTY - 1) / (32 * kTY);
    // with tensor-map staging the element path (edge tiles only) re-derives
    // its offsets from the tables instead of holding them (CH_EXPLICIT_TMA_RECOMPUTE)
    constexpr bool kRecompute = TMA && CH_EXPLICIT_TMA_RECOMPUTE;
    int soff[kRecompute ? 1 : kStageN];
    if constexpr (!kRecompute) {
#pragma unroll
        for (int m = 0; m < kStageN; ++m) {
            const int e = tid + m * 32 * kTY;
            const int row = e / PX, cc = e - row * PX;
            soff[m] = e < PX * PY ? gj_tab[row] * a.nx + gi_tab[cc] : 0;
        }
    }
    // plane kk of C into buffer b: a tile load (TMA tiles) or per-thread copies
    auto stage_c = [&](int kk, int b) {
        const T* Ck = C + kk * plane;
        T* dst = &Cs[b][0][0];
        if (TMA && use_tma) {
            if (tid == 0) {
                mbar_expect_tx(&mbar[b], (unsigned)(PX * PY * sizeof(T)));
                tma_load_3d(dst, tmap, i0 - kHL2, j0 - kHalo, kk, &mbar[b]);
            }
        } else {
#pragma unroll
            for (int m = 0; m < kStageN; ++m) {
                const int e = tid + m * 32 * kTY;
                if constexpr (kRecompute) {
                    const int row = e / PX, cc = e - row * PX;
                    if (e < PX * PY) cp_async_elem(dst + e, Ck + (gj_tab[row] * a.nx + gi_tab[cc]));
                } else {
                    if (e < PX * PY) cp_async_elem(dst + e, Ck + soff[m]);
                }
            }
        }
    };
#else
    auto stage_c = [&](int kk, int b) {
        const T* Ck = C + (int64_t)kk * plane;
        for (int e = tid; e < PX * PY; e += 32 * kTY) {
            const int row = e / PX, cc = e - row * PX;
            cp_async_elem(&Cs[b][row][cc], Ck + (int64_t)gj_tab[row] * a.nx + gi_tab[cc]);
        }
    };
#endif
    // one commit group per plane: its C (per-thread copies) and its velocity
    // and H^{l-1} slots
    auto stage_rest = [&](int kk) {
        prefetch(kk);
        cp_async_commit();
    };
    const bool tma_tile = TMA && use_tma;
    stage_c(k0, 0);
    if (tma_tile && k0 + 1 < kend) stage_c(k0 + 1, 1);
    stage_rest(k0);
    for (int k = k0, buf = 0, it = 0; k < kend; ++k, ++it, buf = (buf + 1 == NB ? 0 : buf + 1)) {
        const int b1 = buf + 1 == NB ? 0 : buf + 1;
        if (tma_tile && k + 2 < kend) stage_c(k + 2, b1 + 1 == NB ? 0 : b1 + 1);
        if (k + 1 < kend) {
            if (!tma_tile) stage_c(k + 1, b1);
            stage_rest(k + 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        if constexpr (TMA) {
            static_assert(!TMA || CH_EXPLICIT_STAGE_OFFSETS, "tensor-map staging uses the offset-table stage");
            // buffer buf's it / NB-th fill.  A wait that gives up (after
            // 2 s) flags the launch and goes on: the results are void then,
            // and every thread still meets every barrier of the tile.
            if (use_tma && !mbar_wait_bounded(&mbar[buf], (unsigned)((it / NB) & 1), 2000000000ull) && status)
                atomicOr(status, 4u);
        }
        // per-thread global inputs of this plane (issued before the barrier)
        Pr<T> qnext = ldp(C + (bc_near(k + 4, a.nz, a.bcz) * plane + col));
        if (DIRI && bc_negate(k + 4, a.nz, a.bcz)) qnext = sub(sp<T>(T(0)), qnext);
        const int kp = k * a.ny;
        T uxa = T(0), uxb = T(0), uxe_a = T(0), uxe_b = T(0);
        Pr<T> vy = sp<T>(T(0)), vye = sp<T>(T(0)), wz = sp<T>(T(0)), hp = sp<T>(T(0));
        const bool zwall = (a.bcz != CH_PERIODIC) && (k + 1 >= a.nz);
        if (ADV && !kSlots) {
            uxa = wxa ? T(0) : u[(kp + jc) * a.nfx + fxa];
            uxb = wxb ? T(0) : u[(kp + jc) * a.nfx + fxb];
            if (!wy) vy = ldp(v + ((k * a.nfy + fy) * a.nx + ic));
            if (ty == 0 && !wye) vye = ldp(v + ((k * a.nfy + fye) * a.nx + ic));
            if (ty == 1 && tx < 4 && !wxe) {
                uxe_a = u[(kp + jea) * a.nfx + fxe];
                uxe_b = u[(kp + jeb) * a.nfx + fxe];
            }
            if (!zwall) wz = ldp(w + (((k + 1 < a.nz) ? k + 1 : 0) * plane + col));
        }
        if (!kSlots && a.has_prev && in_xy) hp = ldp(Hprev + (k * plane + j * a.nx + ia));
        __syncthreads();
        if constexpr (kSlots) {
            const T* S = &Ps[(k - k0) & 1][0][2 * tid];
            if (!wxa) uxa = S[0];
            if (!wxb) uxb = S[1];
            if (!wy) vy = ldp(S + 2 * kNT);
            if (!zwall) wz = ldp(S + 4 * kNT);
            if (a.has_prev && in_xy) hp = ldp(S + 6 * kNT);
            if (ty == 0 && !wye) vye = ldp(S + 8 * kNT);
            if (ty == 1 && tx < 4 && !wxe) {
                uxe_a = S[8 * kNT];
                uxe_b = S[8 * kNT + 1];
            }
        }

        const T(*P)[PX] = Cs[buf];
        const int cy = ty + kHalo, cx = 2 * tx + kHL2;  // smem position of cell ia
        // row of 7 cells ia-3 .. ia+3 and the y-column pairs rows j-3 .. j+2
        const T s1 = P[cy][cx - 3], s2 = P[cy][cx - 2], s3 = P[cy][cx - 1], s4 = P[cy][cx], s5 = P[cy][cx + 1],
                s6 = P[cy][cx + 2], s7 = P[cy][cx + 3];
        const Pr<T> ym3 = ldp(&P[cy - 3][cx]), ym2 = ldp(&P[cy - 2][cx]), ym1 = ldp(&P[cy - 1][cx]);
        const Pr<T> c0 = mk(s4, s5);
        const Pr<T> yp1 = ldp(&P[cy + 1][cx]), yp2 = ldp(&P[cy + 2][cx]);
        Pr<T> fz_up = sp<T>(T(0));
        if (ADV) {
            // x: lower faces of the two cells (faces ia, ia+1)
            const Pr<T> fx = face_flux_p(mk(uxa, uxb), mk(s1, s2), mk(s2, s3), mk(s3, s4), mk(s4, s5), mk(s5, s6),
                                         mk(s6, s7), eps);
            Fx[ty][2 * tx] = wxa ? T(0) : fx.x();
            Fx[ty][2 * tx + 1] = wxb ? T(0) : fx.y();
            // y: lower faces (face j) of the two cells
            Pr<T> fyp = sp<T>(T(0));
            if (!wy) fyp = face_flux_p(vy, ym3, ym2, ym1, c0, yp1, yp2, eps);
            stp(&Fy[ty][2 * tx], fyp);
            // extra faces
            if (ty == 0) {
                Pr<T> f = sp<T>(T(0));
                if (!wye) {
                    const int yy = kTY + kHalo;
                    f = face_flux_p(vye, ldp(&P[yy - 3][cx]), ldp(&P[yy - 2][cx]), ldp(&P[yy - 1][cx]),
                                    ldp(&P[yy][cx]), ldp(&P[yy + 1][cx]), ldp(&P[yy + 2][cx]), eps);
                }
                stp(&Fy[kTY][2 * tx], f);
            }
            if (ty == 1 && tx < 4) {
                // x-face i0+64 of rows ra = 2(tx) and rb = 2(tx)+1 of the tile
                const int ra = 2 * tx + kHalo, rb = ra + 1, xx = kTX2 + kHL2;
                Pr<T> f = sp<T>(T(0));
                if (!wxe) {
                    f = face_flux_p(mk(uxe_a, uxe_b), mk(P[ra][xx - 3], P[rb][xx - 3]), mk(P[ra][xx - 2], P[rb][xx - 2]),
                                    mk(P[ra][xx - 1], P[rb][xx - 1]), mk(P[ra][xx], P[rb][xx]),
                                    mk(P[ra][xx + 1], P[rb][xx + 1]), mk(P[ra][xx + 2], P[rb][xx + 2]), eps);
                }
                Fx[2 * tx][kTX2] = f.x();
                Fx[2 * tx + 1][kTX2] = f.y();
            }
            // z: upper face k+1 of the two cells
            if (!zwall) fz_up = face_flux_p(wz, q[0], q[1], q[2], q[3], q[4], q[5], eps);
            __syncthreads();
        }

        // M lap(psi'(C)), 7-point central (Sec. 3); neighbour differences are
        // formed first, so FP32 keeps the accuracy of the small differences
        const Pr<T> xl = mk(s3, s4), xr = mk(s5, s6);
        const Pr<T> pc = psi_pp(c0);
        Pr<T> pzm = psi_pp(q[1]), pzp = psi_pp(q[3]);
        if (DIRI && a.bcz == CH_DIRICHLET) {  // the ghost of psi' is its own negated mirror (psi' = 0 on the wall)
            if (k == 0) pzm = sub(sp<T>(T(0)), psi_pp(sub(sp<T>(T(0)), q[1])));
            if (k + 1 == a.nz) pzp = sub(sp<T>(T(0)), psi_pp(sub(sp<T>(T(0)), q[3])));
        }
        const Pr<T> lap = mul(add(add(add(sub(psi_pp(xl), pc), sub(psi_pp(xr), pc)),
                                      add(sub(psi_pp(ym1), pc), sub(psi_pp(yp1), pc))),
                                  add(sub(pzm, pc), sub(pzp, pc))),
                              sp<T>(a.inv_h2));
        // [1,-4,6,-4,1] sums of A_x + A_y + A_z (Eq. eq-a3d) as differences of
        // second differences: D2(i-1) - 2 D2(i) + D2(i+1)
        auto fourth = [&](Pr<T> m2, Pr<T> m1, Pr<T> p1, Pr<T> p2) {
            const Pr<T> da = sub(m1, c0), db = sub(p1, c0);
            const Pr<T> dm = sub(sub(m2, m1), da), dp = sub(sub(p2, p1), db);
            return fma2(sp<T>(T(-2)), add(da, db), add(dm, dp));
        };
        const Pr<T> astar = add(add(fourth(mk(s2, s3), xl, xr, mk(s6, s7)), fourth(ym2, ym1, yp1, yp2)),
                                fourth(q[0], q[1], q[3], q[4]));

        Pr<T> H = mul(sp<T>(a.mob), lap);
        if (ADV) {
            const T f0 = Fx[ty][2 * tx], f1 = Fx[ty][2 * tx + 1], f2 = Fx[ty][2 * tx + 2];
            const Pr<T> dxf = mk(f1 - f0, f2 - f1);
            const Pr<T> dyf = sub(ldp(&Fy[ty + 1][2 * tx]), ldp(&Fy[ty][2 * tx]));
            const Pr<T> div = add(add(dxf, dyf), sub(fz_up, fz_lo));
            H = fma2(sp<T>(-a.inv_h), div, H);
        }
        if (in_xy) {
            const int idx = k * plane + j * a.nx + ia;
            Pr<T> rhs = fma2(sp<T>(-a.impl), astar, mul(sp<T>(a.dtg), H));
            if (a.has_prev) rhs = fma2(sp<T>(a.dtr), hp, rhs);
            stp(Hout + idx, H);
            if (r) stp(r + idx, rhs);
        }
#pragma unroll
        for (int m = 0; m < 5; ++m) q[m] = q[m + 1];
        q[5] = qnext;
        fz_lo = fz_up;
    }
}

// TZ: z-planes per CTA, a compile-time constant (a runtime depth cost 2 % on
// the 256 x 256 x 128 shear drop).  TMA: stage C through the tensor map tmap
// (of this C) where a tile allows.
template <typename T, bool ADV, bool DIRI, int TZ, bool TMA>
__global__ void __launch_bounds__(32 * kTY, sizeof(T) == 4 ? CH_EXPLICIT_MIN_BLOCKS : 2)
ch_explicit_rhs2(const T* __restrict__ C, const T* __restrict__ u, const T* __restrict__ v,
                 const T* __restrict__ w, const T* __restrict__ Hprev, T* __restrict__ Hout, T* __restrict__ r,
                 RhsArgs<T> a, const __grid_constant__ CUtensorMap tmap, unsigned int* status) {
    pdl_wait();
    pdl_launch_dependents();
    explicit_tile2<T, ADV, DIRI, TMA>(C, u, v, w, Hprev, Hout, r, a, blockIdx.x, blockIdx.y, blockIdx.z, TZ,
                                      TMA ? (const void*)&tmap : nullptr, status);
}

}  // namespace chg
