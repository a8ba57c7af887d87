// Two-column form of the column line solver (y- and z-lines; Eqs.
// eq-fac-2, eq-fac-3 of arXiv 2105.01865).  Lane l of a warp owns the two
// adjacent lines at x = i0 + 2l, i0 + 2l + 1, so a tile covers 64 lines and
// every row access is one 256-byte coalesced pair access; both lines advance
// with one paired instruction (FFMA2 for FP32) per multiply-add, and each
// broadcast coefficient load serves two lines.  Warp w owns rows
// [w R, w R + R) in registers; the chunk end states are composed across warps
// through shared memory with the host-precomputed 2x2 chunk transfer
// matrices, as in ch_solve_cols.
//
// With UPDATE the solved increment is added to C (q^{l+1} = q^l + dq), C
// having been prefetched into shared memory by cp.async at kernel entry when
// it fits, so its latency hides behind the solve.  Requires even nx (pairs
// are 8/16-byte aligned).
#pragma once

#include <cooperative_groups.h>

#include "ch_explicit2.cuh"

namespace chg {

// dynamic shared memory of ch_solve_cols2 (in bytes), by part
template <typename T, int R, int NW, bool UPDATE>
struct Cols2Smem {
    static constexpr size_t kPair = 2 * sizeof(T);
    static constexpr size_t kQueues = (size_t)NW * 2 * 32 * kPair * 2;  // forward + backward chunk states
    static constexpr size_t kCorner = (size_t)4 * 32 * kPair;           // corner rows (periodic)
    static constexpr size_t kRows = (size_t)NW * R;
    static constexpr bool kPrefetch = UPDATE && kRows * 32 * kPair <= 96 * 1024;
    static constexpr size_t kCbuf = kPrefetch ? kRows * 32 * kPair : 0;
    static constexpr size_t bytes(bool) { return kQueues + kCorner + kCbuf; }
    static constexpr size_t kMax = kQueues + kCorner + kCbuf;
};

__device__ __forceinline__ void cp_async_pair(Pr<float>* dst, const float* src) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_pair(Pr<double>* dst, const double* src) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(src) : "memory");
}

// Coefficient loads: volatile (issued in program order, so the compiler
// does not keep R rows of coefficients live) unless CH_COLS2_PLAIN_LOADS.
#ifndef CH_COLS2_PLAIN_LOADS
#define CH_COLS2_PLAIN_LOADS 0
#endif

// two duplicated pairs (a, a, b, b) from a coefficient table row
template <typename T>
__device__ __forceinline__ void ld_pairs(const T* p, Pr<T>& a, Pr<T>& b) {
    const V4<T> c = CH_COLS2_PLAIN_LOADS ? ld4(p) : ldv4(p);
    a = mk(c.x, c.y);
    b = mk(c.z, c.w);
}
template <typename T>
__device__ __forceinline__ void ld_pair(const T* p, T& a, T& b) {
    if (CH_COLS2_PLAIN_LOADS)
        ld2(p, a, b);
    else
        ldv2(p, a, b);
}

// One 64-line tile (tile index = x-block + xblocks * outer) solved by the NW
// warps of a CTA; raw is the CTA's dynamic shared memory (Cols2Smem bytes).
template <typename T, int R, int NW, bool UPDATE>
__device__ __forceinline__ void solve_cols2_tile(T* a, T* Cf, int nx, int64_t outer_stride, int64_t line_stride,
                                                 const CCoef<T>& cf, unsigned int* status, int64_t tile,
                                                 unsigned char* raw) {
    using SM = Cols2Smem<T, R, NW, UPDATE>;
    __syncthreads();  // the buffers may still be read by a previous tile of this CTA
    Pr<T>* fq = reinterpret_cast<Pr<T>*>(raw);  // [NW][2][32]
    Pr<T>* bq = fq + NW * 2 * 32;               // [NW][2][32]
    Pr<T>* corner = bq + NW * 2 * 32;           // [4][32] (periodic)
    Pr<T>* cbuf = corner + 4 * 32;              // [rows][32] (prefetched C)
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int xblocks = (nx + 63) >> 6;
    const int xb = (int)(tile % xblocks);
    const int64_t outer = tile / xblocks;
    const int ia = xb * 64 + 2 * lane;
    const bool valid = ia < nx;  // nx even: ia + 1 < nx as well
    const int n = cf.n;
    const int j0 = w * R;
    const bool per = cf.periodic;
    const int64_t g = outer * outer_stride + ia + (int64_t)j0 * line_stride;

    if (SM::kPrefetch) {
#pragma unroll
        for (int i = 0; i < R; ++i)
            if (valid && j0 + i < n) cp_async_pair(&cbuf[(j0 + i) * 32 + lane], Cf + g + (int64_t)i * line_stride);
        cp_async_commit();
    }
    Pr<T> v[R];
#pragma unroll
    for (int i = 0; i < R; ++i)
        v[i] = (valid && j0 + i < n) ? ldp(a + g + (int64_t)i * line_stride) : sp<T>(T(0));

    // forward elimination from a zero state over this warp's rows
    Pr<T> y1 = sp<T>(T(0)), y2 = sp<T>(T(0));
#pragma unroll
    for (int i = 0; i < R; ++i) {
        Pr<T> nl1, nl2;
        ld_pairs(cf.fwdp + 4 * (j0 + i), nl1, nl2);
        const Pr<T> y = fma2(nl1, y1, fma2(nl2, y2, v[i]));
        y2 = y1;
        y1 = y;
    }
    fq[(w * 2 + 0) * 32 + lane] = y1;
    fq[(w * 2 + 1) * 32 + lane] = y2;
    __syncthreads();
    // incoming state: compose the chunks of warps 0 .. w-1
    Pr<T> s0 = sp<T>(T(0)), s1 = sp<T>(T(0));
    for (int u = 0; u < w; ++u) {
        const V4<T> Pm = ld4(cf.P + 4 * u);
        const Pr<T> n0 = fma2(sp<T>(Pm.x), s0, fma2(sp<T>(Pm.y), s1, fq[(u * 2 + 0) * 32 + lane]));
        const Pr<T> n1 = fma2(sp<T>(Pm.z), s0, fma2(sp<T>(Pm.w), s1, fq[(u * 2 + 1) * 32 + lane]));
        s0 = n0;
        s1 = n1;
    }
    y1 = s0;
    y2 = s1;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        Pr<T> nl1, nl2;
        ld_pairs(cf.fwdp + 4 * (j0 + i), nl1, nl2);
        const Pr<T> y = fma2(nl1, y1, fma2(nl2, y2, v[i]));
        y2 = y1;
        y1 = y;
        T d0, d1;
        ld_pair(cf.dinvp + 2 * (j0 + i), d0, d1);
        v[i] = mul(y, mk(d0, d1));
    }
    // back substitution from a zero state over this warp's rows
    Pr<T> x1 = sp<T>(T(0)), x2 = sp<T>(T(0));
#pragma unroll
    for (int i = R - 1; i >= 0; --i) {
        Pr<T> nu1, nu2;
        ld_pairs(cf.bwdp + 4 * (j0 + i), nu1, nu2);
        const Pr<T> x = fma2(nu1, x1, fma2(nu2, x2, v[i]));
        x2 = x1;
        x1 = x;
    }
    bq[(w * 2 + 0) * 32 + lane] = x1;
    bq[(w * 2 + 1) * 32 + lane] = x2;
    if (SM::kPrefetch) cp_async_wait<0>();
    __syncthreads();
    s0 = sp<T>(T(0));
    s1 = sp<T>(T(0));
    for (int u = NW - 1; u > w; --u) {
        const V4<T> Qm = ld4(cf.Q + 4 * u);
        const Pr<T> n0 = fma2(sp<T>(Qm.x), s0, fma2(sp<T>(Qm.y), s1, bq[(u * 2 + 0) * 32 + lane]));
        const Pr<T> n1 = fma2(sp<T>(Qm.z), s0, fma2(sp<T>(Qm.w), s1, bq[(u * 2 + 1) * 32 + lane]));
        s0 = n0;
        s1 = n1;
    }
    x1 = s0;
    x2 = s1;
#pragma unroll
    for (int i = R - 1; i >= 0; --i) {
        Pr<T> nu1, nu2;
        ld_pairs(cf.bwdp + 4 * (j0 + i), nu1, nu2);
        const Pr<T> x = fma2(nu1, x1, fma2(nu2, x2, v[i]));
        x2 = x1;
        x1 = x;
        v[i] = x;
        if (per) {  // corner rows 0, 1 -> slots 0, 1; rows n-2, n-1 -> slots 2, 3
            const int j = j0 + i;
            if (j < 2) corner[j * 32 + lane] = x;
            else if (j >= n - 2 && j < n) corner[(j - n + 4) * 32 + lane] = x;
        }
    }
    // periodic: the Woodbury correction from the corner rows (0, 1, n-2, n-1)
    // of the banded solution, s = K y_c, then x -= Z s
    Pr<T> sv0 = sp<T>(T(0)), sv1 = sv0, sv2 = sv0, sv3 = sv0;
    if (per) {
        __syncthreads();
        const Pr<T> c0 = corner[lane], c1 = corner[32 + lane], c2 = corner[64 + lane], c3 = corner[96 + lane];
        const V4<T> k0 = ld4(cf.K), k1 = ld4(cf.K + 4), k2 = ld4(cf.K + 8), k3 = ld4(cf.K + 12);
        sv0 = fma2(sp<T>(k0.x), c0, fma2(sp<T>(k0.y), c1, fma2(sp<T>(k0.z), c2, mul(sp<T>(k0.w), c3))));
        sv1 = fma2(sp<T>(k1.x), c0, fma2(sp<T>(k1.y), c1, fma2(sp<T>(k1.z), c2, mul(sp<T>(k1.w), c3))));
        sv2 = fma2(sp<T>(k2.x), c0, fma2(sp<T>(k2.y), c1, fma2(sp<T>(k2.z), c2, mul(sp<T>(k2.w), c3))));
        sv3 = fma2(sp<T>(k3.x), c0, fma2(sp<T>(k3.y), c1, fma2(sp<T>(k3.z), c2, mul(sp<T>(k3.w), c3))));
    }
    bool bad = false;
    T* dst = (UPDATE ? Cf : a) + g;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        Pr<T> o = v[i];
        if (per) {
            Pr<T> z0, z1, z2, z3;
            ld_pairs(cf.Zp + 8 * (j0 + i), z0, z1);
            ld_pairs(cf.Zp + 8 * (j0 + i) + 4, z2, z3);
            o = fma2(z0, sv0, fma2(z1, sv1, fma2(z2, sv2, fma2(z3, sv3, o))));
        }
        if (valid && j0 + i < n) {
            T* pd = dst + (int64_t)i * line_stride;
            if (UPDATE) {
                const Pr<T> cold = SM::kPrefetch ? cbuf[(j0 + i) * 32 + lane] : ldp(pd);
                const Pr<T> cnew = add(cold, o);
                bad |= !isfinite(cnew.x()) || !isfinite(cnew.y());
                stp(pd, cnew);
            } else {
                stp(pd, o);
            }
        }
    }
    if (UPDATE && bad) atomicOr(status, 1u);
}

// Up to 128 registers a thread (a lane holds R row pairs); shapes of 16 or
// more warps with 8 rows target 64 registers, for twice the resident warps.
template <int R, int NW>
struct Cols2MinBlocks {
    static constexpr int kThreadsPerSm = (R <= 8 && NW >= 16) ? 1024 : 512;
    static constexpr int value = kThreadsPerSm / (NW * 32) > 0 ? kThreadsPerSm / (NW * 32) : 1;
};
template <typename T, int R, int NW, bool UPDATE>
__global__ void __launch_bounds__(NW * 32, Cols2MinBlocks<R, NW>::value)
ch_solve_cols2(T* __restrict__ a, T* __restrict__ Cf, int nx, int64_t outer_stride, int64_t line_stride,
               CCoef<T> cf, unsigned int* status) {
    extern __shared__ __align__(16) unsigned char cols2_raw[];
    pdl_wait();
    pdl_launch_dependents();
    solve_cols2_tile<T, R, NW, UPDATE>(a, Cf, nx, outer_stride, line_stride, cf, status, blockIdx.x, cols2_raw);
}

// ---------------------------------------------------------------------------
// Cluster form for lines longer than one CTA holds (n in (256, 1024]): a
// 64-line tile is split over the CL CTAs of a thread-block cluster, CTA r
// owning rows [r NW R, (r+1) NW R).  Inside a CTA the warps compose their
// chunk states through shared memory as in solve_cols2_tile; across CTAs each
// CTA publishes its zero-start total state, and after a cluster barrier CTA r
// reads the totals of the CTAs before it (forward) or after it (backward)
// from their shared memory (distributed shared memory) and composes them with
// the products of those CTAs' warp matrices, which each CTA also publishes.  Periodic lines read the four
// corner rows from the CTAs that own them the same way.  A last cluster
// barrier keeps every CTA's shared memory alive until the remote reads end.
// ---------------------------------------------------------------------------
template <typename T, int R, int NW, int CL, bool UPDATE>
struct Cols2cSmem {
    static constexpr size_t kPair = 2 * sizeof(T);
    static constexpr size_t kQueues = (size_t)NW * 2 * 32 * kPair * 2;
    static constexpr size_t kTot = (size_t)2 * 2 * 32 * kPair;     // forward / backward totals
    static constexpr size_t kCorner = (size_t)4 * 32 * kPair;
    static constexpr size_t kRows = (size_t)NW * R;
    static constexpr size_t kCbuf = UPDATE ? kRows * 32 * kPair : 0;
    static constexpr size_t kBytes = kQueues + kTot + kCorner + kCbuf;
};

template <typename T, int R, int NW, int CL, bool UPDATE>
__global__ void __launch_bounds__(NW * 32, Cols2MinBlocks<R, NW>::value)
ch_solve_cols2c(T* __restrict__ a, T* __restrict__ Cf, int nx, int64_t outer_stride, int64_t line_stride,
                CCoef<T> cf, unsigned int* status) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char c2c_raw[];
    pdl_wait();
    Pr<T>* fq = reinterpret_cast<Pr<T>*>(c2c_raw);  // [NW][2][32]
    Pr<T>* bq = fq + NW * 2 * 32;                    // [NW][2][32]
    Pr<T>* tot = bq + NW * 2 * 32;                   // [2 (fwd, bwd)][2][32]
    Pr<T>* corner = tot + 2 * 2 * 32;                // [4][32]
    Pr<T>* cbuf = corner + 4 * 32;                   // [rows of this CTA][32]
    __shared__ T prod[8];                            // this CTA's forward and backward matrix products
    const int rank = (int)cluster.block_rank();
    const int64_t tile = blockIdx.x / CL;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int xblocks = (nx + 63) >> 6;
    const int xb = (int)(tile % xblocks);
    const int64_t outer = tile / xblocks;
    const int ia = xb * 64 + 2 * lane;
    const bool valid = ia < nx;
    const int n = cf.n;
    const int gw0 = rank * NW;           // first global warp of this CTA
    const int jc0 = gw0 * R;             // first row of this CTA
    const int j0 = jc0 + w * R;          // first row of this warp
    const bool per = cf.periodic;
    const int64_t g = outer * outer_stride + ia + (int64_t)j0 * line_stride;

    if (UPDATE) {
#pragma unroll
        for (int i = 0; i < R; ++i)
            if (valid && j0 + i < n)
                cp_async_pair(&cbuf[(w * R + i) * 32 + lane], Cf + g + (int64_t)i * line_stride);
        cp_async_commit();
    }
    Pr<T> v[R];
#pragma unroll
    for (int i = 0; i < R; ++i)
        v[i] = (valid && j0 + i < n) ? ldp(a + g + (int64_t)i * line_stride) : sp<T>(T(0));

    // forward elimination from a zero state over this warp's rows
    Pr<T> y1 = sp<T>(T(0)), y2 = sp<T>(T(0));
#pragma unroll
    for (int i = 0; i < R; ++i) {
        Pr<T> nl1, nl2;
        ld_pairs(cf.fwdp + 4 * (j0 + i), nl1, nl2);
        const Pr<T> y = fma2(nl1, y1, fma2(nl2, y2, v[i]));
        y2 = y1;
        y1 = y;
    }
    fq[(w * 2 + 0) * 32 + lane] = y1;
    fq[(w * 2 + 1) * 32 + lane] = y2;
    __syncthreads();
    if (w == 0) {  // this CTA's zero-start total and the product of its warps' matrices
        Pr<T> t0 = sp<T>(T(0)), t1 = sp<T>(T(0));
        T p00 = T(1), p01 = T(0), p10 = T(0), p11 = T(1);
        for (int u = 0; u < NW; ++u) {
            const V4<T> Pm = ld4(cf.P + 4 * (gw0 + u));
            const Pr<T> n0 = fma2(sp<T>(Pm.x), t0, fma2(sp<T>(Pm.y), t1, fq[(u * 2 + 0) * 32 + lane]));
            const Pr<T> n1 = fma2(sp<T>(Pm.z), t0, fma2(sp<T>(Pm.w), t1, fq[(u * 2 + 1) * 32 + lane]));
            t0 = n0;
            t1 = n1;
            const T q00 = Pm.x * p00 + Pm.y * p10, q01 = Pm.x * p01 + Pm.y * p11;
            const T q10 = Pm.z * p00 + Pm.w * p10, q11 = Pm.z * p01 + Pm.w * p11;
            p00 = q00; p01 = q01; p10 = q10; p11 = q11;
        }
        tot[0 * 32 + lane] = t0;
        tot[1 * 32 + lane] = t1;
        if (lane == 0) {
            prod[0] = p00; prod[1] = p01; prod[2] = p10; prod[3] = p11;
        }
    }
    cluster.sync();
    // incoming state: the totals of the CTAs before this one, then this CTA's warps before w
    Pr<T> s0 = sp<T>(T(0)), s1 = sp<T>(T(0));
    for (int c = 0; c < rank; ++c) {
        const Pr<T>* rt = cluster.map_shared_rank(tot, c);
        const T* rp = cluster.map_shared_rank(prod, c);
        const T m00 = rp[0], m01 = rp[1], m10 = rp[2], m11 = rp[3];
        const Pr<T> n0 = fma2(sp<T>(m00), s0, fma2(sp<T>(m01), s1, rt[0 * 32 + lane]));
        const Pr<T> n1 = fma2(sp<T>(m10), s0, fma2(sp<T>(m11), s1, rt[1 * 32 + lane]));
        s0 = n0;
        s1 = n1;
    }
    for (int u = 0; u < w; ++u) {
        const V4<T> Pm = ld4(cf.P + 4 * (gw0 + u));
        const Pr<T> n0 = fma2(sp<T>(Pm.x), s0, fma2(sp<T>(Pm.y), s1, fq[(u * 2 + 0) * 32 + lane]));
        const Pr<T> n1 = fma2(sp<T>(Pm.z), s0, fma2(sp<T>(Pm.w), s1, fq[(u * 2 + 1) * 32 + lane]));
        s0 = n0;
        s1 = n1;
    }
    y1 = s0;
    y2 = s1;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        Pr<T> nl1, nl2;
        ld_pairs(cf.fwdp + 4 * (j0 + i), nl1, nl2);
        const Pr<T> y = fma2(nl1, y1, fma2(nl2, y2, v[i]));
        y2 = y1;
        y1 = y;
        T d0, d1;
        ld_pair(cf.dinvp + 2 * (j0 + i), d0, d1);
        v[i] = mul(y, mk(d0, d1));
    }
    // back substitution from a zero state over this warp's rows
    Pr<T> x1 = sp<T>(T(0)), x2 = sp<T>(T(0));
#pragma unroll
    for (int i = R - 1; i >= 0; --i) {
        Pr<T> nu1, nu2;
        ld_pairs(cf.bwdp + 4 * (j0 + i), nu1, nu2);
        const Pr<T> x = fma2(nu1, x1, fma2(nu2, x2, v[i]));
        x2 = x1;
        x1 = x;
    }
    bq[(w * 2 + 0) * 32 + lane] = x1;
    bq[(w * 2 + 1) * 32 + lane] = x2;
    if (UPDATE) cp_async_wait<0>();
    __syncthreads();
    if (w == NW - 1) {  // this CTA's zero-start backward total and the product of its warps' matrices
        Pr<T> t0 = sp<T>(T(0)), t1 = sp<T>(T(0));
        T p00 = T(1), p01 = T(0), p10 = T(0), p11 = T(1);
        for (int u = NW - 1; u >= 0; --u) {
            const V4<T> Qm = ld4(cf.Q + 4 * (gw0 + u));
            const Pr<T> n0 = fma2(sp<T>(Qm.x), t0, fma2(sp<T>(Qm.y), t1, bq[(u * 2 + 0) * 32 + lane]));
            const Pr<T> n1 = fma2(sp<T>(Qm.z), t0, fma2(sp<T>(Qm.w), t1, bq[(u * 2 + 1) * 32 + lane]));
            t0 = n0;
            t1 = n1;
            const T q00 = Qm.x * p00 + Qm.y * p10, q01 = Qm.x * p01 + Qm.y * p11;
            const T q10 = Qm.z * p00 + Qm.w * p10, q11 = Qm.z * p01 + Qm.w * p11;
            p00 = q00; p01 = q01; p10 = q10; p11 = q11;
        }
        tot[2 * 32 + lane] = t0;
        tot[3 * 32 + lane] = t1;
        if (lane == 0) {
            prod[4] = p00; prod[5] = p01; prod[6] = p10; prod[7] = p11;
        }
    }
    cluster.sync();
    s0 = sp<T>(T(0));
    s1 = sp<T>(T(0));
    for (int c = CL - 1; c > rank; --c) {
        const Pr<T>* rt = cluster.map_shared_rank(tot, c);
        const T* rp = cluster.map_shared_rank(prod, c);
        const T m00 = rp[4], m01 = rp[5], m10 = rp[6], m11 = rp[7];
        const Pr<T> n0 = fma2(sp<T>(m00), s0, fma2(sp<T>(m01), s1, rt[2 * 32 + lane]));
        const Pr<T> n1 = fma2(sp<T>(m10), s0, fma2(sp<T>(m11), s1, rt[3 * 32 + lane]));
        s0 = n0;
        s1 = n1;
    }
    for (int u = NW - 1; u > w; --u) {
        const V4<T> Qm = ld4(cf.Q + 4 * (gw0 + u));
        const Pr<T> n0 = fma2(sp<T>(Qm.x), s0, fma2(sp<T>(Qm.y), s1, bq[(u * 2 + 0) * 32 + lane]));
        const Pr<T> n1 = fma2(sp<T>(Qm.z), s0, fma2(sp<T>(Qm.w), s1, bq[(u * 2 + 1) * 32 + lane]));
        s0 = n0;
        s1 = n1;
    }
    x1 = s0;
    x2 = s1;
#pragma unroll
    for (int i = R - 1; i >= 0; --i) {
        Pr<T> nu1, nu2;
        ld_pairs(cf.bwdp + 4 * (j0 + i), nu1, nu2);
        const Pr<T> x = fma2(nu1, x1, fma2(nu2, x2, v[i]));
        x2 = x1;
        x1 = x;
        v[i] = x;
        if (per) {  // corner rows 0, 1 -> slots 0, 1; rows n-2, n-1 -> slots 2, 3 (in the owning CTA)
            const int j = j0 + i;
            if (j < 2) corner[j * 32 + lane] = x;
            else if (j >= n - 2 && j < n) corner[(j - n + 4) * 32 + lane] = x;
        }
    }
    Pr<T> sv0 = sp<T>(T(0)), sv1 = sv0, sv2 = sv0, sv3 = sv0;
    if (per) {
        cluster.sync();
        Pr<T> cv[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int row = m < 2 ? m : n - 4 + m;
            const Pr<T>* rc = cluster.map_shared_rank(corner, row / (NW * R));
            cv[m] = rc[m * 32 + lane];
        }
        const V4<T> k0 = ld4(cf.K), k1 = ld4(cf.K + 4), k2 = ld4(cf.K + 8), k3 = ld4(cf.K + 12);
        sv0 = fma2(sp<T>(k0.x), cv[0], fma2(sp<T>(k0.y), cv[1], fma2(sp<T>(k0.z), cv[2], mul(sp<T>(k0.w), cv[3]))));
        sv1 = fma2(sp<T>(k1.x), cv[0], fma2(sp<T>(k1.y), cv[1], fma2(sp<T>(k1.z), cv[2], mul(sp<T>(k1.w), cv[3]))));
        sv2 = fma2(sp<T>(k2.x), cv[0], fma2(sp<T>(k2.y), cv[1], fma2(sp<T>(k2.z), cv[2], mul(sp<T>(k2.w), cv[3]))));
        sv3 = fma2(sp<T>(k3.x), cv[0], fma2(sp<T>(k3.y), cv[1], fma2(sp<T>(k3.z), cv[2], mul(sp<T>(k3.w), cv[3]))));
    }
    bool bad = false;
    T* dst = (UPDATE ? Cf : a) + g;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        Pr<T> o = v[i];
        if (per) {
            Pr<T> z0, z1, z2, z3;
            ld_pairs(cf.Zp + 8 * (j0 + i), z0, z1);
            ld_pairs(cf.Zp + 8 * (j0 + i) + 4, z2, z3);
            o = fma2(z0, sv0, fma2(z1, sv1, fma2(z2, sv2, fma2(z3, sv3, o))));
        }
        if (valid && j0 + i < n) {
            T* pd = dst + (int64_t)i * line_stride;
            if (UPDATE) {
                const Pr<T> cnew = add(cbuf[(w * R + i) * 32 + lane], o);
                bad |= !isfinite(cnew.x()) || !isfinite(cnew.y());
                stp(pd, cnew);
            } else {
                stp(pd, o);
            }
        }
    }
    if (UPDATE && bad) atomicOr(status, 1u);
    cluster.sync();  // no CTA leaves while another may still read its shared memory
}

}  // namespace chg
