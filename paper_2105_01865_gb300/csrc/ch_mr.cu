// Multiple-resolution velocity transfer (arXiv 2105.01865, Sec. 3.4): the
// face velocity of a stretched coarse mesh is carried to the uniform fine
// mesh of C through its face-normal gradients, a tri-cubic Hermite spline of
// four points per direction (64-point stencil, tables built once), and an
// integration along every fine line from a reference plane.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "ch_internal.h"

using namespace chg;

namespace {

constexpr int kThreads = 256;

// ---------------------------------------------------------------------------
// Tables: for every fine cell centre x = (i + 1/2) h of one direction, the
// first of its four coarse nodes and the four weights of the cubic Hermite
// segment that contains x.  Nodes are coarse cell centres; the base node is
// the last node at or left of x; slopes are central differences over the
// neighbouring nodes (one-sided at the ends of a walled direction, whose
// stencil is clamped into the node range); periodic directions wrap.
// ---------------------------------------------------------------------------
__global__ void mr_tables_kernel(const double* __restrict__ faces, int nc, int periodic, int nfine, double h,
                                 const double* __restrict__ queries, int32_t* __restrict__ start_out,
                                 double* __restrict__ w_out, float* __restrict__ wf_out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nfine) return;
    // query point: the fine cell centre, or an explicit coordinate (restriction tables)
    const double x = queries ? queries[i] : ((double)i + 0.5) * h;
    const double P = faces[nc] - faces[0];
    auto node = [&](int k) { return 0.5 * (faces[k] + faces[k + 1]); };
    // j = max{j : node_j <= x}, -1 if none (binary search)
    int lo = 0, hi = nc;  // invariant: node(lo-1) <= x < node(hi) in the extended sense
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (node(mid) <= x)
            lo = mid + 1;
        else
            hi = mid;
    }
    const int j = lo - 1;
    double wgt[4] = {0.0, 0.0, 0.0, 0.0};
    int start;
    double xs[4];
    int a, b, la, ha, lb, hb;  // segment nodes and slope neighbours, as slots 0..3
    if (periodic) {
        start = ((j - 1) % nc + nc) % nc;
        for (int m = 0; m < 4; ++m) {
            const int k = j - 1 + m;
            const int q = (k >= 0) ? k / nc : -((-k + nc - 1) / nc);
            const int kk = k - q * nc;
            xs[m] = node(kk) + P * (double)q;
        }
        a = 1; b = 2; la = 0; ha = 2; lb = 1; hb = 3;
    } else {
        const int seg = min(max(j, 0), nc - 2);
        start = min(max(seg - 1, 0), nc - 4);
        for (int m = 0; m < 4; ++m) xs[m] = node(start + m);
        a = seg - start;
        b = a + 1;
        la = max(seg - 1, 0) - start;
        ha = seg + 1 - start;
        lb = seg - start;
        hb = min(seg + 2, nc - 1) - start;
    }
    const double dx = xs[b] - xs[a];
    const double t = (x - xs[a]) / dx;
    const double h00 = 2 * t * t * t - 3 * t * t + 1;
    const double h10 = t * t * t - 2 * t * t + t;
    const double h01 = -2 * t * t * t + 3 * t * t;
    const double h11 = t * t * t - t * t;
    wgt[a] += h00;
    wgt[b] += h01;
    const double sa = h10 * dx / (xs[ha] - xs[la]);
    wgt[ha] += sa;
    wgt[la] -= sa;
    const double sb = h11 * dx / (xs[hb] - xs[lb]);
    wgt[hb] += sb;
    wgt[lb] -= sb;
    start_out[i] = start;
    for (int m = 0; m < 4; ++m) {
        w_out[4 * i + m] = wgt[m];
        wf_out[4 * i + m] = (float)wgt[m];
    }
}

// Step (1) of Sec. 3.4: normal gradients at coarse cell centres.
template <typename T>
__global__ void mr_gradients_kernel(const T* __restrict__ uc, const T* __restrict__ vc, const T* __restrict__ wc,
                                    const double* __restrict__ xf, const double* __restrict__ yf,
                                    const double* __restrict__ zf, int ncx, int ncy, int ncz, int ncfx, int ncfy,
                                    int per_x, int per_y, int per_z, T* __restrict__ gx, T* __restrict__ gy,
                                    T* __restrict__ gz) {
    const int64_t N = (int64_t)ncx * ncy * ncz;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % ncx);
        const int64_t t = e / ncx;
        const int j = (int)(t % ncy), k = (int)(t / ncy);
        const int ip = per_x ? (i + 1) % ncx : i + 1;
        const int jp = per_y ? (j + 1) % ncy : j + 1;
        const int kp = per_z ? (k + 1) % ncz : k + 1;
        const T du = uc[((int64_t)k * ncy + j) * ncfx + ip] - uc[((int64_t)k * ncy + j) * ncfx + i];
        const T dv = vc[((int64_t)k * ncfy + jp) * ncx + i] - vc[((int64_t)k * ncfy + j) * ncx + i];
        const T dw = wc[((int64_t)kp * ncy + j) * ncx + i] - wc[((int64_t)k * ncy + j) * ncx + i];
        gx[e] = du / T(xf[i + 1] - xf[i]);
        gy[e] = dv / T(yf[j + 1] - yf[j]);
        gz[e] = dw / T(zf[k + 1] - zf[k]);
    }
}

template <typename T>
struct Tab {
    const int32_t* __restrict__ s;
    const T* __restrict__ w;
};

// 2D Hermite of a coarse face plane P[row][col] (row stride `stride`).
template <typename T>
__device__ __forceinline__ T hermite2(const T* __restrict__ P, int64_t row_stride, int64_t col_stride, int nr,
                                      int ncol, int sr, const T* wr, int sc, const T* wc) {
    T acc = T(0);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        int kr = sr + b;
        kr -= (kr >= nr) ? nr : 0;
        T accc = T(0);
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            int kc = sc + a;
            kc -= (kc >= ncol) ? ncol : 0;
            accc += wc[a] * P[kr * row_stride + kc * col_stride];
        }
        acc += wr[b] * accc;
    }
    return acc;
}

struct MrArgs {
    int nx, ny, nz;       // fine cells
    int nfx, nfy, nfz;    // fine face planes
    int ncx, ncy, ncz;    // coarse cells
    int ncfx, ncfy, ncfz; // coarse face planes
    int wall[3];
    double h;
};

// The 4 weights of entry i of a table (16-byte aligned rows in FP32).
__device__ __forceinline__ void load_w(const float* __restrict__ w, int i, float* out) {
    const float4 v = *reinterpret_cast<const float4*>(w + 4 * i);
    out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
}
__device__ __forceinline__ void load_w(const double* __restrict__ w, int i, double* out) {
    const double2 a = *reinterpret_cast<const double2*>(w + 4 * i), b = *reinterpret_cast<const double2*>(w + 4 * i + 2);
    out[0] = a.x; out[1] = a.y; out[2] = b.x; out[3] = b.y;
}

// Running sum of the integration (step 3).  FP32 keeps a compensation term
// (Kahan's summation: the rounding error of every addition is carried and
// fed back), so a 1024-term prefix sum stays within a few FP32 roundings of
// the exact sum without FP64 arithmetic, which is slow on this GPU; FP64 sums
// plainly.
template <typename T>
struct RunSum {
    T s = T(0), c = T(0);  // sum and the negated lost low-order part
    __device__ __forceinline__ void add(T x) {
        const T y = __fsub_rn(x, c);
        const T t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ T value() const { return __fsub_rn(s, c); }
    __device__ __forceinline__ T plus(T x) const { return __fadd_rn(s, __fsub_rn(x, c)); }
};
template <>
struct RunSum<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double value() const { return s; }
    __device__ __forceinline__ double plus(double x) const { return s + x; }
};

__device__ __forceinline__ int wrap_add(int s, int m, int n) {
    const int k = s + m;
    return k >= n ? k - n : k;
}

// Running sum of the integration along a line, carried in blocks: the terms
// of the current block of up to 32 cells add to a plain partial p, and every
// full block is folded into a compensated carry (Kahan's summation in FP32,
// plain in FP64).  A prefix of a 1024-cell line is then within a few
// roundings of the exact sum without FP64 arithmetic, which is slow on this
// GPU.
template <typename T>
struct BlockSum {
    RunSum<T> carry;
    T p = T(0);
    int n = 0;
    __device__ __forceinline__ T value() const { return carry.plus(p); }
    __device__ __forceinline__ void add(T x) {
        p += x;
        if (++n == 32) {
            carry.add(p);
            p = T(0);
            n = 0;
        }
    }
};

// Steps (2)-(3) along x: one warp per fine x-line (j, k).  The 64-point
// stencil is sum-factorised: the warp first contracts the 16 coarse rows of
// its (y, z) stencil into one coarse x-line g(ix) = sum_{b,c} wy_b wz_c
// G(ix, sy+b, sz+c) (coalesced over ix, kept in shared memory), then walks the
// fine line in chunks of 128 cells, 4 consecutive cells per lane: each cell's
// gradient is the 4-point x-stencil of g; a lane sums its 4 terms, a warp
// scan of the lane sums gives the chunk's prefix, and a compensated carry
// joins the chunks (R20).  u(face i) = u_ref(j, k) + h sum_{i' < i} Gx(i').
//
// The 8 warps of a CTA take 8 consecutive j of one k, whose y-stencils start
// within a few coarse rows of each other.  When they all start within
// qrows - 4 rows of the first (qrows > 0), the CTA first contracts the 4
// coarse z-rows once for each of those y-rows into shared memory,
// Q(r, ix) = sum_c wz_c G(ix, sy0 + r, sz + c), and each warp then forms
// g(ix) = sum_b wy_b Q(sy - sy0 + b, ix): about 6 instead of 32 coarse-row
// reads per ix per CTA.  Otherwise each warp contracts its 16 rows itself.
constexpr int kMrWarps = 8;
constexpr int kMrQRows = 8;
// adjacent fine columns per thread of the y/z line march (1, 2 or 4)
#ifndef CH_MR_CPT
#define CH_MR_CPT 4
#endif
constexpr size_t kMrMaxSmem = 226 * 1024;  // dynamic shared memory per CTA (227 KB on sm_103a, less the static)

template <typename T>
__global__ void __launch_bounds__(kMrWarps * 32, 4)
mr_integrate_x(const T* __restrict__ gx, const T* __restrict__ uc, Tab<T> tx, Tab<T> ty, Tab<T> tz, MrArgs a,
               T* __restrict__ u, int qrows) {
    // kMrWarps coarse lines of ncx + 4 values, then qrows rows of Q
    extern __shared__ __align__(16) unsigned char mr_smem[];
    __shared__ int dmax;
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nlines = a.ny * a.nz;
    const int warp = blockIdx.x * kMrWarps + wib;
    const bool live = warp < nlines;
    const int wl = live ? warp : nlines - 1;  // a warp past the last line stands in for it until it leaves
    const int j = wl % a.ny, k = wl / a.ny;
    T wy[4], wz[4];
    load_w(ty.w, j, wy);
    load_w(tz.w, k, wz);
    const int sy = ty.s[j], sz = tz.s[k];
    const int ld = a.ncx + 4;
    // the coarse line, followed by copies of its first 4 values, so a stencil
    // starting at sx <= ncx - 1 reads g[sx .. sx + 4] without wrapping
    T* g = reinterpret_cast<T*>(mr_smem) + (int64_t)wib * ld;
    const int w0 = blockIdx.x * kMrWarps, wlast = min(w0 + kMrWarps - 1, nlines - 1);
    const int sy0 = ty.s[w0 % a.ny];
    const int d = sy >= sy0 ? sy - sy0 : sy - sy0 + a.ncy;  // this line's first y-row, counted from sy0
    bool shared_q = false;
    if (qrows > 0 && w0 / a.ny == wlast / a.ny) {  // one k (and so one sz, wz) for the whole CTA
        if (threadIdx.x == 0) dmax = 0;
        __syncthreads();
        if (lane == 0) atomicMax(&dmax, d);
        __syncthreads();
        shared_q = dmax + 4 <= qrows;
    }
    if (shared_q) {
        const int nq = dmax + 4;
        T* Q = reinterpret_cast<T*>(mr_smem) + (int64_t)kMrWarps * ld;
        for (int r = 0; r < nq; ++r) {
            const int ky = (sy0 + r) % a.ncy;
            int zr[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) zr[c] = (wrap_add(sz, c, a.ncz) * a.ncy + ky) * a.ncx;
            for (int ix = threadIdx.x; ix < a.ncx + 4; ix += kMrWarps * 32) {
                const int cx = ix < a.ncx ? ix : ix - a.ncx;
                Q[r * ld + ix] = wz[0] * gx[zr[0] + cx] + wz[1] * gx[zr[1] + cx] + wz[2] * gx[zr[2] + cx] +
                                 wz[3] * gx[zr[3] + cx];
            }
        }
        __syncthreads();
        if (!live) return;  // whole warp
        const T* q0 = Q + d * ld;
        for (int ix = lane; ix < a.ncx + 4; ix += 32)
            g[ix] = wy[0] * q0[ix] + wy[1] * q0[ld + ix] + wy[2] * q0[2 * ld + ix] + wy[3] * q0[3 * ld + ix];
    } else {
        if (!live) return;  // whole warp
        int rows[4][4];  // element offsets of the 16 coarse rows (the coarse mesh has < 2^31 cells)
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int b = 0; b < 4; ++b)
                rows[c][b] = (wrap_add(sz, c, a.ncz) * a.ncy + wrap_add(sy, b, a.ncy)) * a.ncx;
        for (int ix = lane; ix < a.ncx + 4; ix += 32) {
            const int cx = ix < a.ncx ? ix : ix - a.ncx;
            T acc = T(0);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const T accy = wy[0] * gx[rows[c][0] + cx] + wy[1] * gx[rows[c][1] + cx] +
                               wy[2] * gx[rows[c][2] + cx] + wy[3] * gx[rows[c][3] + cx];
                acc += wz[c] * accy;
            }
            g[ix] = acc;
        }
    }
    T uref = T(0);
    if (!a.wall[0]) uref = hermite2(uc, (int64_t)a.ncy * a.ncfx, (int64_t)a.ncfx, a.ncz, a.ncy, sz, wz, sy, wy);
    __syncwarp();
    T* row = u + ((int64_t)k * a.ny + j) * a.nfx;
    const T hT = (T)a.h;
    const bool vec = (a.nx % 4 == 0) && (a.nfx % 4 == 0);
    RunSum<T> carry;  // sum over the previous chunks
    for (int i0 = 0; i0 < a.nx; i0 += 128) {
        const int ib = i0 + 4 * lane;
        T gv[4];
        int sxq[4];
        if (ib + 3 < a.nx) {
            const int4 s4 = *reinterpret_cast<const int4*>(tx.s + ib);  // 16-byte aligned: ib % 4 == 0
            sxq[0] = s4.x; sxq[1] = s4.y; sxq[2] = s4.z; sxq[3] = s4.w;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) sxq[q] = ib + q < a.nx ? tx.s[ib + q] : 0;
        }
        int span = sxq[3] - sxq[0];  // the starts are non-decreasing modulo ncx
        if (span < 0) span += a.ncx;
        if (ib + 3 < a.nx && span <= 1) {
            // the 4 cells' stencils start at s0 or s0 + 1 modulo ncx (a coarse
            // mesh at least twice as coarse as the fine one): 5 shared loads
            // serve them, instead of 16 (g[s0 + 1 + m] is g[m] past the wrap)
            const T* gs = g + sxq[0];
            const T g0 = gs[0], g1 = gs[1], g2 = gs[2], g3 = gs[3], g4 = gs[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                T wx[4];
                load_w(tx.w, ib + q, wx);
                const bool o = sxq[q] != sxq[0];
                gv[q] = wx[0] * (o ? g1 : g0) + wx[1] * (o ? g2 : g1) + wx[2] * (o ? g3 : g2) + wx[3] * (o ? g4 : g3);
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = ib + q;
                gv[q] = T(0);
                if (i < a.nx) {
                    T wx[4];
                    load_w(tx.w, i, wx);
                    const T* gs = g + sxq[q];
                    gv[q] = wx[0] * gs[0] + wx[1] * gs[1] + wx[2] * gs[2] + wx[3] * gs[3];
                }
            }
        }
        const T l1 = gv[0], l2 = l1 + gv[1], l3 = l2 + gv[2], tot = l3 + gv[3];
        T incl = tot;  // inclusive scan of the lane sums
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const T base = carry.plus(incl - tot);
        const T o0 = uref + hT * base, o1 = uref + hT * (base + l1), o2 = uref + hT * (base + l2),
                o3 = uref + hT * (base + l3);
        if (vec && ib < a.nx) {
            if constexpr (sizeof(T) == 4) {
                *reinterpret_cast<float4*>(row + ib) = make_float4(o0, o1, o2, o3);
            } else {
                *reinterpret_cast<double2*>(row + ib) = make_double2(o0, o1);
                *reinterpret_cast<double2*>(row + ib + 2) = make_double2(o2, o3);
            }
        } else {
            if (ib < a.nx) row[ib] = o0;
            if (ib + 1 < a.nx) row[ib + 1] = o1;
            if (ib + 2 < a.nx) row[ib + 2] = o2;
            if (ib + 3 < a.nx) row[ib + 3] = o3;
        }
        carry.add(__shfl_sync(0xffffffffu, incl, 31));
    }
    if (a.wall[0] && lane == 0) row[a.nx] = uref + hT * carry.value();
}

// Step (2) for a strided direction d (y or z), sum-factorised: the coarse
// gradient of d interpolated by the 4-point Hermite stencils of the two
// directions across the d-lines (x, and z for d = y or y for d = z) to the
// fine positions there, at every coarse node along d:
//   d = y: Py[k][ky][i] = sum_c wz_c(k) sum_q wx_q(i) Gy(sx(i) + q, ky, sz(k) + c),
//   d = z: Pz[kz][j][i] = sum_b wy_b(j) sum_q wx_q(i) Gz(sx(i) + q, sy(j) + b, kz).
// One CTA per output row at a time: the non-x contraction of the row's coarse
// x-line goes to shared memory, then every fine i takes its 4-point x-stencil.
// The 64-point tri-cubic value at a fine cell is then the 4-point stencil
// along d of these (mr_line_yz).
template <typename T, int DIR>
__global__ void __launch_bounds__(256)
mr_plane_yz(const T* __restrict__ G, Tab<T> tx, Tab<T> ty, Tab<T> tz, MrArgs a, T* __restrict__ P) {
    extern __shared__ __align__(16) unsigned char mr_smem[];  // one coarse x-line
    T* Z = reinterpret_cast<T*>(mr_smem);
    const int nrows = DIR == 1 ? a.nz * a.ncy : a.ncz * a.ny;
    for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
        int64_t rowoff[4];
        T w[4];
        if (DIR == 1) {  // r = k ncy + ky: contract z
            const int k = r / a.ncy, ky = r - k * a.ncy;
            load_w(tz.w, k, w);
            const int sz = tz.s[k];
#pragma unroll
            for (int c = 0; c < 4; ++c) rowoff[c] = ((int64_t)wrap_add(sz, c, a.ncz) * a.ncy + ky) * a.ncx;
        } else {         // r = kz ny + j: contract y
            const int kz = r / a.ny, j = r - kz * a.ny;
            load_w(ty.w, j, w);
            const int sy = ty.s[j];
#pragma unroll
            for (int b = 0; b < 4; ++b) rowoff[b] = ((int64_t)kz * a.ncy + wrap_add(sy, b, a.ncy)) * a.ncx;
        }
        __syncthreads();  // the previous row's Z is no longer read
        for (int x = threadIdx.x; x < a.ncx; x += blockDim.x)
            Z[x] = w[0] * G[rowoff[0] + x] + w[1] * G[rowoff[1] + x] + w[2] * G[rowoff[2] + x] +
                   w[3] * G[rowoff[3] + x];
        __syncthreads();
        T* out = P + (int64_t)r * a.nx;
        for (int i = threadIdx.x; i < a.nx; i += blockDim.x) {
            T wx[4];
            load_w(tx.w, i, wx);
            const int sx = tx.s[i];
            out[i] = wx[0] * Z[sx] + wx[1] * Z[wrap_add(sx, 1, a.ncx)] + wx[2] * Z[wrap_add(sx, 2, a.ncx)] +
                     wx[3] * Z[wrap_add(sx, 3, a.ncx)];
        }
    }
}

// Step (3) along a strided direction (y: v, or z: w): one thread per fine
// transverse position (i, o), marching the fine line.  The 4 values of Py / Pz
// at the coarse nodes of the current stencil sit in a window that slides with
// it (one coalesced load per coarse node passed), so a fine cell costs its
// 4-point stencil along the line, the running sum and one store.
// CPT adjacent columns i .. i + CPT - 1 per thread (nx a multiple of CPT):
// the loads of the start and weights along the line, the window test and the
// loop serve all CPT columns, and the window loads and stores move CPT values
// at once.
template <typename T, int CPT>
struct MrVec;
template <typename T>
struct MrVec<T, 1> {
    static __device__ __forceinline__ void ld(const T* p, T* v) { v[0] = *p; }
    static __device__ __forceinline__ void st(T* p, const T* v) { *p = v[0]; }
};
template <>
struct MrVec<float, 2> {
    static __device__ __forceinline__ void ld(const float* p, float* v) {
        const float2 t = *reinterpret_cast<const float2*>(p);
        v[0] = t.x; v[1] = t.y;
    }
    static __device__ __forceinline__ void st(float* p, const float* v) {
        *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
    }
};
template <>
struct MrVec<float, 4> {
    static __device__ __forceinline__ void ld(const float* p, float* v) {
        const float4 t = *reinterpret_cast<const float4*>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
    static __device__ __forceinline__ void st(float* p, const float* v) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <>
struct MrVec<double, 2> {
    static __device__ __forceinline__ void ld(const double* p, double* v) {
        const double2 t = *reinterpret_cast<const double2*>(p);
        v[0] = t.x; v[1] = t.y;
    }
    static __device__ __forceinline__ void st(double* p, const double* v) {
        *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    }
};

template <typename T, int DIR, int CPT>
__global__ void __launch_bounds__(256)
mr_line_yz(const T* __restrict__ P, const T* __restrict__ Vc, Tab<T> tx, Tab<T> ty, Tab<T> tz, MrArgs a,
           T* __restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int nlong = DIR == 1 ? a.ny : a.nz;                 // fine cells along the line
    const int ntr = DIR == 1 ? a.nz : a.ny;                   // second transverse fine size
    const int nxc = a.nx / CPT;                               // column groups along x
    if (t >= (int64_t)nxc * ntr) return;
    const int i = (int)(t % nxc) * CPT, o = (int)(t / nxc);   // first fine x and the other transverse index
    const Tab<T>& to = DIR == 1 ? tz : ty;                    // table of the other transverse direction
    const Tab<T>& tl = DIR == 1 ? ty : tz;                    // table along the line
    const int ncl = DIR == 1 ? a.ncy : a.ncz;                 // coarse cells along the line
    // P address of coarse node m along the line for this thread
    const T* p0 = DIR == 1 ? P + (int64_t)o * a.ncy * a.nx + i : P + (int64_t)o * a.nx + i;
    const int64_t pst = DIR == 1 ? (int64_t)a.nx : (int64_t)a.ny * a.nx;
    // reference plane: v at y = 0 (plane [kz][0][kx] of Vc) or w at z = 0
    T ref[CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
        ref[c] = T(0);
        if (!a.wall[DIR]) {
            T wxv[4], wov[4];
            load_w(tx.w, i + c, wxv);
            load_w(to.w, o, wov);
            if (DIR == 1)
                ref[c] = hermite2(Vc, (int64_t)a.ncfy * a.ncx, (int64_t)1, a.ncz, a.ncx, to.s[o], wov, tx.s[i + c], wxv);
            else
                ref[c] = hermite2(Vc, (int64_t)a.ncx, (int64_t)1, a.ncy, a.ncx, to.s[o], wov, tx.s[i + c], wxv);
        }
    }
    T win[4][CPT];
    int ws = -1;  // coarse start index of the window
    const T hT = (T)a.h;
    BlockSum<T> run[CPT];
    int64_t idx = DIR == 1 ? ((int64_t)o * a.nfy) * a.nx + i : (int64_t)o * a.nx + i;
    const int64_t ost = DIR == 1 ? (int64_t)a.nx : (int64_t)a.ny * a.nx;  // output stride along the line
    for (int jl = 0; jl < nlong; ++jl, idx += ost) {
        const int sl = tl.s[jl];
        if (sl != ws) {
            if (ws >= 0 && sl == wrap_add(ws, 1, ncl)) {
#pragma unroll
                for (int c = 0; c < CPT; ++c) {
                    win[0][c] = win[1][c];
                    win[1][c] = win[2][c];
                    win[2][c] = win[3][c];
                }
                MrVec<T, CPT>::ld(p0 + wrap_add(sl, 3, ncl) * pst, win[3]);
            } else {
#pragma unroll
                for (int m = 0; m < 4; ++m) MrVec<T, CPT>::ld(p0 + wrap_add(sl, m, ncl) * pst, win[m]);
            }
            ws = sl;
        }
        T wl[4];
        load_w(tl.w, jl, wl);
        T o_[CPT];
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const T gval = wl[0] * win[0][c] + wl[1] * win[1][c] + wl[2] * win[2][c] + wl[3] * win[3][c];
            o_[c] = ref[c] + hT * run[c].value();
            run[c].add(gval);
        }
        MrVec<T, CPT>::st(out + idx, o_);
    }
    if (a.wall[DIR]) {
        T o_[CPT];
#pragma unroll
        for (int c = 0; c < CPT; ++c) o_[c] = ref[c] + hT * run[c].value();
        MrVec<T, CPT>::st(out + idx, o_);
    }
}

MrArgs mr_args(const ch_handle* h) {
    MrArgs a;
    a.nx = (int)h->n[0];
    a.ny = (int)h->n[1];
    a.nz = (int)h->n[2];
    a.nfx = (int)h->nf[0];
    a.nfy = (int)h->nf[1];
    a.nfz = (int)h->nf[2];
    a.ncx = (int)h->nc[0];
    a.ncy = (int)h->nc[1];
    a.ncz = (int)h->nc[2];
    a.ncfx = (int)h->ncf[0];
    a.ncfy = (int)h->ncf[1];
    a.ncfz = (int)h->ncf[2];
    for (int d = 0; d < 3; ++d) a.wall[d] = h->p.bc[d] != CH_PERIODIC;
    a.h = h->p.h;
    return a;
}

template <typename T>
Tab<T> tab(const ch_handle* h, int d) {
    Tab<T> t;
    t.s = h->mr_start[d];
    t.w = (const T*)(sizeof(T) == 8 ? (const void*)h->mr_w[d] : (const void*)(h->mr_w[d] + 4 * h->n[d]));
    return t;
}

// The transfer's four launches; with ev (5 events) an event is recorded
// before the first and after every launch.
template <typename T>
int interp(ch_handle* h, cudaEvent_t* ev = nullptr) {
    const MrArgs a = mr_args(h);
    const double* xf = h->mr_coords;
    const double* yf = xf + h->nc[0] + 1;
    const double* zf = yf + h->nc[1] + 1;
    const int64_t ncell = h->nc[0] * h->nc[1] * h->nc[2];
    const int gblocks = (int)std::min<int64_t>((ncell + kThreads - 1) / kThreads, 8 * 152);
    if (ev) CHG_CUDA(h, cudaEventRecord(ev[0], h->stream));
    mr_gradients_kernel<T><<<gblocks, kThreads, 0, h->stream>>>(
        (const T*)h->vel_c[0], (const T*)h->vel_c[1], (const T*)h->vel_c[2], xf, yf, zf, a.ncx, a.ncy, a.ncz, a.ncfx,
        a.ncfy, !a.wall[0], !a.wall[1], !a.wall[2], (T*)h->grad_c[0], (T*)h->grad_c[1], (T*)h->grad_c[2]);
    CHG_CUDA(h, cudaGetLastError());
    if (ev) CHG_CUDA(h, cudaEventRecord(ev[1], h->stream));
    const Tab<T> tx = tab<T>(h, 0), ty = tab<T>(h, 1), tz = tab<T>(h, 2);
    {
        const int64_t warps = (int64_t)a.ny * a.nz;
        const unsigned blocks = (unsigned)((warps + kMrWarps - 1) / kMrWarps);
        // the shared z-contraction's rows where they fit beside the warps' lines
        const size_t line_bytes = (size_t)(a.ncx + 4) * sizeof(T);
        const int qrows = (kMrWarps + kMrQRows) * line_bytes <= kMrMaxSmem ? kMrQRows : 0;
        const size_t smem = (kMrWarps + qrows) * line_bytes;
        static bool attr_set = false;  // one instantiation per T
        if (!attr_set) {
            const size_t most = std::min((size_t)(kMrWarps + kMrQRows) * (kMaxCoarseLine + 4) * sizeof(T), kMrMaxSmem);
            CHG_CUDA(h, cudaFuncSetAttribute(mr_integrate_x<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most));
            attr_set = true;
        }
        mr_integrate_x<T><<<blocks, kMrWarps * 32, smem, h->stream>>>((const T*)h->grad_c[0], (const T*)h->vel_c[0],
                                                                      tx, ty, tz, a, (T*)h->vel[0], qrows);
        CHG_CUDA(h, cudaGetLastError());
        if (ev) CHG_CUDA(h, cudaEventRecord(ev[2], h->stream));
    }
    T* P = (T*)h->mr_plane;
    const size_t zsm = (size_t)a.ncx * sizeof(T);
    // the line march with CPT adjacent columns per thread where nx allows
    constexpr int CPT = sizeof(T) == 4 ? CH_MR_CPT : (CH_MR_CPT < 2 ? CH_MR_CPT : 2);
    auto line = [&](auto dirc, const T* Vc, T* out, int64_t ntr) {
        constexpr int DIR = decltype(dirc)::value;
        if (a.nx % CPT == 0) {
            const int64_t thr = (int64_t)(a.nx / CPT) * ntr;
            mr_line_yz<T, DIR, CPT><<<(unsigned)((thr + 255) / 256), 256, 0, h->stream>>>(P, Vc, tx, ty, tz, a, out);
        } else {
            const int64_t thr = (int64_t)a.nx * ntr;
            mr_line_yz<T, DIR, 1><<<(unsigned)((thr + 255) / 256), 256, 0, h->stream>>>(P, Vc, tx, ty, tz, a, out);
        }
    };
    {
        mr_plane_yz<T, 1><<<16 * 152, 256, zsm, h->stream>>>((const T*)h->grad_c[1], tx, ty, tz, a, P);
        CHG_CUDA(h, cudaGetLastError());
        line(std::integral_constant<int, 1>{}, (const T*)h->vel_c[1], (T*)h->vel[1], a.nz);
        CHG_CUDA(h, cudaGetLastError());
        if (ev) CHG_CUDA(h, cudaEventRecord(ev[3], h->stream));
    }
    {
        mr_plane_yz<T, 2><<<16 * 152, 256, zsm, h->stream>>>((const T*)h->grad_c[2], tx, ty, tz, a, P);
        CHG_CUDA(h, cudaGetLastError());
        line(std::integral_constant<int, 2>{}, (const T*)h->vel_c[2], (T*)h->vel[2], a.ny);
        CHG_CUDA(h, cudaGetLastError());
        if (ev) CHG_CUDA(h, cudaEventRecord(ev[4], h->stream));
    }
    return CH_OK;
}

}  // namespace

namespace chg {

void mr_destroy(ch_handle* h) {
    cudaFree(h->mr_coords);
    cudaFree(h->rs_coords);
    for (int d = 0; d < 3; ++d) {
        cudaFree(h->mr_start[d]);
        cudaFree(h->mr_w[d]);
        cudaFree(h->rs_start[d]);
        cudaFree(h->rs_w[d]);
    }
}

// Hermite tables of nq query points against the nodes at the centres of the
// nc cells bounded by faces (device arrays); weights as doubles [nq][4] then
// floats [nq][4] in w.
int mr_tables_launch(ch_handle* h, const double* faces, int nc, int periodic, int nq, const double* queries,
                     int32_t* start, double* w) {
    mr_tables_kernel<<<(unsigned)((nq + kThreads - 1) / kThreads), kThreads, 0, h->stream>>>(
        faces, nc, periodic, nq, h->p.h, queries, start, w, (float*)(w + 4 * (int64_t)nq));
    CHG_CUDA(h, cudaGetLastError());
    return CH_OK;
}

// Called from ch_create with the caller's host face coordinates.
int mr_build_tables(ch_handle* h, const double* xf, const double* yf, const double* zf) {
    const int64_t ncoord = h->nc[0] + h->nc[1] + h->nc[2] + 3;
    std::vector<double> all;
    all.reserve(ncoord);
    all.insert(all.end(), xf, xf + h->nc[0] + 1);
    all.insert(all.end(), yf, yf + h->nc[1] + 1);
    all.insert(all.end(), zf, zf + h->nc[2] + 1);
    if (cudaMalloc(&h->mr_coords, ncoord * sizeof(double)) != cudaSuccess) return CH_ENOMEM;
    CHG_CUDA(h, cudaMemcpy(h->mr_coords, all.data(), ncoord * sizeof(double), cudaMemcpyHostToDevice));
    const double* dev_faces[3] = {h->mr_coords, h->mr_coords + h->nc[0] + 1,
                                  h->mr_coords + h->nc[0] + h->nc[1] + 2};
    for (int d = 0; d < 3; ++d) {
        const int64_t n = h->n[d];
        if (cudaMalloc(&h->mr_start[d], n * sizeof(int32_t)) != cudaSuccess) return CH_ENOMEM;
        // doubles [n][4] followed by floats [n][4]
        if (cudaMalloc(&h->mr_w[d], n * 4 * sizeof(double) + n * 4 * sizeof(float)) != cudaSuccess) return CH_ENOMEM;
        mr_tables_kernel<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, h->stream>>>(
            dev_faces[d], (int)h->nc[d], h->p.bc[d] == CH_PERIODIC, (int)n, h->p.h, nullptr, h->mr_start[d], h->mr_w[d],
            (float*)(h->mr_w[d] + 4 * n));
        CHG_CUDA(h, cudaGetLastError());
    }
    CHG_CUDA(h, cudaStreamSynchronize(h->stream));
    return CH_OK;
}

}  // namespace chg

extern "C" {

int ch_set_velocity_coarse(ch_handle* h, const void* uc, const void* vc, const void* wc) {
    if (!h) return CH_EINVAL;
    if (!h->nc[0]) return fail(h, CH_EINVAL, "ch_set_velocity_coarse: no coarse mesh at create");
    if (!uc || !vc || !wc) return fail(h, CH_EINVAL, "ch_set_velocity_coarse: NULL pointer");
    const void* src[3] = {uc, vc, wc};
    for (int d = 0; d < 3; ++d) {
        int64_t cnt = h->ncf[d];
        for (int e = 0; e < 3; ++e)
            if (e != d) cnt *= h->nc[e];
        CHG_CUDA(h, cudaMemcpyAsync(h->vel_c[d], src[d], (size_t)cnt * h->esz, cudaMemcpyDeviceToDevice, h->stream));
    }
    return CH_OK;
}

int ch_interp_to_fine(ch_handle* h) {
    if (!h) return CH_EINVAL;
    if (!h->nc[0]) return fail(h, CH_EINVAL, "ch_interp_to_fine: no coarse mesh at create");
    return h->prec == CH_F64 ? interp<double>(h) : interp<float>(h);
}

int ch_profile_interp(ch_handle* h, double* ms_out) {
    if (!h) return CH_EINVAL;
    if (!h->nc[0]) return fail(h, CH_EINVAL, "ch_profile_interp: no coarse mesh at create");
    if (!ms_out) return fail(h, CH_EINVAL, "ch_profile_interp: NULL output");
    cudaEvent_t ev[5] = {};
    int rc = CH_OK;
    for (int i = 0; i < 5 && rc == CH_OK; ++i)
        if (cudaEventCreate(&ev[i]) != cudaSuccess) rc = fail(h, CH_ECUDA, "ch_profile_interp: cudaEventCreate failed");
    if (rc == CH_OK) rc = h->prec == CH_F64 ? interp<double>(h, ev) : interp<float>(h, ev);
    if (rc == CH_OK && cudaEventSynchronize(ev[4]) != cudaSuccess)
        rc = fail(h, CH_ECUDA, "ch_profile_interp: event wait failed");
    for (int i = 0; i < 4 && rc == CH_OK; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev[i], ev[i + 1]) != cudaSuccess)
            rc = fail(h, CH_ECUDA, "ch_profile_interp: cudaEventElapsedTime failed");
        ms_out[i] = ms;
    }
    for (int i = 0; i < 5; ++i)
        if (ev[i]) cudaEventDestroy(ev[i]);
    return rc;
}

int ch_get_interp_tables(ch_handle* h, int dir, int32_t* start, double* weights) {
    if (!h) return CH_EINVAL;
    if (!h->nc[0]) return fail(h, CH_EINVAL, "ch_get_interp_tables: no coarse mesh at create");
    if (dir < 0 || dir > 2 || !start || !weights) return fail(h, CH_EINVAL, "ch_get_interp_tables: bad argument");
    const int64_t n = h->n[dir];
    CHG_CUDA(h, cudaMemcpyAsync(start, h->mr_start[dir], n * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    CHG_CUDA(h, cudaMemcpyAsync(weights, h->mr_w[dir], n * 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CHG_CUDA(h, cudaStreamSynchronize(h->stream));
    return CH_OK;
}

}  // extern "C"
