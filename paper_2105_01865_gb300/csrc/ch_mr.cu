// Multiple-resolution velocity transfer (arXiv 2105.01865, Sec. 3.4): the
// face velocity of a stretched coarse mesh is carried to the uniform fine
// mesh of C through its face-normal gradients, a tri-cubic Hermite spline of
// four points per direction (64-point stencil, tables built once), and an
// integration along every fine line from a reference plane.
#include <cuda_runtime.h>

#include <algorithm>
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

template <typename T>
__device__ __forceinline__ void load_w(const T* __restrict__ w, int i, T* out) {
#pragma unroll
    for (int m = 0; m < 4; ++m) out[m] = w[4 * i + m];
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

// Step (3) along x: one warp per fine x-line (j, k).  The 64-point stencil
// is sum-factorised: the warp first contracts the 16 coarse rows of its (y, z)
// stencil into one coarse x-line g(ix) = sum_{b,c} wy_b wz_c G(ix, sy+b, sz+c)
// (coalesced over ix, kept in shared memory), then every fine point needs only
// its 4-point x-stencil of g.  u(face i) = u_ref(j, k) + h sum_{i' < i} Gx(i'),
// a warp scan per 32-point chunk plus a compensated carry (RunSum).
constexpr int kMrWarps = 8;

template <typename T>
__global__ void __launch_bounds__(kMrWarps * 32)
mr_integrate_x(const T* __restrict__ gx, const T* __restrict__ uc, Tab<T> tx, Tab<T> ty, Tab<T> tz, MrArgs a,
               T* __restrict__ u) {
    extern __shared__ __align__(16) unsigned char mr_smem[];  // kMrWarps coarse lines of ncx values
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int warp = blockIdx.x * kMrWarps + wib;
    if (warp >= a.ny * a.nz) return;  // whole warp
    const int j = warp % a.ny, k = warp / a.ny;
    T wy[4], wz[4];
    load_w(ty.w, j, wy);
    load_w(tz.w, k, wz);
    const int sy = ty.s[j], sz = tz.s[k];
    T* g = reinterpret_cast<T*>(mr_smem) + (int64_t)wib * a.ncx;
    for (int ix = lane; ix < a.ncx; ix += 32) {
        T acc = T(0);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            int kz = sz + c;
            kz -= (kz >= a.ncz) ? a.ncz : 0;
            T accy = T(0);
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                int ky = sy + b;
                ky -= (ky >= a.ncy) ? a.ncy : 0;
                accy += wy[b] * gx[((int64_t)kz * a.ncy + ky) * a.ncx + ix];
            }
            acc += wz[c] * accy;
        }
        g[ix] = acc;
    }
    T uref = T(0);
    if (!a.wall[0]) uref = hermite2(uc, (int64_t)a.ncy * a.ncfx, (int64_t)a.ncfx, a.ncz, a.ncy, sz, wz, sy, wy);
    __syncwarp();
    T* row = u + ((int64_t)k * a.ny + j) * a.nfx;
    const T hT = (T)a.h;
    RunSum<T> carry;  // sum over the previous 32-point chunks
    for (int i0 = 0; i0 < a.nx; i0 += 32) {
        const int i = i0 + lane;
        T gv = T(0);
        if (i < a.nx) {
            T wx[4];
            load_w(tx.w, i, wx);
            const int sx = tx.s[i];
            T acc = T(0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int kx = sx + q;
                kx -= (kx >= a.ncx) ? a.ncx : 0;
                acc += wx[q] * g[kx];
            }
            gv = acc;
        }
        T incl = gv;  // inclusive scan of the chunk over lanes
        for (int o = 1; o < 32; o <<= 1) {
            const T t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        T excl = __shfl_up_sync(0xffffffffu, incl, 1);
        if (lane == 0) excl = T(0);
        if (i < a.nx) row[i] = uref + hT * carry.plus(excl);
        carry.add(__shfl_sync(0xffffffffu, incl, 31));
    }
    if (a.wall[0] && lane == 0) row[a.nx] = uref + hT * carry.value();
}

// Contraction of a coarse gradient over the 4 x 4 stencil of the two
// transverse directions at one coarse index along the marching direction:
// value(m) = sum_{p,q} wp_p wq_q G(m, sp + p, sq + q) with the index order
// given by the strides.
template <typename T>
__device__ __forceinline__ T contract16(const T* __restrict__ G, int64_t off_m, int sp, int np, int64_t stride_p,
                                        const T* wp, int sq, int nq, int64_t stride_q, const T* wq) {
    T acc = T(0);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        int kp = sp + p;
        kp -= (kp >= np) ? np : 0;
        T accq = T(0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int kq = sq + q;
            kq -= (kq >= nq) ? nq : 0;
            accq += wq[q] * G[off_m + kp * stride_p + kq * stride_q];
        }
        acc += wp[p] * accq;
    }
    return acc;
}

// Steps (2)-(3) along a strided direction (y: v, or z: w): one thread per
// fine transverse position, marching the fine line.  The transverse 16-point
// contraction of each coarse index along the line is computed once and kept
// in a 4-entry window that slides with the fine point's stencil, so a fine
// point costs 4 FMAs instead of 64 gathers.
template <typename T, int DIR>
__global__ void __launch_bounds__(256)
mr_integrate_yz(const T* __restrict__ G, const T* __restrict__ Vc, Tab<T> tx, Tab<T> ty, Tab<T> tz, MrArgs a,
                T* __restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int nlong = DIR == 1 ? a.ny : a.nz;                 // fine cells along the line
    const int ntr = DIR == 1 ? a.nz : a.ny;                   // second transverse fine size
    if (t >= (int64_t)a.nx * ntr) return;
    const int i = (int)(t % a.nx), o = (int)(t / a.nx);       // fine x and the other transverse index
    T wxv[4], wov[4];
    load_w(tx.w, i, wxv);
    const Tab<T>& to = DIR == 1 ? tz : ty;                    // table of the other transverse direction
    const Tab<T>& tl = DIR == 1 ? ty : tz;                    // table along the line
    load_w(to.w, o, wov);
    const int sx = tx.s[i], so = to.s[o];
    const int ncl = DIR == 1 ? a.ncy : a.ncz;                 // coarse cells along the line
    const int nco = DIR == 1 ? a.ncz : a.ncy;                 // coarse cells of the other transverse dir
    // strides of G[kz][ky][kx]
    const int64_t st_l = DIR == 1 ? (int64_t)a.ncx : (int64_t)a.ncx * a.ncy;
    const int64_t st_o = DIR == 1 ? (int64_t)a.ncx * a.ncy : (int64_t)a.ncx;
    // reference plane: v at y = 0 (plane [kz][0][kx] of Vc) or w at z = 0
    T ref = T(0);
    if (!a.wall[DIR]) {
        if (DIR == 1)
            ref = hermite2(Vc, (int64_t)a.ncfy * a.ncx, (int64_t)1, a.ncz, a.ncx, so, wov, sx, wxv);
        else
            ref = hermite2(Vc, (int64_t)a.ncx, (int64_t)1, a.ncy, a.ncx, so, wov, sx, wxv);
    }
    T win[4];
    int ws = -1;  // coarse start index of the window
    const T hT = (T)a.h;
    RunSum<T> run;
    for (int jl = 0; jl < nlong; ++jl) {
        const int sl = tl.s[jl];
        if (sl != ws) {
            int first = 0;
            if (ws >= 0 && sl == (ws + 1 == ncl ? 0 : ws + 1)) {
                win[0] = win[1];
                win[1] = win[2];
                win[2] = win[3];
                first = 3;
            }
            for (int m = first; m < 4; ++m) {
                int km = sl + m;
                km -= (km >= ncl) ? ncl : 0;
                win[m] = contract16(G, km * st_l, so, nco, st_o, wov, sx, a.ncx, (int64_t)1, wxv);
            }
            ws = sl;
        }
        T wl[4];
        load_w(tl.w, jl, wl);
        const T gval = wl[0] * win[0] + wl[1] * win[1] + wl[2] * win[2] + wl[3] * win[3];
        const int64_t idx = DIR == 1 ? ((int64_t)o * a.nfy + jl) * a.nx + i : ((int64_t)jl * a.ny + o) * a.nx + i;
        out[idx] = ref + hT * run.value();
        run.add(gval);
    }
    if (a.wall[DIR]) {
        const int64_t idx = DIR == 1 ? ((int64_t)o * a.nfy + a.ny) * a.nx + i : ((int64_t)a.nz * a.ny + o) * a.nx + i;
        out[idx] = ref + hT * run.value();
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
        const size_t smem = (size_t)kMrWarps * a.ncx * sizeof(T);
        static bool attr_set = false;  // one instantiation per T
        if (!attr_set) {
            CHG_CUDA(h, cudaFuncSetAttribute(mr_integrate_x<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(kMrWarps * kMaxCoarseLine * sizeof(T))));
            attr_set = true;
        }
        mr_integrate_x<T><<<blocks, kMrWarps * 32, smem, h->stream>>>((const T*)h->grad_c[0], (const T*)h->vel_c[0], tx,
                                                                   ty, tz, a, (T*)h->vel[0]);
        CHG_CUDA(h, cudaGetLastError());
        if (ev) CHG_CUDA(h, cudaEventRecord(ev[2], h->stream));
    }
    {
        const int64_t thr = (int64_t)a.nx * a.nz;
        mr_integrate_yz<T, 1><<<(unsigned)((thr + 255) / 256), 256, 0, h->stream>>>(
            (const T*)h->grad_c[1], (const T*)h->vel_c[1], tx, ty, tz, a, (T*)h->vel[1]);
        CHG_CUDA(h, cudaGetLastError());
        if (ev) CHG_CUDA(h, cudaEventRecord(ev[3], h->stream));
    }
    {
        const int64_t thr = (int64_t)a.nx * a.ny;
        mr_integrate_yz<T, 2><<<(unsigned)((thr + 255) / 256), 256, 0, h->stream>>>(
            (const T*)h->grad_c[2], (const T*)h->vel_c[2], tx, ty, tz, a, (T*)h->vel[2]);
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
