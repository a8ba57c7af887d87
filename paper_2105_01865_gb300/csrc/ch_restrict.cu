// Down-sampling back-coupling of the multiple-resolution method (arXiv
// 2105.01865, Sec. 3.4, last step): the fine C is projected directly to the
// stretched coarse mesh, where it gives the density and viscosity (Sec. 2.2,
// Eqs. eq-rho, eq-mu) and the surface-tension force (Eq. eq-fst).
//
// The projection is the 4-point-per-direction Hermite stencil of the
// velocity transfer with nodes and queries swapped: nodes at the fine cell
// centres, queries at the coarse cell centres (tables built once per mesh
// pair).  It is applied to C and to the fine F_st = 6 sqrt(2) phi grad C / Cn,
// phi = psi'(C) - Cn^2 lap_h C, grad by central differences with the step's
// ghost cells.  The 64-point stencil is sum-factorised in three passes:
//   X: g1[f][k][j][ic] = sum_a wx_a F_f(sx + a, j, k)  (F computed on the fly)
//   Y: g2[f][k][jc][ic] = sum_b wy_b g1[f][k][sy + b][ic]
//   Z: out_f[kc][jc][ic] = sum_c wz_c g2[f][sz + c][jc][ic], then rho and mu.
// f runs over C, F_x, F_y, F_z.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "ch_internal.h"
#include "ch_kernels.cuh"

using namespace chg;

namespace {

constexpr int kRsThreads = 256;

template <typename T>
struct RsTab {
    const int32_t* __restrict__ s;
    const T* __restrict__ w;  // [n][4]
};

template <typename T>
RsTab<T> rs_tab(const ch_handle* h, int d) {
    const int64_t n = h->nc[d];
    RsTab<T> t;
    t.s = h->rs_start[d];
    t.w = (const T*)(sizeof(T) == 8 ? (const void*)h->rs_w[d] : (const void*)(h->rs_w[d] + 4 * n));
    return t;
}

struct RsDims {
    int nx, ny, nz;     // fine
    int ncx, ncy, ncz;  // coarse
    int bcx, bcy, bcz;
};

// neighbour index at +-1 with wrap or the mirror about a wall face
__device__ __forceinline__ int rs_lo(int i, int n, int bc) { return i > 0 ? i - 1 : (bc == CH_PERIODIC ? n - 1 : 0); }
__device__ __forceinline__ int rs_hi(int i, int n, int bc) { return i + 1 < n ? i + 1 : (bc == CH_PERIODIC ? 0 : n - 1); }

// Pass X: one thread per (k, j, ic) of the fine (k, j) rows and coarse x index.
template <typename T>
__global__ void __launch_bounds__(kRsThreads)
rs_pass_x(const T* __restrict__ C, RsTab<T> tx, RsDims d, T cn2_h2, T kfst_2h, T* __restrict__ g1) {
    const int64_t nrow = (int64_t)d.nz * d.ny;
    const int64_t N = nrow * d.ncx;
    const int64_t t = (int64_t)blockIdx.x * kRsThreads + threadIdx.x;
    if (t >= N) return;
    const int ic = (int)(t % d.ncx);
    const int64_t row = t / d.ncx;
    const int j = (int)(row % d.ny), k = (int)(row / d.ny);
    const int64_t plane = (int64_t)d.nx * d.ny;
    const T* Crow = C + (int64_t)k * plane + (int64_t)j * d.nx;
    const T* Cym = C + (int64_t)k * plane + (int64_t)rs_lo(j, d.ny, d.bcy) * d.nx;
    const T* Cyp = C + (int64_t)k * plane + (int64_t)rs_hi(j, d.ny, d.bcy) * d.nx;
    const T* Czm = C + (int64_t)rs_lo(k, d.nz, d.bcz) * plane + (int64_t)j * d.nx;
    const T* Czp = C + (int64_t)rs_hi(k, d.nz, d.bcz) * plane + (int64_t)j * d.nx;
    const int sx = tx.s[ic];
    T acc[4] = {T(0), T(0), T(0), T(0)};
    // the stencil's fine cells inside the row and 16-byte aligned (a uniform
    // coarse mesh 4 times coarser than the fine one puts every stencil there):
    // the cell row and its y and z neighbour rows as 16-byte vectors, the same
    // arithmetic in the same order
    if constexpr (sizeof(T) == 4) {
        if ((sx & 3) == 0 && sx + 4 <= d.nx && (d.nx & 3) == 0) {
            const float4 c4 = *reinterpret_cast<const float4*>(Crow + sx);
            const float4 ym4 = *reinterpret_cast<const float4*>(Cym + sx);
            const float4 yp4 = *reinterpret_cast<const float4*>(Cyp + sx);
            const float4 zm4 = *reinterpret_cast<const float4*>(Czm + sx);
            const float4 zp4 = *reinterpret_cast<const float4*>(Czp + sx);
            const T cv[6] = {Crow[rs_lo(sx, d.nx, d.bcx)], c4.x, c4.y, c4.z, c4.w, Crow[rs_hi(sx + 3, d.nx, d.bcx)]};
            const T ymv[4] = {ym4.x, ym4.y, ym4.z, ym4.w}, ypv[4] = {yp4.x, yp4.y, yp4.z, yp4.w};
            const T zmv[4] = {zm4.x, zm4.y, zm4.z, zm4.w}, zpv[4] = {zp4.x, zp4.y, zp4.z, zp4.w};
            const float4 w4 = *reinterpret_cast<const float4*>(tx.w + 4 * ic);
            const T wv[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const T wa = wv[a];
                const T c = cv[a + 1];
                const T xm = cv[a], xp = cv[a + 2];
                const T ym = ymv[a], yp = ypv[a], zm = zmv[a], zp = zpv[a];
                const T lap = (((xm - c) + (xp - c)) + ((ym - c) + (yp - c))) + ((zm - c) + (zp - c));
                const T phi = c * (c * (c - T(1.5)) + T(0.5)) - cn2_h2 * lap;
                const T kphi = kfst_2h * phi;
                acc[0] += wa * c;
                acc[1] += wa * (kphi * (xp - xm));
                acc[2] += wa * (kphi * (yp - ym));
                acc[3] += wa * (kphi * (zp - zm));
            }
#pragma unroll
            for (int f = 0; f < 4; ++f) g1[(int64_t)f * N + t] = acc[f];
            return;
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        int i = sx + a;
        i -= (i >= d.nx) ? d.nx : 0;
        const T wa = tx.w[4 * ic + a];
        const T c = Crow[i];
        const T xm = Crow[rs_lo(i, d.nx, d.bcx)], xp = Crow[rs_hi(i, d.nx, d.bcx)];
        const T ym = Cym[i], yp = Cyp[i], zm = Czm[i], zp = Czp[i];
        const T lap = (((xm - c) + (xp - c)) + ((ym - c) + (yp - c))) + ((zm - c) + (zp - c));
        const T phi = c * (c * (c - T(1.5)) + T(0.5)) - cn2_h2 * lap;
        const T kphi = kfst_2h * phi;  // 6 sqrt(2) phi / (2 h Cn)
        acc[0] += wa * c;
        acc[1] += wa * (kphi * (xp - xm));
        acc[2] += wa * (kphi * (yp - ym));
        acc[3] += wa * (kphi * (zp - zm));
    }
#pragma unroll
    for (int f = 0; f < 4; ++f) g1[(int64_t)f * N + t] = acc[f];
}

// Pass Y: g2[f][k][jc][ic] from g1[f][k][j][ic].
template <typename T>
__global__ void __launch_bounds__(kRsThreads)
rs_pass_y(const T* __restrict__ g1, RsTab<T> ty, RsDims d, T* __restrict__ g2) {
    const int64_t N = (int64_t)d.nz * d.ncy * d.ncx, N1 = (int64_t)d.nz * d.ny * d.ncx;
    const int64_t t = (int64_t)blockIdx.x * kRsThreads + threadIdx.x;
    if (t >= N) return;
    const int ic = (int)(t % d.ncx);
    const int64_t r = t / d.ncx;
    const int jc = (int)(r % d.ncy), k = (int)(r / d.ncy);
    const int sy = ty.s[jc];
    T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        int j = sy + b;
        j -= (j >= d.ny) ? d.ny : 0;
        const T wb = ty.w[4 * jc + b];
        const int64_t src = ((int64_t)k * d.ny + j) * d.ncx + ic;
#pragma unroll
        for (int f = 0; f < 4; ++f) acc[f] += wb * g1[(int64_t)f * N1 + src];
    }
#pragma unroll
    for (int f = 0; f < 4; ++f) g2[(int64_t)f * N + t] = acc[f];
}

// Pass Z: the coarse fields, then rho and mu from the coarse C.
template <typename T>
__global__ void __launch_bounds__(kRsThreads)
rs_pass_z(const T* __restrict__ g2, RsTab<T> tz, RsDims d, T lam_rho, T lam_mu, T* __restrict__ Cc,
          T* __restrict__ rho, T* __restrict__ mu, T* __restrict__ Fx, T* __restrict__ Fy, T* __restrict__ Fz) {
    const int64_t N = (int64_t)d.ncz * d.ncy * d.ncx, N2 = (int64_t)d.nz * d.ncy * d.ncx;
    const int64_t t = (int64_t)blockIdx.x * kRsThreads + threadIdx.x;
    if (t >= N) return;
    const int64_t cyx = (int64_t)d.ncy * d.ncx;
    const int64_t inner = t % cyx;
    const int kc = (int)(t / cyx);
    const int sz = tz.s[kc];
    T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        int k = sz + c;
        k -= (k >= d.nz) ? d.nz : 0;
        const T wc = tz.w[4 * kc + c];
        const int64_t src = (int64_t)k * cyx + inner;
#pragma unroll
        for (int f = 0; f < 4; ++f) acc[f] += wc * g2[(int64_t)f * N2 + src];
    }
    Cc[t] = acc[0];
    rho[t] = acc[0] + lam_rho * (T(1) - acc[0]);
    mu[t] = acc[0] + lam_mu * (T(1) - acc[0]);
    Fx[t] = acc[1];
    Fy[t] = acc[2];
    Fz[t] = acc[3];
}

size_t rs_work_elems(const ch_handle* h) {
    const int64_t g1 = 4 * h->n[2] * h->n[1] * h->nc[0];
    const int64_t g2 = 4 * h->n[2] * h->nc[1] * h->nc[0];
    return (size_t)(g1 + g2);
}

template <typename T>
int restrict_run(ch_handle* h, double lam_rho, double lam_mu, void* const* out, void* work) {
    RsDims d;
    d.nx = (int)h->n[0];
    d.ny = (int)h->n[1];
    d.nz = (int)h->n[2];
    d.ncx = (int)h->nc[0];
    d.ncy = (int)h->nc[1];
    d.ncz = (int)h->nc[2];
    d.bcx = h->p.bc[0];
    d.bcy = h->p.bc[1];
    d.bcz = h->p.bc[2];
    const ch_params& p = h->p;
    T* g1 = (T*)work;
    T* g2 = g1 + 4 * (int64_t)d.nz * d.ny * d.ncx;
    const int64_t n1 = (int64_t)d.nz * d.ny * d.ncx, n2 = (int64_t)d.nz * d.ncy * d.ncx,
                  n3 = (int64_t)d.ncz * d.ncy * d.ncx;
    const T cn2_h2 = (T)(p.cn * p.cn / (p.h * p.h));
    const T kfst_2h = (T)(6.0 * std::sqrt(2.0) / (p.cn * 2.0 * p.h));
    rs_pass_x<T><<<(unsigned)((n1 + kRsThreads - 1) / kRsThreads), kRsThreads, 0, h->stream>>>(
        (const T*)h->C, rs_tab<T>(h, 0), d, cn2_h2, kfst_2h, g1);
    CHG_CUDA(h, cudaGetLastError());
    rs_pass_y<T><<<(unsigned)((n2 + kRsThreads - 1) / kRsThreads), kRsThreads, 0, h->stream>>>(g1, rs_tab<T>(h, 1),
                                                                                                  d, g2);
    CHG_CUDA(h, cudaGetLastError());
    rs_pass_z<T><<<(unsigned)((n3 + kRsThreads - 1) / kRsThreads), kRsThreads, 0, h->stream>>>(
        g2, rs_tab<T>(h, 2), d, (T)lam_rho, (T)lam_mu, (T*)out[0], (T*)out[1], (T*)out[2], (T*)out[3], (T*)out[4],
        (T*)out[5]);
    CHG_CUDA(h, cudaGetLastError());
    return CH_OK;
}

}  // namespace

namespace chg {

// Tables of the down-sampling: fine faces i h as nodes, coarse centres as
// queries, per direction.
int rs_build_tables(ch_handle* h, const double* xf, const double* yf, const double* zf) {
    const double* cf[3] = {xf, yf, zf};
    std::vector<double> all;
    for (int d = 0; d < 3; ++d)
        for (int64_t i = 0; i <= h->n[d]; ++i) all.push_back((double)i * h->p.h);
    for (int d = 0; d < 3; ++d)
        for (int64_t k = 0; k < h->nc[d]; ++k) all.push_back(0.5 * (cf[d][k] + cf[d][k + 1]));
    if (cudaMalloc(&h->rs_coords, all.size() * sizeof(double)) != cudaSuccess) return CH_ENOMEM;
    CHG_CUDA(h, cudaMemcpy(h->rs_coords, all.data(), all.size() * sizeof(double), cudaMemcpyHostToDevice));
    int64_t off_f = 0, off_c = h->n[0] + h->n[1] + h->n[2] + 3;
    for (int d = 0; d < 3; ++d) {
        const int64_t nq = h->nc[d];
        if (cudaMalloc(&h->rs_start[d], nq * sizeof(int32_t)) != cudaSuccess) return CH_ENOMEM;
        if (cudaMalloc(&h->rs_w[d], nq * 4 * sizeof(double) + nq * 4 * sizeof(float)) != cudaSuccess)
            return CH_ENOMEM;
        const int rc = mr_tables_launch(h, h->rs_coords + off_f, (int)h->n[d], h->p.bc[d] == CH_PERIODIC, (int)nq,
                                        h->rs_coords + off_c, h->rs_start[d], h->rs_w[d]);
        if (rc != CH_OK) return rc;
        off_f += h->n[d] + 1;
        off_c += nq;
    }
    CHG_CUDA(h, cudaStreamSynchronize(h->stream));
    return CH_OK;
}

}  // namespace chg

extern "C" {

size_t ch_restrict_workspace_bytes(const ch_handle* h) {
    if (!h || !h->nc[0]) return 0;
    return rs_work_elems(h) * h->esz;
}

int ch_restrict_to_coarse(ch_handle* h, double lambda_rho, double lambda_mu, void* C_c, void* rho_c, void* mu_c,
                          void* fx_c, void* fy_c, void* fz_c, void* work, size_t work_bytes) {
    if (!h) return CH_EINVAL;
    if (!h->nc[0]) return fail(h, CH_EINVAL, "ch_restrict_to_coarse: the handle has no coarse mesh");
    if (h->p.bc[2] == CH_DIRICHLET)
        return fail(h, CH_EINVAL, "ch_restrict_to_coarse: Dirichlet walls are not supported");
    void* out[6] = {C_c, rho_c, mu_c, fx_c, fy_c, fz_c};
    for (void* o : out)
        if (!o || ((uintptr_t)o % h->esz)) return fail(h, CH_EINVAL, "ch_restrict_to_coarse: bad output pointer");
    if (!work || ((uintptr_t)work % 256)) return fail(h, CH_EINVAL, "ch_restrict_to_coarse: bad workspace pointer");
    if (work_bytes < rs_work_elems(h) * h->esz) return fail(h, CH_ENOMEM, "ch_restrict_to_coarse: workspace too small");
    if (!std::isfinite(lambda_rho) || !std::isfinite(lambda_mu))
        return fail(h, CH_EINVAL, "ch_restrict_to_coarse: non-finite property ratio");
    return h->prec == CH_F64 ? restrict_run<double>(h, lambda_rho, lambda_mu, out, work)
                             : restrict_run<float>(h, lambda_rho, lambda_mu, out, work);
}

}  // extern "C"
