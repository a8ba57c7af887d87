// Adjoint (reverse-mode derivative) of nsteps Cahn-Hilliard steps without
// advection, with checkpointed recomputation (arXiv 2105.01865, Sec. 3 step;
// the derivative itself has no counterpart in the paper).
//
// For substep l with C' = C + P^-1 r, r = dt(gamma H + rho Hp) - alpha dt M A C,
// H = M lap(psi'(C)), P = prod_d (I + c A_d), c = alpha dt M / 2, the reverse
// map of adjoints (lam_C', lam_H' of this H as the next substep's Hp) is
//   lam_r  = P^-1 lam_C'                       (the same line solves)
//   lam_H  = dt gamma lam_r + lam_H',  lam_Hp = dt rho lam_r
//   lam_C  = lam_C' - alpha dt M A lam_r + psi''(C) M lap(lam_H)
//   dL/dM += <lam_H, lap psi'(C)> - alpha dt <lam_r, A C>
//            - (alpha dt / 2) sum_d <A_d lam_r, (I + c A_d)^-1 r>
// (all operators symmetric; the P_d act on different axes and commute).
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "ch_internal.h"
#include "ch_kernels.cuh"

using namespace chg;

namespace {

constexpr int kAThreadsX = 32, kAThreadsY = 8;

template <typename T>
struct AdjArgs {
    int nx, ny, nz, bcx, bcy, bcz;
    double dt, gamma, rho, alpha, mob, kappa, inv_h2;
};

template <typename T>
__device__ __forceinline__ T at(const T* f, int i, int j, int k, const AdjArgs<T>& a) {
    return f[((int64_t)bc_index(k, a.nz, a.bcz) * a.ny + bc_index(j, a.ny, a.bcy)) * a.nx + bc_index(i, a.nx, a.bcx)];
}

template <typename T>
__device__ __forceinline__ T fourth(const T* f, int i, int j, int k, int d, const AdjArgs<T>& a) {
    const int di = d == 0, dj = d == 1, dk = d == 2;
    const T c = f[((int64_t)k * a.ny + j) * a.nx + i];
    const T m1 = at(f, i - di, j - dj, k - dk, a), p1 = at(f, i + di, j + dj, k + dk, a);
    const T m2 = at(f, i - 2 * di, j - 2 * dj, k - 2 * dk, a), p2 = at(f, i + 2 * di, j + 2 * dj, k + 2 * dk, a);
    const T da = m1 - c, db = p1 - c;
    return ((m2 - m1) - da) + ((p2 - p1) - db) - T(2) * (da + db);
}

template <typename T>
__device__ __forceinline__ T psi_prime_t(T c) { return c * (c * (c - T(1.5)) + T(0.5)); }

// One thread per cell: the reverse substep map above, in the field precision,
// with the dL/dM terms accumulated per block in FP64.
template <typename T>
__global__ void __launch_bounds__(kAThreadsX * kAThreadsY)
adj_substep(const T* C, const T* lam_r, const T* lamH_in, const T* lamC_in, const T* s0, const T* s1, const T* s2,
            T* lamC_out, T* lamHp_out, double* partials, AdjArgs<T> a) {
    const int i = blockIdx.x * kAThreadsX + threadIdx.x;
    const int j = blockIdx.y * kAThreadsY + threadIdx.y;
    const int k = blockIdx.z;
    double dm = 0.0;
    if (i < a.nx && j < a.ny) {
        const int64_t e = ((int64_t)k * a.ny + j) * a.nx + i;
        const T dtg = T(a.dt * a.gamma), mob = T(a.mob), inv_h2 = T(a.inv_h2), kap = T(a.kappa);
        auto lamH = [&](int ii, int jj, int kk) { return dtg * at(lam_r, ii, jj, kk, a) + at(lamH_in, ii, jj, kk, a); };
        auto psi_at = [&](int ii, int jj, int kk) { return psi_prime_t(at(C, ii, jj, kk, a)); };
        const T lh0 = lamH(i, j, k);
        const T lap_lh = ((lamH(i - 1, j, k) - lh0) + (lamH(i + 1, j, k) - lh0) + (lamH(i, j - 1, k) - lh0) +
                          (lamH(i, j + 1, k) - lh0) + (lamH(i, j, k - 1) - lh0) + (lamH(i, j, k + 1) - lh0)) *
                         inv_h2;
        const T p0 = psi_at(i, j, k);
        const T lap_psi = ((psi_at(i - 1, j, k) - p0) + (psi_at(i + 1, j, k) - p0) + (psi_at(i, j - 1, k) - p0) +
                           (psi_at(i, j + 1, k) - p0) + (psi_at(i, j, k - 1) - p0) + (psi_at(i, j, k + 1) - p0)) *
                          inv_h2;
        const T A_lr[3] = {kap * fourth(lam_r, i, j, k, 0, a), kap * fourth(lam_r, i, j, k, 1, a),
                           kap * fourth(lam_r, i, j, k, 2, a)};
        const T A_C = kap * (fourth(C, i, j, k, 0, a) + fourth(C, i, j, k, 1, a) + fourth(C, i, j, k, 2, a));
        const T c = C[e];
        const T ppp = (T(3) * c - T(3)) * c + T(0.5);
        const T adt = T(a.alpha * a.dt);
        lamC_out[e] = lamC_in[e] - adt * mob * ((A_lr[0] + A_lr[1]) + A_lr[2]) + ppp * mob * lap_lh;
        lamHp_out[e] = T(a.dt * a.rho) * lam_r[e];
        dm = (double)lh0 * (double)lap_psi - a.alpha * a.dt * (double)lam_r[e] * (double)A_C -
             0.5 * a.alpha * a.dt *
                 ((double)A_lr[0] * (double)s0[e] + (double)A_lr[1] * (double)s1[e] + (double)A_lr[2] * (double)s2[e]);
    }
    __shared__ double ws[kAThreadsX * kAThreadsY / 32];
    for (int o = 16; o > 0; o >>= 1) dm += __shfl_xor_sync(0xffffffffu, dm, o);
    const int tid = threadIdx.y * kAThreadsX + threadIdx.x;
    if ((tid & 31) == 0) ws[tid >> 5] = dm;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < kAThreadsX * kAThreadsY / 32; ++w) t += ws[w];
        partials[((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = t;
    }
}

__global__ void adj_accumulate(const double* partials, int64_t n, double* acc) {
    __shared__ double ws[8];
    double t = 0.0;
    for (int64_t b = threadIdx.x; b < n; b += blockDim.x) t += partials[b];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += ws[w];
        *acc += s;
    }
}

size_t a256(size_t x) { return (x + 255) / 256 * 256; }

struct AdjLayout {
    size_t field, nck, K, total;
};

AdjLayout adj_layout(const ch_handle* h, int64_t nsteps, int64_t K) {
    AdjLayout L;
    L.field = a256((size_t)h->ncell * h->esz);
    L.nck = (size_t)((nsteps + K - 1) / K);
    L.K = (size_t)std::min(K, nsteps);
    const size_t nblocks = (size_t)((h->n[0] + kAThreadsX - 1) / kAThreadsX) *
                           ((h->n[1] + kAThreadsY - 1) / kAThreadsY) * h->n[2];
    L.total = (L.nck + L.K + 15) * L.field + a256(nblocks * sizeof(double)) + 256;
    return L;
}

}  // namespace

extern "C" {

size_t ch_adjoint_workspace_bytes(const ch_handle* h, int64_t nsteps, int64_t ckpt_every) {
    if (!h || nsteps < 1 || ckpt_every < 1 || h->p.advect) return 0;
    return adj_layout(h, nsteps, ckpt_every).total;
}

int ch_step_adjoint(ch_handle* h, const void* C0, int64_t nsteps, int64_t ckpt_every, const void* lam_T, void* lam_0,
                    double* dL_dM, void* work, size_t work_bytes) {
    if (!h) return CH_EINVAL;
    if (h->p.advect) return fail(h, CH_EINVAL, "ch_step_adjoint: only u = 0 (advect = 0) is supported");
    if (h->p.scheme != CH_SCHEME_SPLIT) return fail(h, CH_EINVAL, "ch_step_adjoint: only the split scheme");
    if (h->n[2] < 5) return fail(h, CH_EINVAL, "ch_step_adjoint: needs nz >= 5");
    if (h->p.bc[2] == CH_DIRICHLET) return fail(h, CH_EINVAL, "ch_step_adjoint: Dirichlet walls are not supported");
    if (!C0 || !lam_T || !lam_0 || !dL_dM || !work || nsteps < 1 || ckpt_every < 1 || ((uintptr_t)work % 256))
        return fail(h, CH_EINVAL, "ch_step_adjoint: bad argument");
    const AdjLayout L = adj_layout(h, nsteps, ckpt_every);
    if (work_bytes < L.total) return fail(h, CH_ENOMEM, "ch_step_adjoint: workspace too small");
    const size_t fb = (size_t)h->ncell * h->esz;
    char* w = (char*)work;
    auto field = [&](size_t idx) { return (void*)(w + idx * L.field); };
    size_t q = 0;
    std::vector<void*> ckpt(L.nck), seg(L.K);
    for (auto& p : ckpt) p = field(q++);
    for (auto& p : seg) p = field(q++);
    void* X[3] = {field(q++), field(q++), field(q++)};
    void* Hs[2] = {field(q++), field(q++)};
    void* Htmp = field(q++);
    void* rtmp = field(q++);
    void* lamr = field(q++);
    void* sd[3] = {field(q++), field(q++), field(q++)};
    void* lamC = field(q++);
    void* lamH = field(q++);
    void* lamCn = field(q++);
    void* lamHn = field(q++);
    double* partials = (double*)field(q);
    double* acc = (double*)(w + L.total - 256);
    cudaStream_t st = h->stream;
    const ch_params& p = h->p;
    const int nx = (int)h->n[0], ny = (int)h->n[1], nz = (int)h->n[2];
    dim3 grid((nx + kAThreadsX - 1) / kAThreadsX, (ny + kAThreadsY - 1) / kAThreadsY, nz);
    dim3 block(kAThreadsX, kAThreadsY);
    const int64_t nblk = (int64_t)grid.x * grid.y * grid.z;
    auto cp = [&](void* dst, const void* src) {
        return cudaMemcpyAsync(dst, src, fb, cudaMemcpyDeviceToDevice, st);
    };
    int rc = CH_OK;
    CHG_CUDA(h, cudaMemsetAsync(acc, 0, sizeof(double), st));

    // forward pass: checkpoints every ckpt_every steps
    CHG_CUDA(h, cp(seg[0], C0));
    for (int64_t s = 0; s < nsteps && rc == CH_OK; ++s) {
        if (s % ckpt_every == 0) CHG_CUDA(h, cp(ckpt[s / ckpt_every], seg[0]));
        if (s + 1 < nsteps) rc = launch_step_any(h, seg[0]);
    }
    if (rc != CH_OK) return rc;

    CHG_CUDA(h, cp(lamC, lam_T));
    const double kappa = p.w * p.cn * p.cn / (p.h * p.h * p.h * p.h);
    for (int64_t m = (int64_t)L.nck - 1; m >= 0 && rc == CH_OK; --m) {
        const int64_t s0 = m * ckpt_every, s1 = std::min(s0 + ckpt_every, nsteps);
        // recompute the segment's step-start states
        CHG_CUDA(h, cp(seg[0], ckpt[m]));
        for (int64_t s = s0 + 1; s < s1 && rc == CH_OK; ++s) {
            CHG_CUDA(h, cp(seg[s - s0], seg[s - s0 - 1]));
            rc = launch_step_any(h, seg[s - s0]);
        }
        for (int64_t s = s1 - 1; s >= s0 && rc == CH_OK; --s) {
            // substep start states X[l] and the explicit terms H of substeps 0, 1
            CHG_CUDA(h, cp(X[0], seg[s - s0]));
            for (int l = 0; l < 2 && rc == CH_OK; ++l) {
                rc = launch_explicit_any(h, l, X[l], l ? Hs[l - 1] : nullptr, Hs[l], rtmp);
                CHG_CUDA(h, cp(X[l + 1], X[l]));
                for (int d = 0; d < 3 && rc == CH_OK; ++d) rc = launch_solve_any(h, l, d, rtmp, d == 2 ? X[l + 1] : nullptr);
            }
            CHG_CUDA(h, cudaMemsetAsync(lamH, 0, fb, st));
            for (int l = 2; l >= 0 && rc == CH_OK; --l) {
                rc = launch_explicit_any(h, l, X[l], l ? Hs[l - 1] : nullptr, Htmp, rtmp);
                CHG_CUDA(h, cp(lamr, lamC));
                for (int d = 0; d < 3 && rc == CH_OK; ++d) rc = launch_solve_any(h, l, d, lamr, nullptr);
                for (int d = 0; d < 3 && rc == CH_OK; ++d) {
                    CHG_CUDA(h, cp(sd[d], rtmp));
                    rc = launch_solve_any(h, l, d, sd[d], nullptr);
                }
                if (rc != CH_OK) break;
                if (h->prec == CH_F64) {
                    AdjArgs<double> a{nx, ny, nz, p.bc[0], p.bc[1], p.bc[2], p.dt, kGamma[l], kRho[l], kGamma[l] + kRho[l],
                                      1.0 / p.pe, kappa, 1.0 / (p.h * p.h)};
                    adj_substep<double><<<grid, block, 0, st>>>(
                        (const double*)X[l], (const double*)lamr, (const double*)lamH, (const double*)lamC,
                        (const double*)sd[0], (const double*)sd[1], (const double*)sd[2], (double*)lamCn,
                        (double*)lamHn, partials, a);
                } else {
                    AdjArgs<float> a{nx, ny, nz, p.bc[0], p.bc[1], p.bc[2], p.dt, kGamma[l], kRho[l], kGamma[l] + kRho[l],
                                     1.0 / p.pe, kappa, 1.0 / (p.h * p.h)};
                    adj_substep<float><<<grid, block, 0, st>>>(
                        (const float*)X[l], (const float*)lamr, (const float*)lamH, (const float*)lamC,
                        (const float*)sd[0], (const float*)sd[1], (const float*)sd[2], (float*)lamCn, (float*)lamHn,
                        partials, a);
                }
                CHG_CUDA(h, cudaGetLastError());
                adj_accumulate<<<1, 256, 0, st>>>(partials, nblk, acc);
                CHG_CUDA(h, cudaGetLastError());
                std::swap(lamC, lamCn);
                std::swap(lamH, lamHn);
            }
        }
    }
    if (rc != CH_OK) return rc;
    CHG_CUDA(h, cp(lam_0, lamC));
    CHG_CUDA(h, cudaMemcpyAsync(dL_dM, acc, sizeof(double), cudaMemcpyDeviceToHost, st));
    CHG_CUDA(h, cudaStreamSynchronize(st));
    return CH_OK;
}

}  // extern "C"
