// The standard explicit scheme the paper's split operator replaces
// (arXiv 2105.01865, Sec. 3.1, Eq. eq-disbi; compared in Sec. 4.1).
//
// Every term of Eq. (eq-ch) is explicit in the same low-storage RK3:
//   H^l = -div(uC) + M lap_h(psi'(C) - Cn^2 lap_h C),
//   C  <- C + dt (gamma_l H^l + rho_l H^{l-1}).
// M lap_h(psi' - Cn^2 lap_h C) equals M lap_h psi'(C) - M Cn^2 lap_h^2 C, the
// 25-point biharmonic of Eq. (eq-disbi) (13 points in 2D), so the substep is
// three launches: the chemical potential mu = psi'(C) - Cn^2 lap_h C
// (ch_std_mu), the WENO5 advection of the split scheme's explicit kernel run
// with its diffusive and implicit terms switched off, and the update
// (ch_std_update).  Ghost cells follow the split scheme: periodic wrap or the
// mirror about a wall face, so both Laplacians are conservative.
#include <cuda_runtime.h>

#include "ch_internal.h"
#include "ch_kernels.cuh"

using namespace chg;

namespace {

template <typename T>
struct StdArgs {
    int nx, ny, nz;
    int bcx, bcy, bcz;
    T cn2_h2;   // Cn^2 / h^2
    T mob_h2;   // M / h^2
    T dtg, dtr; // dt gamma_l, dt rho_l
    int has_prev;
};

// Neighbour index at +-1 along a line of n cells: wrap, or the mirror about
// the wall face (ghost C_{-1} = C_0, C_n = C_{n-1}).
__device__ __forceinline__ int nb_lo(int i, int n, int bc) { return i > 0 ? i - 1 : (bc == CH_PERIODIC ? n - 1 : 0); }
__device__ __forceinline__ int nb_hi(int i, int n, int bc) { return i + 1 < n ? i + 1 : (bc == CH_PERIODIC ? 0 : n - 1); }

// Sum of the six neighbour differences of f at (i, j, k) (lap_h times h^2),
// differences formed first as in the split scheme's Laplacian.
template <typename T>
__device__ __forceinline__ T lap_sum(const T* f, int i, int j, int k, const StdArgs<T>& a, T c) {
    const int64_t row = (int64_t)a.nx, plane = (int64_t)a.nx * a.ny;
    const int64_t base = (int64_t)k * plane + (int64_t)j * row;
    const T xm = f[base + nb_lo(i, a.nx, a.bcx)], xp = f[base + nb_hi(i, a.nx, a.bcx)];
    const T ym = f[(int64_t)k * plane + (int64_t)nb_lo(j, a.ny, a.bcy) * row + i];
    const T yp = f[(int64_t)k * plane + (int64_t)nb_hi(j, a.ny, a.bcy) * row + i];
    const T zm = f[(int64_t)nb_lo(k, a.nz, a.bcz) * plane + (int64_t)j * row + i];
    const T zp = f[(int64_t)nb_hi(k, a.nz, a.bcz) * plane + (int64_t)j * row + i];
    return (((xm - c) + (xp - c)) + ((ym - c) + (yp - c))) + ((zm - c) + (zp - c));
}

// mu = psi'(C) - Cn^2 lap_h C, psi'(C) = C (C (C - 1.5) + 0.5)
template <typename T>
__global__ void __launch_bounds__(256) ch_std_mu(const T* __restrict__ C, T* __restrict__ mu, StdArgs<T> a) {
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
    if (i >= a.nx || j >= a.ny) return;
    const int64_t idx = ((int64_t)k * a.ny + j) * a.nx + i;
    const T c = C[idx];
    const T psi_p = c * (c * (c - T(1.5)) + T(0.5));
    mu[idx] = psi_p - a.cn2_h2 * lap_sum(C, i, j, k, a, c);
}

// H = [-div(uC)] + M lap_h mu; C += dt (gamma H + rho H^{l-1}).  Hadv may be
// the same array as Hout (each thread reads its cell before writing it).
template <typename T, bool ADV>
__global__ void __launch_bounds__(256) ch_std_update(const T* __restrict__ mu, const T* Hadv, const T* __restrict__ Hprev,
                                                     T* Hout, T* __restrict__ C, StdArgs<T> a, unsigned int* status) {
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
    if (i >= a.nx || j >= a.ny) return;
    const int64_t idx = ((int64_t)k * a.ny + j) * a.nx + i;
    T H = a.mob_h2 * lap_sum(mu, i, j, k, a, mu[idx]);
    if (ADV) H += Hadv[idx];
    T rhs = a.dtg * H;
    if (a.has_prev) rhs += a.dtr * Hprev[idx];
    Hout[idx] = H;
    const T cnew = C[idx] + rhs;
    C[idx] = cnew;
    if (!isfinite(cnew)) atomicOr(status, 1u);
}

template <typename T>
int substep_standard(ch_handle* h, int l, cudaEvent_t* ev) {
    const ch_params& p = h->p;
    StdArgs<T> a;
    a.nx = (int)h->n[0];
    a.ny = (int)h->n[1];
    a.nz = (int)h->n[2];
    a.bcx = p.bc[0];
    a.bcy = p.bc[1];
    a.bcz = p.bc[2];
    a.cn2_h2 = (T)(p.cn * p.cn / (p.h * p.h));
    a.mob_h2 = (T)(1.0 / (p.pe * p.h * p.h));
    a.dtg = (T)(p.dt * kGamma[l]);
    a.dtr = (T)(p.dt * kRho[l]);
    a.has_prev = kRho[l] != 0.0;
    T* C = (T*)h->C;
    T* mu = (T*)h->r;  // the split scheme's right-hand side buffer holds mu
    T* Hcur = (T*)h->H[l & 1];
    const T* Hprev = (const T*)h->H[(l + 1) & 1];
    const dim3 block(32, 8), grid((unsigned)((a.nx + 31) / 32), (unsigned)((a.ny + 7) / 8), (unsigned)a.nz);
    if (ev) CHG_CUDA(h, cudaEventRecord(ev[0], h->stream));
    ch_std_mu<T><<<grid, block, 0, h->stream>>>(C, mu, a);
    CHG_CUDA(h, cudaGetLastError());
    if (ev) CHG_CUDA(h, cudaEventRecord(ev[1], h->stream));
    if (p.advect) {
        const int rc = launch_advection_any(h, C, Hcur);
        if (rc != CH_OK) return rc;
    }
    if (ev) CHG_CUDA(h, cudaEventRecord(ev[2], h->stream));
    if (p.advect)
        ch_std_update<T, true><<<grid, block, 0, h->stream>>>(mu, Hcur, Hprev, Hcur, C, a, h->status);
    else
        ch_std_update<T, false><<<grid, block, 0, h->stream>>>(mu, nullptr, Hprev, Hcur, C, a, h->status);
    CHG_CUDA(h, cudaGetLastError());
    if (ev) {
        CHG_CUDA(h, cudaEventRecord(ev[3], h->stream));
        CHG_CUDA(h, cudaEventRecord(ev[4], h->stream));
    }
    return CH_OK;
}

}  // namespace

namespace chg {

int launch_substep_standard(ch_handle* h, int l, cudaEvent_t* ev) {
    return h->prec == CH_F64 ? substep_standard<double>(h, l, ev) : substep_standard<float>(h, l, ev);
}

}  // namespace chg
