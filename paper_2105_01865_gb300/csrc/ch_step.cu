// C ABI of the Cahn-Hilliard fine-grid step: handle creation, the host-side
// FP64 factorisation of the line operators, kernel launches and the CUDA
// graph of one full RK3 step (arXiv 2105.01865, Sec. 3 and Eqs. eq-re ..
// eq-fac-3).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <tuple>
#include <vector>

#include "ch_internal.h"
#include "ch_kernels.cuh"

using namespace chg;

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

bool params_valid(const ch_params* p, char* why, size_t wl) {
    auto bad = [&](const char* m) {
        snprintf(why, wl, "%s", m);
        return false;
    };
    if (!p) return bad("params is NULL");
    if (p->nx < 5 || p->ny < 5 || p->nz < 5) return bad("nx, ny, nz must each be >= 5");
    if (p->nx > (1 << 20) || p->ny > (1 << 20) || p->nz > (1 << 20)) return bad("a dimension exceeds 2^20");
    if ((double)p->nx * p->ny * p->nz > 9.0e18 / 8) return bad("grid too large");
    if (!(p->h > 0) || !(p->cn > 0) || !(p->pe > 0) || !(p->dt > 0) || !(p->w > 0) || !(p->weno_eps > 0))
        return bad("h, cn, pe, dt, w, weno_eps must be positive and finite");
    if (!std::isfinite(p->h) || !std::isfinite(p->cn) || !std::isfinite(p->pe) || !std::isfinite(p->dt) ||
        !std::isfinite(p->w) || !std::isfinite(p->weno_eps))
        return bad("non-finite parameter");
    for (int d = 0; d < 3; ++d)
        if (p->bc[d] != CH_PERIODIC && p->bc[d] != CH_NOFLUX) return bad("bc must be CH_PERIODIC or CH_NOFLUX");
    if (p->precision != CH_F32 && p->precision != CH_F64) return bad("precision must be CH_F32 or CH_F64");
    if (p->advect != 0 && p->advect != 1) return bad("advect must be 0 or 1");
    if (p->reserved != 0) return bad("reserved must be 0");
    const bool any_c = p->ncx || p->ncy || p->ncz || p->xf_coarse || p->yf_coarse || p->zf_coarse;
    if (any_c) {
        if (p->ncx < 4 || p->ncy < 4 || p->ncz < 4) return bad("coarse mesh needs >= 4 cells per direction");
        if (!p->xf_coarse || !p->yf_coarse || !p->zf_coarse) return bad("coarse face coordinates missing");
        if (!p->advect) return bad("a coarse mesh requires advect = 1");
        const int64_t nf[3] = {p->nx, p->ny, p->nz};
        const int64_t nc[3] = {p->ncx, p->ncy, p->ncz};
        const double* f[3] = {p->xf_coarse, p->yf_coarse, p->zf_coarse};
        for (int d = 0; d < 3; ++d) {
            const double L = nf[d] * p->h;
            if (f[d][0] != 0.0) return bad("coarse face coordinates must start at 0");
            if (std::fabs(f[d][nc[d]] - L) > 1e-12 * L) return bad("coarse faces must end at n*h of the fine mesh");
            for (int64_t k = 0; k < nc[d]; ++k)
                if (!(f[d][k + 1] > f[d][k])) return bad("coarse face coordinates must increase");
        }
    }
    // line-solve tiles must fit in shared memory (8 lines of the longest direction)
    const size_t esz = p->precision == CH_F64 ? 8 : 4;
    const int64_t nmax = std::max(p->nx + 1, std::max(p->ny, p->nz));
    if ((size_t)nmax * 8 * esz > 200 * 1024) return bad("a line is too long for the shared-memory line solve");
    return true;
}

struct Layout {
    size_t H0, H1, r, vel[3], velc[3], gradc[3], total;
};

Layout layout(const ch_params* p) {
    Layout L{};
    const size_t esz = p->precision == CH_F64 ? 8 : 4;
    const size_t N = (size_t)p->nx * p->ny * p->nz;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align_up(bytes);
        return o;
    };
    L.H0 = take(N * esz);
    L.H1 = take(N * esz);
    L.r = take(N * esz);
    const int64_t n[3] = {p->nx, p->ny, p->nz};
    int64_t nf[3];
    for (int d = 0; d < 3; ++d) nf[d] = n[d] + (p->bc[d] == CH_NOFLUX ? 1 : 0);
    if (p->advect) {
        L.vel[0] = take((size_t)n[2] * n[1] * nf[0] * esz);
        L.vel[1] = take((size_t)n[2] * nf[1] * n[0] * esz);
        L.vel[2] = take((size_t)nf[2] * n[1] * n[0] * esz);
    }
    if (p->ncx) {
        const int64_t nc[3] = {p->ncx, p->ncy, p->ncz};
        int64_t ncf[3];
        for (int d = 0; d < 3; ++d) ncf[d] = nc[d] + (p->bc[d] == CH_NOFLUX ? 1 : 0);
        L.velc[0] = take((size_t)nc[2] * nc[1] * ncf[0] * esz);
        L.velc[1] = take((size_t)nc[2] * ncf[1] * nc[0] * esz);
        L.velc[2] = take((size_t)ncf[2] * nc[1] * nc[0] * esz);
        for (int d = 0; d < 3; ++d) L.gradc[d] = take((size_t)nc[0] * nc[1] * nc[2] * esz);
    }
    L.total = off;
    return L;
}

// Banded LU without pivoting of a pentadiagonal matrix given by its bands
// e (j, j-2), c (j, j-1), d (j, j), a (j, j+1), b (j, j+2).
struct BandLU {
    std::vector<double> l1, l2, u0, u1, u2;
};

BandLU band_lu(const std::vector<double>& e, const std::vector<double>& c, const std::vector<double>& d,
               const std::vector<double>& a, const std::vector<double>& b) {
    const int n = (int)d.size();
    BandLU f;
    f.l1.assign(n, 0.0);
    f.l2.assign(n, 0.0);
    f.u0.assign(n, 0.0);
    f.u1.assign(n, 0.0);
    f.u2.assign(n, 0.0);
    for (int j = 0; j < n; ++j) {
        if (j >= 2) f.l2[j] = e[j] / f.u0[j - 2];
        if (j >= 1) f.l1[j] = (c[j] - (j >= 2 ? f.l2[j] * f.u1[j - 2] : 0.0)) / f.u0[j - 1];
        f.u0[j] = d[j] - (j >= 1 ? f.l1[j] * f.u1[j - 1] : 0.0) - (j >= 2 ? f.l2[j] * f.u2[j - 2] : 0.0);
        f.u1[j] = (j + 1 < n ? a[j] : 0.0) - (j >= 1 ? f.l1[j] * f.u2[j - 1] : 0.0);
        f.u2[j] = (j + 2 < n) ? b[j] : 0.0;
    }
    return f;
}

std::vector<double> band_solve(const BandLU& f, std::vector<double> x) {
    const int n = (int)x.size();
    for (int j = 0; j < n; ++j)
        x[j] -= (j >= 1 ? f.l1[j] * x[j - 1] : 0.0) + (j >= 2 ? f.l2[j] * x[j - 2] : 0.0);
    for (int j = n - 1; j >= 0; --j) {
        double s = x[j];
        if (j + 1 < n) s -= f.u1[j] * x[j + 1];
        if (j + 2 < n) s -= f.u2[j] * x[j + 2];
        x[j] = s / f.u0[j];
    }
    return x;
}

bool invert4(const double* A, double* out) {
    double M[4][8];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 8; ++j) M[i][j] = j < 4 ? A[i * 4 + j] : (j - 4 == i ? 1.0 : 0.0);
    for (int col = 0; col < 4; ++col) {
        int piv = col;
        for (int i = col + 1; i < 4; ++i)
            if (std::fabs(M[i][col]) > std::fabs(M[piv][col])) piv = i;
        if (M[piv][col] == 0.0) return false;
        for (int j = 0; j < 8; ++j) std::swap(M[col][j], M[piv][j]);
        const double inv = 1.0 / M[col][col];
        for (int j = 0; j < 8; ++j) M[col][j] *= inv;
        for (int i = 0; i < 4; ++i) {
            if (i == col) continue;
            const double f = M[i][col];
            for (int j = 0; j < 8; ++j) M[i][j] -= f * M[col][j];
        }
    }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) out[i * 4 + j] = M[i][j + 4];
    return true;
}

// Host FP64 coefficients of (I + c kappa B) for one direction: B applies
// [1,-4,6,-4,1] with wrapped (periodic) or mirrored (wall) neighbours.
// Returns the arrays l1, l2, u1, u2, dinv (n each) and, when periodic,
// W (n x 4), Z (n x 4), S (4 x 4) of the Woodbury correction of the corners.
std::vector<double> line_coefficients(int n, int bc, double ck) {
    std::vector<double> e(n, 0.0), c(n, 0.0), d(n, 1.0), a(n, 0.0), b(n, 0.0);
    // corner (out-of-band) entries for the periodic case: (row, col, value)
    std::vector<std::tuple<int, int, double>> corner;
    const double stencil[5] = {1.0, -4.0, 6.0, -4.0, 1.0};
    for (int i = 0; i < n; ++i) {
        for (int s = -2; s <= 2; ++s) {
            int j = i + s;
            if (bc == CH_PERIODIC) {
                j = ((j % n) + n) % n;
            } else {
                if (j < 0) j = -1 - j;
                if (j >= n) j = 2 * n - 1 - j;
            }
            const double val = ck * stencil[s + 2];
            const int off = j - i;
            switch (off) {
                case -2: e[i] += val; break;
                case -1: c[i] += val; break;
                case 0: d[i] += val; break;
                case 1: a[i] += val; break;
                case 2: b[i] += val; break;
                default: corner.emplace_back(i, j, val);
            }
        }
    }
    const BandLU f = band_lu(e, c, d, a, b);
    std::vector<double> out;
    out.reserve(5 * n + 8 * n + 16);
    out.insert(out.end(), f.l1.begin(), f.l1.end());
    out.insert(out.end(), f.l2.begin(), f.l2.end());
    out.insert(out.end(), f.u1.begin(), f.u1.end());
    out.insert(out.end(), f.u2.begin(), f.u2.end());
    for (int j = 0; j < n; ++j) out.push_back(1.0 / f.u0[j]);
    if (bc != CH_PERIODIC) return out;
    // Woodbury: M = Mb + U V^T with U = [e_r] for the corner rows r in R,
    // V^T = the corner part of those rows.  M^-1 r = y - Z (I + V^T Z)^-1 V^T y,
    // y = Mb^-1 r, Z = Mb^-1 U; V^T y = W^T r with W = Mb^-T V.
    const int R[4] = {0, 1, n - 2, n - 1};
    std::vector<double> Vt(4 * (size_t)n, 0.0);
    for (auto& t : corner) {
        const int row = std::get<0>(t);
        int m = -1;
        for (int q = 0; q < 4; ++q)
            if (R[q] == row) m = q;
        Vt[(size_t)m * n + std::get<1>(t)] += std::get<2>(t);
    }
    // transpose band for Mb^-T
    std::vector<double> et(n, 0.0), ctt(n, 0.0), at(n, 0.0), bt(n, 0.0);
    for (int j = 0; j < n; ++j) {
        if (j >= 2) et[j] = b[j - 2];
        if (j >= 1) ctt[j] = a[j - 1];
        if (j + 1 < n) at[j] = c[j + 1];
        if (j + 2 < n) bt[j] = e[j + 2];
    }
    const BandLU ft = band_lu(et, ctt, d, at, bt);
    std::vector<double> W(4 * (size_t)n), Z(4 * (size_t)n);
    for (int m = 0; m < 4; ++m) {
        std::vector<double> vcol(Vt.begin() + (size_t)m * n, Vt.begin() + (size_t)(m + 1) * n);
        std::vector<double> wcol = band_solve(ft, vcol);
        std::vector<double> ucol(n, 0.0);
        ucol[R[m]] = 1.0;
        std::vector<double> zcol = band_solve(f, ucol);
        for (int j = 0; j < n; ++j) {
            W[(size_t)j * 4 + m] = wcol[j];
            Z[(size_t)j * 4 + m] = zcol[j];
        }
    }
    double cap[16], S[16];
    for (int p = 0; p < 4; ++p)
        for (int q = 0; q < 4; ++q) {
            double s = (p == q) ? 1.0 : 0.0;
            for (int j = 0; j < n; ++j) s += Vt[(size_t)p * n + j] * Z[(size_t)j * 4 + q];
            cap[p * 4 + q] = s;
        }
    if (!invert4(cap, S)) return {};
    out.insert(out.end(), W.begin(), W.end());
    out.insert(out.end(), Z.begin(), Z.end());
    out.insert(out.end(), S, S + 16);
    return out;
}

template <typename T>
Coef<T> coef_of(const LineCoefs& c) {
    Coef<T> k;
    k.l1 = (const T*)c.l1;
    k.l2 = (const T*)c.l2;
    k.u1 = (const T*)c.u1;
    k.u2 = (const T*)c.u2;
    k.dinv = (const T*)c.dinv;
    k.W = (const T*)c.W;
    k.Z = (const T*)c.Z;
    k.S = (const T*)c.S;
    k.n = c.n;
    k.periodic = c.periodic;
    return k;
}

int solve_x_lines(int nx, size_t esz) {
    // lines per CTA for the x solve: up to 32 rows of nx+1 values in <= 96 KB
    int lines = (int)std::min<size_t>(32, (96 * 1024) / ((size_t)(nx + 1) * esz));
    return std::max(lines, 1);
}

int solve_yz_lanes(int n, size_t esz) {
    int lanes = 32;
    while (lanes > 8 && (size_t)n * lanes * esz > 96 * 1024) lanes /= 2;
    return lanes;
}

template <typename T>
int launch_substep(ch_handle* h, int l, cudaEvent_t* ev = nullptr) {
    const ch_params& p = h->p;
    const int nx = (int)h->n[0], ny = (int)h->n[1], nz = (int)h->n[2];
    RhsArgs a;
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    a.bcx = p.bc[0];
    a.bcy = p.bc[1];
    a.bcz = p.bc[2];
    a.nfx = (int)h->nf[0];
    a.nfy = (int)h->nf[1];
    a.nfz = (int)h->nf[2];
    a.inv_h = 1.0 / p.h;
    a.inv_h2 = 1.0 / (p.h * p.h);
    a.mob = 1.0 / p.pe;
    const double alpha = kGamma[l] + kRho[l];
    const double kappa = p.w * p.cn * p.cn / (p.h * p.h * p.h * p.h);
    a.dtg = p.dt * kGamma[l];
    a.dtr = p.dt * kRho[l];
    a.impl = alpha * p.dt * a.mob * kappa;
    a.eps = p.weno_eps;
    a.has_prev = kRho[l] != 0.0;
    T* C = (T*)h->C;
    T* Hout = (T*)h->H[l & 1];
    const T* Hprev = (const T*)h->H[(l + 1) & 1];
    T* r = (T*)h->r;
    dim3 grid((nx + kTX - 1) / kTX, (ny + kTY - 1) / kTY, (nz + kTZ - 1) / kTZ);
    dim3 block(kTX, kTY);
    if (ev) CHG_CUDA(h, cudaEventRecord(ev[0], h->stream));
    if (p.advect)
        ch_explicit_rhs<T, true><<<grid, block, 0, h->stream>>>(C, (const T*)h->vel[0], (const T*)h->vel[1],
                                                                (const T*)h->vel[2], Hprev, Hout, r, a);
    else
        ch_explicit_rhs<T, false><<<grid, block, 0, h->stream>>>(C, nullptr, nullptr, nullptr, Hprev, Hout, r, a);
    CHG_CUDA(h, cudaGetLastError());
    if (ev) CHG_CUDA(h, cudaEventRecord(ev[1], h->stream));

    // x solve (Eq. eq-fac-1)
    {
        const int lines = solve_x_lines(nx, sizeof(T));
        const int64_t nlines = (int64_t)ny * nz;
        const size_t shm = (size_t)lines * (nx + 1) * sizeof(T);
        ch_solve_x<T><<<(unsigned)((nlines + lines - 1) / lines), kSolveThreads, shm, h->stream>>>(
            r, nlines, nx, lines, coef_of<T>(h->coefs[0][l]));
        CHG_CUDA(h, cudaGetLastError());
        if (ev) CHG_CUDA(h, cudaEventRecord(ev[2], h->stream));
    }
    // y solve (Eq. eq-fac-2)
    {
        const int lanes = solve_yz_lanes(ny, sizeof(T));
        const size_t shm = (size_t)ny * lanes * sizeof(T);
        const unsigned blocks = (unsigned)(((nx + lanes - 1) / lanes) * (int64_t)nz);
        ch_solve_yz<T, false><<<blocks, kSolveThreads, shm, h->stream>>>(
            r, nullptr, nx, (int64_t)nx * ny, nx, lanes, coef_of<T>(h->coefs[1][l]), h->status);
        CHG_CUDA(h, cudaGetLastError());
        if (ev) CHG_CUDA(h, cudaEventRecord(ev[3], h->stream));
    }
    // z solve + update (Eq. eq-fac-3)
    {
        const int lanes = solve_yz_lanes(nz, sizeof(T));
        const size_t shm = (size_t)nz * lanes * sizeof(T);
        const unsigned blocks = (unsigned)(((nx + lanes - 1) / lanes) * (int64_t)ny);
        ch_solve_yz<T, true><<<blocks, kSolveThreads, shm, h->stream>>>(
            r, C, nx, nx, (int64_t)nx * ny, lanes, coef_of<T>(h->coefs[2][l]), h->status);
        CHG_CUDA(h, cudaGetLastError());
        if (ev) CHG_CUDA(h, cudaEventRecord(ev[4], h->stream));
    }
    return CH_OK;
}

template <typename T>
int set_smem_attrs(ch_handle* h) {
    CHG_CUDA(h, cudaFuncSetAttribute(ch_solve_x<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    CHG_CUDA(h, cudaFuncSetAttribute(ch_solve_yz<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    CHG_CUDA(h, cudaFuncSetAttribute(ch_solve_yz<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    return CH_OK;
}

int launch_step(ch_handle* h) {
    for (int l = 0; l < kRK; ++l) {
        const int rc = h->prec == CH_F64 ? launch_substep<double>(h, l) : launch_substep<float>(h, l);
        if (rc != CH_OK) return rc;
    }
    return CH_OK;
}

template <typename T>
int reduce(ch_handle* h, bool energy, double* out) {
    const ch_params& p = h->p;
    if (energy)
        ch_reduce_energy<T><<<h->red_blocks, kRedThreads, 0, h->stream>>>(
            (const T*)h->C, (int)h->n[0], (int)h->n[1], (int)h->n[2], p.bc[0], p.bc[1], p.bc[2], 1.0 / p.h,
            0.5 * p.cn * p.cn, h->red_partials, h->status);
    else
        ch_reduce_mass<T><<<h->red_blocks, kRedThreads, 0, h->stream>>>((const T*)h->C, h->ncell, h->red_partials,
                                                                        h->status);
    CHG_CUDA(h, cudaGetLastError());
    ch_reduce_finish<<<1, kRedThreads, 0, h->stream>>>(h->red_partials, h->red_blocks, p.h * p.h * p.h, h->red_out);
    CHG_CUDA(h, cudaGetLastError());
    CHG_CUDA(h, cudaMemcpyAsync(out, h->red_out, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return ch_sync(h);
}

bool aligned(const void* p) { return ((uintptr_t)p % kAlign) == 0; }

}  // namespace

extern "C" {

size_t ch_workspace_bytes(const ch_params* p) {
    char why[256];
    if (!params_valid(p, why, sizeof(why))) return 0;
    return layout(p).total;
}

int ch_create(const ch_params* p, void* C, void* work, size_t work_bytes, void* stream, ch_handle** out) {
    char why[256];
    if (!out) return CH_EINVAL;
    *out = nullptr;
    if (!params_valid(p, why, sizeof(why))) return CH_EINVAL;
    if (!C || !work || !aligned(C) || !aligned(work)) return CH_EINVAL;
    const Layout L = layout(p);
    if (work_bytes < L.total) return CH_ENOMEM;

    ch_handle* h = (ch_handle*)calloc(1, sizeof(ch_handle));
    if (!h) return CH_ENOMEM;
    h->p = *p;
    h->p.xf_coarse = h->p.yf_coarse = h->p.zf_coarse = nullptr;  // host arrays are not kept
    h->prec = p->precision;
    h->esz = p->precision == CH_F64 ? 8 : 4;
    h->n[0] = p->nx;
    h->n[1] = p->ny;
    h->n[2] = p->nz;
    for (int d = 0; d < 3; ++d) h->nf[d] = h->n[d] + (p->bc[d] == CH_NOFLUX ? 1 : 0);
    h->ncell = p->nx * p->ny * p->nz;
    h->stream = (cudaStream_t)stream;
    h->C = C;
    char* wb = (char*)work;
    h->H[0] = wb + L.H0;
    h->H[1] = wb + L.H1;
    h->r = wb + L.r;
    if (p->advect)
        for (int d = 0; d < 3; ++d) h->vel[d] = wb + L.vel[d];
    const int64_t nc[3] = {p->ncx, p->ncy, p->ncz};
    if (p->ncx)
        for (int d = 0; d < 3; ++d) {
            h->vel_c[d] = wb + L.velc[d];
            h->grad_c[d] = wb + L.gradc[d];
            h->nc[d] = nc[d];
            h->ncf[d] = nc[d] + (p->bc[d] == CH_NOFLUX ? 1 : 0);
        }
    h->launches_per_step = 4 * kRK;

    int rc = CH_OK;
    // line-operator coefficients for every direction and substep
    {
        const double M = 1.0 / p->pe;
        const double kappa = p->w * p->cn * p->cn / (p->h * p->h * p->h * p->h);
        std::vector<std::vector<double>> all;
        size_t total = 0;
        for (int d = 0; d < 3; ++d)
            for (int l = 0; l < kRK; ++l) {
                const double ck = (kGamma[l] + kRho[l]) * p->dt * M / 2.0 * kappa;
                all.push_back(line_coefficients((int)h->n[d], p->bc[d], ck));
                if (all.back().empty()) {
                    free(h);
                    return CH_EINVAL;
                }
                total += align_up(all.back().size() * h->esz);
            }
        if (cudaMalloc(&h->coef_buf, total) != cudaSuccess) {
            free(h);
            return CH_ENOMEM;
        }
        std::vector<unsigned char> host(total, 0);
        size_t off = 0;
        for (int d = 0; d < 3; ++d)
            for (int l = 0; l < kRK; ++l) {
                const std::vector<double>& v = all[d * kRK + l];
                const int n = (int)h->n[d];
                unsigned char* dst = host.data() + off;
                for (size_t q = 0; q < v.size(); ++q) {
                    if (h->esz == 8)
                        ((double*)dst)[q] = v[q];
                    else
                        ((float*)dst)[q] = (float)v[q];
                }
                char* base = (char*)h->coef_buf + off;
                LineCoefs& c = h->coefs[d][l];
                c.n = n;
                c.periodic = p->bc[d] == CH_PERIODIC;
                c.l1 = base;
                c.l2 = base + (size_t)n * h->esz;
                c.u1 = base + (size_t)2 * n * h->esz;
                c.u2 = base + (size_t)3 * n * h->esz;
                c.dinv = base + (size_t)4 * n * h->esz;
                if (c.periodic) {
                    c.W = base + (size_t)5 * n * h->esz;
                    c.Z = base + (size_t)9 * n * h->esz;
                    c.S = base + (size_t)13 * n * h->esz;
                }
                off += align_up(v.size() * h->esz);
            }
        if (cudaMemcpy(h->coef_buf, host.data(), total, cudaMemcpyHostToDevice) != cudaSuccess) rc = CH_ECUDA;
    }
    if (rc == CH_OK) {
        h->red_blocks = 4 * 152;
        if (cudaMalloc(&h->red_partials, (size_t)h->red_blocks * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&h->red_out, sizeof(double)) != cudaSuccess ||
            cudaMalloc(&h->status, sizeof(unsigned int)) != cudaSuccess)
            rc = CH_ENOMEM;
        else if (cudaMemset(h->status, 0, sizeof(unsigned int)) != cudaSuccess)
            rc = CH_ECUDA;
    }
    if (rc == CH_OK) rc = h->prec == CH_F64 ? set_smem_attrs<double>(h) : set_smem_attrs<float>(h);
    if (rc == CH_OK && p->ncx) rc = mr_build_tables(h, p->xf_coarse, p->yf_coarse, p->zf_coarse);
    if (rc != CH_OK) {
        ch_free(h);
        return rc;
    }
    *out = h;
    return CH_OK;
}

int ch_free(ch_handle* h) {
    if (!h) return CH_EINVAL;
    if (h->graph_ready) cudaGraphExecDestroy(h->graph);
    mr_destroy(h);
    cudaFree(h->coef_buf);
    cudaFree(h->red_partials);
    cudaFree(h->red_out);
    cudaFree(h->status);
    free(h);
    return CH_OK;
}

int ch_set_velocity_fine(ch_handle* h, const void* u, const void* v, const void* w) {
    if (!h) return CH_EINVAL;
    if (!h->p.advect) return fail(h, CH_EINVAL, "ch_set_velocity_fine: created with advect = 0");
    if (!u || !v || !w) return fail(h, CH_EINVAL, "ch_set_velocity_fine: NULL pointer");
    const void* src[3] = {u, v, w};
    for (int d = 0; d < 3; ++d) {
        int64_t cnt = h->nf[d];
        for (int e = 0; e < 3; ++e)
            if (e != d) cnt *= h->n[e];
        CHG_CUDA(h, cudaMemcpyAsync(h->vel[d], src[d], (size_t)cnt * h->esz, cudaMemcpyDeviceToDevice, h->stream));
    }
    return CH_OK;
}

int ch_get_velocity_fine(ch_handle* h, void* u, void* v, void* w) {
    if (!h) return CH_EINVAL;
    if (!h->p.advect) return fail(h, CH_EINVAL, "ch_get_velocity_fine: created with advect = 0");
    if (!u || !v || !w) return fail(h, CH_EINVAL, "ch_get_velocity_fine: NULL pointer");
    void* dst[3] = {u, v, w};
    for (int d = 0; d < 3; ++d) {
        int64_t cnt = h->nf[d];
        for (int e = 0; e < 3; ++e)
            if (e != d) cnt *= h->n[e];
        CHG_CUDA(h, cudaMemcpyAsync(dst[d], h->vel[d], (size_t)cnt * h->esz, cudaMemcpyDeviceToDevice, h->stream));
    }
    return CH_OK;
}

int ch_step(ch_handle* h, int64_t nsteps) {
    if (!h) return CH_EINVAL;
    if (nsteps < 0) return fail(h, CH_EINVAL, "ch_step: nsteps < 0");
    if (nsteps == 0) return CH_OK;
    if (h->stream == nullptr) {  // the legacy stream cannot be captured: launch directly
        for (int64_t s = 0; s < nsteps; ++s) {
            const int rc = launch_step(h);
            if (rc != CH_OK) return rc;
        }
        return CH_OK;
    }
    if (!h->graph_ready) {
        cudaGraph_t g;
        CHG_CUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        const int rc = launch_step(h);
        cudaError_t e = cudaStreamEndCapture(h->stream, &g);
        if (rc != CH_OK) {
            if (e == cudaSuccess) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return fail(h, CH_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&h->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(h, CH_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
        h->graph_ready = 1;
    }
    for (int64_t s = 0; s < nsteps; ++s) CHG_CUDA(h, cudaGraphLaunch(h->graph, h->stream));
    return CH_OK;
}

int ch_mass(ch_handle* h, double* out) {
    if (!h || !out) return CH_EINVAL;
    return h->prec == CH_F64 ? reduce<double>(h, false, out) : reduce<float>(h, false, out);
}

int ch_free_energy(ch_handle* h, double* out) {
    if (!h || !out) return CH_EINVAL;
    return h->prec == CH_F64 ? reduce<double>(h, true, out) : reduce<float>(h, true, out);
}

int ch_sync(ch_handle* h) {
    if (!h) return CH_EINVAL;
    unsigned int flag = 0;
    CHG_CUDA(h, cudaMemcpyAsync(&flag, h->status, sizeof(flag), cudaMemcpyDeviceToHost, h->stream));
    CHG_CUDA(h, cudaStreamSynchronize(h->stream));
    if (flag) {
        CHG_CUDA(h, cudaMemsetAsync(h->status, 0, sizeof(unsigned int), h->stream));
        CHG_CUDA(h, cudaStreamSynchronize(h->stream));
        return fail(h, CH_ENONFINITE, "non-finite value in C");
    }
    return CH_OK;
}

int ch_launches_per_step(const ch_handle* h) { return h ? h->launches_per_step : 0; }

int ch_profile_step(ch_handle* h, int64_t nsteps, double* ms_out) {
    if (!h) return CH_EINVAL;
    if (nsteps < 1 || !ms_out) return fail(h, CH_EINVAL, "ch_profile_step: nsteps < 1 or NULL output");
    const int nev = 5;
    std::vector<cudaEvent_t> ev((size_t)nsteps * kRK * nev);
    for (auto& e : ev) CHG_CUDA(h, cudaEventCreate(&e));
    int rc = CH_OK;
    for (int64_t s = 0; s < nsteps && rc == CH_OK; ++s)
        for (int l = 0; l < kRK && rc == CH_OK; ++l) {
            cudaEvent_t* e = ev.data() + ((size_t)s * kRK + l) * nev;
            rc = h->prec == CH_F64 ? launch_substep<double>(h, l, e) : launch_substep<float>(h, l, e);
        }
    if (rc == CH_OK) {
        cudaError_t err = cudaStreamSynchronize(h->stream);
        if (err != cudaSuccess) rc = fail(h, CH_ECUDA, "ch_profile_step: %s", cudaGetErrorString(err));
    }
    if (rc == CH_OK) {
        double acc[4] = {0, 0, 0, 0};
        for (size_t b = 0; b < (size_t)nsteps * kRK; ++b)
            for (int k = 0; k < 4; ++k) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ev[b * nev + k], ev[b * nev + k + 1]);
                acc[k] += ms;
            }
        for (int k = 0; k < 4; ++k) ms_out[k] = acc[k] / (double)(nsteps * kRK);
    }
    for (auto& e : ev) cudaEventDestroy(e);
    return rc;
}

const char* ch_error_string(int status) {
    switch (status) {
        case CH_OK: return "CH_OK: success";
        case CH_EINVAL: return "CH_EINVAL: invalid argument";
        case CH_ECUDA: return "CH_ECUDA: CUDA runtime error";
        case CH_ENONFINITE: return "CH_ENONFINITE: non-finite value in C";
        case CH_ETIMEOUT: return "CH_ETIMEOUT: bounded device wait expired";
        case CH_ENOMEM: return "CH_ENOMEM: workspace too small or allocation failed";
        default: return "unknown status";
    }
}

const char* ch_last_error(const ch_handle* h) { return h ? h->err : ""; }

}  // extern "C"
