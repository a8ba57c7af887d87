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
#include <type_traits>
#include <utility>
#include <vector>

#include "ch_internal.h"
#include "ch_explicit2.cuh"
#include "ch_kernels.cuh"
#include "ch_cols2.cuh"
#include "line_tables.h"

using namespace chg;

namespace {

constexpr size_t kAlign = 256;
constexpr size_t kMaxSmem = 227 * 1024;  // dynamic shared memory per CTA (sm_103a)

// Use the two-column form of the column solver when nx is even, and its
// cluster form for y/z lines longer than 256 cells.
#ifndef CH_COLUMN_PAIRS
#define CH_COLUMN_PAIRS 1
#endif
#ifndef CH_COLUMN_CLUSTER
#define CH_COLUMN_CLUSTER 1
#endif
// Lines of 513..1024 cells over clusters of 4 CTAs: measured slower than the
// shared-memory tile solver on the 1024-cell periodic y-lines of the
// 1024x1024x512 box (3.74 against 2.81 ms), so off by default.
#ifndef CH_COLUMN_CLUSTER4
#define CH_COLUMN_CLUSTER4 0
#endif
// x-lines of 257..1024 cells solved in shared memory (ch_solve_x_sm) rather
// than in registers.
#ifndef CH_X_SM
#define CH_X_SM 1
#endif
// FP32 lines of 257..1024 cells: adjacent lines solved together per warp in
// shared memory.  y and z: ch_solve_yz_v with CH_Y_LINES / CH_Z_LINES lines
// per warp over tiles of CH_Y_COLS / CH_Z_COLS columns, at most
// CH_Y_MAX_BLOCKS / CH_Z_MAX_BLOCKS CTAs per SM (lines = 1 keeps the one-line
// tile solver; for z, CH_Z_TILE = 0 keeps the 2-CTA cluster column solver).
// x: ch_solve_x_smv with CH_X_LINES lines per warp, CH_X_WARPS warps per CTA.
// Defaults: the fastest measured on the 1024x1024x512 mesh.
#ifndef CH_Y_LINES
#define CH_Y_LINES 4
#endif
#ifndef CH_Y_COLS
#define CH_Y_COLS 32
#endif
#ifndef CH_Y_MAX_BLOCKS
#define CH_Y_MAX_BLOCKS 2
#endif
#ifndef CH_Z_TILE
#define CH_Z_TILE 1
#endif
#ifndef CH_Z_LINES
#define CH_Z_LINES 4
#endif
#ifndef CH_Z_COLS
#define CH_Z_COLS 32
#endif
#ifndef CH_Z_MAX_BLOCKS
#define CH_Z_MAX_BLOCKS 2
#endif
#ifndef CH_X_LINES
#define CH_X_LINES 2
#endif
#ifndef CH_X_WARPS
#define CH_X_WARPS 2
#endif
// y/z multi-line tiles from persistent CTAs, each tile's write-back fused
// with the staging of the CTA's next tile (0: one CTA per tile, the default:
// the persistent form measured slower, y 1.47 against 1.41 ms and z 1.41
// against 1.38 ms on the 1024x1024x512 mesh)
#ifndef CH_YZ_PERSIST
#define CH_YZ_PERSIST 0
#endif
// shortest lines (in rows per lane, M) that take the multi-line solvers
// FP32 explicit kernel: stage C through a tensor map (TMA tile loads, two
// planes ahead) on the tiles that need no wrapped or mirrored index.  Off by
// default: measured slower than the per-thread copies on the 1024x1024x512
// mesh (5.67 against 5.58 ms per launch; the kernel is bound by instruction
// issue, not by its staging)
#ifndef CH_EXPLICIT_TMA
#define CH_EXPLICIT_TMA 0
#endif
// CTAs per SM of the mass and free-energy reductions
#ifndef CH_RED_BLOCKS_PER_SM
#define CH_RED_BLOCKS_PER_SM 4
#endif
#ifndef CH_MULTI_MIN_M
#define CH_MULTI_MIN_M 16
#endif
// Lines of 65..256 cells also over 2-CTA clusters (CTAs of 4 or 8 warps), so
// that two tiles share an SM.
#ifndef CH_COLUMN_CLUSTER_SMALL
#define CH_COLUMN_CLUSTER_SMALL 0
#endif

// Launch a step kernel, optionally with programmatic stream serialisation
// (CH_PDL = 1): it may then be scheduled while its predecessor on the stream
// drains, and waits (pdl_wait) before touching memory.  Off by default: on the
// shear-drop step the early CTAs slowed the predecessors' tails more than the
// launch gaps they hide (0.628 against 0.619 ms per step).
#ifndef CH_PDL
#define CH_PDL 0
#endif
template <typename... KArgs, typename... Args>
cudaError_t launch_k(cudaStream_t st, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                     Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = CH_PDL;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

bool params_valid(const ch_params* p, char* why, size_t wl) {
    auto bad = [&](const char* m) {
        snprintf(why, wl, "%s", m);
        return false;
    };
    if (!p) return bad("params is NULL");
    if (p->nx < 5 || p->ny < 5) return bad("nx and ny must each be >= 5");
    // nz = 1 with a periodic z: one plane, the 2D scheme (A_x + A_y, Eq. eq-a2d with w = 2)
    if (p->nz < 5 && !(p->nz == 1 && p->bc[2] == CH_PERIODIC))
        return bad("nz must be >= 5, or 1 (a periodic single plane: the 2D scheme)");
    if (p->nx > (1 << 20) || p->ny > (1 << 20) || p->nz > (1 << 20)) return bad("a dimension exceeds 2^20");
    if ((double)p->nx * p->ny * p->nz > 9.0e18 / 8) return bad("grid too large");
    if (!(p->h > 0) || !(p->cn > 0) || !(p->pe > 0) || !(p->dt > 0) || !(p->w > 0) || !(p->weno_eps > 0))
        return bad("h, cn, pe, dt, w, weno_eps must be positive and finite");
    if (!std::isfinite(p->h) || !std::isfinite(p->cn) || !std::isfinite(p->pe) || !std::isfinite(p->dt) ||
        !std::isfinite(p->w) || !std::isfinite(p->weno_eps))
        return bad("non-finite parameter");
    for (int d = 0; d < 3; ++d)
        if (p->bc[d] != CH_PERIODIC && p->bc[d] != CH_NOFLUX && !(d == 2 && p->bc[d] == CH_DIRICHLET))
            return bad("bc must be CH_PERIODIC or CH_NOFLUX (z may also be CH_DIRICHLET)");
    if (p->bc[2] == CH_DIRICHLET && p->scheme != CH_SCHEME_SPLIT)
        return bad("Dirichlet walls are supported by the split scheme only");
    if (p->precision != CH_F32 && p->precision != CH_F64) return bad("precision must be CH_F32 or CH_F64");
    if (p->advect != 0 && p->advect != 1) return bad("advect must be 0 or 1");
    if (p->scheme != CH_SCHEME_SPLIT && p->scheme != CH_SCHEME_STANDARD)
        return bad("scheme must be CH_SCHEME_SPLIT or CH_SCHEME_STANDARD");
    const bool any_c = p->ncx || p->ncy || p->ncz || p->xf_coarse || p->yf_coarse || p->zf_coarse;
    if (any_c) {
        if (p->ncx < 4 || p->ncy < 4 || p->ncz < 4) return bad("coarse mesh needs >= 4 cells per direction");
        if (p->nz < 5) return bad("a coarse mesh needs nz >= 5");
        if (p->ncx > kMaxCoarseLine || p->ncy > kMaxCoarseLine || p->ncz > kMaxCoarseLine)
            return bad("coarse mesh has more than 2048 cells in a direction");
        if ((double)p->ncx * p->ncy * p->ncz >= 2147483647.0) return bad("coarse mesh has 2^31 cells or more");
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
    // warp-scan line solves: at most 32 x 32 rows per line; the y/z tile
    // (32 M rows x 32 columns, 16 for FP64 lines of 1024 cells) fits in
    // shared memory for every supported length
    if (p->nx > 1024 || p->ny > 1024 || p->nz > 1024) return bad("lines longer than 1024 cells are not supported");
    return true;
}

struct Layout {
    size_t H0, H1, r, vel[3], velc[3], gradc[3], mrplane, total;
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
    for (int d = 0; d < 3; ++d) nf[d] = n[d] + (p->bc[d] != CH_PERIODIC ? 1 : 0);
    if (p->advect) {
        L.vel[0] = take((size_t)n[2] * n[1] * nf[0] * esz);
        L.vel[1] = take((size_t)n[2] * nf[1] * n[0] * esz);
        L.vel[2] = take((size_t)nf[2] * n[1] * n[0] * esz);
    }
    if (p->ncx) {
        const int64_t nc[3] = {p->ncx, p->ncy, p->ncz};
        int64_t ncf[3];
        for (int d = 0; d < 3; ++d) ncf[d] = nc[d] + (p->bc[d] != CH_PERIODIC ? 1 : 0);
        L.velc[0] = take((size_t)nc[2] * nc[1] * ncf[0] * esz);
        L.velc[1] = take((size_t)nc[2] * ncf[1] * nc[0] * esz);
        L.velc[2] = take((size_t)ncf[2] * nc[1] * nc[0] * esz);
        for (int d = 0; d < 3; ++d) L.gradc[d] = take((size_t)nc[0] * nc[1] * nc[2] * esz);
        // the transfer's intermediate for y and z (one at a time): the coarse
        // gradient interpolated across the lines, at the coarse nodes along them
        L.mrplane = take((size_t)std::max(n[2] * nc[1], nc[2] * n[1]) * (size_t)n[0] * esz);
    }
    L.total = off;
    return L;
}

template <typename T>
WCoef<T> wcoef(const LineTables& lt) {
    const WarpLayout L = warp_layout(lt.M);
    const T* b = (const T*)lt.base;
    WCoef<T> k;
    k.fwd = b + L.fwd;
    k.bwd = b + L.bwd;
    k.W = b + L.W;
    k.Z = b + L.Z;
    k.Pf = b + L.Pf;
    k.Pb = b + L.Pb;
    k.S = b + L.S;
    k.n = lt.n;
    k.periodic = lt.periodic;
    k.r0 = lt.r0;
    k.r1 = lt.r1;
    for (int m = 0; m < 5; ++m) k.k[m] = (T)lt.k[m];
    return k;
}

// Solve (I + c A_dir) x = a in place along direction dir for substep l's c;
// for dir = 2 with Cupd != nullptr the solution is added to Cupd instead.
// y (dir 1) or z (dir 2) lines through ch_solve_yz_v: L lines per warp,
// NC-column tiles, at most B CTAs per SM.
template <typename T, int M, int L, int NC, int B>
void launch_yz_v(ch_handle* h, int dir, T* r, T* Cupd, const WCoef<T>& cf) {
    using S = YZVShape<T, M, L, NC, B>;
    const int nx = (int)h->n[0], ny = (int)h->n[1], nz = (int)h->n[2];
    const int64_t xblocks = (nx + NC - 1) / NC;
    const int64_t plane = (int64_t)nx * ny;
    const int64_t ntiles = xblocks * (dir == 1 ? nz : ny);
    // persistent CTAs (each runs tiles blockIdx.x, + gridDim.x, ...): as many
    // as fit on the device at once
    int dev = 0, nsm = 152;
    if (CH_YZ_PERSIST && cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const unsigned grid = (unsigned)(CH_YZ_PERSIST ? std::min<int64_t>(ntiles, (int64_t)S::kMinBlocks * nsm) : ntiles);
    if (dir == 1)
        launch_k(h->stream, ch_solve_yz_v<T, M, false, L, NC, B>, dim3(grid), dim3(S::kWarps * 32), S::kTileBytes, r,
                 nullptr, nx, plane, (int64_t)nx, cf, h->status, ntiles);
    else if (Cupd)
        launch_k(h->stream, ch_solve_yz_v<T, M, true, L, NC, B>, dim3(grid), dim3(S::kWarps * 32), S::kTileBytes, r,
                 Cupd, nx, (int64_t)nx, plane, cf, h->status, ntiles);
    else
        launch_k(h->stream, ch_solve_yz_v<T, M, false, L, NC, B>, dim3(grid), dim3(S::kWarps * 32), S::kTileBytes, r,
                 nullptr, nx, (int64_t)nx, plane, cf, h->status, ntiles);
}

// Whether FP32 lines of 257..1024 cells (M = 16, 32) along dir go through the
// multi-line shared-memory solvers (ch_solve_x_smv, ch_solve_yz_v).
template <typename T, int M>
bool multi_line(const ch_handle* h, int dir) {
    if constexpr (sizeof(T) != 4 || M < CH_MULTI_MIN_M || M < 4) {
        return false;
    } else {
        const int64_t nx = h->n[0];
        if (dir == 0) return CH_X_LINES > 1 && nx % 4 == 0;
        if (dir == 1) return CH_Y_LINES > 1 && nx % CH_Y_LINES == 0;
        return CH_Z_TILE && CH_Z_LINES > 1 && nx % CH_Z_LINES == 0;
    }
}

template <typename T, int M>
int launch_solves_m(ch_handle* h, int l, int dir, T* r, T* Cupd, cudaEvent_t ev_after) {
    const int nx = (int)h->n[0], ny = (int)h->n[1], nz = (int)h->n[2];
    const WCoef<T> cf = wcoef<T>(h->lines[dir][l]);
    if constexpr (sizeof(T) == 4 && M >= CH_MULTI_MIN_M && M >= 4) {
        if (multi_line<T, M>(h, dir)) {
            if (dir == 0) {
                constexpr int L = CH_X_LINES, W = CH_X_WARPS;
                using S = XSmvShape<T, M, L, W>;
                const int64_t nlines = (int64_t)ny * nz;
                launch_k(h->stream, ch_solve_x_smv<T, M, L, W>, dim3((unsigned)((nlines + W * L - 1) / (W * L))),
                         dim3(W * 32), W * S::kWarpBytes, r, nlines, nx, cf);
            } else if (dir == 1) {
                launch_yz_v<T, M, CH_Y_LINES, CH_Y_COLS, CH_Y_MAX_BLOCKS>(h, dir, r, Cupd, cf);
            } else {
                launch_yz_v<T, M, CH_Z_LINES, CH_Z_COLS, CH_Z_MAX_BLOCKS>(h, dir, r, Cupd, cf);
            }
            CHG_CUDA(h, cudaGetLastError());
            if (ev_after) CHG_CUDA(h, cudaEventRecord(ev_after, h->stream));
            return CH_OK;
        }
    }
    if (dir == 0) {
        const int64_t nlines = (int64_t)ny * nz;
        constexpr int wpb = 8, lpb = wpb * LinesPerWarp<T, M>::value;
        if constexpr (M >= 16 && CH_X_SM)
            launch_k(h->stream, ch_solve_x_sm<T, M>, dim3((unsigned)((nlines + wpb - 1) / wpb)), dim3(wpb * 32),
                     wpb * XSmShape<T, M>::kWarpBytes, r, nlines, nx, cf);
        else
            launch_k(h->stream, ch_solve_x<T, M>, dim3((unsigned)((nlines + lpb - 1) / lpb)), dim3(wpb * 32), 0, r,
                     nlines, nx, cf);
    } else {
        constexpr int NC = YZShape<T, M>::kCols;
        const unsigned xblocks = (unsigned)((nx + NC - 1) / NC);
        const size_t shm = YZShape<T, M>::kTileBytes;
        if (dir == 1)
            launch_k(h->stream, ch_solve_yz<T, M, false>, dim3(xblocks * (unsigned)nz), dim3(YZShape<T, M>::kWarps * 32), shm,
                r, nullptr, nx, (int64_t)nx * ny, nx, cf, h->status);
        else if (Cupd)
            launch_k(h->stream, ch_solve_yz<T, M, true>, dim3(xblocks * (unsigned)ny), dim3(YZShape<T, M>::kWarps * 32), shm,
                r, Cupd, nx, nx, (int64_t)nx * ny, cf, h->status);
        else
            launch_k(h->stream, ch_solve_yz<T, M, false>, dim3(xblocks * (unsigned)ny), dim3(YZShape<T, M>::kWarps * 32), shm,
                r, nullptr, nx, nx, (int64_t)nx * ny, cf, h->status);
    }
    CHG_CUDA(h, cudaGetLastError());
    if (ev_after) CHG_CUDA(h, cudaEventRecord(ev_after, h->stream));
    return CH_OK;
}

template <typename T>
CCoef<T> ccoef(const LineTables& lt) {
    const ColLayout L = col_layout(lt.nw, lt.R);
    const T* b = (const T*)lt.col;
    CCoef<T> k;
    k.fwd = b + L.fwd;
    k.bwd = b + L.bwd;
    k.W = b + L.W;
    k.Z = b + L.Z;
    k.P = b + L.P;
    k.Q = b + L.Q;
    k.S = b + L.S;
    k.fwdp = b + L.fwdp;
    k.dinvp = b + L.dinvp;
    k.bwdp = b + L.bwdp;
    k.Wp = b + L.Wp;
    k.Zp = b + L.Zp;
    k.K = b + L.K;
    k.n = lt.n;
    k.periodic = lt.periodic;
    return k;
}

template <typename T, int R, int NW>
int launch_cols_rn(ch_handle* h, int l, int dir, T* r, T* Cupd) {
    const int nx = (int)h->n[0], ny = (int)h->n[1], nz = (int)h->n[2];
    const CCoef<T> cf = ccoef<T>(h->lines[dir][l]);
    const unsigned xblocks = (unsigned)((nx + 31) / 32);
    if (dir == 1)
        launch_k(h->stream, ch_solve_cols<T, R, NW, false>, dim3(xblocks * (unsigned)nz), dim3(NW * 32), 0,
            r, nullptr, nx, (int64_t)nx * ny, nx, cf, h->status);
    else if (Cupd)
        launch_k(h->stream, ch_solve_cols<T, R, NW, true>, dim3(xblocks * (unsigned)ny), dim3(NW * 32), 0,
            r, Cupd, nx, nx, (int64_t)nx * ny, cf, h->status);
    else
        launch_k(h->stream, ch_solve_cols<T, R, NW, false>, dim3(xblocks * (unsigned)ny), dim3(NW * 32), 0,
            r, nullptr, nx, nx, (int64_t)nx * ny, cf, h->status);
    CHG_CUDA(h, cudaGetLastError());
    return CH_OK;
}

// Two-column form (even nx): lanes own pairs of adjacent lines.
template <typename T, int R, int NW>
int launch_cols2_rn(ch_handle* h, int l, int dir, T* r, T* Cupd) {
    const int nx = (int)h->n[0], ny = (int)h->n[1], nz = (int)h->n[2];
    const CCoef<T> cf = ccoef<T>(h->lines[dir][l]);
    const unsigned xblocks = (unsigned)((nx + 63) / 64);
    const bool per = cf.periodic != 0;
    if (dir == 1) {
        launch_k(h->stream, ch_solve_cols2<T, R, NW, false>, dim3(xblocks * (unsigned)nz), dim3(NW * 32), Cols2Smem<T, R, NW, false>::bytes(per),
            r, nullptr, nx, (int64_t)nx * ny, nx, cf, h->status);
    } else if (Cupd) {
        launch_k(h->stream, ch_solve_cols2<T, R, NW, true>, dim3(xblocks * (unsigned)ny), dim3(NW * 32), Cols2Smem<T, R, NW, true>::bytes(per),
            r, Cupd, nx, nx, (int64_t)nx * ny, cf, h->status);
    } else {
        launch_k(h->stream, ch_solve_cols2<T, R, NW, false>, dim3(xblocks * (unsigned)ny), dim3(NW * 32), Cols2Smem<T, R, NW, false>::bytes(per),
            r, nullptr, nx, nx, (int64_t)nx * ny, cf, h->status);
    }
    CHG_CUDA(h, cudaGetLastError());
    return CH_OK;
}

// Cluster form: CL CTAs of NW warps per 64-line tile (lines of up to CL NW R cells).
template <typename T, int R, int NW, int CL, bool UPDATE>
int cols2c_launch(ch_handle* h, T* r, T* Cupd, int nx, int64_t outer_stride, int64_t line_stride, int64_t tiles,
                  const CCoef<T>& cf) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(tiles * CL));
    cfg.blockDim = dim3(NW * 32);
    cfg.dynamicSmemBytes = Cols2cSmem<T, R, NW, CL, UPDATE>::kBytes;
    cfg.stream = h->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CHG_CUDA(h, cudaLaunchKernelEx(&cfg, ch_solve_cols2c<T, R, NW, CL, UPDATE>, r, Cupd, nx, outer_stride,
                                   line_stride, cf, h->status));
    return CH_OK;
}

template <typename T, int R, int NW, int CL>
int launch_cols2c_rn(ch_handle* h, int l, int dir, T* r, T* Cupd) {
    const int nx = (int)h->n[0], ny = (int)h->n[1], nz = (int)h->n[2];
    const CCoef<T> cf = ccoef<T>(h->lines[dir][l]);
    const int64_t xblocks = (nx + 63) / 64;
    if (dir == 1)
        return cols2c_launch<T, R, NW, CL, false>(h, r, nullptr, nx, (int64_t)nx * ny, nx, xblocks * nz, cf);
    if (Cupd) return cols2c_launch<T, R, NW, CL, true>(h, r, Cupd, nx, nx, (int64_t)nx * ny, xblocks * ny, cf);
    return cols2c_launch<T, R, NW, CL, false>(h, r, nullptr, nx, nx, (int64_t)nx * ny, xblocks * ny, cf);
}

template <typename T, int R, int NW, int CL>
int set_attrs_cols2c(ch_handle* h) {
    CHG_CUDA(h, cudaFuncSetAttribute(ch_solve_cols2c<T, R, NW, CL, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)Cols2cSmem<T, R, NW, CL, false>::kBytes));
    CHG_CUDA(h, cudaFuncSetAttribute(ch_solve_cols2c<T, R, NW, CL, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)Cols2cSmem<T, R, NW, CL, true>::kBytes));
    return CH_OK;
}

template <typename T, int R, int NW>
int set_attrs_cols2(ch_handle* h) {
    CHG_CUDA(h, cudaFuncSetAttribute(ch_solve_cols2<T, R, NW, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)Cols2Smem<T, R, NW, false>::kMax));
    CHG_CUDA(h, cudaFuncSetAttribute(ch_solve_cols2<T, R, NW, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)Cols2Smem<T, R, NW, true>::kMax));
    return CH_OK;
}

template <typename T>
int set_attrs_cols2_all(ch_handle* h) {
    int rc = set_attrs_cols2<T, 1, 8>(h);
    if (rc == CH_OK) rc = set_attrs_cols2<T, 2, 8>(h);
    if (rc == CH_OK) rc = set_attrs_cols2<T, 4, 8>(h);
    if (rc == CH_OK) rc = set_attrs_cols2<T, 8, 8>(h);
    if (rc == CH_OK) rc = set_attrs_cols2<T, 16, 8>(h);
    if (rc == CH_OK) rc = set_attrs_cols2<T, 16, 16>(h);
    if (rc == CH_OK) rc = set_attrs_cols2<T, 8, 16>(h);
    if (rc == CH_OK) rc = set_attrs_cols2<T, 8, 32>(h);
    if (rc == CH_OK) rc = set_attrs_cols2c<T, 16, kClusterNW, 2>(h);
    if (rc == CH_OK) rc = set_attrs_cols2c<T, 16, 8, 2>(h);
    if (rc == CH_OK) rc = set_attrs_cols2c<T, 16, 4, 2>(h);
    if (rc == CH_OK) rc = set_attrs_cols2c<T, 16, kClusterNW, 4>(h);
    return rc;
}

// Which strided directions use the column solver (bit 1: y, bit 2: z); the
// others use the shared-memory tile solver.  Default: both (measured with the
// two-column form; the one-column form alone was slower than the tile for y).
#ifndef CH_COLUMN_DIRS
#define CH_COLUMN_DIRS 6
#endif


// Column solver for y/z lines (shape chosen by col_shape); -1 if none.
template <typename T>
int launch_cols(ch_handle* h, int l, int dir, T* r, T* Cupd) {
    const LineTables& lt = h->lines[dir][l];
    if (!lt.col || !((CH_COLUMN_DIRS >> dir) & 1)) return -1;
    // two-column form: FP32 only (an FP64 lane would hold 4 R registers of rows)
    if constexpr (sizeof(T) == 4) {
        if (CH_COLUMN_PAIRS && h->n[0] % 2 == 0) {
            if (CH_COLUMN_CLUSTER_SMALL && lt.R == 16 && lt.nw == 16)
                return launch_cols2c_rn<T, 16, 8, 2>(h, l, dir, r, Cupd);
            if (CH_COLUMN_CLUSTER_SMALL && lt.R == 16 && lt.nw == 8)
                return launch_cols2c_rn<T, 16, 4, 2>(h, l, dir, r, Cupd);
            if (lt.nw == 8) {
                switch (lt.R) {
                    case 1: return launch_cols2_rn<T, 1, 8>(h, l, dir, r, Cupd);
                    case 2: return launch_cols2_rn<T, 2, 8>(h, l, dir, r, Cupd);
                    case 4: return launch_cols2_rn<T, 4, 8>(h, l, dir, r, Cupd);
                    case 8: return launch_cols2_rn<T, 8, 8>(h, l, dir, r, Cupd);
                    case 16: return launch_cols2_rn<T, 16, 8>(h, l, dir, r, Cupd);
                    default: return -1;
                }
            }
            if (lt.nw == 16 && lt.R == 16) return launch_cols2_rn<T, 16, 16>(h, l, dir, r, Cupd);
            if (lt.nw == 16 && lt.R == 8) return launch_cols2_rn<T, 8, 16>(h, l, dir, r, Cupd);
            if (lt.nw == 32 && lt.R == 8) return launch_cols2_rn<T, 8, 32>(h, l, dir, r, Cupd);
            if (CH_COLUMN_CLUSTER && lt.R == 16 && lt.nw == 2 * kClusterNW)
                return launch_cols2c_rn<T, 16, kClusterNW, 2>(h, l, dir, r, Cupd);
            if (CH_COLUMN_CLUSTER && lt.R == 16 && lt.nw == 4 * kClusterNW)
                return launch_cols2c_rn<T, 16, kClusterNW, 4>(h, l, dir, r, Cupd);
            // 32 warps leave 64 registers a thread: the one-column form below
        }
    }
    if (lt.nw == 8) {
        switch (lt.R) {
            case 1: return launch_cols_rn<T, 1, 8>(h, l, dir, r, Cupd);
            case 2: return launch_cols_rn<T, 2, 8>(h, l, dir, r, Cupd);
            case 4: return launch_cols_rn<T, 4, 8>(h, l, dir, r, Cupd);
            case 8: return launch_cols_rn<T, 8, 8>(h, l, dir, r, Cupd);
            case 16: return launch_cols_rn<T, 16, 8>(h, l, dir, r, Cupd);
            default: return -1;
        }
    }
    if (lt.nw == 16 && lt.R == 16) return launch_cols_rn<T, 16, 16>(h, l, dir, r, Cupd);
    if (lt.nw == 32 && lt.R == 16) return launch_cols_rn<T, 16, 32>(h, l, dir, r, Cupd);
    if (lt.nw == 16 && lt.R == 8) return launch_cols_rn<T, 8, 16>(h, l, dir, r, Cupd);
    if (lt.nw == 32 && lt.R == 8) return launch_cols_rn<T, 8, 32>(h, l, dir, r, Cupd);
    return -1;
}

template <typename T>
bool multi_line_any(const ch_handle* h, int l, int dir) {
    switch (h->lines[dir][l].M) {
        case 4: return multi_line<T, 4>(h, dir);
        case 8: return multi_line<T, 8>(h, dir);
        case 16: return multi_line<T, 16>(h, dir);
        case 32: return multi_line<T, 32>(h, dir);
        default: return false;
    }
}

template <typename T>
int launch_solve(ch_handle* h, int l, int dir, T* r, T* Cupd, cudaEvent_t ev_after) {
    if (dir > 0 && !multi_line_any<T>(h, l, dir)) {
        const int rc = launch_cols<T>(h, l, dir, r, Cupd);
        if (rc >= 0) {
            if (rc == CH_OK && ev_after) CHG_CUDA(h, cudaEventRecord(ev_after, h->stream));
            return rc;
        }
    }
    switch (h->lines[dir][l].M) {
        case 1: return launch_solves_m<T, 1>(h, l, dir, r, Cupd, ev_after);
        case 2: return launch_solves_m<T, 2>(h, l, dir, r, Cupd, ev_after);
        case 4: return launch_solves_m<T, 4>(h, l, dir, r, Cupd, ev_after);
        case 8: return launch_solves_m<T, 8>(h, l, dir, r, Cupd, ev_after);
        case 16: return launch_solves_m<T, 16>(h, l, dir, r, Cupd, ev_after);
        case 32: return launch_solves_m<T, 32>(h, l, dir, r, Cupd, ev_after);
        default: return fail(h, CH_EINVAL, "unsupported line length");
    }
}

template <typename T, int M>
int set_attrs_m(ch_handle* h) {
    if constexpr (M >= 16)
        CHG_CUDA(h, cudaFuncSetAttribute(ch_solve_x_sm<T, M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(8 * XSmShape<T, M>::kWarpBytes)));
    if constexpr (sizeof(T) == 4 && M >= CH_MULTI_MIN_M && M >= 4) {
        using SX = XSmvShape<T, M, CH_X_LINES, CH_X_WARPS>;
        CHG_CUDA(h, cudaFuncSetAttribute(ch_solve_x_smv<T, M, CH_X_LINES, CH_X_WARPS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(CH_X_WARPS * SX::kWarpBytes)));
        using SY = YZVShape<T, M, CH_Y_LINES, CH_Y_COLS, CH_Y_MAX_BLOCKS>;
        CHG_CUDA(h, cudaFuncSetAttribute(ch_solve_yz_v<T, M, false, CH_Y_LINES, CH_Y_COLS, CH_Y_MAX_BLOCKS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SY::kTileBytes));
        using SZ = YZVShape<T, M, CH_Z_LINES, CH_Z_COLS, CH_Z_MAX_BLOCKS>;
        CHG_CUDA(h, cudaFuncSetAttribute(ch_solve_yz_v<T, M, false, CH_Z_LINES, CH_Z_COLS, CH_Z_MAX_BLOCKS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SZ::kTileBytes));
        CHG_CUDA(h, cudaFuncSetAttribute(ch_solve_yz_v<T, M, true, CH_Z_LINES, CH_Z_COLS, CH_Z_MAX_BLOCKS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SZ::kTileBytes));
    }
    const int shm = (int)YZShape<T, M>::kTileBytes;
    if ((size_t)shm > kMaxSmem) return CH_OK;  // never launched for this precision
    CHG_CUDA(h, cudaFuncSetAttribute(ch_solve_yz<T, M, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, shm));
    CHG_CUDA(h, cudaFuncSetAttribute(ch_solve_yz<T, M, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, shm));
    return CH_OK;
}

// Explicit RHS of substep l from C (and Hprev) into Hout and r.
// With adv_only (the standard scheme's advection): Hout = -div(uC) only, no
// diffusive or implicit term, no right-hand side written.
template <typename T>
int launch_explicit(ch_handle* h, int l, const T* C, const T* Hprev, T* Hout, T* r, cudaEvent_t* ev,
                    bool adv_only = false) {
    const ch_params& p = h->p;
    const int nx = (int)h->n[0], ny = (int)h->n[1], nz = (int)h->n[2];
    RhsArgs<T> a;
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    a.bcx = p.bc[0];
    a.bcy = p.bc[1];
    a.bcz = p.bc[2];
    a.nfx = (int)h->nf[0];
    a.nfy = (int)h->nf[1];
    a.nfz = (int)h->nf[2];
    const double mob = 1.0 / p.pe;
    const double alpha = kGamma[l] + kRho[l];
    const double kappa = p.w * p.cn * p.cn / (p.h * p.h * p.h * p.h);
    a.inv_h = (T)(1.0 / p.h);
    a.inv_h2 = (T)(1.0 / (p.h * p.h));
    a.mob = (T)mob;
    a.dtg = (T)(p.dt * kGamma[l]);
    a.dtr = (T)(p.dt * kRho[l]);
    a.impl = (T)(alpha * p.dt * mob * kappa);
    a.eps = (T)p.weno_eps;
    a.has_prev = kRho[l] != 0.0;
    if (adv_only) {
        a.mob = T(0);
        a.impl = T(0);
        a.dtg = T(1);
        a.dtr = T(0);
        a.has_prev = 0;
        r = nullptr;
    }
    const T* u = p.advect ? (const T*)h->vel[0] : nullptr;
    const T* v = p.advect ? (const T*)h->vel[1] : nullptr;
    const T* w = p.advect ? (const T*)h->vel[2] : nullptr;
    if (ev) CHG_CUDA(h, cudaEventRecord(ev[0], h->stream));
    if (nx % 2 == 0) {  // two cells per thread (paired FP32 arithmetic)
        const int tz = explicit_zchunk(nx, ny, nz, sizeof(T) == 4);
        dim3 grid((nx + kTX2 - 1) / kTX2, (ny + kTY - 1) / kTY, (nz + tz - 1) / tz);
        dim3 block(32, kTY);
        const bool diri = p.bc[2] == CH_DIRICHLET;
        // the tensor map of the handle's C (FP32) when this launch reads that C
        CUtensorMap tm;
        std::memcpy(&tm, h->tmap_c, sizeof(tm));
        // ... and when most tiles (>= 3/4) need no wrapped or mirrored index, so
        // take the tile load; the rest stage element by element
        const int64_t txn = (nx + kTX2 - 1) / kTX2, tyn = (ny + kTY - 1) / kTY;
        const bool mostly_inner = 4 * std::max<int64_t>(txn - 2, 0) * std::max<int64_t>(tyn - 2, 0) >= 3 * txn * tyn;
        const bool tma = sizeof(T) == 4 && h->tmap_ok && (const void*)C == h->C && mostly_inner;
        auto go = [&](auto tzc, auto tmac) {
            constexpr int TZ = decltype(tzc)::value;
            constexpr bool TMA = decltype(tmac)::value;
            if (p.advect && diri)
                launch_k(h->stream, ch_explicit_rhs2<T, true, true, TZ, TMA>, grid, block, 0, C, u, v, w, Hprev, Hout,
                         r, a, tm, h->status);
            else if (p.advect)
                launch_k(h->stream, ch_explicit_rhs2<T, true, false, TZ, TMA>, grid, block, 0, C, u, v, w, Hprev, Hout,
                         r, a, tm, h->status);
            else if (diri)
                launch_k(h->stream, ch_explicit_rhs2<T, false, true, TZ, TMA>, grid, block, 0, C, u, v, w, Hprev, Hout,
                         r, a, tm, h->status);
            else
                launch_k(h->stream, ch_explicit_rhs2<T, false, false, TZ, TMA>, grid, block, 0, C, u, v, w, Hprev,
                         Hout, r, a, tm, h->status);
        };
        using NoTma = std::false_type;
        if constexpr (sizeof(T) == 4) {
            using Tma = std::integral_constant<bool, CH_EXPLICIT_TMA != 0>;
            if (tz == kTZ2Deep) {
                if (tma) go(std::integral_constant<int, kTZ2Deep>{}, Tma{});
                else go(std::integral_constant<int, kTZ2Deep>{}, NoTma{});
            } else {
                if (tma) go(std::integral_constant<int, kTZ2>{}, Tma{});
                else go(std::integral_constant<int, kTZ2>{}, NoTma{});
            }
        } else {
            go(std::integral_constant<int, kTZ2>{}, NoTma{});
        }
    } else {
        dim3 grid((nx + kTX - 1) / kTX, (ny + kTY - 1) / kTY, (nz + kTZ - 1) / kTZ);
        dim3 block(kTX, kTY);
        if (p.advect)
            launch_k(h->stream, ch_explicit_rhs<T, true>, dim3(grid), dim3(block), 0, C, u, v, w, Hprev, Hout, r, a);
        else
            launch_k(h->stream, ch_explicit_rhs<T, false>, dim3(grid), dim3(block), 0, C, u, v, w, Hprev, Hout, r, a);
    }
    CHG_CUDA(h, cudaGetLastError());
    if (ev) CHG_CUDA(h, cudaEventRecord(ev[1], h->stream));
    return CH_OK;
}

template <typename T>
int launch_substep(ch_handle* h, int l, cudaEvent_t* ev = nullptr) {
    if (h->p.scheme == CH_SCHEME_STANDARD) return launch_substep_standard(h, l, ev);
    T* C = (T*)h->C;
    T* r = (T*)h->r;
    int rc = launch_explicit<T>(h, l, C, (const T*)h->H[(l + 1) & 1], (T*)h->H[l & 1], r, ev);
    if (rc != CH_OK) return rc;
    // x solve (Eq. eq-fac-1), y solve (Eq. eq-fac-2), z solve + update (Eq. eq-fac-3);
    // a single plane (2D scheme) has no z-solve: C += dq directly
    for (int dir = 0; dir < 3; ++dir) {
        if (dir == 2 && h->n[2] == 1) {
            const int64_t N = h->ncell;
            const unsigned blocks = (unsigned)std::min<int64_t>((N + 255) / 256, 16 * 152);
            ch_add_increment<T><<<blocks, 256, 0, h->stream>>>(C, r, N, h->status);
            CHG_CUDA(h, cudaGetLastError());
            if (ev) CHG_CUDA(h, cudaEventRecord(ev[4], h->stream));
            continue;
        }
        rc = launch_solve<T>(h, l, dir, r, dir == 2 ? C : nullptr, ev ? ev[2 + dir] : nullptr);
        if (rc != CH_OK) return rc;
    }
    return CH_OK;
}

template <typename T>
int set_smem_attrs(ch_handle* h) {
    int rc = CH_OK;
    if (rc == CH_OK) rc = set_attrs_m<T, 1>(h);
    if (rc == CH_OK) rc = set_attrs_m<T, 2>(h);
    if (rc == CH_OK) rc = set_attrs_m<T, 4>(h);
    if (rc == CH_OK) rc = set_attrs_m<T, 8>(h);
    if (rc == CH_OK) rc = set_attrs_m<T, 16>(h);
    if (rc == CH_OK) rc = set_attrs_m<T, 32>(h);
    if constexpr (sizeof(T) == 4)
        if (rc == CH_OK) rc = set_attrs_cols2_all<T>(h);
    return rc;
}

}  // namespace

namespace chg {

int launch_explicit_any(ch_handle* h, int l, const void* C, const void* Hprev, void* Hout, void* r) {
    if (h->prec == CH_F64)
        return launch_explicit<double>(h, l, (const double*)C, (const double*)Hprev, (double*)Hout, (double*)r, nullptr);
    return launch_explicit<float>(h, l, (const float*)C, (const float*)Hprev, (float*)Hout, (float*)r, nullptr);
}

int launch_advection_any(ch_handle* h, const void* C, void* Hout) {
    if (h->prec == CH_F64)
        return launch_explicit<double>(h, 0, (const double*)C, nullptr, (double*)Hout, nullptr, nullptr, true);
    return launch_explicit<float>(h, 0, (const float*)C, nullptr, (float*)Hout, nullptr, nullptr, true);
}

int launch_solve_any(ch_handle* h, int l, int dir, void* a, void* Cupd) {
    if (h->prec == CH_F64) return launch_solve<double>(h, l, dir, (double*)a, (double*)Cupd, nullptr);
    return launch_solve<float>(h, l, dir, (float*)a, (float*)Cupd, nullptr);
}

int launch_step_any(ch_handle* h, void* C) {
    void* saved = h->C;
    h->C = C;
    int rc = CH_OK;
    for (int l = 0; l < kRK && rc == CH_OK; ++l)
        rc = h->prec == CH_F64 ? launch_substep<double>(h, l) : launch_substep<float>(h, l);
    h->C = saved;
    return rc;
}

}  // namespace chg

namespace {

int launch_step(ch_handle* h) {
    for (int l = 0; l < kRK; ++l) {
        const int rc = h->prec == CH_F64 ? launch_substep<double>(h, l) : launch_substep<float>(h, l);
        if (rc != CH_OK) return rc;
    }
    return CH_OK;
}

// Both diagnostics in one pass over C: out[0] = mass, out[1] = free energy.
template <typename T>
int reduce_both(ch_handle* h, double* out) {
    const ch_params& p = h->p;
    ch_reduce_energy<T, true><<<h->red_blocks, kRedThreads, 0, h->stream>>>(
        (const T*)h->C, (int)h->n[0], (int)h->n[1], (int)h->n[2], p.bc[0], p.bc[1], p.bc[2], (T)(1.0 / p.h),
        (T)(0.5 * p.cn * p.cn), h->red_partials, h->status);
    CHG_CUDA(h, cudaGetLastError());
    const double h3 = p.h * p.h * p.h;
    ch_reduce_finish<<<1, kRedThreads, 0, h->stream>>>(h->red_partials + h->red_blocks, h->red_blocks, h3, h->red_out);
    CHG_CUDA(h, cudaGetLastError());
    ch_reduce_finish<<<1, kRedThreads, 0, h->stream>>>(h->red_partials, h->red_blocks, h3, h->red_out + 1);
    CHG_CUDA(h, cudaGetLastError());
    CHG_CUDA(h, cudaMemcpyAsync(out, h->red_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return ch_sync(h);
}

template <typename T>
int reduce(ch_handle* h, bool energy, double* out) {
    const ch_params& p = h->p;
    if (energy)
        ch_reduce_energy<T><<<h->red_blocks, kRedThreads, 0, h->stream>>>(
            (const T*)h->C, (int)h->n[0], (int)h->n[1], (int)h->n[2], p.bc[0], p.bc[1], p.bc[2], (T)(1.0 / p.h),
            (T)(0.5 * p.cn * p.cn), h->red_partials, h->status);
    else
        ch_reduce_mass<T><<<h->red_blocks, kRedThreads, 0, h->stream>>>((const T*)h->C, (int)h->n[0],
                                                                        h->n[1] * h->n[2], h->red_partials,
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

// The explicit kernel's tensor map of C: FP32, nx a multiple of 4 (16-byte
// row strides), a box of one staged plane (72 x 14 x 1).  Left unset
// (tmap_ok = 0) when the driver entry point or the encoding is unavailable;
// the kernel then stages every tile element by element.
void encode_tmap_c(ch_handle* h) {
    h->tmap_ok = 0;
    if (!CH_EXPLICIT_TMA || h->prec != CH_F32 || h->n[0] % 4 != 0) return;
    using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return;
    }
    const cuuint64_t dims[3] = {(cuuint64_t)h->n[0], (cuuint64_t)h->n[1], (cuuint64_t)h->n[2]};
    const cuuint64_t strides[2] = {(cuuint64_t)h->n[0] * 4, (cuuint64_t)(h->n[0] * h->n[1]) * 4};
    const cuuint32_t box[3] = {(cuuint32_t)(kTX2 + 2 * kHL2), (cuuint32_t)(kTY + 2 * kHalo), 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUtensorMap tm;
    if (((Encode)fn)(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, h->C, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return;
    static_assert(sizeof(tm) == sizeof(h->tmap_c), "tensor map size");
    std::memcpy(h->tmap_c, &tm, sizeof(tm));
    h->tmap_ok = 1;
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
    for (int d = 0; d < 3; ++d) h->nf[d] = h->n[d] + (p->bc[d] != CH_PERIODIC ? 1 : 0);
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
            h->mr_plane = wb + L.mrplane;
            h->nc[d] = nc[d];
            h->ncf[d] = nc[d] + (p->bc[d] != CH_PERIODIC ? 1 : 0);
        }
    h->launches_per_step = p->scheme == CH_SCHEME_STANDARD ? (p->advect ? 3 : 2) * kRK : 4 * kRK;

    int rc = CH_OK;
    // warp-scan line-solve tables for every direction and substep
    {
        const double M = 1.0 / p->pe;
        const double kappa = p->w * p->cn * p->cn / (p->h * p->h * p->h * p->h);
        std::vector<std::vector<double>> all;
        size_t total = 0;
        for (int d = 0; d < 3; ++d)
            for (int l = 0; l < kRK; ++l) {
                const double ck = (kGamma[l] + kRho[l]) * p->dt * M / 2.0 * kappa;
                const int n = (int)h->n[d];
                if (n == 1) {  // a single periodic z-plane (2D scheme): no z-solve
                    LineTables& lt = h->lines[d][l];
                    lt.n = 1;
                    lt.M = 1;
                    lt.periodic = 1;
                    lt.nw = lt.R = 0;
                    all.push_back({});
                    all.push_back({});
                    continue;
                }
                const LineFactors F = line_factors(n, p->bc[d], ck);
                if (!F.ok) {
                    free(h);
                    return CH_EINVAL;
                }
                const int mch = warp_chunk(n);
                all.push_back(warp_tables(F, mch));
                LineTables& lt = h->lines[d][l];
                lt.n = n;
                lt.M = mch;
                lt.periodic = F.periodic;
                const Interior I = h->esz == 8 ? interior_rows<double>(F) : interior_rows<float>(F);
                lt.r0 = I.r0;
                lt.r1 = I.r1;
                for (int m = 0; m < 5; ++m) lt.k[m] = I.k[m];
                total += align_up(all.back().size() * h->esz);
                // y and z lines also get column-solver tables when they fit
                int nw = 0, R = 0;
                // lines over 512 cells run the column solver only in its cluster form (FP32, even nx)
                const bool cluster_ok = CH_COLUMN_PAIRS && CH_COLUMN_CLUSTER && h->esz == 4 && h->n[0] % 2 == 0;
                if (d > 0 && col_shape(n, &nw, &R) && (nw <= 32 || (cluster_ok && CH_COLUMN_CLUSTER4))) {
                    lt.nw = nw;
                    lt.R = R;
                    all.push_back(col_tables(F, nw, R));
                } else {
                    lt.nw = lt.R = 0;
                    all.push_back({});
                }
                total += align_up(all.back().size() * h->esz);
            }
        if (cudaMalloc(&h->coef_buf, total) != cudaSuccess) {
            free(h);
            return CH_ENOMEM;
        }
        std::vector<unsigned char> host(total, 0);
        size_t off = 0;
        for (int q = 0; q < 2 * 3 * kRK; ++q) {
            const std::vector<double>& v = all[q];
            unsigned char* dst = host.data() + off;
            for (size_t e = 0; e < v.size(); ++e) {
                if (h->esz == 8)
                    ((double*)dst)[e] = v[e];
                else
                    ((float*)dst)[e] = (float)v[e];
            }
            LineTables& lt = h->lines[(q / 2) / kRK][(q / 2) % kRK];
            if (q % 2 == 0)
                lt.base = (char*)h->coef_buf + off;
            else
                lt.col = v.empty() ? nullptr : (char*)h->coef_buf + off;
            off += align_up(v.size() * h->esz);
        }
        if (cudaMemcpy(h->coef_buf, host.data(), total, cudaMemcpyHostToDevice) != cudaSuccess) rc = CH_ECUDA;
    }
    if (rc == CH_OK) {
        h->red_blocks = CH_RED_BLOCKS_PER_SM * 152;
        if (cudaMalloc(&h->red_partials, 2 * (size_t)h->red_blocks * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&h->red_out, 2 * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&h->status, sizeof(unsigned int)) != cudaSuccess)
            rc = CH_ENOMEM;
        else if (cudaMemset(h->status, 0, sizeof(unsigned int)) != cudaSuccess)
            rc = CH_ECUDA;
    }
    if (rc == CH_OK) rc = h->prec == CH_F64 ? set_smem_attrs<double>(h) : set_smem_attrs<float>(h);
    if (rc == CH_OK) encode_tmap_c(h);
    if (rc == CH_OK && p->ncx) rc = mr_build_tables(h, p->xf_coarse, p->yf_coarse, p->zf_coarse);
    if (rc == CH_OK && p->ncx) rc = rs_build_tables(h, p->xf_coarse, p->yf_coarse, p->zf_coarse);
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

int ch_diagnostics(ch_handle* h, double* mass, double* free_energy) {
    if (!h || !mass || !free_energy) return CH_EINVAL;
    double out[2] = {0.0, 0.0};
    const int rc = h->prec == CH_F64 ? reduce_both<double>(h, out) : reduce_both<float>(h, out);
    if (rc != CH_OK) return rc;
    *mass = out[0];
    *free_energy = out[1];
    return CH_OK;
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
        if (flag & 4u) return fail(h, CH_ETIMEOUT, "a tile load of the explicit kernel did not complete");
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
