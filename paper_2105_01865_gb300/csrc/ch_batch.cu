// Batched form: many independent Cahn-Hilliard boxes of uneven sizes and
// parameters advanced together (arXiv 2105.01865, Sec. 3 step applied box by
// box; the batching itself has no counterpart in the paper).
//
// One RK3 step of every box is 12 phases (3 substeps x [explicit RHS, x-,
// y-, z-line solve]).  Each phase is a flat list of work items over all
// boxes (explicit tiles, groups of 16 x-lines, y/z tiles of 64 two-column
// lines or 32-column shared-memory tiles).  Two
// schedules run the same item functions:
//  - persistent: one cooperative launch per step; CTAs walk the item list of
//    a phase, then meet at a grid barrier whose spin is bounded in time (on
//    expiry the kernel records CH_ETIMEOUT and returns);
//  - phased: one launch per phase, no device barrier.
// A small autotuner times the schedules, CTAs per SM, the explicit tiles' z
// extent and the item order, and keeps the fastest.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "ch_internal.h"
#include "ch_explicit2.cuh"
#include "ch_kernels.cuh"
#include "ch_cols2.cuh"
#include "line_tables.h"

using namespace chg;

namespace {

constexpr int kBThreads = 256;  // 8 warps per CTA in every phase
constexpr int kBWarps = 8;
constexpr unsigned kTimeoutFlag = 2u;

struct BoxDesc {
    float* C;
    float* H[2];
    float* r;
    int nx, ny, nz;
    int nlines_x;
    int M[3];
    RhsArgs<float> rhs[kRK];
    WCoef<float> lines[3][kRK];
    // y and z: rows per warp of the two-column solver (8 warps of R rows),
    // 0 where the line is too long and the shared-memory tile solver runs
    int colR[2];
    CCoef<float> cols[2][kRK];
};

struct BatchArgs {
    const BoxDesc* boxes;
    const int4* items[4];
    int nitems[4];
    unsigned* bar;          // [0] arrivals, [1] generation
    unsigned* status;
    unsigned expected;      // CTAs that must arrive at a barrier
    long long limit_ns;     // bounded wait per barrier
    int zchunk;
};

__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier with a bounded wait.  Returns false (and sets the timeout bit
// of *status) if the other CTAs did not arrive within limit_ns.
__device__ bool grid_barrier(const BatchArgs& A) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned* gen = A.bar + 1;
        const unsigned g = *gen;  // read before arriving
        __threadfence();
        if (atomicAdd(A.bar, 1u) == A.expected - 1) {
            atomicExch(A.bar, 0u);
            __threadfence();
            atomicAdd(A.bar + 1, 1u);
        } else {
            const long long t0 = global_ns();
            while (*gen == g) {
                if (global_ns() - t0 > A.limit_ns) {
                    atomicOr(A.status, kTimeoutFlag);
                    ok = 0;
                    break;
                }
                __nanosleep(128);
            }
        }
        __threadfence();
    }
    __syncthreads();
    __threadfence();
    return ok != 0;
}

// x-lines solved together by a warp: 2, or more for short lines (a lane then
// holds 8 rows in all), so the scans of short lines are shared by more rows
__host__ __device__ constexpr int x_lines_per_warp(int M) { return M >= 4 ? 2 : 8 / M; }

// kBWarps x x_lines_per_warp(M) consecutive x-lines
template <int M>
__device__ __forceinline__ void x_item(const BoxDesc& B, int line0, int l) {
    constexpr int L = x_lines_per_warp(M);
    const int warp = threadIdx.x >> 5;
    const int64_t line = (int64_t)line0 + L * warp;
    if (line < B.nlines_x) solve_x_lines<float, M, L>(B.r, line, B.nlines_x, B.nx, B.lines[0][l]);
}

// one 64-line tile of the two-column solver (y: UPDATE false, z: true)
template <int R, bool UPDATE>
__device__ __forceinline__ void cols_item(const BoxDesc& B, int tile, int l, unsigned char* smem, unsigned* status) {
    if (!UPDATE)
        solve_cols2_tile<float, R, kBWarps, false>(B.r, nullptr, B.nx, (int64_t)B.nx * B.ny, B.nx, B.cols[0][l],
                                                   status, tile, smem);
    else
        solve_cols2_tile<float, R, kBWarps, true>(B.r, B.C, B.nx, B.nx, (int64_t)B.nx * B.ny, B.cols[1][l], status,
                                                  tile, smem);
}

template <bool UPDATE>
__device__ __forceinline__ void cols_dispatch(const BoxDesc& B, int R, int tile, int l, unsigned char* smem,
                                              unsigned* status) {
    switch (R) {
        case 1: cols_item<1, UPDATE>(B, tile, l, smem, status); break;
        case 2: cols_item<2, UPDATE>(B, tile, l, smem, status); break;
        case 4: cols_item<4, UPDATE>(B, tile, l, smem, status); break;
        case 8: cols_item<8, UPDATE>(B, tile, l, smem, status); break;
        default: cols_item<16, UPDATE>(B, tile, l, smem, status); break;
    }
}

template <int M, bool UPDATE>
__device__ __forceinline__ void yz_item(const BoxDesc& B, int tile, int l, float* smem, unsigned* status) {
    if (!UPDATE)
        solve_yz_tile<float, M, false, kBWarps>(B.r, nullptr, B.nx, (int64_t)B.nx * B.ny, B.nx, B.lines[1][l], status,
                                                tile, smem);
    else
        solve_yz_tile<float, M, true, kBWarps>(B.r, B.C, B.nx, B.nx, (int64_t)B.nx * B.ny, B.lines[2][l], status,
                                               tile, smem);
}

// MAXM: the largest rows-per-lane of any box (4 or 8); smaller builds carry
// fewer solver variants and fewer registers.
template <int MAXM>
__device__ void run_phase(const BatchArgs& A, int ph, int l, float* smem) {
    const int n = A.nitems[ph];
    const int4* items = A.items[ph];
    for (int it = blockIdx.x; it < n; it += gridDim.x) {
        const int4 w = items[it];
        const BoxDesc& B = A.boxes[w.x];
        if (ph == 0) {
            explicit_tile2<float, false>(B.C, nullptr, nullptr, nullptr, B.H[(l + 1) & 1], B.H[l & 1], B.r, B.rhs[l],
                                         w.y, w.z, w.w, A.zchunk);
        } else if (ph == 1) {
            switch (B.M[0]) {
                case 1: x_item<1>(B, w.y, l); break;
                case 2: x_item<2>(B, w.y, l); break;
                case 4: x_item<4>(B, w.y, l); break;
                default: x_item<MAXM>(B, w.y, l); break;
            }
        } else if (w.z) {
            if (ph == 2)
                cols_dispatch<false>(B, B.colR[0], w.y, l, reinterpret_cast<unsigned char*>(smem), A.status);
            else
                cols_dispatch<true>(B, B.colR[1], w.y, l, reinterpret_cast<unsigned char*>(smem), A.status);
        } else {
            const int m = B.M[ph - 1];
            if (ph == 2) {
                switch (m) {
                    case 1: yz_item<1, false>(B, w.y, l, smem, A.status); break;
                    case 2: yz_item<2, false>(B, w.y, l, smem, A.status); break;
                    case 4: yz_item<4, false>(B, w.y, l, smem, A.status); break;
                    default: yz_item<MAXM, false>(B, w.y, l, smem, A.status); break;
                }
            } else {
                switch (m) {
                    case 1: yz_item<1, true>(B, w.y, l, smem, A.status); break;
                    case 2: yz_item<2, true>(B, w.y, l, smem, A.status); break;
                    case 4: yz_item<4, true>(B, w.y, l, smem, A.status); break;
                    default: yz_item<MAXM, true>(B, w.y, l, smem, A.status); break;
                }
            }
        }
    }
}

// One full RK3 step of every box in one cooperative launch.
template <int MAXM>
__global__ void __launch_bounds__(kBThreads, 3) ch_batch_persistent(BatchArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* smem = reinterpret_cast<float*>(smem_raw);
    // A barrier of an earlier launch gave up and left the arrival counter part
    // way: run nothing until ch_batch_sync has reported and cleared it (every
    // CTA reads the same word, written by a launch that has completed).
    if (*(volatile unsigned*)A.status & kTimeoutFlag) return;
    for (int l = 0; l < kRK; ++l)
        for (int ph = 0; ph < 4; ++ph) {
            run_phase<MAXM>(A, ph, l, smem);
            if (l == kRK - 1 && ph == 3) break;
            if (!grid_barrier(A)) return;
        }
}

// One phase of one substep for every box, specialised per phase so that each
// phase gets its own register allocation (the persistent kernel must carry
// the largest of all phases).
template <int PH, int MAXM>
__global__ void __launch_bounds__(kBThreads, PH == 0 ? 3 : 2) ch_batch_phase(BatchArgs A, int l) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    run_phase<MAXM>(A, PH, l, reinterpret_cast<float*>(smem_raw));
}

// FP64 mass of every box: blockIdx.y = box.
__global__ void __launch_bounds__(kRedThreads) batch_mass_partials(const BoxDesc* boxes, double* partials) {
    const BoxDesc& B = boxes[blockIdx.y];
    const int64_t N = (int64_t)B.nx * B.ny * B.nz;
    double acc = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * kRedThreads + threadIdx.x; e < N; e += (int64_t)gridDim.x * kRedThreads)
        acc += (double)B.C[e];
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kRedThreads) batch_mass_finish(const double* partials, int nb, const double* h3,
                                                                 double* out) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += kRedThreads) acc += partials[(size_t)blockIdx.x * nb + b];
    acc = block_sum(acc);
    if (threadIdx.x == 0) out[blockIdx.x] = acc * h3[blockIdx.x];
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// shared memory of the two-column tiles for rows-per-warp up to maxR
size_t cols2_smem_max(int maxR) {
    size_t m = Cols2Smem<float, 1, kBWarps, true>::kMax;
    if (maxR >= 2) m = std::max(m, Cols2Smem<float, 2, kBWarps, true>::kMax);
    if (maxR >= 4) m = std::max(m, Cols2Smem<float, 4, kBWarps, true>::kMax);
    if (maxR >= 8) m = std::max(m, Cols2Smem<float, 8, kBWarps, true>::kMax);
    if (maxR >= 16) m = std::max(m, Cols2Smem<float, 16, kBWarps, true>::kMax);
    return m;
}

bool batch_params_ok(const ch_params* b, int nbox) {
    if (!b || nbox < 1 || nbox > 65535) return false;
    for (int i = 0; i < nbox; ++i) {
        const ch_params& p = b[i];
        if (p.precision != CH_F32 || p.advect != 0 || p.scheme != CH_SCHEME_SPLIT) return false;
        if (p.ncx || p.ncy || p.ncz || p.xf_coarse || p.yf_coarse || p.zf_coarse) return false;
        if (p.nx < 6 || p.ny < 5 || p.nz < 5 || (p.nx & 1)) return false;
        if (p.nx > 256 || p.ny > 256 || p.nz > 256) return false;
        if (!(p.h > 0) || !(p.cn > 0) || !(p.pe > 0) || !(p.dt > 0) || !(p.w > 0)) return false;
        if (!std::isfinite(p.h) || !std::isfinite(p.cn) || !std::isfinite(p.pe) || !std::isfinite(p.dt) ||
            !std::isfinite(p.w))
            return false;
        for (int d = 0; d < 3; ++d)
            if (p.bc[d] != CH_PERIODIC && p.bc[d] != CH_NOFLUX) return false;
    }
    return true;
}

}  // namespace

struct ch_batch {
    int nbox = 0;
    std::vector<ch_params> params;
    cudaStream_t stream = nullptr;
    std::vector<float*> C;
    BoxDesc* d_boxes = nullptr;
    std::vector<BoxDesc> boxes;
    int4* d_items[4] = {nullptr, nullptr, nullptr, nullptr};
    int nitems[4] = {0, 0, 0, 0};
    void* coef_buf = nullptr;
    unsigned* d_bar = nullptr;
    unsigned* d_status = nullptr;
    double* d_partials = nullptr;
    double* d_out = nullptr;
    double* d_h3 = nullptr;
    int red_blocks = 64;
    // schedule
    int mode = 0;  // 0 persistent, 1 phased
    int blocks_per_sm = 2;
    int zchunk = 8;
    int lpt = 1;
    long long limit_ns = 2000000000LL;
    int poison = 0;
    int grid = 0;
    size_t smem = 0;
    int num_sms = 0;
    int max_m = 1;  // largest rows-per-lane of the warp solver over all boxes
    cudaGraphExec_t graph = nullptr;
    bool graph_ready = false;
    char err[512] = {0};
};

namespace {

int bfail(ch_batch* b, int code, const char* msg) {
    if (b) snprintf(b->err, sizeof(b->err), "%s", msg);
    return code;
}

#define CHB_CUDA(b, call)                                                                           \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) {                                                                    \
            snprintf((b)->err, sizeof((b)->err), "%s failed: %s", #call, cudaGetErrorString(e_));   \
            return CH_ECUDA;                                                                        \
        }                                                                                           \
    } while (0)

// Item lists for the current schedule (z extent of explicit tiles, order).
int build_items(ch_batch* b) {
    std::vector<std::pair<double, int4>> lists[4];
    for (int i = 0; i < b->nbox; ++i) {
        const ch_params& p = b->params[i];
        const int nx = (int)p.nx, ny = (int)p.ny, nz = (int)p.nz;
        const int bxn = (nx + kTX2 - 1) / kTX2, byn = (ny + kTY - 1) / kTY, bzn = (nz + b->zchunk - 1) / b->zchunk;
        for (int bz = 0; bz < bzn; ++bz)
            for (int by = 0; by < byn; ++by)
                for (int bx = 0; bx < bxn; ++bx) {
                    const double cost = (double)std::min(kTX2, nx - bx * kTX2) * std::min(kTY, ny - by * kTY) *
                                        std::min(b->zchunk, nz - bz * b->zchunk);
                    lists[0].push_back({cost, make_int4(i, bx, by, bz)});
                }
        const int nlx = ny * nz, xl = x_lines_per_warp(b->boxes[i].M[0]) * kBWarps;
        for (int l0 = 0; l0 < nlx; l0 += xl)
            lists[1].push_back({(double)std::min(xl, nlx - l0) * nx, make_int4(i, l0, 0, 0)});
        // y, z: 64-line two-column tiles (w = 1) or 32-column shared-memory tiles (w = 0)
        const BoxDesc& B = b->boxes[i];
        const int xb = (nx + 31) / 32, xb2 = (nx + 63) / 64;
        if (B.colR[0])
            for (int t = 0; t < xb2 * nz; ++t) lists[2].push_back({64.0 * ny, make_int4(i, t, 1, 0)});
        else
            for (int t = 0; t < xb * nz; ++t) lists[2].push_back({32.0 * warp_chunk(ny) * 32, make_int4(i, t, 0, 0)});
        if (B.colR[1])
            for (int t = 0; t < xb2 * ny; ++t) lists[3].push_back({64.0 * nz, make_int4(i, t, 1, 0)});
        else
            for (int t = 0; t < xb * ny; ++t) lists[3].push_back({32.0 * warp_chunk(nz) * 32, make_int4(i, t, 0, 0)});
    }
    for (int ph = 0; ph < 4; ++ph) {
        if (b->lpt)
            std::stable_sort(lists[ph].begin(), lists[ph].end(),
                             [](const std::pair<double, int4>& a, const std::pair<double, int4>& c) {
                                 return a.first > c.first;
                             });
        std::vector<int4> v(lists[ph].size());
        for (size_t q = 0; q < v.size(); ++q) v[q] = lists[ph][q].second;
        cudaFree(b->d_items[ph]);
        b->d_items[ph] = nullptr;
        b->nitems[ph] = (int)v.size();
        CHB_CUDA(b, cudaMalloc(&b->d_items[ph], std::max<size_t>(1, v.size()) * sizeof(int4)));
        CHB_CUDA(b, cudaMemcpy(b->d_items[ph], v.data(), v.size() * sizeof(int4), cudaMemcpyHostToDevice));
    }
    return CH_OK;
}

BatchArgs batch_args(const ch_batch* b) {
    BatchArgs A;
    A.boxes = b->d_boxes;
    for (int ph = 0; ph < 4; ++ph) {
        A.items[ph] = b->d_items[ph];
        A.nitems[ph] = b->nitems[ph];
    }
    A.bar = b->d_bar;
    A.status = b->d_status;
    A.expected = (unsigned)b->grid + (b->poison ? 1u : 0u);
    A.limit_ns = b->limit_ns;
    A.zchunk = b->zchunk;
    return A;
}

template <int MAXM>
int launch_step_m(ch_batch* b) {
    const BatchArgs A = batch_args(b);
    if (b->mode == 0) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)b->grid);
        cfg.blockDim = dim3(kBThreads);
        cfg.dynamicSmemBytes = b->smem;
        cfg.stream = b->stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        CHB_CUDA(b, cudaLaunchKernelEx(&cfg, ch_batch_persistent<MAXM>, A));
    } else {
        for (int l = 0; l < kRK; ++l)
            for (int ph = 0; ph < 4; ++ph) {
                // one CTA per item: the phase kernels hold no barrier
                const unsigned g = (unsigned)std::max(1, b->nitems[ph]);
                switch (ph) {
                    case 0: ch_batch_phase<0, MAXM><<<g, kBThreads, b->smem, b->stream>>>(A, l); break;
                    case 1: ch_batch_phase<1, MAXM><<<g, kBThreads, b->smem, b->stream>>>(A, l); break;
                    case 2: ch_batch_phase<2, MAXM><<<g, kBThreads, b->smem, b->stream>>>(A, l); break;
                    default: ch_batch_phase<3, MAXM><<<g, kBThreads, b->smem, b->stream>>>(A, l); break;
                }
                CHB_CUDA(b, cudaGetLastError());
            }
    }
    return CH_OK;
}

int launch_step(ch_batch* b) { return b->max_m <= 4 ? launch_step_m<4>(b) : launch_step_m<8>(b); }

template <int MAXM>
int set_attrs_batch(ch_batch* b, int* maxb) {
    CHB_CUDA(b, cudaFuncSetAttribute(ch_batch_persistent<MAXM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)b->smem));
    CHB_CUDA(b, cudaFuncSetAttribute(ch_batch_phase<0, MAXM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
    CHB_CUDA(b, cudaFuncSetAttribute(ch_batch_phase<1, MAXM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
    CHB_CUDA(b, cudaFuncSetAttribute(ch_batch_phase<2, MAXM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
    CHB_CUDA(b, cudaFuncSetAttribute(ch_batch_phase<3, MAXM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
    CHB_CUDA(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(maxb, ch_batch_persistent<MAXM>, kBThreads, b->smem));
    return CH_OK;
}

int configure(ch_batch* b) {
    if (b->graph_ready) {
        cudaGraphExecDestroy(b->graph);
        b->graph_ready = false;
    }
    int rc = build_items(b);
    if (rc != CH_OK) return rc;
    int maxb = 0;
    rc = b->max_m <= 4 ? set_attrs_batch<4>(b, &maxb) : set_attrs_batch<8>(b, &maxb);
    if (rc != CH_OK) return rc;
    if (maxb < 1) return bfail(b, CH_EINVAL, "batch kernel does not fit on an SM");
    b->blocks_per_sm = std::max(1, std::min(b->blocks_per_sm, maxb));
    b->grid = b->blocks_per_sm * b->num_sms;
    return CH_OK;
}

}  // namespace

extern "C" {

size_t ch_batch_workspace_bytes(const ch_params* boxes, int nbox) {
    if (!batch_params_ok(boxes, nbox)) return 0;
    size_t tot = 0;
    for (int i = 0; i < nbox; ++i) tot += 3 * align256((size_t)boxes[i].nx * boxes[i].ny * boxes[i].nz * sizeof(float));
    return tot;
}

int ch_batch_create(const ch_params* boxes, int nbox, void* const* C, void* work, size_t work_bytes, void* stream,
                    ch_batch** out) {
    if (!out) return CH_EINVAL;
    *out = nullptr;
    if (!batch_params_ok(boxes, nbox) || !C || !work || ((uintptr_t)work % 256)) return CH_EINVAL;
    for (int i = 0; i < nbox; ++i)
        if (!C[i] || ((uintptr_t)C[i] % 16)) return CH_EINVAL;
    if (work_bytes < ch_batch_workspace_bytes(boxes, nbox)) return CH_ENOMEM;
    ch_batch* b = new ch_batch();
    b->nbox = nbox;
    b->params.assign(boxes, boxes + nbox);
    for (auto& p : b->params) p.xf_coarse = p.yf_coarse = p.zf_coarse = nullptr;
    b->stream = (cudaStream_t)stream;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (!coop) b->mode = 1;

    // workspace carve + line tables of every box
    char* wb = (char*)work;
    std::vector<std::vector<double>> tabs;
    size_t coef_total = 0;
    b->boxes.resize(nbox);
    int maxM = 1, maxR = 0;
    for (int i = 0; i < nbox; ++i) {
        const ch_params& p = b->params[i];
        BoxDesc& B = b->boxes[i];
        const size_t bytes = align256((size_t)p.nx * p.ny * p.nz * sizeof(float));
        B.C = (float*)C[i];
        B.H[0] = (float*)wb;
        B.H[1] = (float*)(wb + bytes);
        B.r = (float*)(wb + 2 * bytes);
        wb += 3 * bytes;
        B.nx = (int)p.nx;
        B.ny = (int)p.ny;
        B.nz = (int)p.nz;
        B.nlines_x = (int)(p.ny * p.nz);
        const double mob = 1.0 / p.pe;
        const double kappa = p.w * p.cn * p.cn / (p.h * p.h * p.h * p.h);
        for (int l = 0; l < kRK; ++l) {
            RhsArgs<float>& a = B.rhs[l];
            a.nx = B.nx;
            a.ny = B.ny;
            a.nz = B.nz;
            a.bcx = p.bc[0];
            a.bcy = p.bc[1];
            a.bcz = p.bc[2];
            a.nfx = a.nfy = a.nfz = 0;
            a.inv_h = (float)(1.0 / p.h);
            a.inv_h2 = (float)(1.0 / (p.h * p.h));
            a.mob = (float)mob;
            a.dtg = (float)(p.dt * kGamma[l]);
            a.dtr = (float)(p.dt * kRho[l]);
            a.impl = (float)((kGamma[l] + kRho[l]) * p.dt * mob * kappa);
            a.eps = (float)p.weno_eps;
            a.has_prev = kRho[l] != 0.0;
        }
        const int64_t n[3] = {p.nx, p.ny, p.nz};
        for (int d = 0; d < 3; ++d) {
            B.M[d] = warp_chunk((int)n[d]);
            maxM = std::max(maxM, B.M[d]);
            int nw = 0, R = 0;
            if (d > 0) B.colR[d - 1] = (col_shape((int)n[d], &nw, &R) && nw == kBWarps) ? R : 0;
            for (int l = 0; l < kRK; ++l) {
                const double ck = (kGamma[l] + kRho[l]) * p.dt * mob / 2.0 * kappa;
                const LineFactors F = line_factors((int)n[d], p.bc[d], ck);
                if (!F.ok) {
                    delete b;
                    return CH_EINVAL;
                }
                tabs.push_back(warp_tables(F, B.M[d]));
                coef_total += align256(tabs.back().size() * sizeof(float));
                if (d > 0 && B.colR[d - 1]) {
                    tabs.push_back(col_tables(F, kBWarps, B.colR[d - 1]));
                    coef_total += align256(tabs.back().size() * sizeof(float));
                }
            }
            if (d > 0 && B.colR[d - 1]) maxR = std::max(maxR, B.colR[d - 1]);
        }
    }
    // dynamic shared memory: the larger of the y/z tile and the two-column buffers
    b->smem = (size_t)32 * maxM * 32 * sizeof(float);
    if (maxR) b->smem = std::max(b->smem, cols2_smem_max(maxR));
    b->max_m = maxM;
    int rc = CH_OK;
    if (cudaMalloc(&b->coef_buf, coef_total) != cudaSuccess) rc = CH_ENOMEM;
    if (rc == CH_OK) {
        std::vector<float> host(coef_total / sizeof(float), 0.f);
        size_t off = 0;
        int q = 0;
        for (int i = 0; i < nbox; ++i)
            for (int d = 0; d < 3; ++d)
                for (int l = 0; l < kRK; ++l) {
                    const int nd = (int)(d == 0 ? b->params[i].nx : d == 1 ? b->params[i].ny : b->params[i].nz);
                    const int per = b->params[i].bc[d] == CH_PERIODIC;
                    {
                        const std::vector<double>& t = tabs[q++];
                        for (size_t e = 0; e < t.size(); ++e) host[off / sizeof(float) + e] = (float)t[e];
                        const float* base = (const float*)((char*)b->coef_buf + off);
                        const WarpLayout L = warp_layout(b->boxes[i].M[d]);
                        WCoef<float>& w = b->boxes[i].lines[d][l];
                        w.fwd = base + L.fwd;
                        w.bwd = base + L.bwd;
                        w.W = base + L.W;
                        w.Z = base + L.Z;
                        w.Pf = base + L.Pf;
                        w.Pb = base + L.Pb;
                        w.S = base + L.S;
                        w.n = nd;
                        w.periodic = per;
                        off += align256(t.size() * sizeof(float));
                    }
                    if (d > 0 && b->boxes[i].colR[d - 1]) {
                        const std::vector<double>& t = tabs[q++];
                        for (size_t e = 0; e < t.size(); ++e) host[off / sizeof(float) + e] = (float)t[e];
                        const float* base = (const float*)((char*)b->coef_buf + off);
                        const ColLayout L = col_layout(kBWarps, b->boxes[i].colR[d - 1]);
                        CCoef<float>& c = b->boxes[i].cols[d - 1][l];
                        c.fwd = base + L.fwd;
                        c.bwd = base + L.bwd;
                        c.W = base + L.W;
                        c.Z = base + L.Z;
                        c.P = base + L.P;
                        c.Q = base + L.Q;
                        c.S = base + L.S;
                        c.fwdp = base + L.fwdp;
                        c.dinvp = base + L.dinvp;
                        c.bwdp = base + L.bwdp;
                        c.Wp = base + L.Wp;
                        c.Zp = base + L.Zp;
                        c.K = base + L.K;
                        c.n = nd;
                        c.periodic = per;
                        off += align256(t.size() * sizeof(float));
                    }
                }
        if (cudaMemcpy(b->coef_buf, host.data(), coef_total, cudaMemcpyHostToDevice) != cudaSuccess) rc = CH_ECUDA;
    }
    if (rc == CH_OK && (cudaMalloc(&b->d_boxes, nbox * sizeof(BoxDesc)) != cudaSuccess ||
                        cudaMalloc(&b->d_bar, 2 * sizeof(unsigned)) != cudaSuccess ||
                        cudaMalloc(&b->d_status, sizeof(unsigned)) != cudaSuccess ||
                        cudaMalloc(&b->d_partials, (size_t)nbox * b->red_blocks * sizeof(double)) != cudaSuccess ||
                        cudaMalloc(&b->d_out, nbox * sizeof(double)) != cudaSuccess ||
                        cudaMalloc(&b->d_h3, nbox * sizeof(double)) != cudaSuccess))
        rc = CH_ENOMEM;
    if (rc == CH_OK) {
        std::vector<double> h3(nbox);
        for (int i = 0; i < nbox; ++i) h3[i] = b->params[i].h * b->params[i].h * b->params[i].h;
        if (cudaMemcpy(b->d_boxes, b->boxes.data(), nbox * sizeof(BoxDesc), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(b->d_h3, h3.data(), nbox * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemset(b->d_bar, 0, 2 * sizeof(unsigned)) != cudaSuccess ||
            cudaMemset(b->d_status, 0, sizeof(unsigned)) != cudaSuccess)
            rc = CH_ECUDA;
    }
    if (rc == CH_OK) rc = configure(b);
    if (rc != CH_OK) {
        ch_batch_free(b);
        return rc;
    }
    *out = b;
    return CH_OK;
}

int ch_batch_free(ch_batch* b) {
    if (!b) return CH_EINVAL;
    if (b->graph_ready) cudaGraphExecDestroy(b->graph);
    for (int ph = 0; ph < 4; ++ph) cudaFree(b->d_items[ph]);
    cudaFree(b->coef_buf);
    cudaFree(b->d_boxes);
    cudaFree(b->d_bar);
    cudaFree(b->d_status);
    cudaFree(b->d_partials);
    cudaFree(b->d_out);
    cudaFree(b->d_h3);
    delete b;
    return CH_OK;
}

int ch_batch_set_schedule(ch_batch* b, int mode, int blocks_per_sm, int zchunk, int lpt) {
    if (!b) return CH_EINVAL;
    if (mode < 0 || mode > 1 || blocks_per_sm < 1 || blocks_per_sm > 8 || zchunk < 1 || zchunk > 64 || lpt < 0 ||
        lpt > 1)
        return bfail(b, CH_EINVAL, "ch_batch_set_schedule: bad argument");
    int coop = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (mode == 0 && !coop) return bfail(b, CH_EINVAL, "device has no cooperative launch");
    b->mode = mode;
    b->blocks_per_sm = blocks_per_sm;
    b->zchunk = zchunk;
    b->lpt = lpt;
    return configure(b);
}

int ch_batch_get_schedule(const ch_batch* b, int* out4) {
    if (!b || !out4) return CH_EINVAL;
    out4[0] = b->mode;
    out4[1] = b->blocks_per_sm;
    out4[2] = b->zchunk;
    out4[3] = b->lpt;
    return CH_OK;
}

int ch_batch_set_barrier_limit(ch_batch* b, int64_t limit_ns, int poison) {
    if (!b || limit_ns < 1000 || poison < 0 || poison > 1) return CH_EINVAL;
    b->limit_ns = limit_ns;
    b->poison = poison;
    if (b->graph_ready) {
        cudaGraphExecDestroy(b->graph);
        b->graph_ready = false;
    }
    return CH_OK;
}

int ch_batch_step(ch_batch* b, int64_t nsteps) {
    if (!b) return CH_EINVAL;
    if (nsteps < 0) return bfail(b, CH_EINVAL, "ch_batch_step: nsteps < 0");
    if (nsteps == 0) return CH_OK;
    if (b->stream == nullptr) {
        for (int64_t s = 0; s < nsteps; ++s) {
            const int rc = launch_step(b);
            if (rc != CH_OK) return rc;
        }
        return CH_OK;
    }
    if (!b->graph_ready) {
        cudaGraph_t g;
        CHB_CUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        const int rc = launch_step(b);
        cudaError_t e = cudaStreamEndCapture(b->stream, &g);
        if (rc != CH_OK) {
            if (e == cudaSuccess) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return bfail(b, CH_ECUDA, "batch graph capture failed");
        e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return bfail(b, CH_ECUDA, "batch graph instantiate failed");
        b->graph_ready = true;
    }
    for (int64_t s = 0; s < nsteps; ++s) CHB_CUDA(b, cudaGraphLaunch(b->graph, b->stream));
    return CH_OK;
}

int ch_batch_sync(ch_batch* b) {
    if (!b) return CH_EINVAL;
    unsigned flag = 0;
    CHB_CUDA(b, cudaMemcpyAsync(&flag, b->d_status, sizeof(flag), cudaMemcpyDeviceToHost, b->stream));
    CHB_CUDA(b, cudaStreamSynchronize(b->stream));
    if (!flag) return CH_OK;
    // clear the status and the barrier state left by an abandoned wait
    CHB_CUDA(b, cudaMemsetAsync(b->d_status, 0, sizeof(unsigned), b->stream));
    CHB_CUDA(b, cudaMemsetAsync(b->d_bar, 0, 2 * sizeof(unsigned), b->stream));
    CHB_CUDA(b, cudaStreamSynchronize(b->stream));
    if (flag & kTimeoutFlag) return bfail(b, CH_ETIMEOUT, "a batch grid barrier timed out");
    return bfail(b, CH_ENONFINITE, "non-finite value in a batch box");
}

int ch_batch_mass(ch_batch* b, double* out) {
    if (!b || !out) return CH_EINVAL;
    batch_mass_partials<<<dim3((unsigned)b->red_blocks, (unsigned)b->nbox), kRedThreads, 0, b->stream>>>(
        b->d_boxes, b->d_partials);
    CHB_CUDA(b, cudaGetLastError());
    batch_mass_finish<<<(unsigned)b->nbox, kRedThreads, 0, b->stream>>>(b->d_partials, b->red_blocks, b->d_h3,
                                                                        b->d_out);
    CHB_CUDA(b, cudaGetLastError());
    CHB_CUDA(b, cudaMemcpyAsync(out, b->d_out, b->nbox * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    return ch_batch_sync(b);
}

int ch_batch_autotune(ch_batch* b, int steps_per_trial, char* report, size_t report_len) {
    if (!b || steps_per_trial < 1) return CH_EINVAL;
    // keep the fields: trials advance the boxes, so C is saved and restored
    size_t total = 0;
    for (int i = 0; i < b->nbox; ++i) total += align256((size_t)b->params[i].nx * b->params[i].ny * b->params[i].nz * 4);
    void* save = nullptr;
    CHB_CUDA(b, cudaMalloc(&save, total));
    auto copy_all = [&](bool to_save) {
        size_t off = 0;
        for (int i = 0; i < b->nbox; ++i) {
            const size_t bytes = (size_t)b->params[i].nx * b->params[i].ny * b->params[i].nz * 4;
            char* s = (char*)save + off;
            cudaMemcpyAsync(to_save ? (void*)s : (void*)b->boxes[i].C, to_save ? (const void*)b->boxes[i].C : s, bytes,
                            cudaMemcpyDeviceToDevice, b->stream);
            off += align256(bytes);
        }
    };
    copy_all(true);
    struct Cand {
        int mode, bpsm, zc, lpt;
    };
    std::vector<Cand> cands;
    for (int mode = 0; mode < 2; ++mode)
        for (int bpsm : {1, 2, 3})
            for (int zc : {4, 8, 16})
                for (int lpt : {0, 1})
                    if (mode == 0 || bpsm == 1) cands.push_back({mode, bpsm, zc, lpt});
    std::string rep;
    double best = 1e30;
    Cand bc = {b->mode, b->blocks_per_sm, b->zchunk, b->lpt};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = CH_OK;
    for (const Cand& c : cands) {
        rc = ch_batch_set_schedule(b, c.mode, c.bpsm, c.zc, c.lpt);
        if (rc != CH_OK) {
            if (c.mode == 0) continue;  // no cooperative launch here
            break;
        }
        if (b->blocks_per_sm != c.bpsm) continue;  // occupancy cap: duplicate of a smaller setting
        rc = ch_batch_step(b, 1);
        if (rc != CH_OK) break;
        cudaEventRecord(e0, b->stream);
        rc = ch_batch_step(b, steps_per_trial);
        if (rc != CH_OK) break;
        cudaEventRecord(e1, b->stream);
        rc = ch_batch_sync(b);
        if (rc != CH_OK) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= steps_per_trial;
        char line[128];
        snprintf(line, sizeof(line), "mode=%s blocks_per_sm=%d zchunk=%d lpt=%d ms_per_step=%.4f\n",
                 c.mode ? "phased" : "persistent", c.bpsm, c.zc, c.lpt, ms);
        rep += line;
        if (ms < best) {
            best = ms;
            bc = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    copy_all(false);
    cudaStreamSynchronize(b->stream);
    cudaFree(save);
    if (rc != CH_OK) return rc;
    rc = ch_batch_set_schedule(b, bc.mode, bc.bpsm, bc.zc, bc.lpt);
    if (report && report_len) {
        char line[160];
        snprintf(line, sizeof(line), "chosen: mode=%s blocks_per_sm=%d zchunk=%d lpt=%d ms_per_step=%.4f\n",
                 bc.mode ? "phased" : "persistent", bc.bpsm, bc.zc, bc.lpt, best);
        rep += line;
        snprintf(report, report_len, "%s", rep.c_str());
    }
    return rc;
}

int ch_batch_launches_per_step(const ch_batch* b) { return b ? (b->mode == 0 ? 1 : 4 * kRK) : 0; }

const char* ch_batch_last_error(const ch_batch* b) { return b ? b->err : ""; }

}  // extern "C"
