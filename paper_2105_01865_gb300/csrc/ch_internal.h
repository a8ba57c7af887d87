// Internal declarations shared by the translation units of libch.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <vector>

#include "../../include/ch.h"

namespace chg {

constexpr int kRK = 3;  // RK3 substeps (Sec. 3)
constexpr int kMaxCoarseLine = 2048;  // coarse cells per direction (one x-line per warp in shared memory)

// Low-storage RK3 coefficients (Sec. 3 cites the scheme without printing it):
// gamma, rho per substep; alpha = gamma + rho weights the Crank-Nicolson step.
constexpr double kGamma[kRK] = {8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0};
constexpr double kRho[kRK] = {0.0, -17.0 / 60.0, -5.0 / 12.0};

// Warp-scan tables of one factorised line operator (I + c A_d) of one
// direction and substep, in the handle's precision (device memory).
struct LineTables {
    const void* base;  // block laid out by warp_layout(M)
    int n;             // cells along the line
    int M;             // rows per lane (32 M >= n)
    int periodic;
    const void* col;   // column-solver block (col_layout(nw, R)), or null
    int nw, R;         // column-solver warps per CTA and rows per warp
    int r0, r1;        // interior rows with constant factors (interior_rows)
    double k[5];       // their l1, l2, 1/u0, u1/u0, u2/u0
};

}  // namespace chg

struct ch_handle {
    ch_params p;
    int prec;           // CH_F32 / CH_F64
    size_t esz;         // element size
    int64_t n[3];       // nx, ny, nz
    int64_t nf[3];      // face planes per direction
    int64_t ncell;
    cudaStream_t stream;
    void* C;
    // workspace regions
    void* H[2];
    void* r;
    void* vel[3];
    void* vel_c[3];     // coarse face velocity
    void* grad_c[3];    // coarse normal gradients
    void* mr_plane;     // transfer intermediate (y, then z)
    int64_t nc[3];      // coarse cells
    int64_t ncf[3];     // coarse face planes
    // library-owned device memory
    void* coef_buf;
    chg::LineTables lines[3][chg::kRK];
    double* red_partials;
    double* red_out;
    unsigned int* status;
    int red_blocks;
    // multiple-resolution tables (device)
    int32_t* mr_start[3];
    double* mr_w[3];
    double* mr_coords;  // device copy of coarse face coordinates (x, y, z concatenated)
    // down-sampling tables: per coarse cell index, the first of 4 fine nodes and
    // the weights (doubles [nc][4] then floats [nc][4])
    int32_t* rs_start[3];
    double* rs_w[3];
    double* rs_coords;  // fine faces (x, y, z) then coarse centres (x, y, z)
    // CUDA graph of one full step
    cudaGraphExec_t graph;
    int graph_ready;
    int launches_per_step;
    // FP32: a 3D tensor map of C with a 72 x 14 x 1 box for the explicit
    // kernel's tile loads (the bytes of a CUtensorMap; tmap_ok when encoded)
    unsigned char tmap_c[128];
    int tmap_ok;
    char err[512];
};

namespace chg {

inline int fail(ch_handle* h, int code, const char* fmt, ...) {
    if (h) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(h->err, sizeof(h->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

#define CHG_CUDA(h, call)                                                                  \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return chg::fail((h), CH_ECUDA, "%s failed: %s (%s:%d)", #call,                \
                             cudaGetErrorString(e_), __FILE__, __LINE__);                  \
    } while (0)

// launchers shared with the adjoint (ch_step.cu), in the handle's precision
int launch_explicit_any(ch_handle* h, int l, const void* C, const void* Hprev, void* Hout, void* r);
int launch_solve_any(ch_handle* h, int l, int dir, void* a, void* Cupd);
int launch_step_any(ch_handle* h, void* C);  // one full step of the field C (direct launches)
// -div(uC) alone into Hout (the standard scheme's advection; ch_step.cu)
int launch_advection_any(ch_handle* h, const void* C, void* Hout);
// one substep of the standard explicit scheme (ch_standard.cu); ev: 5 events or NULL
int launch_substep_standard(ch_handle* h, int l, cudaEvent_t* ev);

// multi-resolution entry points implemented in ch_mr.cu
int mr_build_tables(ch_handle* h, const double* xf, const double* yf, const double* zf);
void mr_destroy(ch_handle* h);
int mr_tables_launch(ch_handle* h, const double* faces, int nc, int periodic, int nq, const double* queries,
                     int32_t* start, double* w);
// down-sampling tables (ch_restrict.cu), built by ch_create after mr_build_tables
int rs_build_tables(ch_handle* h, const double* xf, const double* yf, const double* zf);

}  // namespace chg
