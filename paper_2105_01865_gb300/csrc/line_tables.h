// Host-side (FP64) factorisation of the line operators (I + c A_d) of the
// approximately factorised Crank-Nicolson step (arXiv 2105.01865, Eqs.
// eq-fac-1..3, with A_d of Eq. eq-a3d) and the tables of the warp-scan line
// solver.  Plain C++, no CUDA: shared by the library and host-only checks.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <tuple>
#include <utility>
#include <vector>

namespace chg {

constexpr int kBcPeriodic = 0;   // same values as CH_PERIODIC / CH_NOFLUX / CH_DIRICHLET
constexpr int kBcDirichlet = 2;
constexpr int kBcNoflux = 1;

// Banded LU without pivoting of a pentadiagonal matrix given by its bands
// e (j, j-2), c (j, j-1), d (j, j), a (j, j+1), b (j, j+2).
struct BandLU {
    std::vector<double> l1, l2, u0, u1, u2;
};

inline BandLU band_lu(const std::vector<double>& e, const std::vector<double>& c, const std::vector<double>& d,
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

inline std::vector<double> band_solve(const BandLU& f, std::vector<double> x) {
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

inline bool invert4(const double* A, double* out) {
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

// Factors of (I + ck B) where B applies [1,-4,6,-4,1] along a line of n
// cells with wrapped (periodic) or mirrored (wall) neighbours: the band LU
// with the diagonal folded in (y_j = r_j - l1 y_{j-1} - l2 y_{j-2};
// x_j = y_j/u0 - (u1/u0) x_{j+1} - (u2/u0) x_{j+2}) and, for periodic lines,
// the Woodbury correction of the corner entries: out = x - Z S (W^T r).
struct LineFactors {
    int n = 0;
    bool periodic = false;
    std::vector<double> l1, l2, dinv, u1s, u2s;
    std::vector<double> W, Z;  // n x 4 each (periodic)
    double S[16] = {0};
    // corner form of the correction: s = K y_c with y_c = (Mb^-1 r) at rows
    // (0, 1, n-2, n-1), K = S V_c (V^T restricted to those columns)
    double K[16] = {0};
    bool ok = false;
};

inline LineFactors line_factors(int n, int bc, double ck) {
    LineFactors F;
    F.n = n;
    F.periodic = bc == kBcPeriodic;
    std::vector<double> e(n, 0.0), c(n, 0.0), d(n, 1.0), a(n, 0.0), b(n, 0.0);
    std::vector<std::tuple<int, int, double>> corner;  // out-of-band (row, col, value)
    const double stencil[5] = {1.0, -4.0, 6.0, -4.0, 1.0};
    for (int i = 0; i < n; ++i) {
        for (int s = -2; s <= 2; ++s) {
            int j = i + s;
            double sign = 1.0;  // a Dirichlet ghost is the negated mirror
            if (F.periodic) {
                j = ((j % n) + n) % n;
            } else {
                if (j < 0) {
                    j = -1 - j;
                    if (bc == kBcDirichlet) sign = -1.0;
                }
                if (j >= n) {
                    j = 2 * n - 1 - j;
                    if (bc == kBcDirichlet) sign = -1.0;
                }
            }
            const double val = sign * ck * stencil[s + 2];
            switch (j - i) {
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
    F.l1 = f.l1;
    F.l2 = f.l2;
    F.dinv.resize(n);
    F.u1s.resize(n);
    F.u2s.resize(n);
    for (int j = 0; j < n; ++j) {
        F.dinv[j] = 1.0 / f.u0[j];
        F.u1s[j] = f.u1[j] / f.u0[j];
        F.u2s[j] = f.u2[j] / f.u0[j];
    }
    if (!F.periodic) {
        F.ok = true;
        return F;
    }
    // M = Mb + U V^T, U = [e_r] for the corner rows r, V^T = those rows' corner
    // part.  M^-1 r = y - Z (I + V^T Z)^-1 V^T y with y = Mb^-1 r, Z = Mb^-1 U,
    // and V^T y = W^T r with W = Mb^-T V.
    const int R[4] = {0, 1, n - 2, n - 1};
    std::vector<double> Vt(4 * (size_t)n, 0.0);
    for (auto& t : corner) {
        int m = -1;
        for (int q = 0; q < 4; ++q)
            if (R[q] == std::get<0>(t)) m = q;
        Vt[(size_t)m * n + std::get<1>(t)] += std::get<2>(t);
    }
    std::vector<double> et(n, 0.0), ct(n, 0.0), at(n, 0.0), bt(n, 0.0);
    for (int j = 0; j < n; ++j) {
        if (j >= 2) et[j] = b[j - 2];
        if (j >= 1) ct[j] = a[j - 1];
        if (j + 1 < n) at[j] = c[j + 1];
        if (j + 2 < n) bt[j] = e[j + 2];
    }
    const BandLU ft = band_lu(et, ct, d, at, bt);
    F.W.assign(4 * (size_t)n, 0.0);
    F.Z.assign(4 * (size_t)n, 0.0);
    for (int m = 0; m < 4; ++m) {
        std::vector<double> vcol(Vt.begin() + (size_t)m * n, Vt.begin() + (size_t)(m + 1) * n);
        const std::vector<double> wcol = band_solve(ft, vcol);
        std::vector<double> ucol(n, 0.0);
        ucol[R[m]] = 1.0;
        const std::vector<double> zcol = band_solve(f, ucol);
        for (int j = 0; j < n; ++j) {
            F.W[(size_t)j * 4 + m] = wcol[j];
            F.Z[(size_t)j * 4 + m] = zcol[j];
        }
    }
    double cap[16];
    for (int p = 0; p < 4; ++p)
        for (int q = 0; q < 4; ++q) {
            double s = (p == q) ? 1.0 : 0.0;
            for (int j = 0; j < n; ++j) s += Vt[(size_t)p * n + j] * F.Z[(size_t)j * 4 + q];
            cap[p * 4 + q] = s;
        }
    F.ok = invert4(cap, F.S);
    // V^T y only reads y at the corner rows: K = S V_c
    const int cols[4] = {0, 1, n - 2, n - 1};
    for (int p = 0; p < 4; ++p)
        for (int q = 0; q < 4; ++q) {
            double acc = 0.0;
            for (int m = 0; m < 4; ++m) acc += F.S[p * 4 + m] * Vt[(size_t)m * n + cols[q]];
            F.K[p * 4 + q] = acc;
        }
    return F;
}

// Interior rows of a factorised line operator: the LU factors of a constant-
// coefficient banded matrix converge geometrically away from the line's ends,
// so in the field precision they are exactly constant over a middle range of
// rows, and the periodic correction vectors W, Z (rows of the inverse banded
// matrix at the corners) decay there below 2^-80 of their largest entry.
// Rows [r0, r1) are those where every factor rounds (to the field precision)
// to its value at row n/2 and W, Z are negligible; k holds those constants
// (l1, l2, 1/u0, u1/u0, u2/u0).  The solver then uses the constants instead of
// the per-row tables there and drops the negligible Woodbury terms (whose
// effect on any output is below 2^-70 of it, far under FP64 rounding).
struct Interior {
    int r0 = 0, r1 = 0;
    double k[5] = {0, 0, 0, 0, 0};
};

template <typename T>
Interior interior_rows(const LineFactors& F) {
    Interior I;
    const int n = F.n, mid = n / 2;
    if (n < 8) return I;
    double wmax = 0.0, zmax = 0.0;
    if (F.periodic)
        for (int j = 0; j < 4 * n; ++j) {
            wmax = std::max(wmax, std::fabs(F.W[j]));
            zmax = std::max(zmax, std::fabs(F.Z[j]));
        }
    const double tiny = std::ldexp(1.0, -80);
    auto same = [&](int j) {
        if ((T)F.l1[j] != (T)F.l1[mid] || (T)F.l2[j] != (T)F.l2[mid] || (T)F.dinv[j] != (T)F.dinv[mid] ||
            (T)F.u1s[j] != (T)F.u1s[mid] || (T)F.u2s[j] != (T)F.u2s[mid])
            return false;
        if (F.periodic)
            for (int m = 0; m < 4; ++m)
                if (std::fabs(F.W[(size_t)j * 4 + m]) > tiny * wmax || std::fabs(F.Z[(size_t)j * 4 + m]) > tiny * zmax)
                    return false;
        return true;
    };
    if (!same(mid)) return I;
    int a = mid, b = mid + 1;
    while (a > 0 && same(a - 1)) --a;
    while (b < n && same(b)) ++b;
    I.r0 = a;
    I.r1 = b;
    I.k[0] = F.l1[mid];
    I.k[1] = F.l2[mid];
    I.k[2] = F.dinv[mid];
    I.k[3] = F.u1s[mid];
    I.k[4] = F.u2s[mid];
    return I;
}

// Rows per lane of the warp-scan solver: the smallest power of two M with
// 32 M >= n (n <= 1024).
inline int warp_chunk(int n) {
    int m = 1;
    while (32 * m < n) m *= 2;
    return m;
}

// Offsets (in elements) of the warp-scan tables inside one block.
struct WarpLayout {
    size_t fwd, bwd, W, Z, Pf, Pb, S, total;
};

inline WarpLayout warp_layout(int M) {
    WarpLayout L;
    size_t off = 0;
    L.fwd = off; off += (size_t)M * 32 * 4;
    L.bwd = off; off += (size_t)M * 32 * 2;
    L.W = off;   off += (size_t)M * 32 * 4;
    L.Z = off;   off += (size_t)M * 32 * 4;
    L.Pf = off;  off += 5 * 32 * 4;
    L.Pb = off;  off += 5 * 32 * 4;
    L.S = off;   off += 16;
    L.total = (off + 63) / 64 * 64;
    return L;
}

// 2x2 row-major matrix product a * b.
inline void mat2_mul(const double* a, const double* b, double* out) {
    const double r0 = a[0] * b[0] + a[1] * b[2], r1 = a[0] * b[1] + a[1] * b[3];
    const double r2 = a[2] * b[0] + a[3] * b[2], r3 = a[2] * b[1] + a[3] * b[3];
    out[0] = r0; out[1] = r1; out[2] = r2; out[3] = r3;
}

// Tables of the warp-scan solver for chunk size M (see warp_line_solve):
// per row (row j = lane*M + i stored at [i][lane]) the forward (l1, l2,
// 1/u0, 0) and backward (u1/u0, u2/u0) coefficients and the Woodbury rows;
// per lane and scan step s the transfer matrices of the lane span.  Rows
// j >= n are padding with zero coefficients.
inline std::vector<double> warp_tables(const LineFactors& F, int M) {
    const WarpLayout L = warp_layout(M);
    std::vector<double> t(L.total, 0.0);
    const int n = F.n;
    auto row = [&](int lane, int i) { return lane * M + i; };
    for (int lane = 0; lane < 32; ++lane)
        for (int i = 0; i < M; ++i) {
            const int j = row(lane, i);
            const size_t k = (size_t)i * 32 + lane;
            if (j >= n) continue;
            t[L.fwd + 4 * k + 0] = F.l1[j];
            t[L.fwd + 4 * k + 1] = F.l2[j];
            t[L.fwd + 4 * k + 2] = F.dinv[j];
            t[L.bwd + 2 * k + 0] = F.u1s[j];
            t[L.bwd + 2 * k + 1] = F.u2s[j];
            if (F.periodic)
                for (int m = 0; m < 4; ++m) {
                    t[L.W + 4 * k + m] = F.W[(size_t)j * 4 + m];
                    t[L.Z + 4 * k + m] = F.Z[(size_t)j * 4 + m];
                }
        }
    // chunk transfer matrices: forward P_l = A_{b-1} ... A_a with
    // A_j = [[-l1_j, -l2_j], [1, 0]]; backward Q_l = B_a ... B_{b-1} with
    // B_j = [[-u1s_j, -u2s_j], [1, 0]]; padding rows are [[0,0],[1,0]].
    std::vector<double> P(32 * 4), Q(32 * 4);
    for (int lane = 0; lane < 32; ++lane) {
        double p[4] = {1, 0, 0, 1}, q[4] = {1, 0, 0, 1};
        for (int i = 0; i < M; ++i) {
            const int j = row(lane, i);
            const double A[4] = {j < n ? -F.l1[j] : 0.0, j < n ? -F.l2[j] : 0.0, 1.0, 0.0};
            mat2_mul(A, p, p);  // p = A_j * p
        }
        for (int i = M - 1; i >= 0; --i) {
            const int j = row(lane, i);
            const double B[4] = {j < n ? -F.u1s[j] : 0.0, j < n ? -F.u2s[j] : 0.0, 1.0, 0.0};
            mat2_mul(B, q, q);  // q = B_j * q, giving B_a ... B_{b-1}
        }
        for (int m = 0; m < 4; ++m) {
            P[lane * 4 + m] = p[m];
            Q[lane * 4 + m] = q[m];
        }
    }
    for (int s = 0; s < 5; ++s) {
        const int d = 1 << s;
        for (int lane = 0; lane < 32; ++lane) {
            // forward span over lanes lane-d+1 .. lane: P_lane ... P_{lane-d+1}
            double sp[4] = {1, 0, 0, 1};
            if (lane >= d)
                for (int k = lane - d + 1; k <= lane; ++k) mat2_mul(&P[k * 4], sp, sp);
            // backward span over lanes lane .. lane+d-1: Q_lane ... Q_{lane+d-1}
            double sq[4] = {1, 0, 0, 1};
            if (lane + d < 32)
                for (int k = lane + d - 1; k >= lane; --k) mat2_mul(&Q[k * 4], sq, sq);
            for (int m = 0; m < 4; ++m) {
                t[L.Pf + ((size_t)s * 32 + lane) * 4 + m] = sp[m];
                t[L.Pb + ((size_t)s * 32 + lane) * 4 + m] = sq[m];
            }
        }
    }
    if (F.periodic)
        for (int m = 0; m < 16; ++m) t[L.S + m] = F.S[m];
    return t;
}

}  // namespace chg

namespace chg {

// Tables of the column solver (lanes = 32 adjacent lines, warp w = rows
// [w R, w R + R)): per row (l1, l2, 1/u0, 0), (u1/u0, u2/u0), Woodbury W and Z
// rows (zero padding past n), then per warp-chunk the forward transfer matrix
// P_w = A_{b-1} ... A_a and the backward one Q_w = B_a ... B_{b-1}.
struct ColLayout {
    size_t fwd, bwd, W, Z, P, Q, S;
    size_t fwdp, dinvp, bwdp, Wp, Zp;  // the same rows as duplicated pairs (two-column form)
    size_t K;                          // corner-form correction matrix (two-column form)
    size_t total;
};

// Cluster form of the two-column solver: lines of 257..1024 cells over CTAs
// of kClusterNW warps.
constexpr int kClusterNW = 16;

inline ColLayout col_layout(int nw, int R) {
    ColLayout L;
    const size_t rows = (size_t)nw * R;
    size_t off = 0;
    L.fwd = off; off += rows * 4;
    L.bwd = off; off += rows * 2;
    L.W = off;   off += rows * 4;
    L.Z = off;   off += rows * 4;
    L.P = off;   off += (size_t)nw * 4;
    L.Q = off;   off += (size_t)nw * 4;
    L.S = off;   off += 16;
    L.fwdp = off;  off += rows * 4;
    L.dinvp = off; off += rows * 2;
    L.bwdp = off;  off += rows * 4;
    L.Wp = off;    off += rows * 8;
    L.Zp = off;    off += rows * 8;
    L.K = off;     off += 16;
    L.total = (off + 63) / 64 * 64;
    return L;
}

inline std::vector<double> col_tables(const LineFactors& F, int nw, int R) {
    const ColLayout L = col_layout(nw, R);
    std::vector<double> t(L.total, 0.0);
    const int n = F.n;
    for (int j = 0; j < n; ++j) {
        t[L.fwd + 4 * (size_t)j + 0] = F.l1[j];
        t[L.fwd + 4 * (size_t)j + 1] = F.l2[j];
        t[L.fwd + 4 * (size_t)j + 2] = F.dinv[j];
        t[L.bwd + 2 * (size_t)j + 0] = F.u1s[j];
        t[L.bwd + 2 * (size_t)j + 1] = F.u2s[j];
        // two-column form: negated multipliers duplicated for paired FMAs
        for (int e = 0; e < 2; ++e) {
            t[L.fwdp + 4 * (size_t)j + e] = -F.l1[j];
            t[L.fwdp + 4 * (size_t)j + 2 + e] = -F.l2[j];
            t[L.dinvp + 2 * (size_t)j + e] = F.dinv[j];
            t[L.bwdp + 4 * (size_t)j + e] = -F.u1s[j];
            t[L.bwdp + 4 * (size_t)j + 2 + e] = -F.u2s[j];
        }
        if (F.periodic)
            for (int m = 0; m < 4; ++m) {
                t[L.W + 4 * (size_t)j + m] = F.W[(size_t)j * 4 + m];
                t[L.Z + 4 * (size_t)j + m] = F.Z[(size_t)j * 4 + m];
                for (int e = 0; e < 2; ++e) {
                    t[L.Wp + 8 * (size_t)j + 2 * m + e] = F.W[(size_t)j * 4 + m];
                    t[L.Zp + 8 * (size_t)j + 2 * m + e] = -F.Z[(size_t)j * 4 + m];
                }
            }
    }
    for (int w = 0; w < nw; ++w) {
        double p[4] = {1, 0, 0, 1}, q[4] = {1, 0, 0, 1};
        for (int i = 0; i < R; ++i) {
            const int j = w * R + i;
            const double A[4] = {j < n ? -F.l1[j] : 0.0, j < n ? -F.l2[j] : 0.0, 1.0, 0.0};
            mat2_mul(A, p, p);
        }
        for (int i = R - 1; i >= 0; --i) {
            const int j = w * R + i;
            const double B[4] = {j < n ? -F.u1s[j] : 0.0, j < n ? -F.u2s[j] : 0.0, 1.0, 0.0};
            mat2_mul(B, q, q);
        }
        for (int m = 0; m < 4; ++m) {
            t[L.P + 4 * (size_t)w + m] = p[m];
            t[L.Q + 4 * (size_t)w + m] = q[m];
        }
    }
    if (F.periodic)
        for (int m = 0; m < 16; ++m) {
            t[L.S + m] = F.S[m];
            t[L.K + m] = F.K[m];
        }
    return t;
}

// Column-solver shape for a line of n cells: nw warps of R rows (powers of
// two; R <= 16 keeps a warp's rows in registers at full occupancy).  Returns
// false for lines longer than 512.
#ifndef CH_COLUMN_MAXR
#define CH_COLUMN_MAXR 16
#endif
inline bool col_shape(int n, int* nw, int* R) {
    if (n <= 128) {
        int r = 1;
        while (8 * r < n) r *= 2;
        *nw = 8;
        *R = r;
        if (r > CH_COLUMN_MAXR) {  // more warps of fewer register rows
            *R = CH_COLUMN_MAXR;
            *nw = 128 / CH_COLUMN_MAXR;
        }
        return true;
    }
    if (n <= 256) {
        *R = CH_COLUMN_MAXR;
        *nw = 256 / CH_COLUMN_MAXR;
        return *nw <= 32;
    }
    if (n <= 512) {
        *nw = 32;
        *R = 16;
        return true;
    }
    if (n <= 1024) {  // cluster form only (four CTAs of 16 warps)
        *nw = 64;
        *R = 16;
        return true;
    }
    return false;
}

}  // namespace chg
