// DIIS code: the canonical blocks of the history (host) and the Pulay
// extrapolation coefficients (host and device).
//
// Pulay (DIIS) extrapolation coefficients.  Given the Gram matrix
// B_ij = Re <e_i|e_j> of the last m update errors, the coefficients c minimise
// |sum_i c_i e_i| subject to sum_i c_i = 1; with a Lagrange multiplier l they solve
//   [ B  -1 ] [c]   [ 0]
//   [-1   0 ] [l] = [-1],
// here by Gaussian elimination with partial pivoting.  The CPU tests build this
// header for the host and check this code itself.
#pragma once
#include <cmath>
#include <utility>
#include <vector>

#include "kgrid.h"

namespace ccsdk {

// The DIIS history holds t1 and the canonical blocks of t2 only: t2 is
// antisymmetric, t2[kj][ki][ka](j, i, a, b) = t2[ki][kj][kb](i, j, b, a)
// = -t2[ki][kj][ka](i, j, a, b) with kb = ki + kj - ka (paper Sec. 2), so the blocks
// with ki <= kj and ka <= kb determine all others.
//   cblk[p]: full block index (ki N + kj) N + ka of canonical block p;
//   cw[p]:   the number of full blocks it stands for (its weight in the full inner
//            product: 2 for ki < kj times 2 for ka < kb);
//   cmap[f]: 4 p + 2 swap_ij + swap_ab for every full block f, where p is the
//            canonical block f is read from with those index swaps (sign -1 when
//            exactly one swap applies).
// Returns false if some block has no canonical partner (not possible on a grid).
inline bool diis_canonical_blocks(const KGrid& kg, std::vector<int>& cblk, std::vector<double>& cw,
                                  std::vector<int>& cmap) {
    const int N = kg.N;
    const long long N3 = (long long)N * N * N;
    cblk.clear(); cw.clear();
    cmap.assign((size_t)N3, 0);
    std::vector<int> canon((size_t)N3, -1);
    for (int ki = 0; ki < N; ++ki) for (int kj = ki; kj < N; ++kj) for (int ka = 0; ka < N; ++ka) {
        const int kb = kg.k4(ki, kj, ka);
        if (ka > kb) continue;
        const int f = (int)(((long long)ki * N + kj) * N + ka);
        canon[(size_t)f] = (int)cblk.size();
        cblk.push_back(f);
        cw.push_back((ki < kj ? 2.0 : 1.0) * (ka < kb ? 2.0 : 1.0));
    }
    for (int ki = 0; ki < N; ++ki) for (int kj = 0; kj < N; ++kj) for (int ka = 0; ka < N; ++ka) {
        const int kb = kg.k4(ki, kj, ka);
        const int sij = ki > kj ? 1 : 0, sab = ka > kb ? 1 : 0;
        const int c = (int)((((long long)(sij ? kj : ki)) * N + (sij ? ki : kj)) * N + (sab ? kb : ka));
        if (canon[(size_t)c] < 0) return false;
        cmap[(size_t)(((long long)ki * N + kj) * N + ka)] = canon[(size_t)c] * 4 + sij * 2 + sab;
    }
    return true;
}

// The inverse of cmap: for canonical block p, ctgt[4 p + t] (t < 4) = 4 f + 2 swap_ij +
// swap_ab for each full block f that is read from p (cmap[f] >> 2 == p), in increasing
// f, and -1 past the last.  The device extrapolation writes each canonical element to
// these blocks.  Returns false if some canonical block would stand for more than four
// full blocks (not possible on a grid: its weight is at most 2 x 2).
inline bool diis_canonical_targets(const std::vector<int>& cmap, long long nc, std::vector<int>& ctgt) {
    ctgt.assign((size_t)nc * 4, -1);
    for (size_t f = 0; f < cmap.size(); ++f) {
        const long long p = cmap[f] >> 2;
        if (p < 0 || p >= nc) return false;
        int t = 0;
        while (t < 4 && ctgt[(size_t)p * 4 + t] >= 0) ++t;
        if (t == 4) return false;
        ctgt[(size_t)p * 4 + t] = (int)(4 * f) + (cmap[f] & 3);
    }
    return true;
}

#ifdef __CUDACC__
#define CCSD_HD __host__ __device__
#else
#define CCSD_HD
#endif

constexpr int DIIS_MAX = 8;     // deepest history

// gram[i][j] for i, j < m <= DIIS_MAX; c receives m coefficients.  Returns false if
// the system is exactly singular (a zero pivot).  The same code runs on the host
// (ccsd_iterate) and on the device (grouped iterations of the batched form).
CCSD_HD inline bool diis_solve(const double (*gram)[DIIS_MAX], int m, double* c) {
    const int S = m + 1;
    double A[DIIS_MAX + 1][DIIS_MAX + 1], b[DIIS_MAX + 1], xs[DIIS_MAX + 1];
    for (int i = 0; i < S; ++i) { b[i] = 0.0; for (int j = 0; j < S; ++j) A[i][j] = 0.0; }
    for (int i = 0; i < m; ++i) for (int j = 0; j < m; ++j) A[i][j] = gram[i][j];
    for (int i = 0; i < m; ++i) { A[i][m] = -1.0; A[m][i] = -1.0; }
    b[m] = -1.0;
    for (int col = 0; col < S; ++col) {
        int p = col;
        for (int r = col + 1; r < S; ++r) {
            const double x = A[r][col] < 0 ? -A[r][col] : A[r][col];
            const double y = A[p][col] < 0 ? -A[p][col] : A[p][col];
            if (x > y) p = r;
        }
        if (p != col) {
            for (int k = 0; k < S; ++k) { const double t = A[col][k]; A[col][k] = A[p][k]; A[p][k] = t; }
            const double t = b[col]; b[col] = b[p]; b[p] = t;
        }
        const double piv = A[col][col];
        if (piv == 0.0) return false;
        for (int r = col + 1; r < S; ++r) {
            const double f = A[r][col] / piv;
            for (int k = col; k < S; ++k) A[r][k] -= f * A[col][k];
            b[r] -= f * b[col];
        }
    }
    for (int r = S - 1; r >= 0; --r) {
        double s = b[r];
        for (int k = r + 1; k < S; ++k) s -= A[r][k] * xs[k];
        xs[r] = s / A[r][r];
    }
    for (int j = 0; j < m; ++j) c[j] = xs[j];
    return true;
}

// The host entry: gram is any row-indexable type (m <= DIIS_MAX).
template <class Gram>
bool diis_coefficients(const Gram& gram, int m, double* c) {
    double g[DIIS_MAX][DIIS_MAX];
    for (int i = 0; i < m; ++i) for (int j = 0; j < m; ++j) g[i][j] = gram[i][j];
    return diis_solve(g, m, c);
}

}  // namespace ccsdk
