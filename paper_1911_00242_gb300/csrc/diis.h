// DIIS host code: the canonical blocks of the history and the Pulay
// extrapolation coefficients.
//
// Pulay (DIIS) extrapolation coefficients.  Given the Gram matrix
// B_ij = Re <e_i|e_j> of the last m update errors, the coefficients c minimise
// |sum_i c_i e_i| subject to sum_i c_i = 1; with a Lagrange multiplier l they solve
//   [ B  -1 ] [c]   [ 0]
//   [-1   0 ] [l] = [-1],
// here by Gaussian elimination with partial pivoting.  Host-only, so that the CPU
// tests check this code itself.
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

// gram[i][j] for i, j < m (any row-indexable type); c receives m coefficients.
// Returns false if the system is exactly singular (a zero pivot).
template <class Gram>
bool diis_coefficients(const Gram& gram, int m, double* c) {
    const int S = m + 1;
    std::vector<double> A((size_t)S * S, 0.0), b((size_t)S, 0.0);
    for (int i = 0; i < m; ++i) for (int j = 0; j < m; ++j) A[(size_t)i * S + j] = gram[i][j];
    for (int i = 0; i < m; ++i) { A[(size_t)i * S + m] = -1.0; A[(size_t)m * S + i] = -1.0; }
    b[(size_t)m] = -1.0;
    for (int col = 0; col < S; ++col) {
        int p = col;
        for (int r = col + 1; r < S; ++r) if (std::fabs(A[(size_t)r * S + col]) > std::fabs(A[(size_t)p * S + col])) p = r;
        if (p != col) { for (int k = 0; k < S; ++k) std::swap(A[(size_t)col * S + k], A[(size_t)p * S + k]); std::swap(b[col], b[p]); }
        const double piv = A[(size_t)col * S + col];
        if (piv == 0.0) return false;
        for (int r = col + 1; r < S; ++r) {
            const double f = A[(size_t)r * S + col] / piv;
            for (int k = col; k < S; ++k) A[(size_t)r * S + k] -= f * A[(size_t)col * S + k];
            b[r] -= f * b[col];
        }
    }
    std::vector<double> xs((size_t)S, 0.0);
    for (int r = S - 1; r >= 0; --r) {
        double s = b[r];
        for (int k = r + 1; k < S; ++k) s -= A[(size_t)r * S + k] * xs[k];
        xs[r] = s / A[(size_t)r * S + r];
    }
    for (int j = 0; j < m; ++j) c[j] = xs[j];
    return true;
}

}  // namespace ccsdk
