// Pulay (DIIS) extrapolation coefficients, host code.  Given the Gram matrix
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

namespace ccsdk {

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
