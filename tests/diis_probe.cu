// Host build of the DIIS coefficient solve (csrc/diis.h), for test_diis_host.py.
#include "../paper_1911_00242_gb300/csrc/diis.h"

#include <vector>

extern "C" int probe_diis(const double* gram, int m, double* c) {
    std::vector<std::vector<double>> g((size_t)m, std::vector<double>((size_t)m));
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) g[(size_t)i][(size_t)j] = gram[(size_t)i * m + j];
    return ccsdk::diis_coefficients(g, m, c) ? 1 : 0;
}
