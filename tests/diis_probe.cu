// Host build of the DIIS coefficient solve (csrc/diis.h), for test_diis_host.py.
#include "../paper_1911_00242_gb300/csrc/diis.h"

#include <vector>

extern "C" int probe_diis(const double* gram, int m, double* c) {
    std::vector<std::vector<double>> g((size_t)m, std::vector<double>((size_t)m));
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) g[(size_t)i][(size_t)j] = gram[(size_t)i * m + j];
    return ccsdk::diis_coefficients(g, m, c) ? 1 : 0;
}

// The canonical blocks of a grid; arrays have room for N^3 entries.
extern "C" int probe_canonical(const int* dims, int* nc, int* cblk, double* cw, int* cmap) {
    ccsdk::KGrid kg;
    kg.init(dims);
    std::vector<int> b, m;
    std::vector<double> w;
    if (!ccsdk::diis_canonical_blocks(kg, b, w, m)) return 0;
    *nc = (int)b.size();
    for (size_t p = 0; p < b.size(); ++p) { cblk[p] = b[p]; cw[p] = w[p]; }
    for (size_t f = 0; f < m.size(); ++f) cmap[f] = m[f];
    return 1;
}

// The canonical blocks' targets (csrc/diis.h, the map the device extrapolation writes by);
// ctgt has room for 4 N^3 entries.
extern "C" int probe_targets(const int* dims, int* nc, int* ctgt) {
    ccsdk::KGrid kg;
    kg.init(dims);
    std::vector<int> b, m, t;
    std::vector<double> w;
    if (!ccsdk::diis_canonical_blocks(kg, b, w, m)) return 0;
    if (!ccsdk::diis_canonical_targets(m, (long long)b.size(), t)) return 0;
    *nc = (int)b.size();
    for (size_t i = 0; i < t.size(); ++i) ctgt[i] = t[i];
    return 1;
}
