// Momentum arithmetic on a regular k grid (host code): flat index k of the grid
// point (c0, c1, c2), and the fourth momentum of a conserving quadruple.
#pragma once
#include <vector>

namespace ccsdk {

struct KGrid {
    int n[3] = {1, 1, 1};
    int N = 1;
    std::vector<int> c0, c1, c2;
    void init(const int* d) {
        n[0] = d[0]; n[1] = d[1]; n[2] = d[2];
        N = n[0] * n[1] * n[2];
        c0.resize(N); c1.resize(N); c2.resize(N);
        for (int k = 0; k < N; ++k) { c0[k] = k / (n[1] * n[2]); c1[k] = (k / n[2]) % n[1]; c2[k] = k % n[2]; }
    }
    static int md(int x, int m) { x %= m; return x < 0 ? x + m : x; }
    int flat(int a, int b, int c) const { return (md(a, n[0]) * n[1] + md(b, n[1])) * n[2] + md(c, n[2]); }
    // k1 + k2 - k3 (momentum conservation k1 + k2 = k3 + k4, paper Sec. 3.2.5)
    int k4(int k1, int k2, int k3) const {
        return flat(c0[k1] + c0[k2] - c0[k3], c1[k1] + c1[k2] - c1[k3], c2[k1] + c2[k2] - c2[k3]);
    }
};

}  // namespace ccsdk
