// Host build of the mixed form's TF32 split (csrc/tf32_split.cuh), for the CPU tests in
// test_tf32_split_host.py.
#include "../paper_1911_00242_gb300/csrc/tf32_split.cuh"

using namespace ccsdk;

extern "C" {

void probe_tf32_round(const float* x, float* out, int n) {
    for (int i = 0; i < n; ++i) out[i] = tf32_round(x[i]);
}

void probe_split_tf32f(const float* x, float* big, float* small, int n) {
    for (int i = 0; i < n; ++i) split_tf32f(x[i], big[i], small[i]);
}

void probe_split_tf32(const double* x, float* big, float* small, int n) {
    for (int i = 0; i < n; ++i) split_tf32(x[i], big[i], small[i]);
}

}  // extern "C"
