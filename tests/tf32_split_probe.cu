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

void probe_f32_rn(const double* x, float* out, int n) {
    for (int i = 0; i < n; ++i) out[i] = f32_rn(x[i]);
}

void probe_f32_residual(const double* x, float* f, float* r, int* ok, int n) {
    for (int i = 0; i < n; ++i) ok[i] = f32_round_with_residual(x[i], f[i], r[i]) ? 1 : 0;
}

}  // extern "C"
