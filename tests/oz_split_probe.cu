// Host build of the Ozaki form's operand splitting (csrc/ozaki_split.cuh) and tile
// schedule (csrc/ozaki_schedule.cuh), for the CPU tests in test_ozaki_scheme.py: the
// row exponent, the fixed-point scales and the BF16 digit patterns, exactly as the
// embedding kernels compute them, and the windows and unit split of the GEMM kernel.
#include "../paper_1911_00242_gb300/csrc/ozaki_split.cuh"
#include "../paper_1911_00242_gb300/csrc/ozaki_schedule.cuh"

using namespace ccsdk;

extern "C" {

int probe_row_exponent(const double* x, int n) {
    unsigned long long m = 0;
    for (int i = 0; i < n; ++i) {
        const unsigned long long a = abs_bits(x[i]);
        m = a > m ? a : m;
    }
    return oz_row_exponent(m);
}

// out[i * s + p] = BF16 pattern of digit p of x[i] under the row exponent E
void probe_split(const double* x, int n, int s, int E, uint16_t* out) {
    const double fx = oz_fixed_scale(s, E);
    for (int i = 0; i < n; ++i) oz_split(x[i], fx, s, out + (long long)i * s);
}

void probe_scales(int s, int E, double* fixed, float* row) {
    *fixed = oz_fixed_scale(s, E);
    *row = oz_row_scale(E);
}

int probe_kwin(int s) { return oz_kwin(s); }

void probe_unit_range(int nch, int S, int kstages, int nsplit, int split, int* u0, int* u1) {
    oz_unit_range(nch, S, kstages, nsplit, split, *u0, *u1);
}

}  // extern "C"
