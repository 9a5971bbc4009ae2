// Host build of the double-float arithmetic of the Ozaki form (csrc/dfloat.cuh), for
// the CPU tests in test_dfloat_host.py.  Compile with -ffp-contract=off so that the
// host operations round once each, as the device intrinsics do.
#include "../paper_1911_00242_gb300/csrc/dfloat.cuh"

using ccsdk::df;

extern "C" {

// x, y, z, out: n pairs (h, l)
void probe_df_add(const float* x, const float* y, float* out, int n) {
    for (int i = 0; i < n; ++i) {
        const df r = df(x[2 * i], x[2 * i + 1]) + df(y[2 * i], y[2 * i + 1]);
        out[2 * i] = r.h; out[2 * i + 1] = r.l;
    }
}

void probe_df_sub(const float* x, const float* y, float* out, int n) {
    for (int i = 0; i < n; ++i) {
        const df r = df(x[2 * i], x[2 * i + 1]) - df(y[2 * i], y[2 * i + 1]);
        out[2 * i] = r.h; out[2 * i + 1] = r.l;
    }
}

void probe_df_mul(const float* x, const float* y, float* out, int n) {
    for (int i = 0; i < n; ++i) {
        const df r = df(x[2 * i], x[2 * i + 1]) * df(y[2 * i], y[2 * i + 1]);
        out[2 * i] = r.h; out[2 * i + 1] = r.l;
    }
}

void probe_df_fma(const float* x, const float* y, const float* z, float* out, int n) {
    for (int i = 0; i < n; ++i) {
        const df r = ccsdk::fma(df(x[2 * i], x[2 * i + 1]), df(y[2 * i], y[2 * i + 1]), df(z[2 * i], z[2 * i + 1]));
        out[2 * i] = r.h; out[2 * i + 1] = r.l;
    }
}

void probe_df_from_double(const double* x, float* out, int n) {
    for (int i = 0; i < n; ++i) {
        const df r(x[i]);
        out[2 * i] = r.h; out[2 * i + 1] = r.l;
    }
}

}  // extern "C"
