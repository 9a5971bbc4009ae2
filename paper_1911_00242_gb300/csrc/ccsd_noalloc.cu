// Correlation energy without any device allocation.
//
// Some callers cannot allocate device memory while they use this library:
//  * code that runs inside a CUDA stream capture, where cudaMalloc is not
//    allowed;
//  * hosts whose allocator owns all device memory and forbids outside
//    allocations;
//  * latency-bound loops that must not pay for an allocation.
// ccsd_energy needs a handle, and ccsd_create allocates.  This entry point
// takes the problem data as plain device pointers instead.  Its only scratch
// -- one partial sum per momentum block -- lives in a fixed array in this
// file, which every GPU that loads the library keeps until the process exits.
#include "../../include/ccsd.h"

#include <cuda_runtime.h>

#include <mutex>

namespace {

constexpr int kMaxPartials = 32768;            // N_k^3 + 1 slots of 16 bytes: 512 KiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double2 g_energy_partials[kMaxPartials];

std::mutex g_mu;
double2* g_partials_addr[kMaxDevices] = {};    // device address of the array, per device

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// One block per momentum block (ki,kj,ka) of t2 writes
//   sum_ijab <ij||ab> (1/4 t_ij^ab + [ka == ki] 1/2 t_i^a t_j^b)
// to partials[block]; the last block writes sum_k sum_ia f_ia t_i^a.
// Every slot is overwritten, so nothing has to be cleared between calls.
__global__ void energy_blocks(const double2* __restrict__ t1, const double2* __restrict__ t2,
                              const double2* __restrict__ fov, const double2* __restrict__ oovv,
                              int N, int o, int v, double2* __restrict__ partials)
{
    __shared__ double sr[256], si[256];
    const int nblk = N * N * N;
    const int b = blockIdx.x;
    double er = 0.0, ei = 0.0;
    if (b < nblk) {
        const long long blk = (long long)o * o * v * v;
        const int ka = b % N, kj = (b / N) % N, ki = b / (N * N);
        const double2* g = oovv + (long long)b * blk;
        const double2* t = t2 + (long long)b * blk;
        for (long long e = threadIdx.x; e < blk; e += blockDim.x) {
            double2 amp = t[e];
            amp.x *= 0.25; amp.y *= 0.25;
            if (ka == ki) {
                long long r = e;                       // o^2 v^2 may exceed 2^31
                const int bb = (int)(r % v); r /= v;
                const int a = (int)(r % v); r /= v;
                const int j = (int)(r % o); const int i = (int)(r / o);
                const double2 q = cmul(t1[((long long)ki * o + i) * v + a], t1[((long long)kj * o + j) * v + bb]);
                amp.x += 0.5 * q.x; amp.y += 0.5 * q.y;
            }
            const double2 p = cmul(g[e], amp);
            er += p.x; ei += p.y;
        }
    } else {
        const long long n1 = (long long)N * o * v;
        for (long long e = threadIdx.x; e < n1; e += blockDim.x) {
            const double2 p = cmul(fov[e], t1[e]);
            er += p.x; ei += p.y;
        }
    }
    sr[threadIdx.x] = er; si[threadIdx.x] = ei;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) { sr[threadIdx.x] += sr[threadIdx.x + s]; si[threadIdx.x] += si[threadIdx.x + s]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[b] = make_double2(sr[0], si[0]);
}

// Fixed-order sum of the partials, divided by N_k (energy per unit cell).
__global__ void energy_finish(const double2* __restrict__ partials, int n, double inv_nk, double* __restrict__ out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double r = 0.0, im = 0.0;
        for (int i = 0; i < n; ++i) { r += partials[i].x; im += partials[i].y; }
        out[0] = r * inv_nk;
        out[1] = im * inv_nk;
    }
}

// Device address of the partials array on the current device, looked up once.
int partials_address(double2** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return CCSD_ERR_CUDA; }
    if (dev < 0 || dev >= kMaxDevices) return CCSD_ERR_INVALID;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_partials_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_energy_partials) != cudaSuccess || !p) { cudaGetLastError(); return CCSD_ERR_CUDA; }
        g_partials_addr[dev] = (double2*)p;
    }
    *out = g_partials_addr[dev];
    return CCSD_OK;
}

}  // namespace

extern "C" int ccsd_energy_noalloc(const int nk_dims[3], int nocc, int nvir, const void* f_ov, const void* oovv,
                                   const void* t1, const void* t2, void* e_out, void* stream)
{
    if (!nk_dims || !f_ov || !oovv || !t1 || !t2 || !e_out) return CCSD_ERR_INVALID;
    long long N = 1;
    for (int d = 0; d < 3; ++d) {
        // the bound ccsd_create applies; it also keeps N^3 below 2^63
        if (nk_dims[d] < 1 || nk_dims[d] > 64) return CCSD_ERR_INVALID;
        N *= nk_dims[d];
    }
    if (nocc < 1 || nvir < 1 || nocc > 256 || nvir > 512) return CCSD_ERR_INVALID;
    // one partial per momentum block of t2 plus one for the singles term
    if (N * N * N + 1 > kMaxPartials) return CCSD_ERR_INVALID;
    double2* partials = nullptr;
    int rc = partials_address(&partials);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int nparts = (int)(N * N * N + 1);
    energy_blocks<<<nparts, 256, 0, st>>>((const double2*)t1, (const double2*)t2, (const double2*)f_ov,
                                          (const double2*)oovv, (int)N, nocc, nvir, partials);
    energy_finish<<<1, 32, 0, st>>>(partials, nparts, 1.0 / (double)N, (double*)e_out);
    if (cudaGetLastError() != cudaSuccess) return CCSD_ERR_CUDA;
    return CCSD_OK;
}
