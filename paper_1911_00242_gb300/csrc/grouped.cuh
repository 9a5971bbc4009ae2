// Grouped launches: one kernel launch runs the same plan step of many independent
// problems (the batched form and the serving loop).
//
// Every elementwise and row-wise step of the iteration is an operation struct with
//   __device__ void run(long long vb, long long nvb) const
// that does the work of block vb of a grid of nvb blocks (grid-stride loops over its
// elements or rows).  A plain launch runs op.run(blockIdx.x, gridDim.x); a grouped
// launch concatenates the members' grids: block w belongs to member m with
// prefix[m] <= w < prefix[m+1] and runs ops[m].run(w - prefix[m], prefix[m+1] - prefix[m]).
// Each member keeps its own grid size, so its partial sums (reductions) come out in
// the same order as in a plain launch.
#pragma once
#include <cuda_runtime.h>

namespace ccsdk {

template <class Op>
__global__ void __launch_bounds__(256) grouped_op_kernel(const Op* __restrict__ ops, const long long* __restrict__ prefix,
                                                         int nmem)
{
    const long long w = blockIdx.x;
    int lo = 0, hi = nmem - 1;
    while (lo < hi) {                       // last member whose prefix <= w
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= w) lo = mid; else hi = mid - 1;
    }
    const Op op = ops[lo];
    op.run(w - prefix[lo], prefix[lo + 1] - prefix[lo]);
}

// A plain launch of one operation: block b of the grid runs op.run(b, gridDim.x).
template <class Op>
__global__ void __launch_bounds__(256) op_kernel(const Op op) { op.run(blockIdx.x, gridDim.x); }

// Zeroes n complex elements (the batched counterpart of a memset step).
struct ZeroOp {
    double2* p; long long n;
    __device__ void run(long long vb, long long nvb) const {
        for (long long e = vb * blockDim.x + threadIdx.x; e < n; e += nvb * blockDim.x) p[e] = make_double2(0.0, 0.0);
    }
};

}  // namespace ccsdk
