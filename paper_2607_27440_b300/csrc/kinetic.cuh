// Device helpers of the kinetic model shared by the pencil build and the BE-BGK base-flow solver:
// the 2-D reduced Maxwellian, block-wide sums and a small dense solve.
#pragma once
#include "common.cuh"

namespace klst {

// g^e = rho / (pi T) exp(-((xi_x - u)^2 + xi_y^2) / T) (transverse bulk velocity zero)
__device__ __forceinline__ double maxw(double rho, double u, double T, double xx, double xy) {
    double dx = xx - u;
    return rho / (M_PI * T) * exp(-(dx * dx + xy * xy) / T);
}

// Block-wide sum of NV doubles per thread; result broadcast to all threads.
template <int NV>
__device__ void block_sum(double (&v)[NV], double* sm /* >= 32*NV */) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        double a = v[i];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) sm[wid * NV + i] = a;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            double a = lane < nw ? sm[lane * NV + i] : 0.0;
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane == 0) sm[32 * NV + i] = a;
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = sm[32 * NV + i];
    __syncthreads();
}

// Solve the small dense system J d = r (n <= 4) by Gaussian elimination with partial pivoting.
__device__ inline void small_solve(int n, double* J /* n*n row-major */, double* r) {
    for (int p = 0; p < n; ++p) {
        int piv = p;
        for (int i = p + 1; i < n; ++i)
            if (fabs(J[i * n + p]) > fabs(J[piv * n + p])) piv = i;
        if (piv != p) {
            for (int c = 0; c < n; ++c) { double t = J[p * n + c]; J[p * n + c] = J[piv * n + c]; J[piv * n + c] = t; }
            double t = r[p]; r[p] = r[piv]; r[piv] = t;
        }
        for (int i = p + 1; i < n; ++i) {
            double f = J[i * n + p] / J[p * n + p];
            for (int c = p; c < n; ++c) J[i * n + c] -= f * J[p * n + c];
            r[i] -= f * r[p];
        }
    }
    for (int p = n - 1; p >= 0; --p) {
        double s = r[p];
        for (int c = p + 1; c < n; ++c) s -= J[p * n + c] * r[c];
        r[p] = s / J[p * n + p];
    }
}

}  // namespace klst
