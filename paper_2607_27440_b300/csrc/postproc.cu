// Post-processing of the base flow and of eigenvectors (Sec. 5): the translational non-equilibrium
// measure E_neq of Eq. L2norm (formed with the base state, see k_base_state), and for eigenvectors the
// macroscopic perturbations (rho^, u^, v^, E^)(x_j) -- the perturbation moments of Sec. 2.2, the same
// functionals V^H the shift-invert apply reduces over the velocity nodes -- with the velocity
// normalisation |U^| = sqrt(|u^|^2 + |v^|^2) of Eq. Unormpert.
#include <vector>

#include "factor.cuh"

namespace klst {

int moments_dev(klst_pencil p, const double2* x, int64_t ldx, int nrhs, double2* mwork, double2* mpart,
                int ngroups, cudaStream_t s, const int* done);

// umax[v] = max_j sqrt(|u^_v(j)|^2 + |v^_v(j)|^2), one warp per vector (fixed reduction order)
__global__ void k_unorm_max(const double2* __restrict__ m, int nx, double* __restrict__ umax) {
    const int v = blockIdx.x, lane = threadIdx.x;
    const double2* mv = m + (size_t)v * 4 * nx;
    double best = 0.0;
    for (int j = lane; j < nx; j += 32) best = fmax(best, sqrt(abs2(mv[nx + j]) + abs2(mv[2 * nx + j])));
    for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
    if (lane == 0) umax[v] = best;
}

}  // namespace klst

using namespace klst;

extern "C" int klst_base_noneq(klst_pencil p, double* eneq_host) {
    if (!p || !eneq_host) { set_error("invalid arguments to klst_base_noneq"); return KLST_EINVAL; }
    KLST_CK(cudaMemcpyAsync(eneq_host, p->eneq, sizeof(double) * p->nx, cudaMemcpyDeviceToHost, p->stream));
    KLST_CK(cudaStreamSynchronize(p->stream));
    return KLST_OK;
}

extern "C" int klst_eigvec_macro(klst_pencil p, const void* q, int32_t nvec, double* macro_host, double* umax_host,
                                 klst_stream stream) {
    if (!p || !q || nvec < 1 || !macro_host) { set_error("invalid arguments to klst_eigvec_macro"); return KLST_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    const int ng = pencil_work_groups(p);
    double2 *mw = nullptr, *mp = nullptr;
    double* um = nullptr;
    cudaError_t e;
    if ((e = dmalloc((void**)&mw, sizeof(double2) * 4 * p->nx * (size_t)nvec, s)) != cudaSuccess ||
        (e = dmalloc((void**)&mp, sizeof(double2) * 4 * p->nx * (size_t)ng * nvec, s)) != cudaSuccess ||
        (e = dmalloc((void**)&um, sizeof(double) * nvec, s)) != cudaSuccess) {
        dfree(mw, s);
        dfree(mp, s);
        return cuda_fail(e, "cudaMalloc", __FILE__, __LINE__);
    }
    int rc = moments_dev(p, (const double2*)q, p->n, nvec, mw, mp, ng, s, nullptr);
    if (rc == KLST_OK) {
        k_unorm_max<<<nvec, 32, 0, s>>>(mw, p->nx, um);
        note_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) rc = cuda_fail(e, "unorm", __FILE__, __LINE__);
    }
    if (rc == KLST_OK) {
        if ((e = cudaMemcpyAsync(macro_host, mw, sizeof(double2) * 4 * p->nx * (size_t)nvec, cudaMemcpyDeviceToHost,
                                 s)) != cudaSuccess ||
            (umax_host && (e = cudaMemcpyAsync(umax_host, um, sizeof(double) * nvec, cudaMemcpyDeviceToHost, s)) !=
                              cudaSuccess) ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            rc = cuda_fail(e, "macro copy", __FILE__, __LINE__);
    }
    dfree(mw, s);
    dfree(mp, s);
    dfree(um, s);
    return rc;
}
