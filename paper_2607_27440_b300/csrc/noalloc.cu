// klst_apply_pencil_noalloc: the float64 pencil operator y = (A - omega B) x with its
// workspace in a fixed device array instead of memory allocated per call.
//
// Who needs this: callers that cannot call cudaMalloc at the moment they apply the operator,
// e.g. a host framework that owns all device memory through its own pool and forbids
// allocations from libraries during its steady-state loop, a latency-critical serving loop
// where a device allocation (and the implicit synchronisation it may cause) would stall
// other streams, or code that must not fail with out-of-memory halfway through a solve.
// klst_apply_pencil allocates its moment workspace on every call; this variant uses the
// array below, which every GPU that loads the library holds until the process exits.
#include <mutex>

#include "factor.cuh"

namespace klst {

int moments_dev(klst_pencil p, const double2* x, int64_t ldx, int nrhs, double2* mwork, double2* mpart,
                int ngroups, cudaStream_t s, const int* done);
int pencil_rows_dev(klst_pencil p, const double2* m, const double2* x, int64_t ldx, int nrhs, const double2* omega,
                    int mode, const double2* b, int mask_b, double2* y, double* normpart, cudaStream_t s,
                    const int* done, int df_arith);

// 4 MiB of scratch per device: shifts [nrhs], moments [nrhs][4 nx] and per-group moment
// partial sums [nrhs][groups][4 nx], all complex128.
constexpr size_t kNoallocScratchBytes = size_t(4) << 20;
constexpr int kNoallocGroups = 32;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array for the current device, resolved once per device.
static int noalloc_scratch(void** out) {
    int dev = -1;
    KLST_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device index %d out of range for the fixed-scratch operator", dev);
        return KLST_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)", __FILE__, __LINE__);
        g_noalloc_ptr[dev] = ptr;
    }
    *out = g_noalloc_ptr[dev];
    return KLST_OK;
}

size_t noalloc_bytes_needed(const klst_pencil p, int nrhs) {
    const int ng = std::min(p->nxi, kNoallocGroups);
    return sizeof(double2) * ((size_t)nrhs + (size_t)nrhs * 4 * p->nx + (size_t)nrhs * ng * 4 * p->nx);
}

}  // namespace klst

using namespace klst;

extern "C" size_t klst_apply_pencil_noalloc_capacity(void) { return kNoallocScratchBytes; }

extern "C" int klst_apply_pencil_noalloc(klst_pencil p, const void* x, void* y, int32_t nrhs, const double* omega,
                                         klst_stream stream) {
    if (!p || !x || !y || nrhs < 1) { set_error("invalid arguments to klst_apply_pencil_noalloc"); return KLST_EINVAL; }
    if (x == y) { set_error("x and y may not alias"); return KLST_EINVAL; }
    const size_t need = noalloc_bytes_needed(p, nrhs);
    if (need > kNoallocScratchBytes) {
        set_error("klst_apply_pencil_noalloc: nx=%d, nrhs=%d needs %zu bytes of scratch; the fixed array holds %zu "
                  "(use fewer right-hand sides per call, or klst_apply_pencil)",
                  p->nx, nrhs, need, kNoallocScratchBytes);
        return KLST_EINVAL;
    }
    void* base = nullptr;
    int rc = noalloc_scratch(&base);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int ng = std::min(p->nxi, kNoallocGroups);
    double2* om = (double2*)base;
    double2* mwork = om + nrhs;
    double2* mpart = mwork + (size_t)nrhs * 4 * p->nx;
    // Every value read below is written first in this call: the shifts by the copy, the moments
    // and partial sums by their kernels, so nothing needs clearing between calls.
    if (omega) KLST_CK(cudaMemcpyAsync(om, omega, sizeof(double2) * nrhs, cudaMemcpyHostToDevice, s));
    rc = moments_dev(p, (const double2*)x, p->n, nrhs, mwork, mpart, ng, s, nullptr);
    if (rc) return rc;
    return pencil_rows_dev(p, mwork, (const double2*)x, p->n, nrhs, omega ? om : nullptr, 0, nullptr, 0, (double2*)y,
                           nullptr, s, nullptr, 0);
}
