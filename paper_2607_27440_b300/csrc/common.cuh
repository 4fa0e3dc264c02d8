// Internal helpers shared by the kLST CUDA sources (not part of the public ABI).
#pragma once
#include <atomic>
#include <mutex>

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

#include "klst.h"

namespace klst {

// ------------------------------------------------------------------ errors
void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define KLST_CK(call)                                                            \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) return ::klst::cuda_fail(e_, #call, __FILE__, __LINE__); \
    } while (0)

#define KLST_CK_LAUNCH() KLST_CK(cudaGetLastError())

// device status bits (klst::Status::flags)
enum : int {
    ST_SINGULAR = 1,   // zero pivot in a block or capacitance inverse
    ST_NOCONV_QR = 4,  // small Schur QR iteration limit
    ST_BREAKDOWN = 8,  // Arnoldi breakdown (invariant subspace)
    ST_REFINE = 16,    // a mixed-precision apply ended its refinement sweeps above refine_tol
    ST_TIMEOUT = 32    // a bounded device-side wait gave up
};

// ------------------------------------------------------------------ complex arithmetic
template <typename T> struct cplx;
template <> struct cplx<double> { using type = double2; };
template <> struct cplx<float> { using type = float2; };

__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
__host__ __device__ __forceinline__ float2 mkf(float a, float b) { return make_float2(a, b); }

__host__ __device__ __forceinline__ double2 operator+(double2 a, double2 b) { return mk(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 operator-(double2 a, double2 b) { return mk(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 operator-(double2 a) { return mk(-a.x, -a.y); }
__host__ __device__ __forceinline__ double2 operator*(double2 a, double2 b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 operator*(double s, double2 a) { return mk(s * a.x, s * a.y); }
__host__ __device__ __forceinline__ double2 conj(double2 a) { return mk(a.x, -a.y); }
__host__ __device__ __forceinline__ double abs2(double2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ double2 cinv(double2 a) {
    double d = 1.0 / abs2(a);
    return mk(a.x * d, -a.y * d);
}
// a += b * c
__host__ __device__ __forceinline__ void cfma(double2& a, double2 b, double2 c) {
    a.x = fma(b.x, c.x, a.x); a.x = fma(-b.y, c.y, a.x);
    a.y = fma(b.x, c.y, a.y); a.y = fma(b.y, c.x, a.y);
}
// a += conj(b) * c
__host__ __device__ __forceinline__ void cfma_conj(double2& a, double2 b, double2 c) {
    a.x = fma(b.x, c.x, a.x); a.x = fma(b.y, c.y, a.x);
    a.y = fma(b.x, c.y, a.y); a.y = fma(-b.y, c.x, a.y);
}

__host__ __device__ __forceinline__ float2 operator+(float2 a, float2 b) { return mkf(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 operator-(float2 a, float2 b) { return mkf(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 operator-(float2 a) { return mkf(-a.x, -a.y); }
__host__ __device__ __forceinline__ float2 operator*(float2 a, float2 b) {
    return mkf(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float abs2(float2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ float2 cinv(float2 a) {
    float d = 1.0f / abs2(a);
    return mkf(a.x * d, -a.y * d);
}
__host__ __device__ __forceinline__ void cfma(float2& a, float2 b, float2 c) {
    a.x = fmaf(b.x, c.x, a.x); a.x = fmaf(-b.y, c.y, a.x);
    a.y = fmaf(b.x, c.y, a.y); a.y = fmaf(b.y, c.x, a.y);
}

template <typename C> __device__ __forceinline__ C to_c(double2 v);
template <typename C> __device__ __forceinline__ C czero() {
    C z;
    memset(&z, 0, sizeof(C));
    return z;
}
template <> __device__ __forceinline__ double2 to_c<double2>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 to_c<float2>(double2 v) { return mkf((float)v.x, (float)v.y); }
__device__ __forceinline__ double2 to_d(double2 v) { return v; }
__device__ __forceinline__ double2 to_d(float2 v) { return mk(v.x, v.y); }

// ------------------------------------------------------------------ handles
struct Status {            // device-resident status word
    int flags;
    int pad[31];
};

}  // namespace klst

struct klst_pencil_s {
    klst_pencil_desc desc;
    int nx, nxi, qx, qy;
    int64_t n;
    // device tables (float64)
    double* x;      // [nx] mapped collocation points (j = 0 is +s_inf)
    double* Dx;     // [nx*nx] row-major D_x
    double* DxT;    // [nx*nx] column-major D_x (DxT[m*nx + j] = D_x[j][m])
    double* xi_x;   // [nxi]
    double* xi_y;   // [nxi]
    double* W;      // [nxi] full-line product weights
    double* nu;     // [nx] collision frequency P/mu
    double* macro;  // [4*nx] rho, u, E, T of the base state
    double* G;      // [((k*2 + c)*4 + a)*nx + j] coupling coefficients (zero on inflow rows)
    double* w;      // [((k*2 + c)*4 + a)*nx + j] moment functionals
    void* dx_oz;    // D_x cut into the tensor-core GEMM's integer slices (A operand) and row exponents
    double* eneq;   // [nx] non-equilibrium measure of the base flow (Eq. L2norm)
    klst::Status* status;
    int64_t footprint;
    cudaStream_t stream;  // stream of the last call (the handle's memory is released on it)
};

namespace klst {

// inflow boundary row test (Sec. 2.2): j = nx-1 (x = -s_inf) with xi_x > 0, j = 0 (x = +s_inf) with xi_x < 0
__host__ __device__ __forceinline__ bool is_bc(int j, int nx, double xix) {
    return (j == nx - 1 && xix > 0.0) || (j == 0 && xix < 0.0);
}

int device_sm_count();

// Deterministic warp sum: every lane adds its values in a fixed order, then a fixed xor tree.
__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Kernel launches issued by this library (process-wide counter, read by klst_launch_count).
void note_launch();
// Runs set() (a cudaFuncSetAttribute call or a few) once per device and flag word, before any
// caller returns: a caller that finds the flag unset takes a process-wide lock and re-checks it, so
// no thread can launch a kernel ahead of the attribute the launch needs.  Returns set()'s error (the
// flag stays unset then).
std::mutex& attr_mutex();
template <class F>
cudaError_t set_once_per_device(std::atomic<unsigned long long>& mask, F&& set) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return set();
    const unsigned long long bit = 1ull << dev;
    if (mask.load(std::memory_order_acquire) & bit) return cudaSuccess;
    std::lock_guard<std::mutex> lk(attr_mutex());
    if (mask.load(std::memory_order_acquire) & bit) return cudaSuccess;
    const cudaError_t e = set();
    if (e == cudaSuccess) mask.fetch_or(bit, std::memory_order_release);
    return e;
}
void note_launches(unsigned long long k);
void set_capturing(bool on);

// Stream-ordered device memory (cudaMallocAsync on the device's default pool, whose release
// threshold is raised once so freed blocks stay cached): allocations on different streams do
// not serialise the device the way cudaMalloc/cudaFree do.
cudaError_t dmalloc(void** ptr, size_t bytes, cudaStream_t s);
void dfree(void* ptr, cudaStream_t s);

// ------------------------------------------------------------------ Gilbarg-Paolucci shock (gp.cu)
// One thread per case; cases, results and the [3][n][npts] profile in device memory, cidx the
// caller's index of each case, xs (device) in decreasing order, perm the output column of each sorted
// point (null: the identity).
int gp_shock_device(const klst_gp_case* cases, const int* cidx, int n, double step, double eps, int max_steps,
                    const double* xs, const int* perm, int npts, double* prof, klst_gp_result* res, cudaStream_t s);
bool gp_case_valid(const klst_gp_case& c);
// test hook behind klst_debug_fail_alloc_after: the n-th next dmalloc fails (n < 0: off)
void fail_alloc_after(long long n);

}  // namespace klst

namespace klst {
// Opt-in per-kernel-group timing (environment KLST_TIMING=1): CUDA events around launch groups,
// summed per name and printed to stderr by klst_eigs.  Off by default; no cost when off.
bool prof_enabled();
void prof_begin(const char* name, cudaStream_t s);
void prof_end(const char* name, cudaStream_t s);
void prof_report(cudaStream_t s);
}  // namespace klst
