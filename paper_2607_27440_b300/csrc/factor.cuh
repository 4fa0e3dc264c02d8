// Internal factor handle shared by factor.cu, apply.cu and eigs.cu.
#pragma once
#include "common.cuh"

struct klst_factor_s {
    klst_pencil p;
    double2 sigma;
    int precision;     // KLST_FP64 / KLST_MIXED
    int nx, nxi, r;    // r = 4 nx (capacitance size)
    int64_t n;
    void* KinvT;       // [nxi][nx(m)][nx(j)] column-major inverse blocks, double2 or float2
    void* kslices;     // FP64 with tc_solve: bfloat16 integer slices of every K_k^{-1} + row exponents
    int tc_solve;      // 1: the float64 block solves run on the tensor cores (float64-accurate split)
    int tc_factor;     // 1: K_k^{-1} by a float32 inverse + tensor-core Newton-Schulz steps
    int ns_steps;      // Newton-Schulz steps taken (largest over the block ranges)
    int ns_fallback;   // block ranges inverted by float64 Gauss-Jordan instead
    double ns_resid;   // largest |I - K X| entry before the last step
    double2* Cinv;     // [r][r] row-major capacitance inverse (float64)
    // apply workspace (sized for nrhs_cap right-hand sides)
    int nrhs_cap;
    int ngroups;       // k-groups of the moment reductions
    double2* tpart;    // [nrhs][ngroups][r]
    double2* t;        // [nrhs][r]
    double2* sv;       // [nrhs][r]
    double2* bwork;    // [nrhs][n] masked right-hand side B x (mixed)
    double2* rwork;    // [nrhs][n] refinement residual
    double2* zwork;    // [nrhs][n] D_x products of the refinement residual (tensor-core path)
    void* ozws;        // tensor-core D_x product workspace (integer slices of the iterate)
    int tc_resid;      // 1: the float64 refinement residual forms its D_x products on the tensor cores
    double* normpart;  // [nrhs][nblk][2]
    int* done;         // [nrhs] refinement converged flags
    double2* sigma_dev;// [nrhs] the shift replicated per right-hand side
    double* worst;     // [1] worst final refinement residual since the last reset
    int* sweeps;       // [1] refinement sweeps executed since the last reset
    int max_refine;
    double refine_tol;
    int arith;         // refinement residual: 0 float64, 1 double-float (set per eigs call)
    double t_factor_ms;
    int64_t footprint;
    klst::Status* status;
    cudaStream_t stream;  // stream of the last call (the handle's memory is released on it)
};

namespace klst {
struct Rot {           // rotation [c s; -conj(s) c] of rows/columns (i, i+1), in double-float
    float4 s;          // complex s: {re.hi, re.lo, im.hi, im.lo}
    float2 c;          // real c: {hi, lo}
    int i;
    int pad;
};
struct SchurArgs {
    int m;             // current basis size (columns of S)
    int lds;           // leading dimension of S (>= m + 1)
    double2* S;        // (m+1) x m Rayleigh quotient + last row, column-major; overwritten by the truncation
    double2* H;        // m x m scratch -> T
    double2* Q;        // m x m scratch -> Schur vectors
    double2* Yc;       // m x m scratch: eigenvectors y_p of T for p < keep
    double2* Ysel;     // m x nev: Ritz vector coefficients Q y / ||y|| of the selected pairs
    double2* mu;       // m Ritz values (sorted)
    double2* mu_sel;   // nev selected Ritz values
    double* est;       // keep residual estimates (sorted positions)
    double* est_sel;   // nev residual estimates of the selected pairs
    int* nconv;        // out: converged among the first nev
    int keep;          // columns kept by the truncation (nev <= keep < m)
    int nev;
    double tol;
    int conv;          // 0: est <= tol |mu|, 1: est <= tol |mu|^2
    Status* st;
    float4* Vh;        // m x m: Householder vectors (column c, rows c+1..m-1), double-float
    double* tau;       // m: Householder scalars (0 = no reflection)
    Rot* log;          // Givens rotations of the QR sweeps and the reordering, in order
    int log_cap;
    int* log_count;    // [0] rotations, [1] QR sweeps, [2] swaps, [3] replay levels (float64 step)
    // float64 step: the log sorted by replay level (rotations of one level act on disjoint index
    // pairs), the level ends, and the per-index level counters the sweeps and swaps update
    Rot* log2;
    int* loff;         // log_cap + 1
    int* rdy;          // 256
};

int launch_schur(const SchurArgs& a, cudaStream_t s);    // double-float sweeps (schur.cu)
int launch_schur64(const SchurArgs& a, cudaStream_t s);  // float64 sweeps (schur64.cu)
void launch_schur_post(const SchurArgs& a, cudaStream_t s);

// float64-accurate GEMMs on the tensor cores (ozaki.cu)
size_t oz_workspace_bytes(int M, int N, int K);
// V'[:, 0:keep] = V[:, 0:m] Q[:, 0:keep]: complex, column-major (ld n for V, V'; m for Q); 2 m <= 256
int oz_rotate(const double2* V, int64_t n, int m, const double2* Q, int keep, double2* Vout, void* ws, Status* st,
              cudaStream_t s);

// D_x products of the pencil operator on the tensor cores: D_x slices once per pencil (oz_dx_bytes,
// oz_split_dx), then z = blockwise D_x x for nrhs vectors (workspace oz_dx_ws_bytes)
size_t oz_dx_bytes(int nx);
int oz_split_dx(const double* Dx, int nx, void* buf, cudaStream_t s);
size_t oz_dx_ws_bytes(int nx, int nxi, int nrhs);
int oz_dx_apply(const void* dxbuf, int nx, int nxi, const double2* x, int64_t ldx, int nrhs, double2* z, void* ws,
                Status* st, cudaStream_t s, const int* done = nullptr);  // done[rhs] != 0: skip that vector

// float64 Gram-Schmidt of one Arnoldi step (orth64.cu)
struct Orth64Args {
    double2* V;        // basis, n x (m + 1) column-major (ld n)
    int64_t n;
    int m;             // ncv
    double2* w;        // the vector to orthogonalise (overwritten)
    double2* vcur;     // receives the new basis vector (input of the next apply)
    int chunk, nchunks, ldp;
    double2* part;     // [nchunks][ldp] per-chunk partial coefficients
    double2 *h1, *h2;  // first- and second-pass coefficients (m + 1 each)
    int nupd;          // CTAs of the updates (and entries of npart)
    double* npart;     // [nupd] partial sums of |w''|^2
    int nscale;        // CTAs of the scaling kernel
    double2* S;        // Krylov-Schur matrix, (m + 1) x m column-major
    int lds;
    double* beta;      // out: ||w''||
    Status* st;
    unsigned short* sl;  // non-NULL: integer slices of V, the float64 passes run on the tensor cores
    float2* v32;         // with sl: V truncated to complex float32 (the first-pass coefficients' operand)
    int ntc;             // CTAs of the tensor-core passes (gs_tc_groups)
};
int orth64_step(const Orth64Args& a, int j, const int* jd, cudaStream_t s);
// tensor-core Gram-Schmidt (orth_tc.cu): slices of the float64 basis and the products with them
size_t basis_slices_bytes(int64_t n);
bool basis_slices_supported(int m);
int gs_tc_groups(int64_t n);
int split_basis(const double2* V, int64_t n, int c0, int c1, unsigned short* SL, float2* V32, cudaStream_t s);
int gs_update_tc(const unsigned short* SL, int64_t n, const double2* h, double2* w, double* npart, bool second,
                 int j, const int* jd, Status* st, cudaStream_t s);
int gs_dots_tc(const unsigned short* SL, int64_t n, const double2* w, double2* part, int ldp, int j, const int* jd,
               Status* st, cudaStream_t s);
void finish_scale64_split(const double2* h1, const double2* h2, const double* npart, int nparts, double2* S, int lds,
                          double* beta, Status* st, const double2* w, int64_t n, double2* V, double2* vcopy, int col,
                          unsigned short* SL, float2* V32, const int* jd, int nblk, cudaStream_t s);
// vcol = vcopy = w / *beta (the first basis vector)
void k_scale64_ext(const double2* w, int64_t n, const double* beta, double2* vcol, double2* vcopy, int64_t ldv,
                   int nblk, cudaStream_t s);
int factor_reserve(klst_factor f, int nrhs, cudaStream_t s);
// y = T x on the factor's stream; x, y complex128 n x nrhs
int apply_T(klst_factor f, const double2* x, double2* y, int nrhs, cudaStream_t s);
// y = (A - omega_r B) x_r (omega on device, nrhs entries)
int apply_pencil_dev(klst_pencil p, const double2* x, double2* y, int nrhs, const double2* omega_dev,
                     cudaStream_t s, double2* mwork, double2* mpart, int ngroups);
int pencil_work_groups(klst_pencil p);
int pencil_rows_z_dev(klst_pencil p, const double2* m, const double2* z, const double2* x, int64_t ldx, int nrhs,
                      const double2* omega, int mode, const double2* b, int mask_b, double2* y, double* normpart,
                      cudaStream_t s, const int* done);
// klst_eigs's option rules (KLST_EINVAL with a message); n = unknowns of the pencil
int validate_eigs_opts(const klst_eigs_opts* o, int64_t n);
void k_reduce_groups_ext(int len, int ngroups, const double2* part, double2* out, const int* done, int nrhs,
                         cudaStream_t s);
// float64-accurate tensor-core block solves (solve_tc.cu)
bool tc_solve_supported(int nx);
size_t tc_kinv_bytes(int nx, int nxi);
int tc_split_kinv(const double2* KinvT, int nx, int nxi, void* buf, cudaStream_t s);
int tc_solve_groups(int nxi, int ngroups_cap);
// tensor-core block inverses (factor_tc.cu)
bool ns_inverse_supported(int nx);
size_t ns_scratch_bytes(int nx, int nxi);
int ns_block_inverses(klst_factor f, double2* K64, cudaStream_t s, int info[2], double* rlast);
int tc_solve_pass(int pass, klst_factor f, const double2* b, int mask, double2* y, int accumulate, int nrhs,
                  cudaStream_t s, const int* done);
}  // namespace klst
