/*
 * klst.h -- C ABI of the B300 kLST shift-and-invert eigensolver.
 *
 * The library computes eigenpairs of the kinetic linear-stability pencil
 *     A q = omega B q                               (Sec. 4, Eq. MatrixProblem)
 * of the linearised Boltzmann-BGK equations for a 1-D normal shock: the
 * perturbed reduced distributions q = [g^; h^] are discretised by mapped
 * Chebyshev collocation in x (Sec. 3.1) and Gauss-Hermite micro-velocity nodes
 * (Sec. 3.2); the rows are Eqs. comp_ghat1Dshock / comp_hhat1Dshock with the
 * inflow boundary rows of Sec. 2.2.  omega is the paper's i*varpi.
 *
 * Unknown ordering: q[(c * Nxi + k) * Nx + j], component c in {g^, h^},
 * micro-velocity node k = kx * qy + ky, collocation point j (fastest).
 * Complex numbers are interleaved (re, im) float64 pairs (C99 double complex,
 * cuDoubleComplex, torch.complex128) unless stated otherwise.
 *
 * Conventions
 *  - Every call returns an int status (klst_status); no exception crosses the ABI.
 *  - Handles (klst_pencil, klst_factor, klst_batch, klst_server) own their device
 *    memory.  The caller owns every buffer it passes.  A failed create call
 *    leaves *out == NULL and frees what it allocated.
 *  - "device" buffers are CUDA global-memory pointers on the current device;
 *    "host" buffers are ordinary host memory.
 *  - Calls are ordered on the given stream (a cudaStream_t; NULL = legacy default
 *    stream).  Calls documented as synchronising wait for the stream.
 *  - Handles are not thread-safe; klst_server_* is internally locked.
 *  - klst_last_error() returns a thread-local message for the last failure.
 */
#ifndef KLST_H
#define KLST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* klst_stream; /* same type as cudaStream_t */

typedef enum {
    KLST_OK = 0,
    KLST_EINVAL = -1,     /* bad argument (sizes, NULL pointers, unsupported shape) */
    KLST_ENOMEM = -2,     /* device allocation failed */
    KLST_ESINGULAR = -3,  /* zero pivot: a shifted block or the capacitance matrix is singular */
    KLST_ENOCONV = -4,    /* eigensolver reached max_restarts before nev pairs converged */
    KLST_EREFINE = -5,    /* mixed-precision refinement did not reach its tolerance */
    KLST_ETIMEOUT = -6,   /* a bounded device-side wait gave up (the tensor-core GEMM's pipeline waits) */
    KLST_ECUDA = -7       /* a CUDA runtime call failed */
} klst_status;

typedef enum { KLST_FP64 = 0, KLST_MIXED = 1, KLST_DF64 = 2 } klst_precision;
/* Synthetic base flows of klst_build_pencil: a tanh-profile local Maxwellian, the bimodal Mott-Smith
 * mixture of the two end-state Maxwellians, or the local Maxwellian of the Gilbarg-Paolucci
 * continuum shock profile (klst_gp_shock with Re = re_delta, s = visc_s, Pr = 1; gamma must be 5/3;
 * width is not used), each with its steepest point at x = 0. */
typedef enum { KLST_BASE_TANH_MAXWELL = 0, KLST_BASE_MOTT_SMITH = 1, KLST_BASE_GILBARG_PAOLUCCI = 2 } klst_base;

/* Pencil description (all nondimensional: T by T_inf, rho by rho_inf, velocity by
 * sqrt(2 R T_inf), length by the shock thickness; Sec. 2.2). */
typedef struct {
    int32_t nx;          /* Chebyshev-Gauss-Lobatto points (N + 1), 4 <= nx <= 128 */
    int32_t qx, qy;      /* Gauss-Hermite nodes in xi_x and xi_y, 1..256 each */
    double map_L;        /* algebraic map length scale L (Eq. Chebmapping) */
    double map_sinf;     /* domain half-width s_inf (Eq. Chebmapping) */
    double mach;         /* free-stream Mach number */
    double gamma;        /* ratio of specific heats (5/3 for argon) */
    double visc_s;       /* viscosity exponent s in mu ~ T^s */
    double re_delta;     /* Reynolds number on the shock thickness */
    double beta;         /* transverse wavenumber (normal-mode ansatz, Sec. 2.2) */
    double width;        /* tanh width of the synthetic base flow */
    int32_t base;        /* klst_base */
    int32_t noneq;       /* 0: EQ (f_c := f_c^e), 1: NONEQ base flow */
    int32_t conservative;/* 1: discrete-conservative equilibrium and coefficients */
} klst_pencil_desc;

typedef struct {
    int32_t nev;          /* eigenpairs wanted (nearest sigma), >= 1 */
    int32_t ncv;          /* Krylov basis size, nev + 2 <= ncv <= 160 */
    int32_t max_restarts; /* Krylov-Schur restarts before KLST_ENOCONV */
    int32_t max_refine;   /* mixed precision: refinement sweeps per solve (>= 0) */
    double tol;           /* Ritz residual tolerance relative to |mu| */
    double refine_tol;    /* mixed precision: target ||r|| / ||rhs|| of each solve */
    const void* v0;       /* device complex128 start vector (length n) or NULL */
    uint64_t seed;        /* start vector seed when v0 == NULL */
    int32_t conv;         /* KLST_CONV_REL: est <= tol |mu|;  KLST_CONV_RESID: est <= tol |mu|^2, which
                             bounds the purified residual ||A q - omega B q|| (||q|| = 1) by ~tol */
    double* est_out;      /* host float64[nev] or NULL: final Ritz residual estimates ||T x - mu x|| */
    int32_t keep;         /* Ritz vectors kept at each restart, nev <= keep < ncv; 0 = nev + (ncv - nev) / 2 */
    int32_t arith;        /* KLST_ARITH_F64: Krylov basis, Gram-Schmidt and rotations in native float64;
                             KLST_ARITH_DF64: basis stored and combined in double-float (two float32 per
                             real, error-free products and compensated sums, ~2^-48 unit roundoff) on the
                             float32 pipes, which the B300 runs ~60x faster than float64 */
} klst_eigs_opts;

typedef enum { KLST_ARITH_F64 = 0, KLST_ARITH_DF64 = 1 } klst_arith;

typedef enum { KLST_CONV_REL = 0, KLST_CONV_RESID = 1 } klst_conv;

typedef struct {
    int32_t nconv;        /* converged pairs returned (<= nev) */
    int32_t restarts;     /* Krylov-Schur restarts performed */
    int32_t applies;      /* shift-invert operator applications */
    int32_t refine_sweeps;/* refinement sweeps executed in total (mixed) */
    double t_factor_ms;   /* time of klst_factor_shift for this factor */
    double t_eigs_ms;     /* wall time of the eigs call */
    double max_resid;     /* max explicit ||A q - omega B q|| over returned pairs, ||q|| = 1 */
    double max_refine_resid; /* worst final relative refinement residual (mixed) */
    double t_apply_ms;    /* device time in shift-invert applies (CUDA events; 0 in graph mode) */
    double t_orth_ms;     /* device time in Gram-Schmidt (graph mode: applies + Gram-Schmidt) */
    double t_restart_ms;  /* device time in Schur restarts and basis rotations */
    double t_schur_ms;    /* of which the small Schur/reorder step */
    int32_t reorths;      /* Arnoldi steps that ran the second Gram-Schmidt pass (float64 basis: every step) */
    int32_t schur_sweeps; /* shifted QR sweeps of the small Schur step, summed over restarts (float64 basis) */
    int32_t schur_swaps;  /* adjacent swaps of the reordering, summed over restarts (float64 basis) */
    int64_t schur_rotations; /* Givens rotations logged by the Schur step, summed over restarts */
} klst_eigs_info;

/* Jacobi-Davidson options (klst_jd_eigs; Sec. 4.2 and the solver table of the paper) */
typedef enum { KLST_JD_PREC_FULL = 0, KLST_JD_PREC_BLOCK = 1 } klst_jd_precond;
typedef struct {
    int32_t nev;          /* eigenpairs wanted (nearest sigma), 1..64 */
    int32_t ncv;          /* largest search space, 4..64 (the paper: 150-200 at 281,088 unknowns) */
    int32_t kmin;         /* search directions kept at a restart, 1 <= kmin < ncv (the paper's k_min = 6) */
    int32_t max_outer;    /* outer iterations before KLST_ENOCONV */
    double tol;           /* a harmonic Ritz pair locks when ||r|| <= tol |theta| (||u|| = 1) */
    int32_t gmres_m;      /* GMRES restart length of the correction equation, 1..64 (the paper: 30) */
    int32_t gmres_max;    /* GMRES iterations per correction equation (the paper: 200) */
    double gmres_rtol;    /* relative tolerance on the preconditioned correction residual (1e-6) */
    double gmres_atol;    /* absolute tolerance (1e-12) */
    int32_t precond;      /* KLST_JD_PREC_FULL: the factored (A - sigma B)^{-1} (Woodbury);
                             KLST_JD_PREC_BLOCK: the block inverses K_k^{-1} alone (no moment coupling) */
    const void* v0;       /* device complex128 start vector (length n) or NULL */
    uint64_t seed;        /* start vector seed when v0 == NULL */
} klst_jd_opts;
typedef struct {
    int32_t nconv;        /* eigenpairs returned (locked) */
    int32_t outer;        /* outer iterations */
    int32_t inner;        /* GMRES iterations in total */
    int32_t restarts;     /* search-space restarts */
    int64_t applies_op;   /* applications of A - theta B */
    int64_t applies_prec; /* preconditioner applications */
    double t_ms;          /* wall time */
    double max_resid;     /* max ||A x - omega B x|| over the returned pairs, ||x|| = 1 */
} klst_jd_info;

/* BE-BGK base-flow solver options and report (klst_bgk_base_flow; Sec. 3.3) */
typedef struct {
    int32_t max_steps;      /* RK4 steps at most (whole multiples of check_every are taken) */
    double cfl;             /* dt = cfl min(dx) / max|xi_x|, and at most 2 / max(nu); e.g. 0.5 */
    double dt;              /* > 0: this fixed time step instead */
    double tol;             /* stop once max|RHS| <= tol max|g| at a check; 0: run max_steps */
    int32_t check_every;    /* RK4 steps per residual check (one CUDA graph launch), >= 1 */
    int32_t recentre_every; /* steps between re-centring checks, a multiple of check_every; 0: off */
    double recentre_tol;    /* re-centre when the shock has moved more than this from the map centre */
    int32_t start;          /* 0: Mott-Smith profile (desc->width); 1: local Maxwellian of the
                               Gilbarg-Paolucci profile (Re = re_delta, s = visc_s, Pr = 1; gamma 5/3) */
} klst_bgk_opts;
typedef struct {
    int32_t steps;          /* RK4 steps taken */
    int32_t recentres;      /* grid rebuilds */
    double resid;           /* max|RHS| / max|g| at the last check */
    double centre;          /* final map centre: the shock's position in the solve's frame */
    double dt;              /* time step of the last check interval */
    double t_ms;            /* wall time */
    double newton_avg;      /* Newton updates per node and equilibrium evaluation */
} klst_bgk_info;

/* Gilbarg-Paolucci continuum shock (klst_gp_shock; Sec. 2.1, Eqs. GB1DShockeqn, ShockThickness) */
typedef struct {
    double mach;            /* free-stream Mach number, 1.01..100 (monatomic: gamma = 5/3) */
    double re;              /* Reynolds number of the length unit: mu = (u_inf / re) T^visc_s */
    double visc_s;          /* viscosity exponent s, 0..2 */
    double prandtl;         /* Prandtl number (1 for the BGK model), 0 < Pr <= 10 */
} klst_gp_case;
typedef struct {
    double step;            /* RK4 step times the largest end-state eigenvalue modulus (0: 0.02) */
    double eps;             /* start offset from the downstream state, relative to u_2 (0: 1e-6) */
    int32_t max_steps;      /* RK4 steps per case at most (0: 2^20) */
} klst_gp_opts;
typedef struct {
    double delta;           /* thickness (u_inf - u_2) / max|du/dx| in the length unit (= Re_Delta at re = 1) */
    double x_shock;         /* the steepest point, measured from the start point (x < 0: upstream) */
    double x_up;            /* where the upstream state was reached, from the start point */
    double lambda_s;        /* the saddle's stable eigenvalue (< 0) */
    int32_t steps;          /* RK4 steps taken */
    int32_t status;         /* KLST_OK or KLST_ENOCONV (max_steps reached first) */
} klst_gp_result;

typedef struct klst_pencil_s* klst_pencil;
typedef struct klst_factor_s* klst_factor;

/* Number of CUDA kernels this library has launched in the process so far (all threads). */
unsigned long long klst_launch_count(void);

/*
 * Per-kernel-group device timing (instrumentation; the paper has no counterpart).
 * klst_prof_enable(1) makes the library record a pair of CUDA events on the launching stream
 * around each group of launches it names (for example "solve_pass1_df64", "orth_pass1",
 * "schur_qr"); klst_prof_enable(0) stops recording.  Totals accumulate across calls until
 * klst_prof_reset().  klst_prof_entry(i, ...) waits for the recorded events, copies group i's
 * name (NUL-terminated, truncated to name_cap bytes), total milliseconds and number of timed
 * groups, and returns the number of groups; an i outside [0, count) only returns the count.
 * Thread-safe; with recording off the library's launch path is unchanged.
 */
void klst_prof_enable(int32_t on);
void klst_prof_reset(void);
int32_t klst_prof_entry(int32_t i, char* name, int32_t name_cap, double* total_ms, int64_t* calls);

/*
 * klst_debug_fail_alloc_after -- test hook (the paper has no counterpart): the n-th next device
 * allocation the library makes (n = 0: the next one) fails as if the device were out of memory, so
 * callers can check that every entry point returns KLST_ENOMEM, leaves its out-handle NULL and frees
 * what it had allocated.  n < 0 switches the hook off (the default).  Process-wide, thread-safe.
 */
void klst_debug_fail_alloc_after(int64_t n);

/* Status text ("KLST_OK", ...) and the calling thread's last error message. */
const char* klst_status_string(int status);
const char* klst_last_error(void);

/*
 * klst_gemm_f64_tc -- C = A B in float64 accuracy on the tensor cores (the building block of the
 * float64 basis rotation of the Krylov-Schur restart, Sec. 4.1; the paper has no counterpart as a
 * separate call).  A: device float64 M x K column-major (leading dimension lda >= M), B: device
 * float64 K x N column-major (ldb >= K), C: device float64 M x N column-major (ldc >= M), no
 * aliasing; 1 <= K <= 256.  Method: each row of A and each column of B is scaled by a power of two
 * and cut into eight 7-bit integer slices held exactly in bfloat16; the 36 slice products with
 * s + t <= 9 are accumulated by tcgen05 MMAs in float32 tensor memory, exactly per diagonal s + t,
 * and combined in float64.  Error: |C - AB|_rc <= ~K 2^-54 max_k |A_rk| max_k |B_kc| (float64-level
 * relative to the row and column maxima).  Allocates a workspace of ~16 (M + N) K bytes per call.
 * Errors: KLST_EINVAL, KLST_ENOMEM, KLST_ETIMEOUT (a bounded device wait gave up; C is then
 * unspecified).  Synchronising.
 */
int klst_gemm_f64_tc(const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc, int32_t M,
                     int32_t N, int32_t K, klst_stream stream);

/*
 * klst_build_pencil -- assemble the structured pencil on the device (Sec. 2.2, 3.1, 3.2).
 * Builds the Gauss-Hermite grid (Golub-Welsch nodes, full-line weights), the mapped
 * Chebyshev derivative D_x = diag(dy/dx) D_y, the synthetic base flow, its discrete
 * moments and equilibrium, the moment functionals w^c_a(j,k), the coupling
 * coefficients G^c_a(j,k) of Eq. Comp1DHarm and the inflow boundary mask.
 * desc: host.  Errors: KLST_EINVAL for out-of-range sizes, KLST_ENOMEM.
 * Synchronising (the handle is usable on any stream afterwards).
 */
int klst_build_pencil(const klst_pencil_desc* desc, klst_stream stream, klst_pencil* out);
void klst_pencil_destroy(klst_pencil p);

/* Sizes: n = 2 nx nxi unknowns; footprint = device bytes the handle owns. Any out may be NULL. */
int klst_pencil_dims(klst_pencil p, int64_t* n, int32_t* nx, int32_t* nxi, int64_t* footprint_bytes);

/*
 * klst_pencil_tables -- copy the assembled tables to host float64 buffers (tests, diagnostics).
 * x[nx], Dx[nx*nx] (row-major), xi_x[nxi], xi_y[nxi], W[nxi], nu[nx],
 * G[nxi*2*4*nx] and w[nxi*2*4*nx] (index ((k*2 + c)*4 + a)*nx + j), bc[nx*nxi] (j*nxi + k, 1 = inflow row).
 * Any pointer may be NULL.  Synchronising.
 */
int klst_pencil_tables(klst_pencil p, double* x, double* Dx, double* xi_x, double* xi_y, double* W,
                       double* nu, double* G, double* w, uint8_t* bc);

/*
 * klst_export_dense -- write the dense pencil to host memory (n <= 16384):
 * A_host[n*n] = A - sigma B (row-major complex128), B_host[n] = diag(B) as float64 (0/1).
 * Either pointer may be NULL.  Synchronising.
 */
int klst_export_dense(klst_pencil p, double sigma_re, double sigma_im, double* A_host, double* B_host);

/*
 * klst_apply_pencil -- y[:, r] = (A - omega_r B) x[:, r] in float64 without forming A
 * (the residual operator of Eq. MatrixProblem).  x, y: device complex128, n x nrhs
 * column-major (column stride n); omega: host complex128[nrhs] (NULL = all zero).
 */
int klst_apply_pencil(klst_pencil p, const void* x, void* y, int32_t nrhs, const double* omega,
                      klst_stream stream);

/*
 * klst_apply_pencil_noalloc -- the same operator as klst_apply_pencil, y[:, r] = (A - omega_r B) x[:, r],
 * without allocating any device memory.  (The paper has no counterpart: this is a library service.)
 * For callers that cannot allocate when they apply the operator: hosts whose device memory is owned
 * by their own pool and who forbid library allocations in their steady-state loop, latency-critical
 * serving loops in which an allocation may synchronise or stall other streams, and code that must not
 * run out of memory halfway through a solve.  The call uses a fixed scratch array of
 * klst_apply_pencil_noalloc_capacity() bytes (4 MiB) that every GPU that loads this library holds
 * until the process exits; it needs 16 * (nrhs + 4 nx nrhs (1 + min(nxi, 32))) bytes and returns
 * KLST_EINVAL, with a message naming the limit, when that exceeds the capacity (e.g. nrhs > 15 at
 * nx = 128).  The first call on each device resolves the array's device address with that device
 * current; make that first call before any stream capture.  All calls share the one array, so calls
 * that may overlap on the GPU (different streams, or different threads without ordering) race: order
 * them on one stream.  Nothing is carried between calls.  x, y: device complex128, n x nrhs
 * column-major, no aliasing; omega: host complex128[nrhs] or NULL (all zero); a page-locked omega
 * must stay valid until the stream reaches the call.
 */
int klst_apply_pencil_noalloc(klst_pencil p, const void* x, void* y, int32_t nrhs, const double* omega,
                              klst_stream stream);
size_t klst_apply_pencil_noalloc_capacity(void);

/*
 * klst_base_noneq -- the base flow's translational non-equilibrium measure (Sec. 5, Eq. L2norm):
 * eneq_host[j] = sqrt( sum_k W_k (g_c(x_j, xi_k) - g_c^e(x_j, xi_k))^2 ) for the nx collocation points,
 * with g_c the base reduced distribution, g_c^e its discrete local equilibrium and W_k the full-line
 * Gauss-Hermite product weights (0 for an EQ base).  eneq_host: host float64[nx].  Synchronising.
 */
int klst_base_noneq(klst_pencil p, double* eneq_host);

/*
 * klst_eigvec_macro -- macroscopic perturbations of nvec vectors q (device complex128, n x nvec
 * column-major, e.g. the evecs of klst_eigs): macro_host (host complex128 [nvec][4][nx]) receives
 * (rho^, u^, v^, E^)(x_j), the perturbation moments of Sec. 2.2 (rho^ = sum W g^, u^ = sum W (xi_x - u)
 * g^ / rho, v^ = sum W xi_y g^ / rho, E^ = [sum W (|xi|^2 - 2E) g^ + sum W h^] / (2 rho)), and umax_host
 * (host float64[nvec], may be NULL) max_j |U^| with |U^| = sqrt(|u^|^2 + |v^|^2) (Eq. Unormpert), the
 * normalisation the paper applies to velocity eigenvectors.  Errors: KLST_EINVAL, KLST_ENOMEM.
 * Synchronising.
 */
int klst_eigvec_macro(klst_pencil p, const void* q, int32_t nvec, double* macro_host, double* umax_host,
                      klst_stream stream);

/*
 * klst_bgk_base_flow -- the steady 1-D shock of the reduced 1D2V BGK equations (Sec. 3.3, Eq.
 * BoltzmannBGK_reduced) on the pencil's mapped Chebyshev nodes and velocity grid (desc; base, noneq
 * and width only shape the Mott-Smith start).  dq/dt = nu (q^e - q) - xi_x dq/dx for q = (g, h):
 * second-order finite volumes with MUSCL reconstruction and the minmod limiter (the paper's form:
 * plain neighbour differences), relaxation toward the discrete equilibrium of each node's moments
 * (the one klst_build_pencil linearises), nu = P / mu(T); Dirichlet ends: the upstream Maxwellian and
 * the Rankine-Hugoniot Maxwellian refined so that its discrete mass, momentum and energy fluxes equal
 * the upstream ones; classical RK4; optional adaptive re-centring (the interval of largest |dU/dx|
 * locates the shock; past recentre_tol the nodes are rebuilt about it and g, h moved by linear
 * interpolation in x).  Starts from a Mott-Smith profile about x = 0 or (opts->start = 1) from the
 * Gilbarg-Paolucci profile with its steepest point at x = 0 (klst_gp_shock).  g_out, h_out: device
 * float64 [Nx][Nxi], node j = 0 at the downstream end (the pencil's order), in the frame centred on
 * the final map centre (info->centre), ready for klst_build_pencil_base.  Errors: KLST_EINVAL,
 * KLST_ENOMEM, KLST_ENOCONV (non-finite residual; a Gilbarg-Paolucci start that did not reach the
 * upstream state).  Synchronising.
 */
int klst_bgk_base_flow(const klst_pencil_desc* desc, const klst_bgk_opts* opts, void* g_out, void* h_out,
                       klst_bgk_info* info, klst_stream stream);

/*
 * klst_build_pencil_base -- klst_build_pencil with given base distributions in place of the
 * synthetic base flow (e.g. the BE-BGK steady state of klst_bgk_base_flow): gc, hc are device float64
 * [Nx][Nxi] (node j = 0 downstream); with desc->noneq = 0 the pencil uses their discrete equilibrium
 * instead (EQ).  The caller keeps gc, hc (they are read during the call).  Errors as klst_build_pencil.
 */
int klst_build_pencil_base(const klst_pencil_desc* desc, const void* gc, const void* hc, klst_stream stream,
                           klst_pencil* out);

/*
 * klst_gp_shock -- the Gilbarg-Paolucci continuum shock structure (Sec. 2.1, Eq. GB1DShockeqn) and
 * its thickness (Eq. ShockThickness) for a batch of cases, one device thread per case.  The printed
 * pair is restated from the steady 1-D Navier-Stokes balances it comes from (monatomic gas, R = 1/2,
 * rho_inf = T_inf = 1, u_inf = M sqrt(5/6)):
 *     (4/3) mu du/dx = m u + m T/(2u) - P,   (5/4)(mu/Pr) dT/dx = (3/4) m T - m u^2/2 + P u - m H
 * (m, P, H the fluxes of mass, momentum and enthalpy; their ratio in the paper's Omega, theta is the
 * printed dtheta/dOmega with the constant (4/5) Pr).  Classical RK4 with a fixed step from the
 * downstream Rankine-Hugoniot state displaced by eps u_2 along the saddle's stable eigenvector,
 * backward in x until the upstream state is reached to 1e-13; the steepest point is the sign change
 * of d^2u/dx^2 next to the largest sampled |du/dx|.  With re = 1, delta is the self-consistent
 * Re_Delta.  cases (host, ncases >= 0), opts (host; NULL: defaults), x (host float64[npts]: points
 * measured from the steepest point, any order), profile (device float64 [3][ncases][npts]: rho, u, T
 * at the points; past the start point the saddle's linear solution, past x_up the upstream state;
 * may be NULL when npts = 0), results (host, ncases).  Errors: KLST_EINVAL (a case or option out of
 * range), KLST_ENOCONV (a case's status; all results are written), KLST_ENOMEM.  Synchronising.
 */
int klst_gp_shock(const klst_gp_case* cases, int32_t ncases, const klst_gp_opts* opts, const double* x,
                  int32_t npts, void* profile, klst_gp_result* results, klst_stream stream);

/*
 * klst_factor_shift -- factor A - sigma B for the shift-and-invert transform
 * (Eqs. parShiftInvert, parLUfactor).  A - sigma B = K - U V^H where K is block
 * diagonal with one Nx x Nx block per node k (xi_x,k D_x + nu + i beta xi_y,k - sigma,
 * inflow rows replaced by identity rows; shared by g^ and h^) and U V^H is the
 * rank-4-per-point BGK moment coupling.  Computes every K_k^{-1} (for Nx <= 128 a complex float32
 * Gauss-Jordan inverse refined to float64 accuracy by Newton-Schulz steps on the tensor cores, see
 * klst_factor_inverse_info; otherwise batched float64 Gauss-Jordan with partial pivoting), the
 * capacitance C = I - V^H K^{-1} U (4 Nx x 4 Nx) and C^{-1} (Gauss-Jordan with partial pivoting: for 4 Nx <= 384 one launch of one
 * thread-block cluster holding the matrix in its CTAs' shared memory, otherwise one launch per
 * pivot; both give the same result).  KLST_NO_CLUSTER_GJ=1 in the environment selects the
 * per-pivot launches.  precision: KLST_FP64 (all float64),
 * KLST_MIXED (K_k^{-1} stored in complex float32, each apply corrected by float64 iterative refinement)
 * or KLST_DF64 (K_k^{-1} stored as double-float pairs, the same bytes as float64, and the block solves
 * run in double-float arithmetic on the float32 pipes; ~2^-48 accuracy without refinement).
 * K_k^{-1} and the capacitance are always formed to float64 accuracy.
 * Errors: KLST_ESINGULAR (zero pivot), KLST_ENOMEM.  Synchronising.
 */
int klst_factor_shift(klst_pencil p, double sigma_re, double sigma_im, int32_t precision,
                      klst_stream stream, klst_factor* out);
void klst_factor_destroy(klst_factor f);

/* Factor metadata: the pencil it belongs to, its shift and precision; any out may be NULL. */
int klst_factor_info(klst_factor f, double* sigma_re, double* sigma_im, int32_t* precision,
                     int64_t* footprint_bytes, double* t_factor_ms);

/*
 * klst_factor_inverse_info -- how the block inverses K_k^{-1} of f were formed (Eq. parLUfactor for
 * the blocks K_k).  *method: 1 = a complex float32 Gauss-Jordan inverse X_0 refined by Newton-Schulz
 * steps X <- X + X (I - K_k X), whose products run as float64-accurate integer-slice GEMMs on the
 * tensor cores (Nx <= 128; each step squares I - K_k X); 0 = float64 Gauss-Jordan with partial
 * pivoting (Nx > 128, or KLST_NO_TC=1 in the environment).  *steps: Newton-Schulz steps taken (the
 * largest over the block ranges processed together); *fallback: block ranges whose float32 inverse
 * was too poor for the iteration to converge (max |I - K X_0| Nx >= 1/2) and that were inverted by
 * float64 Gauss-Jordan instead; *resid: the largest |I - K_k X| entry computed before the last step
 * (the entries after it are bounded by (Nx resid)^2 plus float64 rounding).  The blocks are processed
 * in ranges sized to 768 MB of scratch (KLST_NS_RANGE=n in the environment: n blocks per range); the
 * result does not depend on the range size.  Any out may be NULL.  Errors: KLST_EINVAL (f NULL).
 */
int klst_factor_inverse_info(klst_factor f, int32_t* method, int32_t* steps, int32_t* fallback, double* resid);

/*
 * klst_apply_shift_invert -- y = (A - sigma B)^{-1} B x  (the operator T of Eq. parShiftInvert).
 * x, y: device complex128, n x nrhs column-major, may not alias.  Woodbury form:
 * z = K^{-1} B x, s = C^{-1} V^H z, y = K^{-1} (B x + U s).  MIXED factors run the two
 * block solves in complex float32 and then max_refine sweeps of float64 iterative
 * refinement y += T~ (B x - (A - sigma B) y) (stopping early at refine_tol).
 * Stream-ordered, not synchronising.
 */
int klst_apply_shift_invert(klst_factor f, const void* x, void* y, int32_t nrhs, klst_stream stream);

/* Refinement controls for klst_apply_shift_invert on MIXED factors (defaults 4 sweeps and 1e-12). */
int klst_factor_set_refine(klst_factor f, int32_t max_refine, double refine_tol);

/*
 * klst_factor_check -- waits for stream and reports whether any klst_apply_shift_invert on this MIXED
 * factor since the last check ended its max_refine refinement sweeps with ||r|| / ||B x|| still above
 * refine_tol: KLST_EREFINE (the flag is then cleared; the applies' outputs were still written and are
 * the best iterates reached), else KLST_OK.  klst_eigs reports the same condition for the applies it
 * makes by returning KLST_EREFINE after filling every output.  Synchronising.
 */
int klst_factor_check(klst_factor f, klst_stream stream);

/*
 * klst_eigs -- the nev eigenvalues nearest sigma by Krylov-Schur restarted Arnoldi on T
 * (Sec. 4.1: implicitly restarted Arnoldi with shift-and-invert), with classical
 * Gram-Schmidt (a second pass when the DGKS test ||w'|| < ||w|| / sqrt 2 asks for it) in
 * float64 (opts->arith = KLST_ARITH_F64) or double-float (KLST_ARITH_DF64), and the small
 * Schur/reorder step on the device (Householder, QR sweeps and Q rebuild in double-float).
 * With KLST_ARITH_DF64 on a stream other than the legacy default stream, each Arnoldi step is
 * captured once into a CUDA graph and launched as one graph per step (not when the stream is
 * already capturing, when klst_prof_enable is on, or with KLST_NO_GRAPH=1 in the environment);
 * results are the same either way, and info->t_apply_ms is then 0 with the whole expansion in
 * info->t_orth_ms.  Eigenvalues omega = sigma + 1/mu are returned
 * nearest-first in evals_host (host complex128[nev]); evecs (device complex128,
 * n x nev column-major, may be NULL) receive unit-norm purified eigenvectors
 * q = T x / ||T x||; resid_host (host float64[nev], may be NULL) receives
 * ||A q - omega B q||_2.  info may be NULL.
 * Stopping rule: the nev Ritz pairs nearest sigma that meet the convergence test (opts->conv);
 * an unconverged Ritz value nearer sigma may be passed over only when its |omega - sigma| is
 * within 1% of the last returned one (a cluster straddling the nev boundary, whose internal
 * order is not resolved); any separated nearer Ritz value keeps the iteration going.
 * Errors: KLST_ENOCONV (fewer than nev converged; the converged ones are still
 * returned and info->nconv says how many), KLST_EREFINE (MIXED factors: every pair converged but at
 * least one apply ended its refinement above refine_tol; all outputs are filled and resid_host holds
 * each pair's explicit residual), KLST_EINVAL.  Synchronising.
 */
int klst_eigs(klst_factor f, const klst_eigs_opts* opts, double* evals_host, void* evecs,
              double* resid_host, klst_eigs_info* info, klst_stream stream);

/*
 * klst_jd_eigs -- the nev eigenvalues nearest sigma by Jacobi-Davidson with harmonic Ritz extraction
 * (Sec. 4.2, the paper's second solver; JDQZ form for A q = omega B q with target tau = sigma):
 * search space V and test space W with (A - tau B) V = Z C + W R, harmonic pairs from
 * G = R^{-1} W^H B V (mu = 1 / (theta - tau), the largest |mu| nearest tau; the float64 Schur step
 * of klst_eigs), residual r = (I - Z Z^H)(A - theta B) u; ||r|| <= tol |theta| locks u and its test
 * vector into the partial Schur bases Q, Z; otherwise the correction equation
 * (I - z~ z~^H)(A - theta B)(I - q~ q~^H) t = -r is solved by GMRES(gmres_m) (rtol, atol, at most
 * gmres_max iterations) preconditioned by K = A - sigma B (precond FULL, the factor's exact Woodbury
 * solve) or by the block inverses alone (BLOCK), projected onto q~'s complement, and t expands V.  A
 * full search space (ncv) restarts to its kmin leading Schur directions.  The returned pairs come from
 * the harmonic extraction on the locked space, with explicit residuals ||A x - omega B x||, ||x|| = 1,
 * nearest sigma first.  f must be a KLST_FP64 factor.  evals_host: complex float64[nev] (re, im);
 * evecs: device complex128 n x nev (column-major) or NULL; resid_host: float64[nev] or NULL.  All
 * float64 on the device.  Errors: KLST_EINVAL (options, non-FP64 factor), KLST_ENOCONV (fewer than nev
 * pairs locked within max_outer iterations, or a breakdown; the locked pairs are returned), KLST_ENOMEM.
 * Synchronising.
 */
int klst_jd_eigs(klst_factor f, const klst_jd_opts* opts, double* evals_host, void* evecs, double* resid_host,
                 klst_jd_info* info, klst_stream stream);

/*
 * klst_batch_eigs -- many independent pencils at once (wavenumber, shift and Mach sweeps): pencil i
 * (descs[i], shift sigmas[2i] + i sigmas[2i+1]) is built, factored and solved for the opts->nev
 * eigenvalues nearest its shift, exactly as klst_build_pencil + klst_factor_shift + klst_eigs would,
 * with its start vector seeded by opts->seed + i (opts->v0 must be NULL).  nworkers host threads
 * (0 = 16) each own one non-blocking stream, so pencils overlap on the device; each pencil's result
 * is bit-for-bit the one it gets alone.  Outputs (host): evals_host complex128[npencils * nev]
 * (pencil-major), resid_host float64[npencils * nev] (may be NULL), status_host int32[npencils],
 * infos[npencils] (may be NULL).  Returns KLST_OK when every pencil succeeded, otherwise the first
 * failing status (each pencil's own status is in status_host).  Synchronising.
 */
int klst_batch_eigs(int32_t npencils, const klst_pencil_desc* descs, const double* sigmas, int32_t precision,
                    const klst_eigs_opts* opts, int32_t nworkers, double* evals_host, double* resid_host,
                    int32_t* status_host, klst_eigs_info* infos);

/*
 * Serving: a request loop that admits eigensolve requests by device-memory footprint.
 * klst_server_create starts max_slots worker threads (one stream each); a submitted request waits in
 * arrival order until a slot is free and its footprint fits in hbm_budget_bytes together with the
 * requests already running (a later, smaller request may pass a head request that must wait for
 * memory).  Requests run concurrently, each on its worker's stream, with results bit-for-bit equal to
 * a solve alone.  klst_server_submit copies its arguments (opts->v0 must be NULL; the seed is
 * opts->seed); KLST_ENOMEM if the request alone exceeds the budget.  klst_server_poll (wait != 0
 * blocks) reports done = 1 once finished, copies evals_host complex128[nev], resid_host float64[nev],
 * info, and the latency from submit to completion in ms, releases the ticket and returns the solve's
 * status; a finished ticket can be polled once.  Thread-safe (internally locked).
 */
/*
 * klst_solve_footprint -- device bytes one build + factor + eigs of this request holds at its peak:
 * the admission size klst_server uses (the paper has no counterpart: a serving service).  Returns the
 * byte count (> 0), or KLST_EINVAL (< 0) when the request is invalid (the klst_eigs option rules).
 */
int64_t klst_solve_footprint(const klst_pencil_desc* desc, int32_t precision, const klst_eigs_opts* opts);

typedef struct klst_server_s* klst_server;
int klst_server_create(int64_t hbm_budget_bytes, int32_t max_slots, klst_server* out);
int klst_server_submit(klst_server s, const klst_pencil_desc* desc, double sigma_re, double sigma_im,
                       int32_t precision, const klst_eigs_opts* opts, uint64_t* ticket);
int klst_server_poll(klst_server s, uint64_t ticket, int32_t wait, int32_t* done, double* evals_host,
                     double* resid_host, klst_eigs_info* info, double* latency_ms);
int klst_server_stats(klst_server s, int32_t* queued, int32_t* running, int64_t* bytes_in_flight);
void klst_server_destroy(klst_server s);

#ifdef __cplusplus
}
#endif

#endif /* KLST_H */
