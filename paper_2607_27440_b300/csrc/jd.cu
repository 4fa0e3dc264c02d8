// Jacobi-Davidson with harmonic Ritz extraction (Sec. 4.2, the paper's second solver), in the
// JDQZ form for the generalized problem A q = omega B q with target tau = sigma of the factor.
//
// Search space V (orthonormal, V ⟂ Q) and test space W (orthonormal, W ⟂ Z): every new search
// vector v gives w~ = (A - tau B) v, Gram-Schmidt against Z and then W, so that
//     (A - tau B) V = Z C + W R,   R upper triangular (its coefficients),   M_B = W^H B V.
// Harmonic Ritz (Petrov) pairs ask W^H (A - theta B) V y = 0, i.e. R y = (theta - tau) M_B y, so
// mu = 1 / (theta - tau) is an eigenvalue of G = R^{-1} M_B; the pair nearest tau has the largest
// |mu|.  G's Schur form (the float64 Schur step of the Krylov-Schur solver, sorted by |mu|) gives
// the Ritz vector u = V y, its test vector z = W R y / ||R y|| and the residual
// r = (I - Z Z^H)(A - theta B) u.  ||r|| <= tol |theta| locks u and z into the partial Schur bases
// Q and Z; otherwise the correction equation
//     (I - z~ z~^H)(A - theta B)(I - q~ q~^H) t = -r,   q~ = [Q u], z~ = [Z z],   t ⟂ q~
// is solved approximately by GMRES(m) with the projected preconditioner
//     K~^{-1} y = K^{-1} y - Y^ H^{-1} q~^H K^{-1} y,   Y^ = K^{-1} z~,   H = q~^H Y^,
// K^{-1} the factored (A - sigma B)^{-1} (Woodbury, exact) or the block inverses K_k^{-1} alone,
// and t expands V.  A full search space restarts to its k_min leading Schur directions.  Restart
// and locking rotate V by G's Schur vectors U and W by Q_r from R U = Q_r R'; the rotated M_B is
// Q_r^H M_B U.  The returned eigenpairs come from the harmonic extraction on the locked space:
// G_Q = (Z^H (A - tau B) Q)^{-1} Z^H B Q, omega = tau + 1/mu, x = Q y, with explicit residuals.
//
// Everything runs on the device: float64 vector kernels, the pencil operator and the Woodbury
// solves of the library, the tensor-core basis rotations, and single-CTA kernels for the small
// dense steps; the host reads a few scalars per iteration to steer the loop.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "factor.cuh"

namespace klst {

int apply_inv(klst_factor f, const double2* x, double2* y, int mode, cudaStream_t s);

namespace {

constexpr int kJdMaxM = 64;     // search space
constexpr int kJdMaxNev = 64;   // locked pairs
constexpr int kJdMaxIn = 64;    // GMRES restart length

__host__ __device__ inline double2 cmulj(double2 a, double2 b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__host__ __device__ inline double2 conjj(double2 a) { return mk(a.x, -a.y); }

// ------------------------------------------------------------------ vector kernels
// part[i * gridDim.x + b] = sum over CTA b's rows of conj(X[r, i]) y[r]
__global__ void __launch_bounds__(256) k_jd_dots(const double2* __restrict__ X, int64_t ldx, const double2* __restrict__ y,
                                                 int64_t n, double2* __restrict__ part) {
    const int i = blockIdx.y;
    const double2* xi = X + (int64_t)i * ldx;
    double sr = 0.0, si = 0.0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const double2 a = xi[r], b = y[r];
        sr = fma(a.x, b.x, fma(a.y, b.y, sr));
        si = fma(a.x, b.y, fma(-a.y, b.x, si));
    }
    __shared__ double rr[8], ri[8];
    sr = warp_sum(sr);
    si = warp_sum(si);
    if ((threadIdx.x & 31) == 0) { rr[threadIdx.x >> 5] = sr; ri[threadIdx.x >> 5] = si; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { a += rr[q]; b += ri[q]; }
        part[(size_t)i * gridDim.x + blockIdx.x] = mk(a, b);
    }
}

// out[i] (+)= sign * sum_b part[i * nb + b], one warp per column, fixed order
__global__ void k_jd_dots_fin(const double2* __restrict__ part, int nb, int k, double2* __restrict__ out, double sign,
                              int accumulate) {
    const int lane = threadIdx.x & 31, i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= k) return;
    double a = 0, b = 0;
    for (int q = lane; q < nb; q += 32) { a += part[(size_t)i * nb + q].x; b += part[(size_t)i * nb + q].y; }
    a = warp_sum(a);
    b = warp_sum(b);
    if (lane == 0) {
        const double2 v = mk(sign * a, sign * b);
        out[i] = accumulate ? mk(out[i].x + v.x, out[i].y + v.y) : v;
    }
}

// y -= X c (k columns, c on the device)
__global__ void __launch_bounds__(256) k_jd_update(const double2* __restrict__ X, int64_t ldx, int k,
                                                   const double2* __restrict__ c, double2* __restrict__ y, int64_t n) {
    __shared__ double2 cs[2 * kJdMaxM + 2];
    for (int i = threadIdx.x; i < k; i += blockDim.x) cs[i] = c[i];
    __syncthreads();
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        double2 acc = y[r];
        for (int i = 0; i < k; ++i) {
            const double2 a = X[(int64_t)i * ldx + r];
            acc.x -= a.x * cs[i].x - a.y * cs[i].y;
            acc.y -= a.x * cs[i].y + a.y * cs[i].x;
        }
        y[r] = acc;
    }
}

// y = X c
__global__ void __launch_bounds__(256) k_jd_gemv(const double2* __restrict__ X, int64_t ldx, int k,
                                                 const double2* __restrict__ c, double2* __restrict__ y, int64_t n) {
    __shared__ double2 cs[2 * kJdMaxM + 2];
    for (int i = threadIdx.x; i < k; i += blockDim.x) cs[i] = c[i];
    __syncthreads();
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        double2 acc = mk(0, 0);
        for (int i = 0; i < k; ++i) {
            const double2 a = X[(int64_t)i * ldx + r];
            acc.x += a.x * cs[i].x - a.y * cs[i].y;
            acc.y += a.x * cs[i].y + a.y * cs[i].x;
        }
        y[r] = acc;
    }
}

// y = x * (scale / *nrm) (scale = +-1), nrm on the device; a zero norm leaves zeros
__global__ void k_jd_scale(const double2* __restrict__ x, double2* __restrict__ y, int64_t n, const double* __restrict__ nrm,
                           double scale) {
    const double d = *nrm;
    const double f = d > 0 ? scale / d : 0.0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = x[r];
        y[r] = mk(v.x * f, v.y * f);
    }
}

// y = B x: the inflow boundary rows of every block zeroed (B is the identity elsewhere)
__global__ void k_jd_bmask(const double2* __restrict__ x, double2* __restrict__ y, int64_t n, int nx, int nxi,
                           const double* __restrict__ xi_x) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(r % nx), k = (int)((r / nx) % nxi);
        y[r] = is_bc(j, nx, xi_x[k]) ? mk(0, 0) : x[r];
    }
}

// seeded complex normal entries (splitmix64 counter hash, Box-Muller)
__device__ __forceinline__ uint64_t jd_mix(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__global__ void k_jd_randn(double2* x, int64_t n, uint64_t seed) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t a = jd_mix(seed * 0x100000001b3ull + 2 * i), b = jd_mix(seed * 0x100000001b3ull + 2 * i + 1);
        const double u1 = ((a >> 11) + 0.5) * (1.0 / 9007199254740992.0), u2 = (b >> 11) * (1.0 / 9007199254740992.0);
        const double rr = sqrt(-2.0 * log(u1));
        x[i] = mk(rr * cospi(2.0 * u2), rr * sinpi(2.0 * u2));
    }
}

// ------------------------------------------------------------------ small dense kernels (one CTA)
// S = [R^{-1} M_B; 0] ((m + 1) x m, column-major, ld m + 1) for the Schur step; R, M_B column-major
// with leading dimension ld; m_pad >= m: columns/rows m..m_pad-1 are zero (a padded problem gets
// the extra eigenvalues mu = 0, which sort last)
__global__ void k_jd_small_g(const double2* __restrict__ R, const double2* __restrict__ MB, int ld, int m, int m_pad,
                             double2* __restrict__ S, int* __restrict__ flag) {
    const int lds = m_pad + 1;
    for (int idx = threadIdx.x; idx < lds * m_pad; idx += blockDim.x) S[idx] = mk(0, 0);
    __syncthreads();
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        // back substitution R x = M_B[:, j]
        double2* x = S + (size_t)j * lds;
        for (int i = m - 1; i >= 0; --i) {
            double2 acc = MB[(size_t)j * ld + i];
            for (int l = i + 1; l < m; ++l) {
                const double2 rv = R[(size_t)l * ld + i];
                acc.x -= rv.x * x[l].x - rv.y * x[l].y;
                acc.y -= rv.x * x[l].y + rv.y * x[l].x;
            }
            const double2 d = R[(size_t)i * ld + i];
            const double dd = d.x * d.x + d.y * d.y;
            if (!(dd > 0)) { atomicOr(flag, 1); x[i] = mk(0, 0); continue; }
            x[i] = mk((acc.x * d.x + acc.y * d.y) / dd, (acc.y * d.x - acc.x * d.y) / dd);
        }
    }
}

// After the Schur step: y = Ysel[:, 0] (unit, m entries), ry = R y, ‖ry‖; out: zc = ry / ‖ry‖,
// theta = tau + 1 / mu, and scal[0] = ‖ry‖ (0: breakdown)
__global__ void k_jd_pick(const double2* __restrict__ R, int ld, int m, const double2* __restrict__ Ysel, int ldy,
                          const double2* __restrict__ musel, double2 tau, double2* __restrict__ zc,
                          double2* __restrict__ theta, double* __restrict__ scal) {
    __shared__ double2 ry[kJdMaxM];
    __shared__ double s_n;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double2 acc = mk(0, 0);
        for (int l = i; l < m; ++l) {
            const double2 rv = R[(size_t)l * ld + i], yv = Ysel[l];
            acc.x += rv.x * yv.x - rv.y * yv.y;
            acc.y += rv.x * yv.y + rv.y * yv.x;
        }
        ry[i] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int i = 0; i < m; ++i) s += ry[i].x * ry[i].x + ry[i].y * ry[i].y;
        s_n = sqrt(s);
        scal[0] = s_n;
        const double2 mu = musel[0];
        const double dm = mu.x * mu.x + mu.y * mu.y;
        theta[0] = dm > 0 ? mk(tau.x + mu.x / dm, tau.y - mu.y / dm) : tau;
    }
    __syncthreads();
    const double f = s_n > 0 ? 1.0 / s_n : 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) zc[i] = mk(ry[i].x * f, ry[i].y * f);
    (void)ldy;
}

// Rotation of the projected quantities by the Schur vectors U (m x m, ld m): RU = R U, its QR
// RU = Q_r R' (modified Gram-Schmidt, twice), M_B' = Q_r^H M_B U.  Outputs the columns c0 .. c0+kk-1:
// Ur = U[:, c0:], Qr[:, c0:] (m x kk, ld m each), R' and M_B' blocks [c0:c0+kk, c0:c0+kk] into R and
// MB (ld), overwriting them.  Shared-memory work arrays of m x m complex.
__global__ void __launch_bounds__(256) k_jd_rotate_small(double2* __restrict__ R, double2* __restrict__ MB, int ld, int m,
                                                         const double2* __restrict__ U, double2* __restrict__ Qr,
                                                         int c0, int kk) {
    extern __shared__ double2 sm[];
    double2* A = sm;            // RU, then Q_r (in place)
    double2* Rp = sm + m * m;   // R'
    double2* T = Rp + m * m;    // M_B U, then Q_r^H M_B U
    __shared__ double2 s_dot;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int idx = tid; idx < m * m; idx += nt) {
        const int i = idx % m, j = idx / m;
        double2 a = mk(0, 0), t = mk(0, 0);
        for (int l = 0; l < m; ++l) {
            const double2 u = U[(size_t)j * m + l];
            if (l >= i) a = a + cmulj(R[(size_t)l * ld + i], u);
            t = t + cmulj(MB[(size_t)l * ld + i], u);
        }
        A[idx] = a;
        T[idx] = t;
        Rp[idx] = mk(0, 0);
    }
    __syncthreads();
    // modified Gram-Schmidt on the columns of A, each projection applied twice
    for (int j = 0; j < m; ++j) {
        for (int pass = 0; pass < 2; ++pass) {
            for (int l = 0; l < j; ++l) {
                if (tid < 32) {
                    double2 d = mk(0, 0);
                    for (int i = tid; i < m; i += 32) d = d + cmulj(conjj(A[(size_t)l * m + i]), A[(size_t)j * m + i]);
                    d.x = warp_sum(d.x);
                    d.y = warp_sum(d.y);
                    if (tid == 0) { s_dot = d; Rp[(size_t)j * m + l] = Rp[(size_t)j * m + l] + d; }
                }
                __syncthreads();
                const double2 d = s_dot;
                for (int i = tid; i < m; i += nt) A[(size_t)j * m + i] = A[(size_t)j * m + i] - cmulj(A[(size_t)l * m + i], d);
                __syncthreads();
            }
        }
        if (tid < 32) {
            double s = 0;
            for (int i = tid; i < m; i += 32) s += abs2(A[(size_t)j * m + i]);
            s = warp_sum(s);
            if (tid == 0) { s = sqrt(s); s_dot = mk(s, 0); Rp[(size_t)j * m + j] = mk(s, 0); }
        }
        __syncthreads();
        const double nrm = s_dot.x;
        const double f = nrm > 0 ? 1.0 / nrm : 0.0;
        for (int i = tid; i < m; i += nt) A[(size_t)j * m + i] = mk(A[(size_t)j * m + i].x * f, A[(size_t)j * m + i].y * f);
        __syncthreads();
    }
    // T <- Q_r^H T (column by column into R's storage is avoided: compute into registers per entry)
    for (int idx = tid; idx < kk * kk; idx += nt) {
        const int i = c0 + idx % kk, j = c0 + idx / kk;
        double2 acc = mk(0, 0);
        for (int l = 0; l < m; ++l) acc = acc + cmulj(conjj(A[(size_t)i * m + l]), T[(size_t)j * m + l]);
        MB[(size_t)(j - c0) * ld + (i - c0)] = acc;
        R[(size_t)(j - c0) * ld + (i - c0)] = (i <= j) ? Rp[(size_t)j * m + i] : mk(0, 0);
    }
    for (int idx = tid; idx < m * kk; idx += nt) {
        const int i = idx % m, j = idx / m;
        Qr[(size_t)j * m + i] = A[(size_t)(c0 + j) * m + i];
    }
}

// the small (k1 x k1) matrix H = q~^H Y^ from its dots (column-major, ld kJdMaxNev + 1), inverted
// in place by Gauss-Jordan with partial pivoting (one thread: k1 <= 65)
__global__ void k_jd_hinv(double2* __restrict__ H, int k1, int* __restrict__ flag) {
    if (threadIdx.x != 0) return;
    const int ld = kJdMaxNev + 1;
    int perm[kJdMaxNev + 1];
    for (int p = 0; p < k1; ++p) {
        int piv = p;
        double best = -1;
        for (int i = p; i < k1; ++i) {
            const double v = abs2(H[(size_t)p * ld + i]);
            if (v > best) { best = v; piv = i; }
        }
        perm[p] = piv;
        if (!(best > 0)) { atomicOr(flag, 1); return; }
        if (piv != p)
            for (int c = 0; c < k1; ++c) { const double2 t = H[(size_t)c * ld + p]; H[(size_t)c * ld + p] = H[(size_t)c * ld + piv]; H[(size_t)c * ld + piv] = t; }
        const double2 inv = cinv(H[(size_t)p * ld + p]);
        for (int c = 0; c < k1; ++c) H[(size_t)c * ld + p] = (c == p) ? inv : cmulj(H[(size_t)c * ld + p], inv);
        for (int i = 0; i < k1; ++i) {
            if (i == p) continue;
            const double2 f = H[(size_t)p * ld + i];
            for (int c = 0; c < k1; ++c) {
                if (c == p) H[(size_t)c * ld + i] = mk(-(f.x * inv.x - f.y * inv.y), -(f.x * inv.y + f.y * inv.x));
                else H[(size_t)c * ld + i] = H[(size_t)c * ld + i] - cmulj(f, H[(size_t)c * ld + p]);
            }
        }
    }
    for (int p = k1 - 1; p >= 0; --p)
        if (perm[p] != p)
            for (int i = 0; i < k1; ++i) {
                const double2 t = H[(size_t)p * ld + i];
                H[(size_t)p * ld + i] = H[(size_t)perm[p] * ld + i];
                H[(size_t)perm[p] * ld + i] = t;
            }
}

// c = Hinv d (k1 x k1, ld kJdMaxNev + 1)
__global__ void k_jd_hsolve(const double2* __restrict__ Hinv, int k1, const double2* __restrict__ d, double2* __restrict__ c) {
    const int i = threadIdx.x;
    if (i >= k1) return;
    double2 acc = mk(0, 0);
    for (int l = 0; l < k1; ++l) acc = acc + cmulj(Hinv[(size_t)l * (kJdMaxNev + 1) + i], d[l]);
    c[i] = acc;
}

// GMRES: column j of the Hessenberg matrix (h[0..j+1], h[j+1] = ||w||) gets the earlier Givens
// rotations, a new rotation zeroes h[j+1], and g is updated; res[0] = |g[j+1]|
__global__ void k_jd_givens(double2* __restrict__ Hg, int ldh, int j, double2* __restrict__ cs, double2* __restrict__ sn,
                            double2* __restrict__ g, double* __restrict__ res) {
    if (threadIdx.x != 0) return;
    double2* h = Hg + (size_t)j * ldh;
    for (int i = 0; i < j; ++i) {
        const double2 c = cs[i], s = sn[i];
        const double2 a = h[i], b = h[i + 1];
        // [c s; -conj(s) c] with real c
        h[i] = mk(c.x * a.x + (s.x * b.x - s.y * b.y), c.x * a.y + (s.x * b.y + s.y * b.x));
        h[i + 1] = mk(c.x * b.x - (s.x * a.x + s.y * a.y), c.x * b.y - (s.x * a.y - s.y * a.x));
    }
    const double2 a = h[j], b = h[j + 1];
    const double na = sqrt(abs2(a)), nb = sqrt(abs2(b));
    double2 c, s;
    if (nb == 0) { c = mk(1, 0); s = mk(0, 0); }
    else if (na == 0) { c = mk(0, 0); s = mk(b.x / nb, -b.y / nb); }
    else {
        const double t = sqrt(na * na + nb * nb);
        c = mk(na / t, 0);
        // s = (a / |a|) conj(b) / t
        const double2 ph = mk(a.x / na, a.y / na);
        s = mk((ph.x * b.x + ph.y * b.y) / t, (ph.y * b.x - ph.x * b.y) / t);
    }
    cs[j] = c;
    sn[j] = s;
    h[j] = mk(c.x * a.x + (s.x * b.x - s.y * b.y), c.x * a.y + (s.x * b.y + s.y * b.x));
    h[j + 1] = mk(0, 0);
    const double2 gj = g[j];
    g[j] = mk(c.x * gj.x, c.x * gj.y);
    g[j + 1] = mk(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));
    res[0] = sqrt(abs2(g[j + 1]));
}

// GMRES: y = H^{-1} g (upper triangular j1 x j1), into y
__global__ void k_jd_gmres_y(const double2* __restrict__ Hg, int ldh, int j1, const double2* __restrict__ g,
                             double2* __restrict__ y) {
    if (threadIdx.x != 0) return;
    for (int i = j1 - 1; i >= 0; --i) {
        double2 acc = g[i];
        for (int l = i + 1; l < j1; ++l) acc = acc - cmulj(Hg[(size_t)l * ldh + i], y[l]);
        const double2 d = Hg[(size_t)i * ldh + i];
        y[i] = abs2(d) > 0 ? cmulj(acc, cinv(d)) : mk(0, 0);
    }
}

// g = (beta, 0, ...), beta = *nrm
__global__ void k_jd_gmres_init(double2* __restrict__ g, int len, const double* __restrict__ nrm) {
    for (int i = threadIdx.x; i < len; i += blockDim.x) g[i] = i == 0 ? mk(*nrm, 0) : mk(0, 0);
}

// copy a column of coefficients into a matrix column (and the norm below it)
__global__ void k_jd_put_col(double2* __restrict__ dst, const double2* __restrict__ c, int k, const double* __restrict__ nrm,
                             int with_norm) {
    for (int i = threadIdx.x; i < k; i += blockDim.x) dst[i] = c[i];
    if (with_norm && threadIdx.x == 0) dst[k] = mk(*nrm, 0);
}

// M_B row m (entries 0..m-1) = conj(d)
__global__ void k_jd_put_row(double2* __restrict__ MB, int ld, int row, const double2* __restrict__ d, int m) {
    for (int j = threadIdx.x; j < m; j += blockDim.x) MB[(size_t)j * ld + row] = conjj(d[j]);
}

// column norms ||X[:, c]|| into nrm[c]: partial sums per CTA, then one warp per column
__global__ void __launch_bounds__(256) k_jd_nrm_part(const double2* __restrict__ X, int64_t ldx, int64_t n,
                                                     double* __restrict__ part) {
    const int c = blockIdx.y;
    double s = 0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        s += abs2(X[(int64_t)c * ldx + r]);
    __shared__ double red[8];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) a += red[q];
        part[(size_t)c * gridDim.x + blockIdx.x] = a;
    }
}
__global__ void k_jd_nrm_fin(const double* __restrict__ part, int nb, int ncols, double* __restrict__ nrm) {
    const int lane = threadIdx.x & 31, c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (c >= ncols) return;
    double s = 0;
    for (int q = lane; q < nb; q += 32) s += part[(size_t)c * nb + q];
    s = warp_sum(s);
    if (lane == 0) nrm[c] = sqrt(s);
}

// y = a x + b y (a, b by value)
__global__ void k_jd_axpby(double2 a, const double2* __restrict__ x, double2 b, double2* __restrict__ y, int64_t n) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        y[r] = cmulj(a, x[r]) + cmulj(b, y[r]);
}

__global__ void k_jd_add(double2* __restrict__ c, const double2* __restrict__ d, int k) {
    for (int i = threadIdx.x; i < k; i += blockDim.x) c[i] = c[i] + d[i];
}

// S = [Minv MB; 0] (padded to m_pad, ld m_pad + 1) for the final extraction: Minv (k x k, ld ldh),
// MB (k x k, ld k)
__global__ void k_jd_final_g(const double2* __restrict__ Minv, int ldh, const double2* __restrict__ MB, int k, int m_pad,
                             double2* __restrict__ S) {
    const int lds = m_pad + 1;
    for (int idx = threadIdx.x; idx < lds * m_pad; idx += blockDim.x) {
        const int i = idx % lds, j = idx / lds;
        double2 acc = mk(0, 0);
        if (i < k && j < k)
            for (int l = 0; l < k; ++l) acc = acc + cmulj(Minv[(size_t)l * ldh + i], MB[(size_t)j * k + l]);
        S[idx] = acc;
    }
}

// omega_i = tau + 1 / mu_i for the selected harmonic values
__global__ void k_jd_omegas(const double2* __restrict__ musel, int k, double2 tau, double2* __restrict__ om) {
    const int i = threadIdx.x;
    if (i >= k) return;
    const double2 mu = musel[i];
    const double dm = abs2(mu);
    om[i] = dm > 0 ? mk(tau.x + mu.x / dm, tau.y - mu.y / dm) : tau;
}

// the final residuals reuse the (no longer needed) storage of Z^H B Q as doubles
inline double* resid_dev_slot(double2* Mb, int i) { return reinterpret_cast<double*>(Mb) + i; }

// one 256-byte-aligned slab for every workspace array
struct Carver {
    char* base = nullptr;
    size_t off = 0;
    template <typename T>
    void take(T*& ptr, size_t cnt) {
        ptr = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += (sizeof(T) * cnt + 255) & ~size_t(255);
    }
};

}  // namespace
}  // namespace klst

using namespace klst;

extern "C" int klst_jd_eigs(klst_factor f, const klst_jd_opts* o, double* evals_host, void* evecs, double* resid_host,
                            klst_jd_info* info, klst_stream stream) {
    if (!f || !o || !evals_host) { set_error("invalid arguments to klst_jd_eigs"); return KLST_EINVAL; }
    const int nev = o->nev, mmax = o->ncv, kmin = o->kmin, gm = o->gmres_m;
    if (nev < 1 || nev > kJdMaxNev || mmax < 4 || mmax > kJdMaxM || kmin < 1 || kmin >= mmax || gm < 1 ||
        gm > kJdMaxIn || o->gmres_max < 1 || !(o->tol > 0) || !(o->gmres_rtol > 0) || !(o->gmres_atol >= 0) ||
        o->max_outer < 1 || (o->precond != KLST_JD_PREC_FULL && o->precond != KLST_JD_PREC_BLOCK) ||
        (int64_t)mmax + nev + 2 > f->n) {
        set_error("invalid jd options nev=%d ncv=%d kmin=%d gmres_m=%d (need 1 <= nev <= %d, 4 <= ncv <= %d, "
                  "1 <= kmin < ncv, 1 <= gmres_m <= %d)", nev, mmax, kmin, gm, kJdMaxNev, kJdMaxM, kJdMaxIn);
        return KLST_EINVAL;
    }
    if (f->precision != KLST_FP64) {
        set_error("klst_jd_eigs needs a KLST_FP64 factor (its float64 solves are the preconditioner)");
        return KLST_EINVAL;
    }
    auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = (cudaStream_t)stream;
    klst_pencil p = f->p;
    const int64_t n = f->n;
    const int nb = (int)std::min<int64_t>((n + 255) / 256, 2 * device_sm_count());
    const int ng = pencil_work_groups(p);
    const int msch = std::max(mmax, nev + 1);       // largest Schur step (padded sizes included)
    const int log_cap = 31 * msch * msch;
    const int ldH = kJdMaxNev + 1;
    const int prec_mode = o->precond == KLST_JD_PREC_FULL ? 0 : 1;
    const double2 tau = f->sigma;
    // workspace
    double2 *V, *Vb, *Wt, *Wb, *Qs, *Zs, *Ys, *Gm, *r, *t, *y1, *y2, *R, *MB, *Sch, *Hs, *Qsch, *Yc, *Ysel, *mu, *musel;
    double2 *Vh, *Qr, *coef, *coef2, *zc, *theta, *om, *Hq, *Hg, *gcs, *gsn, *gg, *gy, *part, *mw, *mp, *Mt, *Mb;
    double *est, *estsel, *tauh, *npart, *nrm, *scal, *gres;
    Rot *rlog, *rlog2;
    int *rcount, *loff, *rdy, *nconv, *flag;
    char* ozws;
    void* slab = nullptr;
    {
        Carver c;
        for (int pass = 0; pass < 2; ++pass) {
            c.off = 0;
            c.take(V, n * mmax); c.take(Vb, n * mmax); c.take(Wt, n * mmax); c.take(Wb, n * mmax);
            c.take(Qs, n * (nev + 1)); c.take(Zs, n * (nev + 1)); c.take(Ys, n * (nev + 1));
            c.take(Gm, n * (gm + 1));
            c.take(r, n); c.take(t, n); c.take(y1, n); c.take(y2, n);
            c.take(R, (size_t)mmax * mmax); c.take(MB, (size_t)mmax * mmax);
            c.take(Sch, (size_t)(msch + 1) * msch); c.take(Hs, (size_t)msch * msch); c.take(Qsch, (size_t)msch * msch);
            c.take(Yc, (size_t)msch * msch); c.take(Ysel, (size_t)msch * (nev + 1)); c.take(mu, msch);
            c.take(musel, nev + 1); c.take(est, msch); c.take(estsel, nev + 1); c.take(tauh, msch);
            c.take(Vh, (size_t)msch * msch);
            c.take(rlog, log_cap); c.take(rlog2, log_cap); c.take(loff, (size_t)log_cap + 1);
            c.take(rdy, 256); c.take(rcount, 4); c.take(nconv, 4); c.take(flag, 4);
            c.take(Qr, (size_t)mmax * mmax);
            c.take(coef, 2 * (mmax + nev + gm) + 8); c.take(coef2, 2 * (mmax + nev + gm) + 8);
            c.take(zc, mmax); c.take(theta, 4); c.take(om, nev + 4);
            c.take(Hq, (size_t)ldH * ldH);
            c.take(Mt, (size_t)nev * nev); c.take(Mb, (size_t)nev * nev);
            c.take(Hg, (size_t)(gm + 1) * (gm + 1)); c.take(gcs, gm + 1); c.take(gsn, gm + 1);
            c.take(gg, gm + 2); c.take(gy, gm + 1);
            c.take(part, (size_t)nb * (mmax + nev + gm + 8));
            c.take(npart, (size_t)nb * (nev + 4)); c.take(nrm, nev + 4); c.take(scal, 4); c.take(gres, 4);
            c.take(mw, (size_t)4 * p->nx * nev); c.take(mp, (size_t)4 * p->nx * ng * nev);
            c.take(ozws, oz_workspace_bytes((int)n, 2 * mmax, 2 * mmax));
            if (pass == 0) {
                cudaError_t e = dmalloc(&slab, c.off, s);
                if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc", __FILE__, __LINE__);
                c.base = static_cast<char*>(slab);
            }
        }
    }
    int rc = KLST_OK;
    auto fail = [&](int code) { dfree(slab, s); return code; };
#define JD_CK(call)                                                           \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) return fail(cuda_fail(e_, #call, __FILE__, __LINE__)); \
    } while (0)
#define JD_RC(call)                     \
    do {                                \
        if ((rc = (call)) != KLST_OK) return fail(rc); \
    } while (0)
    if ((rc = factor_reserve(f, nev, s)) != KLST_OK) return fail(rc);
    JD_CK(cudaMemsetAsync(f->status, 0, sizeof(Status), s));
    JD_CK(cudaMemsetAsync(flag, 0, sizeof(int) * 4, s));
    JD_CK(cudaMemsetAsync(R, 0, sizeof(double2) * mmax * mmax, s));
    JD_CK(cudaMemsetAsync(MB, 0, sizeof(double2) * mmax * mmax, s));
    int64_t applies_op = 0, applies_prec = 0;
    // ---- primitives
    auto kcheck = [&]() -> int {
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? KLST_OK : cuda_fail(e, "jd kernels", __FILE__, __LINE__);
    };
    auto dots = [&](const double2* X, int k, const double2* y, double2* out) -> int {   // out = X^H y
        if (k <= 0) return KLST_OK;
        k_jd_dots<<<dim3(nb, k), 256, 0, s>>>(X, n, y, n, part); note_launch();
        k_jd_dots_fin<<<(k + 7) / 8, 256, 0, s>>>(part, nb, k, out, 1.0, 0); note_launch();
        return kcheck();
    };
    auto update = [&](const double2* X, int k, const double2* c, double2* y) -> int {   // y -= X c
        if (k <= 0) return KLST_OK;
        k_jd_update<<<nb, 256, 0, s>>>(X, n, k, c, y, n); note_launch();
        return kcheck();
    };
    auto gemv = [&](const double2* X, int k, const double2* c, double2* y) -> int {    // y = X c
        k_jd_gemv<<<nb, 256, 0, s>>>(X, n, k, c, y, n); note_launch();
        return kcheck();
    };
    // y against X, two classical Gram-Schmidt passes; the summed coefficients into c (if given)
    auto cgs2 = [&](const double2* X, int k, double2* y, double2* c) -> int {
        if (k <= 0) return KLST_OK;
        for (int pass = 0; pass < 2; ++pass) {
            int rc2 = dots(X, k, y, pass == 0 && c ? c : coef2);
            if (!rc2) rc2 = update(X, k, pass == 0 && c ? c : coef2, y);
            if (rc2) return rc2;
            if (pass == 1 && c) { k_jd_add<<<1, 128, 0, s>>>(c, coef2, k); note_launch(); }
        }
        return kcheck();
    };
    auto norm = [&](const double2* x, double* out) -> int {
        k_jd_nrm_part<<<dim3(nb, 1), 256, 0, s>>>(x, n, n, npart); note_launch();
        k_jd_nrm_fin<<<1, 32, 0, s>>>(npart, nb, 1, out); note_launch();
        return kcheck();
    };
    auto scale_by = [&](const double2* x, double2* y, const double* d, double sc) -> int {   // y = sc x / *d
        k_jd_scale<<<nb, 256, 0, s>>>(x, y, n, d, sc); note_launch();
        return kcheck();
    };
    auto axpby = [&](double2 a, const double2* x, double2 b, double2* y) -> int {
        k_jd_axpby<<<nb, 256, 0, s>>>(a, x, b, y, n); note_launch();
        return kcheck();
    };
    auto bmask = [&](const double2* x, double2* y) -> int {
        k_jd_bmask<<<nb, 256, 0, s>>>(x, y, n, p->nx, p->nxi, p->xi_x); note_launch();
        return kcheck();
    };
    auto read1 = [&](const double* d, double& h) -> int {
        cudaError_t e = cudaMemcpyAsync(&h, d, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        return e == cudaSuccess ? KLST_OK : cuda_fail(e, "jd read", __FILE__, __LINE__);
    };
    auto set_om = [&](double2 w) -> int {
        const cudaError_t e = cudaMemcpyAsync(om, &w, sizeof(double2), cudaMemcpyHostToDevice, s);
        return e == cudaSuccess ? KLST_OK : cuda_fail(e, "jd omega", __FILE__, __LINE__);
    };
    auto op = [&](const double2* x, double2* y) -> int {   // y = (A - om B) x
        ++applies_op;
        return apply_pencil_dev(p, x, y, 1, om, s, mw, mp, ng);
    };
    auto prec = [&](const double2* x, double2* y) -> int {   // y = K^{-1} x
        ++applies_prec;
        return apply_inv(f, x, y, prec_mode, s);
    };
    auto schur = [&](int m, int keep, int nsel) -> int {
        SchurArgs a;
        a.m = m; a.lds = m + 1; a.S = Sch; a.H = Hs; a.Q = Qsch; a.Yc = Yc; a.mu = mu; a.est = est;
        a.Ysel = Ysel; a.mu_sel = musel; a.est_sel = estsel;
        a.Vh = (float4*)Vh; a.tau = tauh; a.log = rlog; a.log_cap = log_cap; a.log_count = rcount;
        a.log2 = rlog2; a.loff = loff; a.rdy = rdy;
        a.nconv = nconv; a.keep = keep; a.nev = nsel; a.tol = 1.0; a.conv = 0; a.st = f->status;
        const cudaError_t e = cudaMemsetAsync(rcount, 0, sizeof(int) * 4, s);
        if (e != cudaSuccess) return cuda_fail(e, "jd schur", __FILE__, __LINE__);
        return launch_schur64(a, s);
    };
    // rotation of the bases by the Schur vectors: keep columns c0 .. c0 + kk - 1 of V U and W Q_r
    auto rotate = [&](int m, int c0, int kk) -> int {
        const size_t smem = sizeof(double2) * 3 * m * m;
        k_jd_rotate_small<<<1, 256, smem, s>>>(R, MB, mmax, m, Qsch, Qr, c0, kk); note_launch();
        if ((rc = kcheck())) return rc;
        if ((rc = oz_rotate(V, n, m, Qsch + (size_t)c0 * m, kk, Vb, ozws, f->status, s))) return rc;
        if ((rc = oz_rotate(Wt, n, m, Qr, kk, Wb, ozws, f->status, s))) return rc;
        std::swap(V, Vb);
        std::swap(Wt, Wb);
        return KLST_OK;
    };
    {
        static std::atomic<unsigned long long> attr{0};
        JD_CK(set_once_per_device(attr, [] {
            return cudaFuncSetAttribute(k_jd_rotate_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)(sizeof(double2) * 3 * kJdMaxM * kJdMaxM));
        }));
    }
    // ---- the iteration
    int k = 0, m = 0, outer = 0, inner = 0, restarts = 0;
    bool have_t = true;
    if (o->v0) JD_CK(cudaMemcpyAsync(t, o->v0, sizeof(double2) * n, cudaMemcpyDeviceToDevice, s));
    else { k_jd_randn<<<nb, 256, 0, s>>>(t, n, o->seed); note_launch(); }
    while (k < nev && outer < o->max_outer) {
        ++outer;
        if (have_t) {
            // v = t orthonormalised against Q and V
            JD_RC(cgs2(Qs, k, t, nullptr));
            JD_RC(cgs2(V, m, t, nullptr));
            JD_RC(norm(t, scal));
            double tn = 0;
            JD_RC(read1(scal, tn));
            if (!(tn > 0)) { set_error("Jacobi-Davidson: the expansion vector vanished"); return fail(KLST_ENOCONV); }
            double2* vm = V + (int64_t)m * n;
            JD_RC(scale_by(t, vm, scal, 1.0));
            // w~ = (A - tau B) v against Z, then W (coefficients: R[0:m, m]); R[m, m] = ||w~||
            JD_RC(set_om(tau));
            JD_RC(op(vm, y1));
            JD_RC(cgs2(Zs, k, y1, nullptr));
            JD_RC(cgs2(Wt, m, y1, coef));
            JD_RC(norm(y1, scal));
            k_jd_put_col<<<1, 64, 0, s>>>(R + (size_t)m * mmax, coef, m, scal, 1); note_launch();
            double2* wm = Wt + (int64_t)m * n;
            JD_RC(scale_by(y1, wm, scal, 1.0));
            // M_B: column m = W^H B v; row m = conj(V^H B w)
            JD_RC(bmask(vm, y2));
            JD_RC(dots(Wt, m + 1, y2, MB + (size_t)m * mmax));
            if (m > 0) {
                JD_RC(bmask(wm, y2));
                JD_RC(dots(V, m, y2, coef));
                k_jd_put_row<<<1, 64, 0, s>>>(MB, mmax, m, coef, m); note_launch();
            }
            ++m;
            have_t = false;
        }
        // harmonic pairs: G = R^{-1} M_B (padded to 2 when m = 1), Schur form sorted by |mu|
        const int mpad = std::max(m, 2);
        k_jd_small_g<<<1, 64, 0, s>>>(R, MB, mmax, m, mpad, Sch, flag); note_launch();
        JD_RC(schur(mpad, std::min(mpad - 1, kmin), 1));
        k_jd_pick<<<1, 64, 0, s>>>(R, mmax, m, Ysel, mpad, musel, tau, zc, theta, scal); note_launch();
        // u = V y and z = W zc at column k of Q and Z (the projectors' q~ = [Q u], z~ = [Z z])
        double2* uq = Qs + (int64_t)k * n;
        double2* zz = Zs + (int64_t)k * n;
        JD_RC(gemv(V, m, Ysel, uq));
        JD_RC(gemv(Wt, m, zc, zz));
        double2 th;
        int hflag[2] = {0, 0}, hconv = 0;
        JD_CK(cudaMemcpyAsync(&th, theta, sizeof(double2), cudaMemcpyDeviceToHost, s));
        JD_CK(cudaMemcpyAsync(hflag, flag, sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
        JD_CK(cudaMemcpyAsync(&hconv, nconv, sizeof(int), cudaMemcpyDeviceToHost, s));
        JD_CK(cudaStreamSynchronize(s));
        if (hflag[0] || hflag[1] || hconv < 0) {
            set_error("Jacobi-Davidson: breakdown of the projected problem");
            return fail(KLST_ENOCONV);
        }
        // r = (I - Z Z^H)(A - theta B) u
        JD_RC(set_om(th));
        JD_RC(op(uq, r));
        JD_RC(cgs2(Zs, k, r, nullptr));
        double rn = 0;
        JD_RC(norm(r, scal));
        JD_RC(read1(scal, rn));
        if (rn <= o->tol * sqrt(abs2(th))) {
            // lock u and z; drop the first Schur direction from V and W
            ++k;
            if (m >= 2) JD_RC(rotate(m, 1, m - 1));
            --m;
            if (m == 0) { k_jd_randn<<<nb, 256, 0, s>>>(t, n, o->seed + 7919 * (uint64_t)k); note_launch(); have_t = true; }
            continue;
        }
        if (m == mmax) {   // restart to the kmin leading directions (u stays first)
            JD_RC(rotate(m, 0, kmin));
            m = kmin;
            ++restarts;
        }
        // correction equation, GMRES on the left-preconditioned projected operator
        const int k1 = k + 1;
        JD_RC(prec(zz, Ys + (int64_t)k * n));
        for (int c = 0; c < k1; ++c) JD_RC(dots(Qs, k1, Ys + (int64_t)c * n, Hq + (size_t)c * ldH));
        k_jd_hinv<<<1, 1, 0, s>>>(Hq, k1, flag + 1); note_launch();
        {
            int hf = 0;
            JD_CK(cudaMemcpyAsync(&hf, flag + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
            JD_CK(cudaStreamSynchronize(s));
            if (hf) {
                set_error("Jacobi-Davidson: the projected preconditioner q~^H K^{-1} z~ is singular");
                return fail(KLST_ENOCONV);
            }
        }
        auto kproj = [&](const double2* in, double2* out) -> int {   // out = K~^{-1} in
            int rc2 = prec(in, out);
            if (!rc2) rc2 = dots(Qs, k1, out, coef2);
            if (rc2) return rc2;
            k_jd_hsolve<<<1, 128, 0, s>>>(Hq, k1, coef2, coef); note_launch();
            return update(Ys, k1, coef, out);
        };
        auto opx = [&](const double2* x, double2* out) -> int {      // out = K~^{-1} (I - z~ z~^H)(A - theta B) x
            int rc2 = op(x, y1);
            if (!rc2) rc2 = dots(Zs, k1, y1, coef2);
            if (!rc2) rc2 = update(Zs, k1, coef2, y1);
            if (!rc2) rc2 = kproj(y1, out);
            return rc2;
        };
        JD_CK(cudaMemsetAsync(t, 0, sizeof(double2) * n, s));
        JD_RC(kproj(r, y2));                            // b = -y2
        JD_RC(axpby(mk(0, 0), y2, mk(-1, 0), y2));      // y2 = b: the residual of t = 0
        double bn = 0;
        JD_RC(norm(y2, scal));
        JD_RC(read1(scal, bn));
        const double target = std::max(o->gmres_rtol * bn, o->gmres_atol);
        double res = bn;
        int its = 0;
        while (its < o->gmres_max && res > target) {
            // the cycle starts from the residual in y2 (its norm in scal)
            JD_RC(scale_by(y2, Gm, scal, 1.0));
            k_jd_gmres_init<<<1, 64, 0, s>>>(gg, gm + 2, scal); note_launch();
            int j = 0;
            while (j < gm && its < o->gmres_max) {
                double2* gw = Gm + (int64_t)(j + 1) * n;
                JD_RC(opx(Gm + (int64_t)j * n, gw));
                JD_RC(cgs2(Gm, j + 1, gw, coef));
                JD_RC(norm(gw, scal));
                k_jd_put_col<<<1, 64, 0, s>>>(Hg + (size_t)j * (gm + 1), coef, j + 1, scal, 1); note_launch();
                JD_RC(scale_by(gw, gw, scal, 1.0));
                k_jd_givens<<<1, 1, 0, s>>>(Hg, gm + 1, j, gcs, gsn, gg, gres); note_launch();
                ++j;
                ++its;
                ++inner;
                JD_RC(read1(gres, res));
                if (res <= target) break;
            }
            // t += Gm[:, 0:j] H^{-1} g
            k_jd_gmres_y<<<1, 1, 0, s>>>(Hg, gm + 1, j, gg, gy); note_launch();
            JD_RC(gemv(Gm, j, gy, y1));
            JD_RC(axpby(mk(1, 0), y1, mk(1, 0), t));
            if (res <= target || its >= o->gmres_max) break;
            // next cycle: residual b - Op t = -(K~^{-1} r) - Op t
            JD_RC(opx(t, y2));
            JD_RC(kproj(r, y1));
            JD_RC(axpby(mk(-1, 0), y1, mk(-1, 0), y2));
            JD_RC(norm(y2, scal));
            JD_RC(read1(scal, res));
        }
        have_t = true;
    }
    // ---- the eigenpairs: harmonic extraction on the locked space Q (k columns)
    const int kk = k;
    std::vector<double2> omh(std::max(kk, 1));
    std::vector<double> resh(std::max(kk, 1), 0.0);
    if (kk > 0) {
        // Mt = Z^H (A - tau B) Q, Mb = Z^H B Q (kk x kk); (A - tau B) Q into Ys, B Q into Gm/Vb
        std::vector<double2> taus(kk, tau);
        JD_CK(cudaMemcpyAsync(om, taus.data(), sizeof(double2) * kk, cudaMemcpyHostToDevice, s));
        applies_op += kk;
        JD_RC(apply_pencil_dev(p, Qs, Ys, kk, om, s, mw, mp, ng));
        for (int c = 0; c < kk; ++c) {
            JD_RC(dots(Zs, kk, Ys + (int64_t)c * n, Mt + (size_t)c * kk));
            JD_RC(bmask(Qs + (int64_t)c * n, y2));
            JD_RC(dots(Zs, kk, y2, Mb + (size_t)c * kk));
        }
        // Hq <- Mt, inverted; S = [Mt^{-1} Mb; 0] padded to kk + 1
        JD_CK(cudaMemsetAsync(Hq, 0, sizeof(double2) * ldH * ldH, s));
        JD_CK(cudaMemcpy2DAsync(Hq, sizeof(double2) * ldH, Mt, sizeof(double2) * kk, sizeof(double2) * kk, kk,
                                cudaMemcpyDeviceToDevice, s));
        k_jd_hinv<<<1, 1, 0, s>>>(Hq, kk, flag + 1); note_launch();
        const int mf = kk + 1;
        k_jd_final_g<<<1, 256, 0, s>>>(Hq, ldH, Mb, kk, mf, Sch); note_launch();
        JD_RC(kcheck());
        JD_RC(schur(mf, kk, kk));
        k_jd_omegas<<<1, 64, 0, s>>>(musel, kk, tau, om); note_launch();
        // x_i = Q Ysel[:, i] normalised, into Gm/Ys storage (Ys is free now)
        for (int i = 0; i < kk; ++i) JD_RC(gemv(Qs, kk, Ysel + (size_t)i * mf, Ys + (int64_t)i * n));
        k_jd_nrm_part<<<dim3(nb, kk), 256, 0, s>>>(Ys, n, n, npart); note_launch();
        k_jd_nrm_fin<<<(kk + 7) / 8, 256, 0, s>>>(npart, nb, kk, nrm); note_launch();
        for (int i = 0; i < kk; ++i) JD_RC(scale_by(Ys + (int64_t)i * n, Ys + (int64_t)i * n, nrm + i, 1.0));
        // explicit residuals ||(A - omega_i B) x_i||
        for (int i = 0; i < kk; ++i) {
            ++applies_op;
            JD_RC(apply_pencil_dev(p, Ys + (int64_t)i * n, y1, 1, om + i, s, mw, mp, ng));
            JD_RC(norm(y1, nrm + nev + 2));
            JD_CK(cudaMemcpyAsync(resid_dev_slot(Mb, i), nrm + nev + 2, sizeof(double), cudaMemcpyDeviceToDevice, s));
        }
        JD_RC(kcheck());
        JD_CK(cudaMemcpyAsync(omh.data(), om, sizeof(double2) * kk, cudaMemcpyDeviceToHost, s));
        JD_CK(cudaMemcpyAsync(resh.data(), resid_dev_slot(Mb, 0), sizeof(double) * kk, cudaMemcpyDeviceToHost, s));
        if (evecs) JD_CK(cudaMemcpyAsync(evecs, Ys, sizeof(double2) * n * kk, cudaMemcpyDeviceToDevice, s));
        int hflag[2] = {0, 0}, hconv = 0;
        JD_CK(cudaMemcpyAsync(hflag, flag, sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
        JD_CK(cudaMemcpyAsync(&hconv, nconv, sizeof(int), cudaMemcpyDeviceToHost, s));
        JD_CK(cudaStreamSynchronize(s));
        if (hflag[1] || hconv < 0) { set_error("Jacobi-Davidson: singular projected problem on the locked space"); return fail(KLST_ENOCONV); }
    }
    Status fst;
    JD_CK(cudaMemcpyAsync(&fst, f->status, sizeof(Status), cudaMemcpyDeviceToHost, s));
    JD_CK(cudaStreamSynchronize(s));
    double maxres = 0;
    for (int i = 0; i < kk; ++i) {
        evals_host[2 * i] = omh[i].x;
        evals_host[2 * i + 1] = omh[i].y;
        if (resid_host) resid_host[i] = resh[i];
        maxres = std::max(maxres, resh[i]);
    }
    if (info) {
        info->nconv = kk;
        info->outer = outer;
        info->inner = inner;
        info->restarts = restarts;
        info->applies_op = applies_op;
        info->applies_prec = applies_prec;
        info->t_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        info->max_resid = maxres;
    }
    dfree(slab, s);
#undef JD_CK
#undef JD_RC
    if (fst.flags & ST_TIMEOUT) { set_error("Jacobi-Davidson: a bounded device wait gave up"); return KLST_ETIMEOUT; }
    if (kk < nev) { set_error("Jacobi-Davidson: %d of %d eigenpairs converged in %d outer iterations", kk, nev, outer); return KLST_ENOCONV; }
    return KLST_OK;
}
