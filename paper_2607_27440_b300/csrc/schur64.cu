// The small dense step of the Krylov-Schur restart (Sec. 4.1) in float64: Householder reduction of
// the (keep + 1)-spiked Krylov-Schur matrix to Hessenberg form, shifted QR sweeps with Givens
// rotations to the complex Schur form, reordering so the Ritz values of largest |mu| lead, and the
// Schur vectors rebuilt from the reflectors and the logged rotations.  Same algorithm and data flow
// as the double-float kernels of schur.cu, with float64 operands, float64 deflation (unit
// roundoff 2^-53) and float64 rotations; k_schur_post (Ritz estimates, selection, truncation) is
// shared.
#include "factor.cuh"

namespace klst {

struct Rot64 {         // rotation [c s; -conj(s) c] of rows/columns (i, i+1), float64
    double2 s;
    double c;
    int i;
    int pad;
};
static_assert(sizeof(Rot64) == sizeof(Rot), "the rotation log is shared by both arithmetics");

__device__ __forceinline__ double cabs1_64(double2 a) { return fabs(a.x) + fabs(a.y); }

// x' = c x + s y, y' = c y - conj(s) x (real c).  The terms without x are formed first, so a
// caller that carries y' into the next rotation as its x waits on two float64 operations only.
__device__ __forceinline__ void crot64(double2& x, double2& y, double c, double2 s) {
    const double2 sy = make_double2(fma(s.x, y.x, -s.y * y.y), fma(s.x, y.y, s.y * y.x));
    const double2 cy = make_double2(c * y.x, c * y.y);
    const double2 tx = make_double2(fma(c, x.x, sy.x), fma(c, x.y, sy.y));
    const double2 ty = make_double2(fma(-s.x, x.x, fma(-s.y, x.y, cy.x)), fma(-s.x, x.y, fma(s.y, x.x, cy.y)));
    x = tx;
    y = ty;
}

// 1 / sqrt(x) for a normal x > 0 to float64 accuracy with four dependent float64 operations: x is
// scaled by an even power of two into [1, 4) (integer operations on its bits), the float32
// reciprocal square root gives y0 with |1 - x y0^2| = e ~ 2^-22, and the exact value
// y0 (1 - e)^(-1/2) = y0 (1 + e/2 + 3 e^2/8 + O(e^3)) is taken to second order (error ~2^-66).
// The float32 value and the float64 it feeds are built from bits, off the float64 pipe.
__device__ __forceinline__ double rsqrt64(double x) {
    const long long b = __double_as_longlong(x);
    const int k = ((int)((b >> 52) & 0x7FF) - 1023) >> 1;                 // x = xm 4^k, xm in [1, 4)
    const double xm = __longlong_as_double(b - ((long long)(2 * k) << 52));
    const long long bm = __double_as_longlong(xm);
    const float xf = __uint_as_float((unsigned)(((bm >> 52) - 1023 + 127) << 23) | (unsigned)((bm >> 29) & 0x7FFFFF));
    const unsigned yb = __float_as_uint(rsqrtf(xf));
    const double y0 = __longlong_as_double(((long long)(((yb >> 23) & 0xFF) - 127 + 1023) << 52) |
                                           ((long long)(yb & 0x7FFFFF) << 29));
    const double e = fma(-(xm * y0), y0, 1.0);
    const double y = fma(y0 * e, fma(0.375, e, 0.5), y0);
    return __longlong_as_double(__double_as_longlong(y) - ((long long)k << 52));  // y 2^-k
}

// [c s; -conj(s) c] [f; g] = [r; 0] with real c = |f| / r, s = f conj(g) / (|f| r),
// r = sqrt(|f|^2 + |g|^2) (the LAPACK zlartg convention), from two independent reciprocal square
// roots (no float64 division or square root on the dependent chain).  The entries of the
// Krylov-Schur matrix are far inside the float64 range, so no scaling is needed; an |f|^2 or |g|^2
// below 1e-290 is treated as zero.
__device__ void givens64(double2 f, double2 g, double& c, double2& s) {
    const double ag2 = abs2(g), af2 = abs2(f);
    if (!(ag2 > 1e-290)) { c = 1.0; s = make_double2(0.0, 0.0); return; }
    if (!(af2 > 1e-290)) {  // |f| negligible: c = 0, s = conj(g) / |g|
        const double ig = rsqrt64(ag2);
        c = 0.0;
        s = make_double2(g.x * ig, -g.y * ig);
        return;
    }
    const double ir = rsqrt64(af2 + ag2), iaf = rsqrt64(af2);
    c = (af2 * iaf) * ir;
    const double q = iaf * ir;
    s = make_double2((f.x * g.x + f.y * g.y) * q, (f.y * g.x - f.x * g.y) * q);
}

__device__ double block_sum64(double v, double* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    for (int i = 0; i < nw; ++i) s += red[i];
    __syncthreads();
    return s;
}

// ---------------------------------------------------------------- 1. Householder reduction
// H_c = I - tau_c v_c v_c^H zeroes column c below the subdiagonal; H (global, column-major)
// receives the Hessenberg matrix, v_c is kept in Vh for the Q rebuild.
__global__ void __launch_bounds__(256) k_schur_house64(SchurArgs a) {
    const int m = a.m, tid = threadIdx.x, nt = blockDim.x;
    double2* H = a.H;
    double2* Vh = reinterpret_cast<double2*>(a.Vh);
    __shared__ double2 v[192];
    __shared__ double red[8];
#define HH(i, j) H[(size_t)(j) * m + (i)]
    for (int idx = tid; idx < m * m; idx += nt) {
        const int i = idx % m, j = idx / m;
        H[idx] = a.S[(size_t)j * a.lds + i];
    }
    for (int i = tid; i < m; i += nt) a.tau[i] = 0.0;
    if (tid == 0) { *a.nconv = 0; *a.log_count = 0; }
    __syncthreads();
    for (int c = 0; c + 2 < m; ++c) {
        double tail = 0.0;
        for (int i = c + 2 + tid; i < m; i += nt) tail += abs2(HH(i, c));
        tail = block_sum64(tail, red);
        if (tail == 0.0) continue;
        const double2 x0 = HH(c + 1, c);
        const double ax02 = abs2(x0), s2 = tail + ax02;
        if (s2 < 1e-60) {  // every subdiagonal entry below 1e-30: negligible, set to zero
            __syncthreads();
            for (int i = c + 2 + tid; i < m; i += nt) HH(i, c) = make_double2(0.0, 0.0);
            __syncthreads();
            continue;
        }
        const double alpha = sqrt(s2);
        double ax0 = 0.0;
        double2 ph = make_double2(1.0, 0.0);
        if (ax02 > 1e-200) {
            ax0 = sqrt(ax02);
            ph = make_double2(x0.x / ax0, x0.y / ax0);
        }
        const double2 bet = make_double2(-alpha * ph.x, -alpha * ph.y);  // new subdiagonal entry
        const int len = m - c - 1;
        for (int i = tid; i < len; i += nt) {
            const double2 vi = (i == 0) ? x0 - bet : HH(c + 1 + i, c);
            v[i] = vi;
            Vh[(size_t)c * m + c + 1 + i] = vi;
        }
        __syncthreads();
        const double tau = 1.0 / (alpha * (alpha + ax0));  // 2 / ||v||^2
        if (tid == 0) a.tau[c] = tau;
        // left: H[c+1:, col] -= tau v (v^H H[c+1:, col]) for col > c
        for (int col = c + 1 + tid; col < m; col += nt) {
            double2 g0 = make_double2(0.0, 0.0), g1 = g0;
            int i = 0;
            for (; i + 1 < len; i += 2) {
                cfma_conj(g0, v[i], HH(c + 1 + i, col));
                cfma_conj(g1, v[i + 1], HH(c + 2 + i, col));
            }
            if (i < len) cfma_conj(g0, v[i], HH(c + 1 + i, col));
            const double2 g = (-tau) * (g0 + g1);
            for (i = 0; i < len; ++i) {
                double2 hv = HH(c + 1 + i, col);
                cfma(hv, v[i], g);
                HH(c + 1 + i, col) = hv;
            }
        }
        if (tid == 0) {
            HH(c + 1, c) = bet;
            for (int i = c + 2; i < m; ++i) HH(i, c) = make_double2(0.0, 0.0);
        }
        __syncthreads();
        // right: row[c+1:] -= tau (row[c+1:] v) v^H for every row of H
        for (int row = tid; row < m; row += nt) {
            double2 g0 = make_double2(0.0, 0.0), g1 = g0;
            int i = 0;
            for (; i + 1 < len; i += 2) {
                cfma(g0, HH(row, c + 1 + i), v[i]);
                cfma(g1, HH(row, c + 2 + i), v[i + 1]);
            }
            if (i < len) cfma(g0, HH(row, c + 1 + i), v[i]);
            const double2 g = (-tau) * (g0 + g1);
            for (i = 0; i < len; ++i) {
                double2 hv = HH(row, c + 1 + i);
                cfma(hv, g, conj(v[i]));
                HH(row, c + 1 + i) = hv;
            }
        }
        __syncthreads();
    }
#undef HH
}

// ---------------------------------------------------------------- 2. QR sweeps + reordering
// Packed upper-Hessenberg storage in shared memory: column j keeps rows 0..j+1 at offset j(j+3)/2.
__device__ __forceinline__ int pk64(int i, int j) { return j * (j + 3) / 2 + i; }

__global__ void __launch_bounds__(256) k_schur_qr64(SchurArgs a) {
    extern __shared__ double2 sT64[];
    const int m = a.m, tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
    Rot64* log = reinterpret_cast<Rot64*>(a.log);
    __shared__ double rc[192];
    __shared__ double2 rs[192];
    __shared__ double2 s_mu;
    __shared__ int s_lo, s_fail, s_cnt;
#define TT(i, j) sT64[pk64(i, j)]
    for (int j = 0; j < m; ++j)
        for (int i = tid; i <= min(j + 1, m - 1); i += nt) TT(i, j) = a.H[(size_t)j * m + i];
    if (tid == 0) { s_fail = 0; s_cnt = 0; }
    __syncthreads();
    const double2 zero2 = make_double2(0.0, 0.0);
    const double eps = 2.220446049250313e-16;  // float64 ulp(1): LAPACK's deflation threshold
    int hi = m - 1, its = 0, total = 0;
    const int max_total = 30 * m;
    while (hi > 0) {
        if (wid == 0) {
            // deflation: the largest l in [1, hi] whose subdiagonal entry is negligible (0 if none)
            int l = 0;
            for (int base = hi; base >= 1; base -= 32) {
                const int ll = base - lane;
                bool neg = false;
                if (ll >= 1) {
                    const double sub = cabs1_64(TT(ll, ll - 1));
                    double sc = cabs1_64(TT(ll - 1, ll - 1)) + cabs1_64(TT(ll, ll));
                    if (sc == 0.0) sc = 1.0;
                    neg = sub <= eps * sc;
                }
                const unsigned b = __ballot_sync(0xffffffffu, neg);
                if (b) { l = base - (__ffs(b) - 1); break; }
            }
            if (lane == 0) {
                if (l >= 1) TT(l, l - 1) = zero2;
                s_lo = l;
                if (l < hi) {
                    const double2 aa = TT(hi - 1, hi - 1), bb = TT(hi - 1, hi), cc = TT(hi, hi - 1), dd = TT(hi, hi);
                    double2 mu;
                    if (its > 0 && its % 11 == 0) {
                        mu = dd + make_double2(0.75 * cabs1_64(cc), 0.0);  // exceptional shift
                    } else {
                        // Wilkinson shift: the eigenvalue of the trailing 2x2 nearer dd
                        const double2 hd = 0.5 * (aa - dd);
                        const double2 disc = hd * hd + bb * cc;
                        const double r = sqrt(abs2(disc));
                        const double sr = sqrt(0.5 * (r + fabs(disc.x)));
                        double2 sq;
                        if (sr == 0.0) sq = zero2;
                        else if (disc.x >= 0) sq = make_double2(sr, disc.y / (2.0 * sr));
                        else sq = make_double2(fabs(disc.y) / (2.0 * sr), disc.y >= 0 ? sr : -sr);
                        const double2 m1 = 0.5 * (aa + dd) + sq, m2 = 0.5 * (aa + dd) - sq;
                        mu = abs2(m1 - dd) < abs2(m2 - dd) ? m1 : m2;
                    }
                    s_mu = mu;
                    if (s_cnt + (hi - l) > a.log_cap) s_fail = 2;
                }
            }
        }
        __syncthreads();
        const int lo = s_lo;
        if (lo == hi) { hi -= 1; its = 0; __syncthreads(); continue; }
        if (s_fail || ++total > max_total) { if (tid == 0) s_fail = s_fail ? s_fail : 1; break; }
        ++its;
        const double2 mu = s_mu;
        for (int i = lo + tid; i <= hi; i += nt) TT(i, i) = TT(i, i) - mu;
        __syncthreads();
        if (tid == 0) {
            double c;
            double2 sv;
            givens64(TT(lo, lo), TT(lo + 1, lo), c, sv);
            rc[lo] = c;
            rs[lo] = sv;
        }
        __syncthreads();
        // left sweep: rotation i on rows i, i+1 (columns i..m-1); the thread holding column i+1
        // forms rotation i+1 from its freshly rotated diagonal entry.  (Restricting the sweeps to
        // the active window and replaying the rest from the log on other SMs was measured slower:
        // the sweep's cost is its chain of float64 instructions, which the window does not shorten.)
        for (int i = lo; i < hi; ++i) {
            const int col = i + tid;
            if (col < m) {
                const double c = rc[i];
                const double2 sv = rs[i];
                double2 x = TT(i, col), y = TT(i + 1, col);
                crot64(x, y, c, sv);
                TT(i, col) = x;
                TT(i + 1, col) = (col == i) ? zero2 : y;
                if (col == i + 1 && i + 1 < hi) {
                    double c2;
                    double2 s2;
                    givens64(y, TT(i + 2, i + 1), c2, s2);
                    rc[i + 1] = c2;
                    rs[i + 1] = s2;
                }
            }
            __syncthreads();
        }
        // right sweep in bulk: row r receives rotations i >= max(lo, r - 1), in order
        for (int r = tid; r <= hi; r += nt) {
            const int i0 = max(lo, r - 1);
            if (i0 >= hi) continue;
            double2 x = TT(r, i0);
            for (int i = i0; i < hi; ++i) {
                double2 y = TT(r, i + 1);
                crot64(x, y, rc[i], conj(rs[i]));
                TT(r, i) = x;
                x = y;
            }
            TT(r, hi) = x;
        }
        __syncthreads();
        for (int i = lo + tid; i <= hi; i += nt) TT(i, i) = TT(i, i) + mu;
        const int base = s_cnt;
        for (int t = tid; t < hi - lo; t += nt) {
            Rot64 g;
            g.s = rs[lo + t]; g.c = rc[lo + t]; g.i = lo + t; g.pad = 0;
            log[base + t] = g;
        }
        __syncthreads();
        if (tid == 0) s_cnt = base + (hi - lo);
        __syncthreads();
    }
    __syncthreads();
    if (s_fail) {
        if (tid == 0) { atomicOr(&a.st->flags, ST_NOCONV_QR); *a.nconv = -1; *a.log_count = 0; }
        return;
    }
    for (int j = tid; j + 1 < m; j += nt) TT(j + 1, j) = zero2;
    __syncthreads();
    for (int idx = tid; idx < m * m; idx += nt) {
        const int i = idx % m, j = idx / m;
        a.H[idx] = (i <= j) ? TT(i, j) : zero2;
    }
    if (tid == 0) { *a.log_count = s_cnt; a.log_count[1] = total; }
#undef TT
}

constexpr int kLogChunk = 256;  // rotation-log entries staged in shared memory at a time

// Reordering: bring the keep Ritz values of largest |mu| to the front of the upper triangular T by
// adjacent swaps (ties resolve to the lower index), appending each swap's rotation to the log.
__global__ void __launch_bounds__(256) k_schur_reorder64(SchurArgs a) {
    extern __shared__ double2 sT64[];
    const int m = a.m, tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
    if (*a.nconv < 0) return;  // the QR sweeps failed; the host reports it
    Rot64* log = reinterpret_cast<Rot64*>(a.log);
    __shared__ double s_c;
    __shared__ double2 s_s;
    __shared__ int s_q, s_fail, s_cnt, s_swaps;
#define TT(i, j) sT64[pk64(i, j)]
    for (int j = 0; j < m; ++j)
        for (int i = tid; i <= min(j + 1, m - 1); i += nt) TT(i, j) = a.H[(size_t)j * m + i];
    if (tid == 0) { s_fail = 0; s_cnt = *a.log_count; s_swaps = 0; }
    __syncthreads();
    const double2 zero2 = make_double2(0.0, 0.0);
    for (int p = 0; p < a.keep; ++p) {
        if (wid == 0) {
            double bv = -1.0;
            int q = p;
            for (int i = p + lane; i < m; i += 32) {
                const double v = abs2(TT(i, i));
                if (v > bv) { bv = v; q = i; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
                const int oq = __shfl_xor_sync(0xffffffffu, q, o);
                if (ov > bv || (ov == bv && oq < q)) { bv = ov; q = oq; }
            }
            if (lane == 0) {
                s_q = q;
                if (s_cnt + (q - p) > a.log_cap) { s_fail = 2; s_q = p; }
            }
        }
        __syncthreads();
        const int q = s_q;
        for (int i = q - 1; i >= p; --i) {
            if (tid == 0) {
                double c;
                double2 sv;
                givens64(TT(i, i + 1), TT(i + 1, i + 1) - TT(i, i), c, sv);
                s_c = c;
                s_s = sv;
                Rot64 g;
                g.s = sv; g.c = c; g.i = i; g.pad = 0;
                log[s_cnt] = g;
                s_cnt = s_cnt + 1;
                s_swaps = s_swaps + 1;
            }
            __syncthreads();
            const double c = s_c;
            const double2 sv = s_s, sc = conj(sv);
            const double2 t11 = TT(i, i), t22 = TT(i + 1, i + 1);
            for (int idx = tid; idx < (m - i - 2) + i; idx += nt) {
                if (idx < m - i - 2) {
                    const int col = i + 2 + idx;
                    double2 x = TT(i, col), y = TT(i + 1, col);
                    crot64(x, y, c, sv);
                    TT(i, col) = x; TT(i + 1, col) = y;
                } else {
                    const int row = idx - (m - i - 2);
                    double2 x = TT(row, i), y = TT(row, i + 1);
                    crot64(x, y, c, sc);
                    TT(row, i) = x; TT(row, i + 1) = y;
                }
            }
            __syncthreads();
            if (tid == 0) { TT(i, i) = t22; TT(i + 1, i + 1) = t11; }
            __syncthreads();
        }
    }
    if (s_fail) {
        if (tid == 0) { atomicOr(&a.st->flags, ST_NOCONV_QR); *a.nconv = -1; *a.log_count = 0; }
        return;
    }
    for (int idx = tid; idx < m * m; idx += nt) {
        const int i = idx % m, j = idx / m;
        a.H[idx] = (i <= j) ? TT(i, j) : zero2;
    }
    if (tid == 0) { *a.log_count = s_cnt; a.log_count[2] = s_swaps; }
#undef TT
}

// ---------------------------------------------------------------- 3. Schur vectors
// Row r of Q = e_r^T H_0 H_1 ... H_{m-3} G_1^H G_2^H ...: the reflectors, then every logged rotation
// in order.  One warp per CTA, four rows per CTA (the float64 pipe of one SM serves few lanes, so
// the rows are spread over many SMs); a row lives in shared memory.  The rotation log is staged
// into shared memory 256 entries at a time by the whole warp, so the serial replay of the four
// rows reads its rotations from shared memory instead of waiting on L2 for each one.
__global__ void __launch_bounds__(32) k_schur_q64(SchurArgs a) {
    extern __shared__ double2 q64[];  // [m][RPC], then the log chunk
    constexpr int RPC = 4;
    const int m = a.m, t = threadIdx.x, r = blockIdx.x * RPC + t;
    const bool row_lane = t < RPC;
    Rot64* slog = reinterpret_cast<Rot64*>(q64 + (size_t)m * RPC);
    const Rot64* log = reinterpret_cast<const Rot64*>(a.log);
    const double2* Vh = reinterpret_cast<const double2*>(a.Vh);
    if (row_lane) {
        for (int col = 0; col < m; ++col) q64[col * RPC + t] = make_double2(col == r ? 1.0 : 0.0, 0.0);
        for (int c = 0; c + 2 < m; ++c) {
            const double tau = a.tau[c];
            if (tau == 0.0) continue;
            const double2* vc = Vh + (size_t)c * m;
            double2 g0 = make_double2(0.0, 0.0), g1 = g0;
            int i = c + 1;
            for (; i + 1 < m; i += 2) {
                cfma(g0, q64[i * RPC + t], vc[i]);
                cfma(g1, q64[(i + 1) * RPC + t], vc[i + 1]);
            }
            if (i < m) cfma(g0, q64[i * RPC + t], vc[i]);
            const double2 g = (-tau) * (g0 + g1);
            for (i = c + 1; i < m; ++i) {
                double2 qi = q64[i * RPC + t];
                cfma(qi, g, conj(vc[i]));
                q64[i * RPC + t] = qi;
            }
        }
    }
    // runs of rotations in planes (i, i+1), (i+1, i+2), ... carry column i+1 in registers
    const int nrot = *a.log_count;
    int ci = -1;
    double2 cx = make_double2(0.0, 0.0);
    for (int k0 = 0; k0 < nrot; k0 += kLogChunk) {
        const int cnt = min(kLogChunk, nrot - k0);
        for (int i = t; i < cnt; i += 32) slog[i] = log[k0 + i];  // the whole warp stages the chunk
        __syncwarp();
        if (row_lane) {
            for (int k = 0; k < cnt; ++k) {
                const Rot64 g = slog[k];
                double2 x;
                if (g.i == ci) x = cx;
                else {
                    if (ci >= 0) q64[ci * RPC + t] = cx;
                    x = q64[g.i * RPC + t];
                }
                double2 y = q64[(g.i + 1) * RPC + t];
                crot64(x, y, g.c, conj(g.s));
                q64[g.i * RPC + t] = x;
                ci = g.i + 1;
                cx = y;
            }
        }
        __syncwarp();  // the chunk is consumed before the next one overwrites it
    }
    if (!row_lane) return;
    if (ci >= 0) q64[ci * RPC + t] = cx;
    if (r < m)
        for (int col = 0; col < m; ++col) a.Q[(size_t)col * m + r] = q64[col * RPC + t];
}

int launch_schur64(const SchurArgs& a, cudaStream_t s) {
    static std::atomic<unsigned long long> attr{0};
    if (once_per_device(attr)) {
        KLST_CK(cudaFuncSetAttribute(k_schur_qr64, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024));
        KLST_CK(cudaFuncSetAttribute(k_schur_reorder64, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024));
    }
    const int m = a.m;
    const size_t packed = sizeof(double2) * (size_t)m * (m + 3) / 2;
    prof_begin("schur_house", s);
    k_schur_house64<<<1, 256, 0, s>>>(a); note_launch();
    prof_end("schur_house", s);
    prof_begin("schur_qr", s);
    k_schur_qr64<<<1, 256, packed, s>>>(a); note_launch();
    prof_end("schur_qr", s);
    prof_begin("schur_reorder", s);
    k_schur_reorder64<<<1, 256, packed, s>>>(a); note_launch();
    prof_end("schur_reorder", s);
    prof_begin("schur_q", s);
    k_schur_q64<<<(m + 3) / 4, 32, sizeof(double2) * 4 * m + sizeof(Rot64) * kLogChunk, s>>>(a); note_launch();
    prof_end("schur_q", s);
    launch_schur_post(a, s);
    KLST_CK_LAUNCH();
    return KLST_OK;
}

}  // namespace klst
