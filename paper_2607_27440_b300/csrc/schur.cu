// Small dense step of the Krylov-Schur restart (Sec. 4.1: restarted Arnoldi with a filter that
// keeps the wanted Ritz values), on the device:
//   S_m = Q T Q^H: Householder reduction to Hessenberg form, then shifted QR with Givens
//   rotations to the complex Schur form; T is reordered so the Ritz values mu with the largest
//   |mu| (eigenvalues omega = sigma + 1/mu nearest the shift) lead; Ritz residual estimates
//   beta |e_m^T Q y_i|; the truncated Krylov-Schur relation for the next cycle.
// Four kernels: k_schur_house (one CTA, df64) reduces S and keeps the reflectors; k_schur_qr (one CTA)
// runs the QR sweeps and the reordering on a packed copy of the Hessenberg matrix in shared
// memory and logs every rotation; k_schur_q rebuilds Q from the reflectors and the rotation log,
// one thread per row; k_schur_post forms the Ritz estimates, the selection and the truncation.
#include "df64.cuh"
#include "factor.cuh"

namespace klst {

__device__ __forceinline__ double cabs1(double2 a) { return fabs(a.x) + fabs(a.y); }
__device__ __forceinline__ double cabs(double2 a) { return hypot(a.x, a.y); }


// ---------------------------------------------------------------- 1. Householder reduction
// df64 sum over the block (fixed xor tree within warps, then warps in order)
__device__ df block_sum_df(df v, float2* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v = df_add(v, df_shfl_xor(v, o));
    __syncthreads();
    if (lane == 0) red[wid] = df_pack(v);
    __syncthreads();
    df s = df{0.f, 0.f};
    for (int i = 0; i < nw; ++i) s = df_add(s, df_unpack(red[i]));
    __syncthreads();
    return s;
}

// Reduction of S (m x m block of the Krylov-Schur matrix) to upper Hessenberg form with
// Householder reflectors H_c = I - tau_c v_c v_c^H, in df64: H (global, column-major) holds the
// matrix as float4 df64 values for the QR kernel, v_c is kept in Vh for the Q rebuild.
__global__ void __launch_bounds__(256) k_schur_house(SchurArgs a) {
    const int m = a.m, tid = threadIdx.x, nt = blockDim.x;
    float4* H = reinterpret_cast<float4*>(a.H);
    __shared__ float4 v[192];
    __shared__ float2 red[8];
#define HH(i, j) H[(size_t)(j) * m + (i)]
#define HL(i, j) cdf_unpack(H[(size_t)(j) * m + (i)])
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int idx = tid; idx < m * m; idx += nt) {
        const int i = idx % m, j = idx / m;
        H[idx] = cdf_pack(cdf_from(a.S[(size_t)j * a.lds + i]));
    }
    for (int i = tid; i < m; i += nt) a.tau[i] = 0.0;
    if (tid == 0) { *a.nconv = 0; *a.log_count = 0; }  // k_schur_qr sets nconv = -1 on failure
    __syncthreads();
    for (int c = 0; c + 2 < m; ++c) {
        df tail = df{0.f, 0.f};
        for (int i = c + 2 + tid; i < m; i += nt) tail = df_add(tail, cdf_abs2(HL(i, c)));
        tail = block_sum_df(tail, red);
        if (tail.hi == 0.f) continue;
        const cdf x0 = HL(c + 1, c);
        const df ax02 = cdf_abs2(x0);
        const df s2 = df_add(tail, ax02);
        if (s2.hi < 1e-28f) {  // every subdiagonal entry below 1e-14: negligible, set to zero
            __syncthreads();
            for (int i = c + 2 + tid; i < m; i += nt) HH(i, c) = zero4;
            __syncthreads();
            continue;
        }
        const df alpha = df_mul(s2, df_rsqrt(s2));  // sqrt(|x|^2)
        df ax0 = df{0.f, 0.f};
        cdf ph = cdf{df{1.f, 0.f}, df{0.f, 0.f}};
        if (ax02.hi > 1e-36f) {
            const df ri = df_rsqrt(ax02);
            ax0 = df_mul(ax02, ri);
            ph = cdf_rmul(ri, x0);  // x0 / |x0|
        }
        const cdf bet = cdf_neg(cdf_rmul(alpha, ph));  // new subdiagonal entry
        const int len = m - c - 1;
        for (int i = tid; i < len; i += nt) {
            const cdf vi = (i == 0) ? cdf_sub(x0, bet) : HL(c + 1 + i, c);
            v[i] = cdf_pack(vi);
            a.Vh[(size_t)c * m + c + 1 + i] = cdf_pack(vi);
        }
        __syncthreads();
        const df rt = df_rsqrt(df_mul(alpha, df_add(alpha, ax0)));
        const df tau = df_mul(rt, rt);  // 2 / ||v||^2 = 1 / (alpha (alpha + |x0|))
        if (tid == 0) a.tau[c] = df_to(tau);
        // left: H[c+1:, col] -= tau v (v^H H[c+1:, col]) for col > c
        for (int col = c + 1 + tid; col < m; col += nt) {
            cdf g0 = cdf_zero(), g1 = cdf_zero();
            int i = 0;
            for (; i + 1 < len; i += 2) {
                cdf_fma_conj(g0, cdf_unpack(v[i]), HL(c + 1 + i, col));
                cdf_fma_conj(g1, cdf_unpack(v[i + 1]), HL(c + 2 + i, col));
            }
            if (i < len) cdf_fma_conj(g0, cdf_unpack(v[i]), HL(c + 1 + i, col));
            const cdf g = cdf_neg(cdf_rmul(tau, cdf_add(g0, g1)));
            for (i = 0; i < len; ++i) {
                cdf hv = HL(c + 1 + i, col);
                cdf_fma(hv, cdf_unpack(v[i]), g);
                HH(c + 1 + i, col) = cdf_pack(hv);
            }
        }
        if (tid == 0) {
            HH(c + 1, c) = cdf_pack(bet);
            for (int i = c + 2; i < m; ++i) HH(i, c) = zero4;
        }
        __syncthreads();
        // right: row[c+1:] -= tau (row[c+1:] v) v^H for every row of H
        for (int row = tid; row < m; row += nt) {
            cdf g0 = cdf_zero(), g1 = cdf_zero();
            int i = 0;
            for (; i + 1 < len; i += 2) {
                cdf_fma(g0, HL(row, c + 1 + i), cdf_unpack(v[i]));
                cdf_fma(g1, HL(row, c + 2 + i), cdf_unpack(v[i + 1]));
            }
            if (i < len) cdf_fma(g0, HL(row, c + 1 + i), cdf_unpack(v[i]));
            const cdf g = cdf_neg(cdf_rmul(tau, cdf_add(g0, g1)));
            for (i = 0; i < len; ++i) {
                cdf hv = HL(row, c + 1 + i);
                cdf_fma(hv, g, cdf_conj(cdf_unpack(v[i])));
                HH(row, c + 1 + i) = cdf_pack(hv);
            }
        }
        __syncthreads();
    }
#undef HL
#undef HH
}

// ---------------------------------------------------------------- 2. QR sweeps + reordering
// The sweeps run in double-float (df64) arithmetic on the float32 pipes: a complex rotation costs
// about 150 float32 instructions against 12 float64 ones, and the B300 issues float64 at about
// 1/64 of the float32 rate, so both the rotation chains and the serial scans stay off the float64
// unit.  Packed upper-Hessenberg storage: column j keeps rows 0..j+1 at offset j(j+3)/2.
__device__ __forceinline__ int pk(int i, int j) { return j * (j + 3) / 2 + i; }

// df64 unit roundoff is 2^-48; a subdiagonal entry below 2^-47 (|h_{l-1,l-1}| + |h_{l,l}|) is
// set to zero (the float64 form of the test uses the float64 ulp)
constexpr float kDeflEps = 7.105427357601002e-15f;  // 2^-47

// Givens rotation [c s; -conj(s) c] [f; g] = [r; 0] with real c = |f| / r and
// s = f conj(g) / (|f| r), r = sqrt(|f|^2 + |g|^2) (the LAPACK zlartg convention), in df64.
// f and g are first scaled by one power of two (exact) so the squares stay in float32 range.
__device__ void givens_df(cdf f, cdf g, df& c, cdf& s) {
    const float mg = fmaxf(fabsf(g.re.hi), fabsf(g.im.hi));
    const float mf = fmaxf(fabsf(f.re.hi), fabsf(f.im.hi));
    if (mg == 0.f || mg < 1e-30f * mf) { c = df{1.f, 0.f}; s = cdf_zero(); return; }
    int e;
    frexpf(fmaxf(mf, mg), &e);
    e = max(-120, min(120, e));
    const float sc = ldexpf(1.f, -e);
    f = cdf_scale(f, sc);
    g = cdf_scale(g, sc);
    const df ag2 = cdf_abs2(g), af2 = cdf_abs2(f);
    if (af2.hi < 1e-30f) {  // |f| < 1e-15 |g|: c = 0 and s = conj(g) / |g|
        c = df{0.f, 0.f};
        s = cdf_rmul(df_rsqrt(ag2), cdf_conj(g));
        return;
    }
    const df ir = df_rsqrt(df_add(af2, ag2)), iaf = df_rsqrt(af2);
    c = df_mul(df_mul(af2, iaf), ir);
    s = cdf_rmul(df_mul(iaf, ir), cdf_mul(f, cdf_conj(g)));
}

__global__ void __launch_bounds__(256) k_schur_qr(SchurArgs a) {
    extern __shared__ float4 sT[];
    const int m = a.m, tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
    __shared__ float2 rc[192];
    __shared__ float4 rs[192];
    __shared__ float2 s_c;
    __shared__ float4 s_s, s_mu;
    __shared__ int s_lo, s_q, s_fail, s_cnt;
#define TT(i, j) sT[pk(i, j)]
#define LD(i, j) cdf_unpack(sT[pk(i, j)])
    for (int j = 0; j < m; ++j)
        for (int i = tid; i <= min(j + 1, m - 1); i += nt) TT(i, j) = reinterpret_cast<const float4*>(a.H)[(size_t)j * m + i];
    if (tid == 0) { s_fail = 0; s_cnt = 0; }
    __syncthreads();
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    int hi = m - 1, its = 0, total = 0;
    const int max_total = 30 * m;
    while (hi > 0) {
        if (wid == 0) {
            // deflation: the largest l in [1, hi] whose subdiagonal entry is negligible (0 if none),
            // 32 candidates per ballot
            int l = 0;
            for (int base = hi; base >= 1; base -= 32) {
                const int ll = base - lane;
                bool neg = false;
                if (ll >= 1) {
                    const float sub = cdf_abs1f(LD(ll, ll - 1));
                    float sc = cdf_abs1f(LD(ll - 1, ll - 1)) + cdf_abs1f(LD(ll, ll));
                    if (sc == 0.f) sc = 1.f;
                    neg = sub <= kDeflEps * sc;
                }
                const unsigned b = __ballot_sync(0xffffffffu, neg);
                if (b) { l = base - (__ffs(b) - 1); break; }
            }
            if (lane == 0) {
                if (l >= 1) TT(l, l - 1) = zero4;
                s_lo = l;
                if (l < hi) {
                    // shift from the trailing 2x2 block, in float64 (once per sweep)
                    const double2 aa = cdf_to(LD(hi - 1, hi - 1)), bb = cdf_to(LD(hi - 1, hi)),
                                  cc = cdf_to(LD(hi, hi - 1)), dd = cdf_to(LD(hi, hi));
                    double2 mu;
                    if (its > 0 && its % 11 == 0) {
                        mu = dd + mk(0.75 * cabs1(cc), 0.0);  // exceptional shift
                    } else {
                        // Wilkinson shift: eigenvalue of the trailing 2x2 nearer dd
                        const double2 hd = 0.5 * (aa - dd);
                        const double2 disc = hd * hd + bb * cc;
                        const double r = cabs(disc);
                        const double sr = sqrt(0.5 * (r + fabs(disc.x)));
                        double2 sq;
                        if (sr == 0.0) sq = mk(0, 0);
                        else if (disc.x >= 0) sq = mk(sr, disc.y / (2.0 * sr));
                        else sq = mk(fabs(disc.y) / (2.0 * sr), disc.y >= 0 ? sr : -sr);
                        const double2 m1 = 0.5 * (aa + dd) + sq, m2 = 0.5 * (aa + dd) - sq;
                        mu = cabs(m1 - dd) < cabs(m2 - dd) ? m1 : m2;
                    }
                    s_mu = cdf_pack(cdf_from(mu));
                    if (s_cnt + (hi - l) > a.log_cap) s_fail = 2;
                }
            }
        }
        __syncthreads();
        const int lo = s_lo;
        if (lo == hi) { hi -= 1; its = 0; __syncthreads(); continue; }
        if (s_fail || ++total > max_total) { if (tid == 0) s_fail = s_fail ? s_fail : 1; break; }
        ++its;
        const cdf mu = cdf_unpack(s_mu);
        for (int i = lo + tid; i <= hi; i += nt) TT(i, i) = cdf_pack(cdf_sub(LD(i, i), mu));
        __syncthreads();
        if (tid == 0) {
            df c;
            cdf sv;
            givens_df(LD(lo, lo), LD(lo + 1, lo), c, sv);
            rc[lo] = df_pack(c);
            rs[lo] = cdf_pack(sv);
        }
        __syncthreads();
        // left sweep: rotation i on rows i, i+1 (columns i..m-1); the thread holding column i+1
        // forms rotation i+1 from its freshly rotated diagonal entry
        for (int i = lo; i < hi; ++i) {
            const int col = i + tid;
            if (col < m) {
                const df c = df_unpack(rc[i]);
                const cdf sv = cdf_unpack(rs[i]);
                cdf x = LD(i, col), y = LD(i + 1, col);
                cdf_rot(x, y, c, sv);
                TT(i, col) = cdf_pack(x);
                TT(i + 1, col) = (col == i) ? zero4 : cdf_pack(y);
                if (col == i + 1 && i + 1 < hi) {
                    df c2;
                    cdf s2;
                    givens_df(y, LD(i + 2, i + 1), c2, s2);
                    rc[i + 1] = df_pack(c2);
                    rs[i + 1] = cdf_pack(s2);
                }
            }
            __syncthreads();
        }
        // right sweep in bulk: row r receives rotations i >= max(lo, r - 1), in order
        for (int r = tid; r <= hi; r += nt) {
            const int i0 = max(lo, r - 1);
            if (i0 >= hi) continue;
            cdf x = LD(r, i0);
            for (int i = i0; i < hi; ++i) {
                cdf y = LD(r, i + 1);
                cdf_rot(x, y, df_unpack(rc[i]), cdf_conj(cdf_unpack(rs[i])));
                TT(r, i) = cdf_pack(x);
                x = y;
            }
            TT(r, hi) = cdf_pack(x);
        }
        __syncthreads();
        for (int i = lo + tid; i <= hi; i += nt) TT(i, i) = cdf_pack(cdf_add(LD(i, i), mu));
        const int base = s_cnt;
        for (int t = tid; t < hi - lo; t += nt) {
            Rot g;
            g.s = rs[lo + t]; g.c = rc[lo + t]; g.i = lo + t; g.pad = 0;
            a.log[base + t] = g;
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
    for (int j = tid; j + 1 < m; j += nt) TT(j + 1, j) = zero4;
    __syncthreads();
    // reorder: bring the keep Ritz values of largest |mu| to the front by adjacent swaps; the
    // maximum is found by warp 0 on |T_ii|^2 in df64 (ties resolve to the lower index)
    for (int p = 0; p < a.keep; ++p) {
        if (wid == 0) {
            df bv = df{-1.f, 0.f};
            int q = p;
            for (int i = p + lane; i < m; i += 32) {
                const df v = cdf_abs2(LD(i, i));
                if (v.hi > bv.hi || (v.hi == bv.hi && v.lo > bv.lo)) { bv = v; q = i; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const float oh = __shfl_xor_sync(0xffffffffu, bv.hi, o), ol = __shfl_xor_sync(0xffffffffu, bv.lo, o);
                const int oq = __shfl_xor_sync(0xffffffffu, q, o);
                if (oh > bv.hi || (oh == bv.hi && (ol > bv.lo || (ol == bv.lo && oq < q)))) { bv = df{oh, ol}; q = oq; }
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
                df c;
                cdf sv;
                givens_df(LD(i, i + 1), cdf_sub(LD(i + 1, i + 1), LD(i, i)), c, sv);
                s_c = df_pack(c);
                s_s = cdf_pack(sv);
                Rot g;
                g.s = s_s; g.c = s_c; g.i = i; g.pad = 0;
                a.log[s_cnt] = g;
                s_cnt = s_cnt + 1;
            }
            __syncthreads();
            const df c = df_unpack(s_c);
            const cdf sv = cdf_unpack(s_s), sc = cdf_conj(sv);
            const float4 t11 = TT(i, i), t22 = TT(i + 1, i + 1);
            for (int idx = tid; idx < (m - i - 2) + i; idx += nt) {
                if (idx < m - i - 2) {
                    const int col = i + 2 + idx;
                    cdf x = LD(i, col), y = LD(i + 1, col);
                    cdf_rot(x, y, c, sv);
                    TT(i, col) = cdf_pack(x); TT(i + 1, col) = cdf_pack(y);
                } else {
                    const int row = idx - (m - i - 2);
                    cdf x = LD(row, i), y = LD(row, i + 1);
                    cdf_rot(x, y, c, sc);
                    TT(row, i) = cdf_pack(x); TT(row, i + 1) = cdf_pack(y);
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
    // write T (upper triangular) back to global in float64
    for (int idx = tid; idx < m * m; idx += nt) {
        const int i = idx % m, j = idx / m;
        a.H[idx] = (i <= j) ? cdf_to(LD(i, j)) : mk(0, 0);
    }
    if (tid == 0) *a.log_count = s_cnt;
#undef LD
#undef TT
}

// ---------------------------------------------------------------- 3. Schur vectors
// Row r of Q = e_r^T H_0 H_1 ... H_{m-3} G_1^H G_2^H ...: the reflectors, then every logged
// rotation in order, in df64.  One thread per row; the row lives in shared memory (column-major
// over the block's rows, so the 32 threads hit distinct banks).
__global__ void __launch_bounds__(32) k_schur_q(SchurArgs a) {
    extern __shared__ float4 q4[];  // [m][32]
    const int m = a.m, t = threadIdx.x, r = blockIdx.x * 32 + t;
    for (int col = 0; col < m; ++col) q4[col * 32 + t] = make_float4(col == r ? 1.f : 0.f, 0.f, 0.f, 0.f);
    for (int c = 0; c + 2 < m; ++c) {
        const double tau = a.tau[c];
        if (tau == 0.0) continue;
        const float4* vc = a.Vh + (size_t)c * m;
        // g = tau sum_i q_i v_i, two accumulators
        cdf g0 = cdf_zero(), g1 = cdf_zero();
        int i = c + 1;
        for (; i + 1 < m; i += 2) {
            cdf_fma(g0, cdf_unpack(q4[i * 32 + t]), cdf_unpack(vc[i]));
            cdf_fma(g1, cdf_unpack(q4[(i + 1) * 32 + t]), cdf_unpack(vc[i + 1]));
        }
        if (i < m) cdf_fma(g0, cdf_unpack(q4[i * 32 + t]), cdf_unpack(vc[i]));
        const cdf g = cdf_neg(cdf_rmul(df_from(tau), cdf_add(g0, g1)));
        for (i = c + 1; i < m; ++i) {
            cdf qi = cdf_unpack(q4[i * 32 + t]);
            cdf_fma(qi, g, cdf_conj(cdf_unpack(vc[i])));
            q4[i * 32 + t] = cdf_pack(qi);
        }
    }
    // runs of rotations in planes (i, i+1), (i+1, i+2), ... carry column i+1 in registers; the log
    // is staged into shared memory 256 entries at a time by the whole warp
    Rot* slog = reinterpret_cast<Rot*>(q4 + (size_t)m * 32);
    const int nrot = *a.log_count;
    int ci = -1;
    cdf cx = cdf_zero();
    for (int k0 = 0; k0 < nrot; k0 += 256) {
        const int cnt = min(256, nrot - k0);
        for (int i = t; i < cnt; i += 32) slog[i] = a.log[k0 + i];
        __syncwarp();
        for (int k = 0; k < cnt; ++k) {
            const Rot g = slog[k];
            cdf x;
            if (g.i == ci) x = cx;
            else {
                if (ci >= 0) q4[ci * 32 + t] = cdf_pack(cx);
                x = cdf_unpack(q4[g.i * 32 + t]);
            }
            cdf y = cdf_unpack(q4[(g.i + 1) * 32 + t]);
            cdf_rot(x, y, df_unpack(g.c), cdf_conj(cdf_unpack(g.s)));
            q4[g.i * 32 + t] = cdf_pack(x);
            ci = g.i + 1;
            cx = y;
        }
        __syncwarp();
    }
    if (ci >= 0) q4[ci * 32 + t] = cdf_pack(cx);
    if (r < m)
        for (int col = 0; col < m; ++col) a.Q[(size_t)col * m + r] = cdf_to(cdf_unpack(q4[col * 32 + t]));
}

// ---------------------------------------------------------------- 4. Ritz pairs, selection, truncation
__global__ void __launch_bounds__(256) k_schur_post(SchurArgs a) {
    const int m = a.m, tid = threadIdx.x, nt = blockDim.x;
    if (*a.nconv < 0) return;  // the QR step failed; the host reports it
    double2 *H = a.H, *Q = a.Q;
    const double2 beta = a.S[(size_t)(m - 1) * a.lds + m];
#define HH(i, j) H[(size_t)(j) * m + (i)]
#define QQ(i, j) Q[(size_t)(j) * m + (i)]
    // Ritz values, eigenvectors y of T (back substitution) and residual estimates for the
    // first keep positions (sorted by |mu|, largest first)
    __shared__ int s_sel[192];
    for (int i = tid; i < m; i += nt) a.mu[i] = HH(i, i);
    const double ulp = 2.220446049250313e-16;
    const int npos = a.keep;
    for (int p = tid; p < npos; p += nt) {
        const double2 tp = HH(p, p);
        double2* y = a.Yc + (size_t)p * m;  // y_p in column p of the scratch
        for (int i = p + 1; i < m; ++i) y[i] = mk(0, 0);
        y[p] = mk(1, 0);
        double nrm = 1.0;
        for (int i = p - 1; i >= 0; --i) {
            double2 sacc = mk(0, 0);
            for (int c2 = i + 1; c2 <= p; ++c2) cfma(sacc, HH(i, c2), y[c2]);
            double2 den = HH(i, i) - tp;
            if (cabs(den) < ulp * cabs(tp)) den = mk(ulp * cabs(tp) + 1e-300, 0.0);
            y[i] = -(cinv(den) * sacc);
            nrm += abs2(y[i]);
        }
        nrm = sqrt(nrm);
        double2 e = mk(0, 0);
        for (int i = 0; i <= p; ++i) cfma(e, QQ(m - 1, i), y[i]);
        a.est[p] = cabs(beta) * cabs(e) / nrm;
        for (int i = 0; i <= p; ++i) y[i] = (1.0 / nrm) * y[i];
    }
    __syncthreads();
    // selection: the nev nearest converged Ritz pairs.  An unconverged Ritz value nearer the
    // shift may only be passed over when it lies in a cluster with the last selected one
    // (|omega - sigma| within 1%), where the order inside the cluster is not resolved.
    if (tid == 0) {
        int ns = 0, lead = 0;
        bool leading = true;
        for (int p = 0; p < npos && ns < a.nev; ++p) {
            const double am = cabs(HH(p, p));
            const bool ok = a.est[p] <= a.tol * (a.conv ? am * am : am);
            if (ok) { s_sel[ns++] = p; if (leading) ++lead; }
            else leading = false;
        }
        bool done = ns == a.nev;
        if (done) {
            const double mlast = cabs(HH(s_sel[a.nev - 1], s_sel[a.nev - 1]));
            for (int p = 0; p < s_sel[a.nev - 1]; ++p) {
                const double am = cabs(HH(p, p));
                const bool ok = a.est[p] <= a.tol * (a.conv ? am * am : am);
                if (!ok && am > mlast / 0.99) { done = false; break; }
            }
        }
        if (!done) {
            for (int i = 0; i < a.nev; ++i) s_sel[i] = i;
            *a.nconv = lead;
        } else {
            *a.nconv = a.nev;
        }
        for (int i = 0; i < a.nev; ++i) {
            a.mu_sel[i] = HH(s_sel[i], s_sel[i]);
            a.est_sel[i] = a.est[s_sel[i]];
        }
    }
    __syncthreads();
    // Ritz vector coefficients of the selected pairs: Ysel[:, i] = Q y_{sel_i}
    for (int idx = tid; idx < m * a.nev; idx += nt) {
        const int row = idx % m, i = idx / m, p = s_sel[i];
        double2 acc = mk(0, 0);
        for (int l = 0; l <= p; ++l) cfma(acc, QQ(row, l), a.Yc[(size_t)p * m + l]);
        a.Ysel[(size_t)i * m + row] = acc;
    }
    __syncthreads();
    // truncated Krylov-Schur relation: S[0:k,0:k] = T_kk, S[k,0:k] = b = beta Q[m-1, 0:k].
    // Locking: the leading Schur vectors whose coupling |b_j| already meets the convergence test
    // get b_j = 0 (an exact deflation up to that tolerance), so the next restart's Householder
    // reduction skips their columns and the QR sweeps deflate them without iterating.
    __shared__ int s_lock;
    if (tid == 0) {
        int L = 0;
        for (; L < a.keep; ++L) {
            const double am = cabs(HH(L, L));
            const double bj = cabs(beta) * cabs(QQ(m - 1, L));
            if (!(bj <= a.tol * (a.conv ? am * am : am))) break;
        }
        s_lock = L;
    }
    __syncthreads();
    const int k = a.keep;
    for (int idx = tid; idx < a.lds * m; idx += nt) {
        const int i = idx % a.lds, j = idx / a.lds;
        double2 val = mk(0, 0);
        if (j < k) {
            if (i < k) val = (i <= j) ? HH(i, j) : mk(0, 0);
            else if (i == k) val = (j < s_lock) ? mk(0, 0) : beta * QQ(m - 1, j);
        }
        a.S[(size_t)j * a.lds + i] = val;
    }
#undef HH
#undef QQ
}

int launch_schur(const SchurArgs& a, cudaStream_t s) {
    static std::atomic<unsigned long long> attr{0};
    KLST_CK(set_once_per_device(attr, [] {
        cudaError_t e = cudaFuncSetAttribute(k_schur_qr, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_schur_q, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
        return e;
    }));
    const int m = a.m;
    const size_t packed = sizeof(double2) * (size_t)m * (m + 3) / 2;
    prof_begin("schur_house", s);
    k_schur_house<<<1, 256, 0, s>>>(a);
    klst::note_launch();
    prof_end("schur_house", s);
    prof_begin("schur_qr", s);
    k_schur_qr<<<1, 256, packed, s>>>(a); klst::note_launch();
    prof_end("schur_qr", s);
    prof_begin("schur_q", s);
    k_schur_q<<<(m + 31) / 32, 32, sizeof(double2) * 32 * m + sizeof(Rot) * 256, s>>>(a); klst::note_launch();
    prof_end("schur_q", s);
    launch_schur_post(a, s);
    KLST_CK_LAUNCH();
    return KLST_OK;
}

void launch_schur_post(const SchurArgs& a, cudaStream_t s) {
    prof_begin("schur_post", s);
    k_schur_post<<<1, 256, 0, s>>>(a); klst::note_launch();
    prof_end("schur_post", s);
}

}  // namespace klst
