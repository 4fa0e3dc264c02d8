// Small dense float64 step of the Krylov-Schur restart (Sec. 4.1: restarted Arnoldi with a
// filter that keeps the wanted Ritz values), run by one CTA on the device:
//   S_m = Q T Q^H (Householder reduction to Hessenberg form, then shifted QR with Givens
//   rotations to the complex Schur form), reorder T so the Ritz values mu with the largest
//   |mu| (eigenvalues omega = sigma + 1/mu nearest the shift) lead, Ritz residual estimates
//   beta |e_m^T Q y_i|, and the truncated Krylov-Schur relation for the next cycle.
#include "factor.cuh"

namespace klst {


__device__ __forceinline__ double cabs1(double2 a) { return fabs(a.x) + fabs(a.y); }
__device__ __forceinline__ double cabs(double2 a) { return hypot(a.x, a.y); }

// Givens rotation [c s; -conj(s) c] [f; g] = [r; 0] with real c (the LAPACK zlartg convention).
__device__ void givens(double2 f, double2 g, double& c, double2& s) {
    const double af = cabs(f), ag = cabs(g);
    if (ag == 0.0) { c = 1.0; s = mk(0, 0); return; }
    if (af == 0.0) { c = 0.0; s = (1.0 / ag) * conj(g); return; }
    const double nr = hypot(af, ag);
    c = af / nr;
    const double2 ph = (1.0 / af) * f;  // f / |f|
    s = (1.0 / nr) * (ph * conj(g));
}

// x' = c x + s y ; y' = c y - conj(s) x
__device__ __forceinline__ void rot(double2& x, double2& y, double c, double2 s) {
    const double2 t = c * x + s * y;
    y = c * y - conj(s) * x;
    x = t;
}

__device__ double block_sum1(double v, double* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0;
    for (int i = 0; i < nw; ++i) s += red[i];
    __syncthreads();
    return s;
}

__global__ void __launch_bounds__(256) k_schur(SchurArgs a) {
    const int m = a.m, tid = threadIdx.x, nt = blockDim.x;
    double2 *H = a.H, *Q = a.Q;
    __shared__ double2 v[192];
    __shared__ double rc[192];
    __shared__ double2 rs[192];
    __shared__ double red[8];
    __shared__ double s_c;
    __shared__ double2 s_s, s_mu;
    __shared__ int s_lo, s_q, s_fail;
    const double2 beta = a.S[(size_t)(m - 1) * a.lds + m];
#define HH(i, j) H[(size_t)(j) * m + (i)]
#define QQ(i, j) Q[(size_t)(j) * m + (i)]
    for (int idx = tid; idx < m * m; idx += nt) {
        const int i = idx % m, j = idx / m;
        H[idx] = a.S[(size_t)j * a.lds + i];
        Q[idx] = mk(i == j ? 1.0 : 0.0, 0.0);
    }
    if (tid == 0) s_fail = 0;
    __syncthreads();
    // ---- Householder reduction to upper Hessenberg form
    for (int c = 0; c + 2 < m; ++c) {
        double tail = 0.0;
        for (int i = c + 2 + tid; i < m; i += nt) tail += abs2(HH(i, c));
        tail = block_sum1(tail, red);
        if (tail == 0.0) continue;
        const double2 x0 = HH(c + 1, c);
        const double alpha = sqrt(tail + abs2(x0));
        const double ax0 = cabs(x0);
        const double2 ph = ax0 > 0 ? (1.0 / ax0) * x0 : mk(1, 0);
        const double2 bet = (-alpha) * ph;  // new subdiagonal entry
        const int len = m - c - 1;
        for (int i = tid; i < len; i += nt) v[i] = (i == 0) ? x0 - bet : HH(c + 1 + i, c);
        __syncthreads();
        const double tau = 1.0 / (alpha * (alpha + ax0));  // 2 / ||v||^2
        // left: H[c+1:, col] -= tau v (v^H H[c+1:, col]) for col > c
        for (int col = c + 1 + tid; col < m; col += nt) {
            double2 g = mk(0, 0);
            for (int i = 0; i < len; ++i) cfma_conj(g, v[i], HH(c + 1 + i, col));
            g = tau * g;
            for (int i = 0; i < len; ++i) HH(c + 1 + i, col) = HH(c + 1 + i, col) - v[i] * g;
        }
        if (tid == 0) {
            HH(c + 1, c) = bet;
            for (int i = c + 2; i < m; ++i) HH(i, c) = mk(0, 0);
        }
        __syncthreads();
        // right: row[c+1:] -= tau (row[c+1:] v) v^H for H (all rows) and Q (all rows)
        for (int row = tid; row < 2 * m; row += nt) {
            double2* M = row < m ? H : Q;
            const int rr = row < m ? row : row - m;
            double2 g = mk(0, 0);
            for (int i = 0; i < len; ++i) cfma(g, M[(size_t)(c + 1 + i) * m + rr], v[i]);
            g = tau * g;
            for (int i = 0; i < len; ++i) M[(size_t)(c + 1 + i) * m + rr] = M[(size_t)(c + 1 + i) * m + rr] - g * conj(v[i]);
        }
        __syncthreads();
    }
    // ---- shifted QR iteration to the complex Schur form (full T and Q updates)
    int hi = m - 1, its = 0, total = 0;
    const int max_total = 60 * m;
    while (hi > 0) {
        if (tid == 0) {
            int l = hi;
            for (; l > 0; --l) {
                const double sub = cabs1(HH(l, l - 1));
                double sc = cabs1(HH(l - 1, l - 1)) + cabs1(HH(l, l));
                if (sc == 0.0) sc = 1.0;
                if (sub <= 2.220446049250313e-16 * sc || sub < 1e-300) { HH(l, l - 1) = mk(0, 0); break; }
            }
            s_lo = l;
            if (l < hi) {
                // Wilkinson shift from the trailing 2x2 of the active window; exceptional shifts
                const double2 aa = HH(hi - 1, hi - 1), bb = HH(hi - 1, hi), cc = HH(hi, hi - 1), dd = HH(hi, hi);
                double2 mu;
                if (its > 0 && its % 11 == 0) {
                    mu = dd + mk(0.75 * cabs1(cc), 0.0);
                } else {
                    const double2 hd = 0.5 * (aa - dd);
                    double2 disc = hd * hd + bb * cc;
                    // complex sqrt
                    const double r = cabs(disc);
                    double sr = sqrt(0.5 * (r + fabs(disc.x)));
                    double2 sq;
                    if (sr == 0.0) sq = mk(0, 0);
                    else if (disc.x >= 0) sq = mk(sr, disc.y / (2.0 * sr));
                    else sq = mk(fabs(disc.y) / (2.0 * sr), disc.y >= 0 ? sr : -sr);
                    const double2 m1 = 0.5 * (aa + dd) + sq, m2 = 0.5 * (aa + dd) - sq;
                    mu = cabs(m1 - dd) < cabs(m2 - dd) ? m1 : m2;
                }
                s_mu = mu;
            }
        }
        __syncthreads();
        const int lo = s_lo;
        if (lo == hi) { hi -= 1; its = 0; __syncthreads(); continue; }
        if (++total > max_total) { if (tid == 0) { s_fail = 1; atomicOr(&a.st->flags, ST_NOCONV_QR); } break; }
        ++its;
        const double2 mu = s_mu;
        for (int i = lo + tid; i <= hi; i += nt) HH(i, i) = HH(i, i) - mu;
        __syncthreads();
        // left rotations: triangularise the window of H - mu I
        for (int i = lo; i < hi; ++i) {
            if (tid == 0) {
                double c; double2 s;
                givens(HH(i, i), HH(i + 1, i), c, s);
                s_c = c; s_s = s;
                rc[i] = c; rs[i] = s;
            }
            __syncthreads();
            const double c = s_c; const double2 s = s_s;
            for (int col = i + tid; col < m; col += nt) {
                double2 x = HH(i, col), y = HH(i + 1, col);
                rot(x, y, c, s);
                HH(i, col) = x; HH(i + 1, col) = y;
            }
            __syncthreads();
        }
        // right rotations: R Q^H, columns i, i+1, rows 0..i+1; accumulate into Q
        for (int i = lo; i < hi; ++i) {
            const double c = rc[i];
            const double2 s = rs[i];
            const double2 sc = conj(s);
            for (int row = tid; row < m + (i + 2); row += nt) {
                if (row < i + 2) {
                    double2 x = HH(row, i), y = HH(row, i + 1);
                    rot(x, y, c, sc);
                    HH(row, i) = x; HH(row, i + 1) = y;
                } else {
                    const int qr = row - (i + 2);
                    double2 x = QQ(qr, i), y = QQ(qr, i + 1);
                    rot(x, y, c, sc);
                    QQ(qr, i) = x; QQ(qr, i + 1) = y;
                }
            }
            __syncthreads();
        }
        for (int i = lo + tid; i <= hi; i += nt) HH(i, i) = HH(i, i) + mu;
        __syncthreads();
    }
    __syncthreads();
    if (s_fail) { if (tid == 0) *a.nconv = -1; return; }
    for (int idx = tid; idx < m * m; idx += nt) {
        const int i = idx % m, j = idx / m;
        if (i > j) H[idx] = mk(0, 0);
    }
    __syncthreads();
    // ---- reorder: bring the keep Ritz values of largest |mu| to the front (adjacent swaps)
    for (int p = 0; p < a.keep; ++p) {
        if (tid == 0) {
            int q = p;
            double bv = cabs(HH(p, p));
            for (int i = p + 1; i < m; ++i) {
                const double vv = cabs(HH(i, i));
                if (vv > bv) { bv = vv; q = i; }
            }
            s_q = q;
        }
        __syncthreads();
        const int q = s_q;
        for (int i = q - 1; i >= p; --i) {
            if (tid == 0) {
                double c; double2 s;
                givens(HH(i, i + 1), HH(i + 1, i + 1) - HH(i, i), c, s);
                s_c = c; s_s = s;
            }
            __syncthreads();
            const double c = s_c; const double2 s = s_s, sc = conj(s);
            const double2 t11 = HH(i, i), t22 = HH(i + 1, i + 1);
            __syncthreads();
            for (int idx = tid; idx < (m - i - 2) + i + m; idx += nt) {
                if (idx < m - i - 2) {
                    const int col = i + 2 + idx;
                    double2 x = HH(i, col), y = HH(i + 1, col);
                    rot(x, y, c, s);
                    HH(i, col) = x; HH(i + 1, col) = y;
                } else if (idx < (m - i - 2) + i) {
                    const int row = idx - (m - i - 2);
                    double2 x = HH(row, i), y = HH(row, i + 1);
                    rot(x, y, c, sc);
                    HH(row, i) = x; HH(row, i + 1) = y;
                } else {
                    const int row = idx - (m - i - 2) - i;
                    double2 x = QQ(row, i), y = QQ(row, i + 1);
                    rot(x, y, c, sc);
                    QQ(row, i) = x; QQ(row, i + 1) = y;
                }
            }
            if (tid == 0) { HH(i, i) = t22; HH(i + 1, i + 1) = t11; }
            __syncthreads();
        }
    }
    // ---- Ritz values, eigenvectors y of T (back substitution) and residual estimates for the
    //      first keep positions (sorted by |mu|, largest first)
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
    // ---- selection: the nev nearest converged Ritz pairs.  An unconverged Ritz value nearer the
    //      shift may only be passed over when it lies in a cluster with the last selected one
    //      (|omega - sigma| within 1%), where the order inside the cluster is not resolved.
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
    // ---- truncated Krylov-Schur relation: S[0:k,0:k] = T_kk, S[k,0:k] = beta Q[m-1, 0:k]
    const int k = a.keep;
    for (int idx = tid; idx < a.lds * m; idx += nt) {
        const int i = idx % a.lds, j = idx / a.lds;
        double2 val = mk(0, 0);
        if (j < k) {
            if (i < k) val = (i <= j) ? HH(i, j) : mk(0, 0);
            else if (i == k) val = beta * QQ(m - 1, j);
        }
        a.S[(size_t)j * a.lds + i] = val;
    }
#undef HH
#undef QQ
}

int launch_schur(const SchurArgs& a, cudaStream_t s) {
    k_schur<<<1, 256, 0, s>>>(a);
    KLST_CK_LAUNCH();
    return KLST_OK;
}

}  // namespace klst
