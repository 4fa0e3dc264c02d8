// The small dense step of the Krylov-Schur restart (Sec. 4.1) in float64: Householder reduction of
// the (keep + 1)-spiked Krylov-Schur matrix to Hessenberg form, shifted QR sweeps with Givens
// rotations to the complex Schur form, reordering so the Ritz values of largest |mu| lead, and the
// Schur vectors rebuilt from the reflectors and the logged rotations.  Same algorithm and data flow
// as the double-float kernels of schur.cu, with float64 operands, float64 deflation (unit
// roundoff 2^-53) and float64 rotations; k_schur_post (Ritz estimates, selection, truncation) is
// shared.
#include <cooperative_groups.h>
#include <cstdlib>
#include <mutex>

#include "factor.cuh"

namespace klst {

struct Rot64 {         // rotation [c s; -conj(s) c] of rows/columns (i, i+1), float64
    double2 s;
    double c;
    int i;             // bits 0..7: i; 8..15 and 16..23: the QR sweep's window lo, hi (0, m - 1 for swaps)
    int pad;           // replay level
};
__device__ __forceinline__ int rot_i(const Rot64& g) { return g.i & 0xFF; }
__device__ __forceinline__ int rot_lo(const Rot64& g) { return (g.i >> 8) & 0xFF; }
__device__ __forceinline__ int rot_hi(const Rot64& g) { return (g.i >> 16) & 0xFF; }
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

// The same reduction spread over one thread-block cluster of NC CTAs (one SM's float64 pipe is
// the bound of the single-CTA kernel).  CTA q keeps the columns j with j % NC == q in shared
// memory (cyclic, so the work stays spread as the reduction moves right).  Per column c:
//   1. the owner of column c forms v, tau and the new subdiagonal entry exactly as above and
//      publishes a decision (0: nothing to do, 1: the tail is negligible and zeroed, 2: reflect);
//   2. every CTA copies the decision, tau and v through distributed shared memory and applies the
//      left reflection to its columns > c, one warp per column;
//   3. every CTA forms, for every row r, the partial sum of H[r, col] v over its columns col > c;
//      the NC partials of each row are read back through distributed shared memory and added in
//      rank order, and every CTA applies the right reflection to its columns.
// Three cluster barriers per column, taken by every CTA whatever the decision.
template <int NC>
__global__ void __launch_bounds__(256) k_schur_house64_cl(SchurArgs a) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int m = a.m, q = (int)cl.block_rank(), tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    const int ncol = (m - q + NC - 1) / NC;          // this CTA's columns: q, q + NC, ...
    const int ncmax = (m + NC - 1) / NC;             // the most any CTA keeps: the same layout in every CTA
    extern __shared__ __align__(16) unsigned char hsm[];
    double2* hs = reinterpret_cast<double2*>(hsm);   // [ncol][m], column-major
    double2* part = hs + (size_t)ncmax * m;          // [m] this CTA's partial row sums (read by the others)
    double2* prow = part + m;                        // [m] the summed row products
    double2* Vh = reinterpret_cast<double2*>(a.Vh);
    __shared__ double2 v[192];
    __shared__ double2 s_bet;
    __shared__ double s_tau;
    __shared__ int s_flag;
    __shared__ double red[8];
#define HL(i, lc) hs[(size_t)(lc) * m + (i)]
    for (int idx = tid; idx < ncol * m; idx += nt) {
        const int lc = idx / m, i = idx - lc * m;
        HL(i, lc) = a.S[(size_t)(q + lc * NC) * a.lds + i];
    }
    if (q == 0) {
        for (int i = tid; i < m; i += nt) a.tau[i] = 0.0;
        if (tid == 0) { *a.nconv = 0; *a.log_count = 0; }
    }
    cl.sync();
    for (int c = 0; c + 2 < m; ++c) {
        const int owner = c % NC, len = m - c - 1;
        if (q == owner) {
            const int lcc = c / NC;
            double tail = 0.0;
            for (int i = c + 2 + tid; i < m; i += nt) tail += abs2(HL(i, lcc));
            tail = block_sum64(tail, red);
            const double2 x0 = HL(c + 1, lcc);
            const double ax02 = abs2(x0), s2 = tail + ax02;
            int flag = 2;
            if (tail == 0.0) flag = 0;
            else if (s2 < 1e-60) flag = 1;  // every subdiagonal entry below 1e-30: negligible, zeroed
            if (flag == 2) {
                const double alpha = sqrt(s2);
                double ax0 = 0.0;
                double2 ph = make_double2(1.0, 0.0);
                if (ax02 > 1e-200) {
                    ax0 = sqrt(ax02);
                    ph = make_double2(x0.x / ax0, x0.y / ax0);
                }
                const double2 bet = make_double2(-alpha * ph.x, -alpha * ph.y);
                for (int i = tid; i < len; i += nt) {
                    const double2 vi = (i == 0) ? x0 - bet : HL(c + 1 + i, lcc);
                    v[i] = vi;
                    Vh[(size_t)c * m + c + 1 + i] = vi;
                }
                if (tid == 0) {
                    s_tau = 1.0 / (alpha * (alpha + ax0));  // 2 / ||v||^2
                    s_bet = bet;
                    a.tau[c] = s_tau;
                }
            }
            if (tid == 0) s_flag = flag;
            __syncthreads();
            if (flag == 2) {
                if (tid == 0) HL(c + 1, lcc) = s_bet;
                for (int i = c + 2 + tid; i < m; i += nt) HL(i, lcc) = make_double2(0.0, 0.0);
            } else if (flag == 1) {
                for (int i = c + 2 + tid; i < m; i += nt) HL(i, lcc) = make_double2(0.0, 0.0);
            }
        }
        cl.sync();  // 1: the owner's decision, tau and v are published
        const int flag = *cl.map_shared_rank(&s_flag, owner);
        const double tau = *cl.map_shared_rank(&s_tau, owner);
        if (flag == 2 && q != owner) {
            const double2* vo = cl.map_shared_rank(v, owner);
            for (int i = tid; i < len; i += nt) v[i] = vo[i];
        }
        __syncthreads();
        if (flag == 2) {
            // left: H[c+1:, col] -= tau v (v^H H[c+1:, col]) for this CTA's columns col > c
            for (int lc = wid; lc < ncol; lc += nw) {
                const int col = q + lc * NC;
                if (col <= c) continue;
                double2 g = make_double2(0.0, 0.0);
                for (int i = lane; i < len; i += 32) cfma_conj(g, v[i], HL(c + 1 + i, lc));
                g = make_double2(warp_sum(g.x), warp_sum(g.y));
                g = (-tau) * g;
                for (int i = lane; i < len; i += 32) {
                    double2 hv = HL(c + 1 + i, lc);
                    cfma(hv, v[i], g);
                    HL(c + 1 + i, lc) = hv;
                }
            }
            __syncthreads();
            // right, partial: part[r] = sum over this CTA's columns col > c of H[r, col] v[col - c - 1]
            for (int r = tid; r < m; r += nt) {
                double2 acc = make_double2(0.0, 0.0);
                for (int lc = 0; lc < ncol; ++lc) {
                    const int col = q + lc * NC;
                    if (col > c) cfma(acc, HL(r, lc), v[col - c - 1]);
                }
                part[r] = acc;
            }
        }
        cl.sync();  // 2: every CTA's partial row sums are published
        if (flag == 2) {
            for (int r = tid; r < m; r += nt) {
                double2 sum = make_double2(0.0, 0.0);
                for (int k = 0; k < NC; ++k) sum = sum + cl.map_shared_rank(part, k)[r];
                prow[r] = (-tau) * sum;
            }
            __syncthreads();
            for (int idx = tid; idx < ncol * m; idx += nt) {
                const int lc = idx / m, r = idx - lc * m, col = q + lc * NC;
                if (col <= c) continue;
                double2 hv = HL(r, lc);
                cfma(hv, prow[r], conj(v[col - c - 1]));
                HL(r, lc) = hv;
            }
        }
        cl.sync();  // 3: the partials and v may be overwritten by the next column
    }
    for (int idx = tid; idx < ncol * m; idx += nt) {
        const int lc = idx / m, i = idx - lc * m;
        a.H[(size_t)(q + lc * NC) * m + i] = HL(i, lc);
    }
#undef HL
}

// Launches the cluster reduction when one cluster of NC CTAs with its shared memory fits on the
// device (checked once), else returns false and launches nothing.  KLST_NO_CLUSTER_HOUSE=1 keeps
// the single-CTA kernel.
template <int NC>
static bool launch_house_cluster(const SchurArgs& a, cudaStream_t s) {
    static std::mutex mu;
    static int ok = -1;
    const int m = a.m, ncmax = (m + NC - 1) / NC;
    const size_t smem = sizeof(double2) * ((size_t)ncmax * m + 2 * (size_t)m);
    if (m > 192 || smem > 160 * 1024) return false;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = NC;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(NC, 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (ok < 0) {
            ok = 0;
            const char* off = getenv("KLST_NO_CLUSTER_HOUSE");
            if (!(off && off[0] == '1') &&
                cudaFuncSetAttribute(k_schur_house64_cl<NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024) ==
                    cudaSuccess) {
                cudaLaunchConfig_t probe = cfg;
                probe.dynamicSmemBytes = 160 * 1024;
                int nclusters = 0;
                if (cudaOccupancyMaxActiveClusters(&nclusters, k_schur_house64_cl<NC>, &probe) == cudaSuccess &&
                    nclusters > 0)
                    ok = 1;
            }
            cudaGetLastError();
        }
    }
    if (!ok) return false;
    if (cudaLaunchKernelEx(&cfg, k_schur_house64_cl<NC>, a) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    note_launch();
    return true;
}

// ---------------------------------------------------------------- 2. QR sweeps + reordering
// Packed upper-Hessenberg storage in shared memory: column j keeps rows 0..j+1 at offset j(j+3)/2.
__device__ __forceinline__ int pk64(int i, int j) { return j * (j + 3) / 2 + i; }

// One component of the rotation [x; y] <- [c s; -conj(s) c] [x; y] (crot64's operation order):
// q = 0, 1: Re x', Im x'; q = 2, 3: Re y', Im y' -- three float64 operations each, so four lanes
// rotate one pair at a quarter of the float64 instructions per warp.  Every lane runs the same
// w = P1 Q1 + (P2 Q2 + P3 Q3) with its operands picked by selects (off the float64 pipe): lanes
// taking different arithmetic paths would each issue their own float64 instructions.
__device__ __forceinline__ double crot64_part(double2 x, double2 y, double c, double2 s, int q) {
    const bool lo = q < 2, odd = q & 1;
    const double p1 = lo ? c : -s.x;
    const double q1 = odd ? x.y : x.x;
    const double p2 = lo ? s.x : (odd ? s.y : -s.y);
    const double q2 = lo ? (odd ? y.y : y.x) : (odd ? x.x : x.y);
    const double p3 = lo ? (odd ? s.y : -s.y) : c;
    const double q3 = lo ? (odd ? y.x : y.y) : (odd ? y.y : y.x);
    return fma(p1, q1, fma(p2, q2, p3 * q3));
}

// givens64 by a whole warp (every lane passes the same f, g): lane parity splits the two squared
// moduli and the two reciprocal square roots, lanes 0, 1, 2 form Re s, Im s and c with one shared
// instruction shape, and the thresholds compare bit patterns (non-negative float64 values order
// like their bits), so the dependent chain holds eleven float64 instructions instead of
// twenty-four.  Same convention and edge cases as givens64.
__device__ void givens64_warp(double2 f, double2 g, double& c, double2& s) {
    const int lane = threadIdx.x & 31, h = lane & 1;
    const double2 u = h ? g : f;
    const double a2 = fma(u.x, u.x, u.y * u.y);
    const double o2 = __shfl_xor_sync(0xffffffffu, a2, 1);
    const double af2 = h ? o2 : a2, ag2 = h ? a2 : o2;
    const long long tiny = 0x03C2000000000000ll;  // bits of 2^-963 ~ 1e-290
    if (__double_as_longlong(ag2) <= tiny) { c = 1.0; s = make_double2(0.0, 0.0); return; }
    if (__double_as_longlong(af2) <= tiny) {
        const double ig = rsqrt64(ag2);
        c = 0.0;
        s = make_double2(g.x * ig, -g.y * ig);
        return;
    }
    const double rr = rsqrt64(h ? af2 : af2 + ag2);  // lane 0: 1 / r, lane 1: 1 / |f|
    const double ro = __shfl_xor_sync(0xffffffffu, rr, 1);
    const double q = rr * ro;                          // 1 / (|f| r)
    // lane 0: Re(f conj g), lane 1: Im(f conj g), lane 2: |f|^2, each times q
    const int k = lane & 3;
    const double p1 = k == 0 ? f.x : (k == 1 ? f.y : af2);
    const double q1 = k == 2 ? 1.0 : g.x;
    const double p2 = k == 0 ? f.y : (k == 1 ? -f.x : 0.0);
    const double v = fma(p1, q1, p2 * g.y) * q;
    c = __shfl_sync(0xffffffffu, v, 2);
    s = make_double2(__shfl_sync(0xffffffffu, v, 0), __shfl_sync(0xffffffffu, v, 1));
}

constexpr int kQrThreads = 512;               // 16 warps; the 12 off the first scheduler rotate
constexpr int kQrSlots = (kQrThreads / 32 / 4) * 3 * 8;  // element pairs per pass (4 lanes each)

// Shifted QR sweeps (explicit single shift, Wilkinson / exceptional shifts, float64 deflation).
// Within a sweep on the active window [lo, hi], step i applies left rotation i to rows (i, i+1)
// of the window's columns i..hi and, pipelined two steps behind, right rotation i-2 to columns
// (i-2, i-1) of the window's rows lo..i-1: column i-1 of R is final once left rotation i-1 is in,
// and the two kinds touch disjoint entries within a step.  The entries right of the window and
// above it receive the sweep's rotations afterwards (k_schur_defer64), since later sweeps read
// only entries inside their own windows, which are nested in or disjoint from this one.  Each entry pair is rotated by four lanes
// of a warp that does not share a scheduler with warp 0 (a float64 instruction holds a warp's
// scheduler for 64 cycles whatever the number of active lanes), while warp 0 rotates the pivot
// column i+1 and forms rotation i+1 from it, the only dependent chain of the step.  The shift is
// added back to each diagonal entry when its last rotation has been applied.
__global__ void __launch_bounds__(kQrThreads) k_schur_qr64(SchurArgs a) {
    extern __shared__ double2 sT64[];
    const int m = a.m, tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
    Rot64* log = reinterpret_cast<Rot64*>(a.log);
    __shared__ double rc[192];
    __shared__ double2 rs[192];
    __shared__ double2 s_mu;
    __shared__ int s_lo, s_fail, s_cnt;
    __shared__ int rdy[192], lvb[192];  // replay level bookkeeping (see k_schur_levels64)
#define TT(i, j) sT64[pk64(i, j)]
    for (int j = 0; j < m; ++j)
        for (int i = tid; i <= min(j + 1, m - 1); i += nt) TT(i, j) = a.H[(size_t)j * m + i];
    for (int i = tid; i < m; i += nt) rdy[i] = 0;
    if (tid == 0) { s_fail = 0; s_cnt = 0; }
    __syncthreads();
    const double2 zero2 = make_double2(0.0, 0.0);
    const double eps = 2.220446049250313e-16;  // float64 ulp(1): LAPACK's deflation threshold
    // rotation lanes: warps not on the first scheduler, four lanes per entry pair
    const bool rot_lane = (wid & 3) != 0;
    const int slot = ((wid >> 2) * 3 + (wid & 3) - 1) * 8 + (lane >> 2), comp = lane & 3;
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
        if (wid == 0) {
            double c;
            double2 sv;
            givens64_warp(TT(lo, lo), TT(lo + 1, lo), c, sv);
            if (lane == 0) { rc[lo] = c; rs[lo] = sv; }
        }
        __syncthreads();
        for (int i = lo; i <= hi + 1; ++i) {
            const int k = i - 2;                                  // right rotation of this step
            const int nl = (i <= hi - 1) ? hi + 1 - i : 0;        // left: columns i..hi of the window
            const int nr = (k >= lo && k <= hi - 1) ? k + 2 - lo : 0;  // right: rows lo..k+1
            if (rot_lane) {
                // at most two passes (m <= 160 < 2 kQrSlots): read and rotate both, then write.  Left
                // and right items take the same instruction path (operands chosen by selects).
                int row[2], col[2];
                double v[2];
                bool on[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int it = slot + u * kQrSlots;
                    on[u] = false;
                    // a warp with no item in this pass issues nothing (uniform over the warp)
                    if ((slot & ~7) + u * kQrSlots >= nl + nr) continue;
                    const bool left = it < nl && i + it != i + 1;  // warp 0 owns the pivot column
                    const bool right = it >= nl && it < nl + nr;
                    on[u] = left || right;
                    // left: rows (i, i+1) of column i+it; right: columns (k, k+1) of row lo+it-nl
                    const int rx = left ? i : lo + it - nl, ry = left ? i + 1 : lo + it - nl;
                    const int cx = left ? i + it : k, cy = left ? i + it : k + 1;
                    const int rr = left ? i : k;  // rotation index
                    double2 x = make_double2(0.0, 0.0), y = x, sv = x;
                    double cv = 1.0;
                    if (on[u]) {
                        x = TT(rx, cx);
                        y = TT(ry, cy);
                        cv = rc[rr];
                        sv = left ? rs[rr] : conj(rs[rr]);
                    }
                    double w = crot64_part(x, y, cv, sv, comp);
                    if (left && cx == i && comp >= 2) w = 0.0;  // the annihilated subdiagonal entry
                    if (right) {
                        // a diagonal entry is final after its last right rotation: add the shift back
                        const int r = lo + it - nl;
                        if (r == k && comp < 2) w += comp == 0 ? mu.x : mu.y;
                        if (r == k + 1 && k + 1 == hi && comp >= 2) w += comp == 2 ? mu.x : mu.y;
                    }
                    row[u] = comp < 2 ? rx : ry;
                    col[u] = comp < 2 ? cx : cy;
                    v[u] = w;
                }
                __syncwarp();
#pragma unroll
                for (int u = 0; u < 2; ++u)
                    if (on[u]) {
                        double* e = reinterpret_cast<double*>(&TT(row[u], col[u]));
                        e[comp & 1] = v[u];
                    }
            } else if (wid == 0 && i <= hi - 1) {
                // the pivot column i+1: rotated by lanes 0..3, then rotation i+1 from its new diagonal
                const double2 x = TT(i, i + 1), y = TT(i + 1, i + 1);
                const double w = crot64_part(x, y, rc[i], rs[i], comp);
                const double yr = __shfl_sync(0xffffffffu, w, 2), yi = __shfl_sync(0xffffffffu, w, 3);
                if (lane < 4) reinterpret_cast<double*>(&TT(comp < 2 ? i : i + 1, i + 1))[comp & 1] = w;
                if (i + 1 <= hi - 1) {
                    double c2;
                    double2 s2;
                    givens64_warp(make_double2(yr, yi), TT(i + 2, i + 1), c2, s2);
                    if (lane == 0) { rc[i + 1] = c2; rs[i + 1] = s2; }
                }
            }
            __syncthreads();
        }
        if (tid == 0) {
            // replay level of rotation j: one past the last level that touched index j or j+1
            int lv = max(rdy[lo], rdy[lo + 1]);
            lvb[lo] = lv;
            for (int j = lo + 1; j < hi; ++j) {
                lv = max(lv + 1, rdy[j + 1]);
                lvb[j] = lv;
            }
            for (int j = lo; j < hi; ++j) rdy[j] = lvb[j] + 1;
            rdy[hi] = lvb[hi - 1] + 1;
        }
        __syncthreads();
        const int base = s_cnt;
        for (int t = tid; t < hi - lo; t += nt) {
            Rot64 g;
            g.s = rs[lo + t]; g.c = rc[lo + t]; g.i = (lo + t) | (lo << 8) | (hi << 16); g.pad = lvb[lo + t];
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
    for (int i = tid; i < m; i += nt) a.rdy[i] = rdy[i];
    if (tid == 0) {
        int nlev = 0;
        for (int i = 0; i < m; ++i) nlev = max(nlev, rdy[i]);
        *a.log_count = s_cnt;
        a.log_count[1] = total;
        a.log_count[3] = nlev;
    }
#undef TT
}

// Reordering: bring the keep Ritz values of largest |mu| to the front of the upper triangular T in
// descending |mu| (ties to the lower index), the others after them in their original order -- the
// order a selection of the largest remaining |mu| with adjacent swaps produces.  Every diagonal
// entry gets its target position, and an odd-even transposition network sorts by it: in each
// round the out-of-order pairs (i, i+1) of one parity swap together (LAPACK ztrexc's rotation for
// each).  Swaps of a round touch disjoint row pairs on the left and disjoint column pairs on the
// right, and their rotations are formed from entries no other swap of the round changes; all
// left rotations go first, then all right ones, since both can hit one entry.  Entry pairs are
// rotated by four lanes each (crot64_part), and every swap's rotation is logged in round order.
constexpr int kReThreads = 512;
__global__ void __launch_bounds__(kReThreads) k_schur_reorder64(SchurArgs a) {
    extern __shared__ double2 sT64[];
    const int m = a.m, tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
    if (*a.nconv < 0) return;  // the QR sweeps failed; the host reports it
    Rot64* log = reinterpret_cast<Rot64*>(a.log);
    __shared__ int tgt[192], rnk[192], sw_i[96], offL[97], offR[97];
    __shared__ unsigned long long key[192];
    __shared__ double sw_c[96];
    __shared__ double2 sw_s[96];
    __shared__ int s_ns, s_fail, s_cnt, s_swaps;
    __shared__ int rdy[192], sw_lv[96];
#define TT(i, j) sT64[pk64(i, j)]
    for (int j = 0; j < m; ++j)
        for (int i = tid; i <= min(j + 1, m - 1); i += nt) TT(i, j) = a.H[(size_t)j * m + i];
    // |mu|^2 as an ordering key (non-negative float64 orders like its bits)
    for (int i = tid; i < m; i += nt) {
        const double2 d = a.H[(size_t)i * m + i];
        key[i] = (unsigned long long)__double_as_longlong(fma(d.x, d.x, d.y * d.y));
    }
    for (int i = tid; i < m; i += nt) rdy[i] = a.rdy[i];
    if (tid == 0) { s_fail = 0; s_cnt = *a.log_count; s_swaps = 0; }
    __syncthreads();
    // target positions: the rank in descending |mu| (ties to the lower index) for the keep largest;
    // keep + the number of unselected entries before i for the others
    for (int i = tid; i < m; i += nt) {
        int rank = 0;
        for (int j = 0; j < m; ++j) rank += (key[j] > key[i] || (key[j] == key[i] && j < i)) ? 1 : 0;
        rnk[i] = rank;
    }
    __syncthreads();
    for (int i = tid; i < m; i += nt) {
        int r = rnk[i];
        if (r >= a.keep) {
            int u = 0;
            for (int j = 0; j < i; ++j) u += rnk[j] >= a.keep ? 1 : 0;
            r = a.keep + u;
        }
        tgt[i] = r;
    }
    const int comp = lane & 3, slot = tid >> 2, nslot = nt >> 2;
    for (int round = 0, parity = 0, quiet = 0; quiet < 2 && round <= m + 1; ++round, parity ^= 1) {
        __syncthreads();  // every thread has read the previous round's s_ns
        // the swaps of this round, in increasing i
        if (tid == 0) {
            int ns = 0;
            for (int i = parity; i + 1 < m; i += 2)
                if (tgt[i] > tgt[i + 1]) sw_i[ns++] = i;
            s_ns = ns;
            if (s_cnt + ns > a.log_cap) { s_fail = 2; s_ns = 0; }
            offL[0] = 0; offR[0] = 0;
            for (int q = 0; q < s_ns; ++q) {
                offL[q + 1] = offL[q] + (m - 2 - sw_i[q]);
                offR[q + 1] = offR[q] + sw_i[q];
            }
        }
        __syncthreads();
        const int ns = s_ns;
        quiet = ns == 0 ? quiet + 1 : 0;
        if (ns == 0) { if (s_fail) break; continue; }
        for (int q = tid; q < ns; q += nt) {
            const int i = sw_i[q];
            double c;
            double2 sv;
            givens64(TT(i, i + 1), TT(i + 1, i + 1) - TT(i, i), c, sv);
            sw_c[q] = c;
            sw_s[q] = sv;
            const int lv = max(rdy[i], rdy[i + 1]);  // the swaps of a round touch disjoint pairs
            sw_lv[q] = lv;
            Rot64 g;
            g.s = sv; g.c = c; g.i = i | ((m - 1) << 16); g.pad = lv;
            log[s_cnt + q] = g;
        }
        __syncthreads();
        // left rotations: rows (i, i+1) of columns i+2..m-1, then right: columns (i, i+1) of rows 0..i-1
        for (int phase = 0; phase < 2; ++phase) {
            const int* off = phase == 0 ? offL : offR;
            const int total = off[ns];
            for (int base = 0; base < total; base += nslot) {
                if (base + (slot & ~7) >= total) continue;  // nothing for this warp (uniform)
                const int it = base + slot;
                int rw = 0, cl = 0;
                double v = 0.0;
                const bool on = it < total;
                if (on) {
                    int lo = 0, hi = ns - 1;  // the swap q with off[q] <= it < off[q + 1]
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (off[mid] <= it) lo = mid; else hi = mid - 1;
                    }
                    const int i = sw_i[lo], u = it - off[lo];
                    if (phase == 0) {
                        const int col = i + 2 + u;
                        v = crot64_part(TT(i, col), TT(i + 1, col), sw_c[lo], sw_s[lo], comp);
                        rw = comp < 2 ? i : i + 1;
                        cl = col;
                    } else {
                        const int row = u;
                        v = crot64_part(TT(row, i), TT(row, i + 1), sw_c[lo], conj(sw_s[lo]), comp);
                        rw = row;
                        cl = comp < 2 ? i : i + 1;
                    }
                }
                __syncwarp();
                if (on) reinterpret_cast<double*>(&TT(rw, cl))[comp & 1] = v;
                __syncwarp();
            }
            __syncthreads();
        }
        for (int q = tid; q < ns; q += nt) {
            const int i = sw_i[q];
            const double2 t11 = TT(i, i);
            TT(i, i) = TT(i + 1, i + 1);
            TT(i + 1, i + 1) = t11;
            const int tg = tgt[i];
            tgt[i] = tgt[i + 1];
            tgt[i + 1] = tg;
            rdy[i] = rdy[i + 1] = sw_lv[q] + 1;
        }
        __syncthreads();
        if (tid == 0) { s_cnt += ns; s_swaps += ns; }
        __syncthreads();
    }
    if (s_fail) {
        if (tid == 0) { atomicOr(&a.st->flags, ST_NOCONV_QR); *a.nconv = -1; *a.log_count = 0; }
        return;
    }
    const double2 zero2 = make_double2(0.0, 0.0);
    for (int idx = tid; idx < m * m; idx += nt) {
        const int i = idx % m, j = idx / m;
        a.H[idx] = (i <= j) ? TT(i, j) : zero2;
    }
    if (tid == 0) {
        int nlev = 0;
        for (int i = 0; i < m; ++i) nlev = max(nlev, rdy[i]);
        *a.log_count = s_cnt;
        a.log_count[2] = s_swaps;
        a.log_count[3] = nlev;
    }
#undef TT
}

// ---------------------------------------------------------------- 3. Schur vectors
// Replay levels.  Row r of Q is e_r^T H_0 H_1 ... H_{m-3} G_1^H G_2^H ... (the reflectors, then every
// logged rotation in order).  A rotation acts on entries (i, i+1) of the row only, so two rotations
// on disjoint pairs commute: the sweeps and swaps above give rotation k the level one past the last
// level that touched i or i+1, every rotation of one level acts on a disjoint pair, and replaying
// the levels in order gives the same product (each entry sees its rotations in log order).  The
// QR sweeps follow one another two indices apart, so the levels number about twice the sweeps
// rather than the rotations.  One CTA sorts the log by level (counting sort; the order within a
// level is immaterial), leaving in loff[l] the end of level l.
__global__ void __launch_bounds__(1024) k_schur_levels64(SchurArgs a) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
    if (*a.nconv < 0) return;
    const int nrot = a.log_count[0], nlev = a.log_count[3];
    const Rot64* log = reinterpret_cast<const Rot64*>(a.log);
    Rot64* out = reinterpret_cast<Rot64*>(a.log2);
    __shared__ int wsum[32];
    __shared__ int s_carry;
    for (int l = tid; l <= nlev; l += nt) a.loff[l] = 0;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (int k = tid; k < nrot; k += nt) atomicAdd(&a.loff[log[k].pad], 1);
    __syncthreads();
    // exclusive scan of the level counts, in place
    for (int base = 0; base < nlev; base += nt) {
        const int l = base + tid;
        const int v = l < nlev ? a.loff[l] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int w = lane < (nt >> 5) ? wsum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            wsum[lane] = w;  // inclusive prefix of the warp totals
        }
        __syncthreads();
        const int incl = x + (wid > 0 ? wsum[wid - 1] : 0);
        if (l < nlev) a.loff[l] = s_carry + incl - v;
        __syncthreads();
        if (tid == nt - 1) s_carry += incl;
        __syncthreads();
    }
    for (int k = tid; k < nrot; k += nt) {
        const Rot64 g = log[k];
        out[atomicAdd(&a.loff[g.pad], 1)] = g;
    }
}

// One CTA per row of Q.  Warp 0 applies the reflectors (the lanes split each reflector's dot
// product and update); then the CTA replays the levels: four lanes per rotation, one component
// each (crot64_part), a level's rotations at once, the next level's bounds and entries loaded
// while the current one is applied.
constexpr int kQThreads = 256;
__global__ void __launch_bounds__(kQThreads) k_schur_q64(SchurArgs a) {
    extern __shared__ double2 qrow[];  // [m]
    const int m = a.m, r = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const double2* Vh = reinterpret_cast<const double2*>(a.Vh);
    const Rot64* lg = reinterpret_cast<const Rot64*>(a.log2);
    if (wid == 0) {
        for (int col = lane; col < m; col += 32) qrow[col] = make_double2(col == r ? 1.0 : 0.0, 0.0);
        __syncwarp();
        for (int c = 0; c + 2 < m; ++c) {
            const double tau = a.tau[c];
            if (tau == 0.0) continue;
            const double2* vc = Vh + (size_t)c * m;
            double2 g = make_double2(0.0, 0.0);
            for (int i = c + 1 + lane; i < m; i += 32) cfma(g, qrow[i], vc[i]);
            g = (-tau) * make_double2(warp_sum(g.x), warp_sum(g.y));
            for (int i = c + 1 + lane; i < m; i += 32) {
                double2 qi = qrow[i];
                cfma(qi, g, conj(vc[i]));
                qrow[i] = qi;
            }
            __syncwarp();
        }
    }
    __syncthreads();
    const int nlev = *a.nconv < 0 ? 0 : a.log_count[3];
    const int grp = tid >> 2, comp = tid & 3, ngrp = kQThreads / 4;
    int beg = 0;
    int end = nlev > 0 ? a.loff[0] : 0;
    Rot64 cur;
    if (nlev > 0 && grp < end) cur = lg[grp];
    for (int l = 0; l < nlev; ++l) {
        // prefetch the next level's end and this thread's entry of it
        const int nend = l + 1 < nlev ? a.loff[l + 1] : end;
        Rot64 nxt;
        if (l + 1 < nlev && end + grp < nend) nxt = lg[end + grp];
        for (int k0 = beg; k0 < end; k0 += ngrp) {
            if (k0 + (grp & ~7) >= end) continue;  // nothing for this warp (uniform)
            const int k = k0 + grp;
            const bool on = k < end;
            const Rot64 g = k0 == beg ? cur : (on ? lg[k] : cur);
            double w = 0.0;
            const int gi = rot_i(g);
            if (on) w = crot64_part(qrow[gi], qrow[gi + 1], g.c, conj(g.s), comp);
            __syncwarp();
            if (on) reinterpret_cast<double*>(&qrow[comp < 2 ? gi : gi + 1])[comp & 1] = w;
            __syncwarp();
        }
        __syncthreads();
        beg = end;
        end = nend;
        cur = nxt;
    }
    for (int col = tid; col < m; col += kQThreads) a.Q[(size_t)col * m + r] = qrow[col];
}

// The updates the window-restricted QR sweeps left out, replayed by level like the Schur vectors:
// phase 0, one CTA per row r of T, applies the right rotations of every sweep whose window starts
// below r (entries (r, i), (r, i+1)); phase 1, one CTA per column c, the left rotations of every
// sweep whose window ends above c (entries (i, c), (i+1, c)).  Left and right rotations commute, so
// applying all the right ones first and then all the left ones gives the full update; within one
// row or column the level order keeps every entry's rotations in log order.
__global__ void __launch_bounds__(kQThreads) k_schur_defer64(SchurArgs a, int phase) {
    extern __shared__ double2 qrow[];  // [m]: the row (phase 0) or column (phase 1)
    const int m = a.m, r = blockIdx.x, tid = threadIdx.x;
    if (*a.nconv < 0) return;
    const Rot64* lg = reinterpret_cast<const Rot64*>(a.log2);
    for (int k = tid; k < m; k += kQThreads) qrow[k] = phase == 0 ? a.H[(size_t)k * m + r] : a.H[(size_t)r * m + k];
    __syncthreads();
    const int nlev = a.log_count[3];
    const int grp = tid >> 2, comp = tid & 3, ngrp = kQThreads / 4;
    int beg = 0;
    for (int l = 0; l < nlev; ++l) {
        const int end = a.loff[l];
        for (int k0 = beg; k0 < end; k0 += ngrp) {
            if (k0 + (grp & ~7) >= end) continue;  // nothing for this warp (uniform)
            const int k = k0 + grp;
            Rot64 g;
            bool on = k < end;
            if (on) {
                g = lg[k];
                on = phase == 0 ? (r < rot_lo(g)) : (r > rot_hi(g));
            }
            double w = 0.0;
            int gi = 0;
            if (on) {
                gi = rot_i(g);
                w = crot64_part(qrow[gi], qrow[gi + 1], g.c, phase == 0 ? conj(g.s) : g.s, comp);
            }
            __syncwarp();
            if (on) reinterpret_cast<double*>(&qrow[comp < 2 ? gi : gi + 1])[comp & 1] = w;
            __syncwarp();
        }
        __syncthreads();
        beg = end;
    }
    for (int k = tid; k < m; k += kQThreads) {
        if (phase == 0) a.H[(size_t)k * m + r] = qrow[k];
        else a.H[(size_t)r * m + k] = qrow[k];
    }
}

int launch_schur64(const SchurArgs& a, cudaStream_t s) {
    static std::atomic<unsigned long long> attr{0};
    KLST_CK(set_once_per_device(attr, [] {
        cudaError_t e = cudaFuncSetAttribute(k_schur_qr64, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_schur_reorder64, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
        return e;
    }));
    const int m = a.m;
    const size_t packed = sizeof(double2) * (size_t)m * (m + 3) / 2;
    prof_begin("schur_house", s);
    if (!launch_house_cluster<8>(a, s)) { k_schur_house64<<<1, 256, 0, s>>>(a); note_launch(); }
    prof_end("schur_house", s);
    prof_begin("schur_qr", s);
    k_schur_qr64<<<1, kQrThreads, packed, s>>>(a); note_launch();
    prof_end("schur_qr", s);
    prof_begin("schur_defer", s);
    k_schur_levels64<<<1, 1024, 0, s>>>(a); note_launch();
    for (int phase = 0; phase < 2; ++phase) {
        k_schur_defer64<<<m, kQThreads, sizeof(double2) * m, s>>>(a, phase);
        note_launch();
    }
    prof_end("schur_defer", s);
    prof_begin("schur_reorder", s);
    k_schur_reorder64<<<1, kReThreads, packed, s>>>(a); note_launch();
    prof_end("schur_reorder", s);
    prof_begin("schur_q", s);
    k_schur_levels64<<<1, 1024, 0, s>>>(a); note_launch();
    k_schur_q64<<<m, kQThreads, sizeof(double2) * m, s>>>(a); note_launch();
    prof_end("schur_q", s);
    launch_schur_post(a, s);
    KLST_CK_LAUNCH();
    return KLST_OK;
}

}  // namespace klst
