// Float64-accurate real GEMM C = A B on the 5th-generation tensor cores (tcgen05), by error-free
// splitting of the operands into small integer slices (the Ozaki scheme: Ozaki, Ogita, Oishi and
// Rump, "Error-free transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012).
//
// Splitting.  Row r of A (over the reduction index k) is scaled by 2^-ea[r] with |A[r, k]| < 2^ea[r]
// and written as a signed fixed-point integer F = A[r, k] 2^(56 - ea[r]) (|F| < 2^56, truncated below
// 2^-56 of the row's largest entry).  F is cut into eight balanced base-128 digits,
//     A[r, k] ~= 2^ea[r] sum_{s=1..8} a_s[r, k] 2^(-7 s),   |a_1| <= 128, |a_s| <= 64 (s >= 2),
// every digit an integer held exactly by bfloat16.  B is split the same way per column (eb[c]).
// Products.  a_s b_t is an integer product; for a fixed diagonal d = s + t the sum over k of every
// pair on that diagonal stays below 2^24 for K <= 256 (at most 2 pairs reach 128 x 64, the others
// 64 x 64: (2 * 8192 + 6 * 4096) * 256 < 2^24), so a float32 tensor-core accumulator holds it
// exactly.  The eight diagonals d = 2..9 (36 slice pairs; pairs with s + t > 9 are dropped, a
// relative error below 2^-55 of the row and column maxima) are accumulated in eight TMEM blocks:
// one MMA per A-slice s multiplies a_s by the B slices t = 1..9-s stacked along N, whose products
// land in the TMEM blocks s+1..9 -- a sliding window, so every diagonal block receives exactly its
// own pairs.  The epilogue sums the eight exact block values in float64 (one rounding each) and
// scales by 2^(ea[r] + eb[c]).  The result carries float64-level error relative to
// max_k |A[r, k]| max_k |B[k, c]| K.
//
// Layouts (K-major, no swizzle: 8-row x 16-byte core matrices).  A slices: [mtile][s][kchunk]
// [128 rows][8], so one slice of one 128-row tile is a contiguous block of K x 256 bytes (core
// matrices adjacent in K 2 KB apart, 8-row groups 128 B apart).  B slices: [ntile][kchunk][s]
// [NT rows][8]: for each k-chunk the eight slices' rows follow one another, so a contiguous run of
// (9 - s) slices is one N-stacked operand (8-row groups 128 B apart, k-chunks 8 NT 16 B apart).
#include <algorithm>
#include <atomic>
#include <cstring>

#include "oz_gemm.cuh"

namespace klst {



// Element sources: the GEMM's A rows and B columns as functions (row, k) -> double
struct SrcColMajor {    // A: A[k * ld + r]  (column-major M x K);  B: B[c * ld + k] (column-major K x N)
    const double* p;
    int64_t ld;
    int rows_are_k;     // 0: element (r, k) = p[k * ld + r]; 1: element (c, k) = p[c * ld + k]
    int R, K;
    __device__ double operator()(int r, int k) const {
        if (r >= R || k >= K) return 0.0;
        return rows_are_k ? p[(int64_t)r * ld + k] : p[(int64_t)k * ld + r];
    }
};
struct SrcBasisRows {   // rows of [Re V | Im V] for a complex column-major basis V (n x m, ld)
    const double2* V;
    int64_t ld;
    int m, R;
    __device__ double operator()(int r, int k) const {
        if (r >= R || k >= 2 * m) return 0.0;
        const double2 v = V[(int64_t)(k < m ? k : k - m) * ld + r];
        return k < m ? v.x : v.y;
    }
};
struct SrcRotCols {     // columns of [[Qr, Qi], [-Qi, Qr]] (2m x 2 keep) for a complex Q (m x keep, ld)
    const double2* Q;
    int ld, m, keep;
    __device__ double operator()(int c, int k) const {
        if (c >= 2 * keep || k >= 2 * m) return 0.0;
        const int cc = c < keep ? c : c - keep, kk = k < m ? k : k - m;
        const double2 q = Q[(int64_t)cc * ld + kk];
        if (c < keep) return k < m ? q.x : -q.y;
        return k < m ? q.y : q.x;
    }
};

struct SrcPencilCols {  // Z = D_x Y: column col = rhs * 4 nxi + 2 p + reim of Y is component reim of block p of x_rhs
    const double* y;     // complex, interleaved; x_rhs starts at rhs * ldy complex entries
    int64_t ldy;
    int nx, nxi, N;
    __device__ double operator()(int col, int kk) const {
        if (col >= N || kk >= nx) return 0.0;
        const int per = 4 * nxi, rhs = col / per, cc = col - rhs * per;
        return y[((int64_t)rhs * ldy + (int64_t)(cc >> 1) * nx + kk) * 2 + (cc & 1)];
    }
};





// Output sinks: where C[r, c] goes
struct DstColMajor {    // C[c * ld + r]
    double* p;
    int64_t ld;
    int R, N;
    __device__ void done() {}
    __device__ void operator()(int r, int c, double v) const {
        if (r < R && c < N) p[(int64_t)c * ld + r] = v;
    }
};
struct DstBasis {       // column c < keep -> Re V'[r, c], c >= keep -> Im V'[r, c - keep] (complex, ld)
    double* p;
    int64_t ld;
    int R, keep;
    __device__ void done() {}
    __device__ void operator()(int r, int c, double v) const {
        if (r < R && c < 2 * keep) p[((int64_t)(c < keep ? c : c - keep) * ld + r) * 2 + (c < keep ? 0 : 1)] = v;
    }
};

struct DstPencilCols {  // C[j, col] -> z_rhs[p nx + j] component reim, the layout of the input vectors
    double* z;
    int64_t ldz;
    int nx, nxi, N;
    __device__ void done() {}
    __device__ void operator()(int r, int col, double v) const {
        if (r >= nx || col >= N) return;
        const int per = 4 * nxi, rhs = col / per, cc = col - rhs * per;
        z[((int64_t)rhs * ldz + (int64_t)(cc >> 1) * nx + r) * 2 + (cc & 1)] = v;
    }
};


// ------------------------------------------------------------------ host side
size_t oz_workspace_bytes(int M, int N, int K) {
    const int Kp = (K + 15) / 16 * 16;
    const size_t mt = (M + 127) / 128, nt = (N + OZ_NT - 1) / OZ_NT;
    const size_t a = mt * 128 * (size_t)Kp * OZ_S * 2, b = nt * OZ_NT * (size_t)Kp * OZ_S * 2;
    return ((a + 255) & ~size_t(255)) + ((b + 255) & ~size_t(255)) + (mt * 128 + nt * OZ_NT) * sizeof(int) + 256;
}

struct OzWork {
    unsigned short *A, *B;
    int *ea, *eb;
};
static OzWork oz_carve(void* ws, int M, int N, int Kp) {
    const size_t mt = (M + 127) / 128, nt = (N + OZ_NT - 1) / OZ_NT;
    char* p = (char*)ws;
    OzWork w;
    w.A = (unsigned short*)p;
    p += ((mt * 128 * (size_t)Kp * OZ_S * 2) + 255) & ~size_t(255);
    w.B = (unsigned short*)p;
    p += ((nt * OZ_NT * (size_t)Kp * OZ_S * 2) + 255) & ~size_t(255);
    w.ea = (int*)p;
    w.eb = w.ea + mt * 128;
    return w;
}

template <class Dst>
static int oz_launch_gemm(const OzWork& w, int M, int N, int Kp, Dst dst, Status* st, cudaStream_t s,
                          const int* skip = nullptr, int cols_per_flag = 1) {
    static std::atomic<unsigned long long> attr{0};
    const size_t bytesB = (size_t)Kp * OZ_NT * 16, bytesA = (size_t)Kp * 256;
    const size_t smem = bytesB + (bytesB + 2 * bytesA <= kOzSmemCap ? 2 : 1) * bytesA;
    KLST_CK(set_once_per_device(attr, [] {
        return cudaFuncSetAttribute(k_oz_gemm<Dst>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOzSmemCap);
    }));
    dim3 grid((N + OZ_NT - 1) / OZ_NT, (M + 127) / 128);
    k_oz_gemm<Dst><<<grid, 128, smem, s>>>(w.A, w.B, w.ea, w.eb, Kp, dst, st, skip, cols_per_flag, N, 0);
    note_launch();
    KLST_CK_LAUNCH();
    return KLST_OK;
}

// V'[:, 0:keep] = V[:, 0:m] Q[:, 0:keep] (complex, column-major, ld n for V and V', m for Q)
int oz_rotate(const double2* V, int64_t n, int m, const double2* Q, int keep, double2* Vout, void* ws, Status* st,
              cudaStream_t s) {
    const int K = 2 * m, Kp = (K + 15) / 16 * 16, N = 2 * keep;
    if (Kp > OZ_KMAX || n > (int64_t)0x7FFFFFFF) { set_error("rotation too large for the tensor-core path"); return KLST_EINVAL; }
    OzWork w = oz_carve(ws, (int)n, N, Kp);
    const int R = (int)n;
    SrcBasisRows sa{V, n, m, R};
    SrcRotCols sb{Q, m, m, keep};
    k_oz_split_a<SrcBasisRows><<<(int)((n + 127) / 128 * 32), 128, 0, s>>>(sa, R, Kp, w.A, w.ea, nullptr);
    note_launch();
    k_oz_split_b<SrcRotCols><<<(N + OZ_NT - 1) / OZ_NT * OZ_NT / 4, 128, 0, s>>>(sb, N, Kp, w.B, w.eb, nullptr, 1);
    note_launch();
    KLST_CK_LAUNCH();
    return oz_launch_gemm(w, R, N, Kp, DstBasis{reinterpret_cast<double*>(Vout), n, R, keep}, st, s);
}

// D_x of a pencil as the A operand (row j, reduction index m: D_x[j][m], row-major nx x nx), once per pencil
size_t oz_dx_bytes(int nx) {
    const int Kp = (nx + 15) / 16 * 16;
    return (size_t)128 * Kp * OZ_S * 2 + 128 * sizeof(int);
}
int oz_split_dx(const double* Dx, int nx, void* buf, cudaStream_t s) {
    const int Kp = (nx + 15) / 16 * 16;
    unsigned short* A = (unsigned short*)buf;
    int* ea = (int*)((char*)buf + (size_t)128 * Kp * OZ_S * 2);
    SrcColMajor sa{Dx, nx, 1, nx, nx};
    k_oz_split_a<SrcColMajor><<<32, 128, 0, s>>>(sa, nx, Kp, A, ea, nullptr);
    note_launch();
    KLST_CK_LAUNCH();
    return KLST_OK;
}
// workspace of oz_dx_apply for nrhs vectors
size_t oz_dx_ws_bytes(int nx, int nxi, int nrhs) {
    const int Kp = (nx + 15) / 16 * 16, N = 4 * nxi * nrhs;
    const size_t nt = (N + OZ_NT - 1) / OZ_NT;
    return ((nt * OZ_NT * (size_t)Kp * OZ_S * 2 + 255) & ~size_t(255)) + nt * OZ_NT * sizeof(int) + 256;
}
// z_rhs[(c nxi + k) nx + j] = sum_m D_x[j][m] x_rhs[(c nxi + k) nx + m] for every block, in float64 accuracy
int oz_dx_apply(const void* dxbuf, int nx, int nxi, const double2* x, int64_t ldx, int nrhs, double2* z, void* ws,
                Status* st, cudaStream_t s, const int* done) {
    const int Kp = (nx + 15) / 16 * 16, N = 4 * nxi * nrhs;
    const size_t nt = (N + OZ_NT - 1) / OZ_NT;
    OzWork w;
    w.A = (unsigned short*)dxbuf;
    w.ea = (int*)((const char*)dxbuf + (size_t)128 * Kp * OZ_S * 2);
    w.B = (unsigned short*)ws;
    w.eb = (int*)((char*)ws + ((nt * OZ_NT * (size_t)Kp * OZ_S * 2 + 255) & ~size_t(255)));
    SrcPencilCols sb{reinterpret_cast<const double*>(x), ldx, nx, nxi, N};
    k_oz_split_b<SrcPencilCols><<<(int)(nt * OZ_NT / 4), 128, 0, s>>>(sb, N, Kp, w.B, w.eb, done, 4 * nxi);
    note_launch();
    KLST_CK_LAUNCH();
    return oz_launch_gemm(w, nx, N, Kp, DstPencilCols{reinterpret_cast<double*>(z), ldx, nx, nxi, N}, st, s, done,
                          4 * nxi);
}

int oz_gemm_f64(const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc, int M, int N, int K,
                void* ws, Status* st, cudaStream_t s) {
    const int Kp = (K + 15) / 16 * 16;
    OzWork w = oz_carve(ws, M, N, Kp);
    SrcColMajor sa{A, lda, 0, M, K};
    SrcColMajor sb{B, ldb, 1, N, K};
    k_oz_split_a<SrcColMajor><<<(M + 127) / 128 * 32, 128, 0, s>>>(sa, M, Kp, w.A, w.ea, nullptr);
    note_launch();
    k_oz_split_b<SrcColMajor><<<(N + OZ_NT - 1) / OZ_NT * OZ_NT / 4, 128, 0, s>>>(sb, N, Kp, w.B, w.eb, nullptr, 1);
    note_launch();
    KLST_CK_LAUNCH();
    return oz_launch_gemm(w, M, N, Kp, DstColMajor{C, ldc, M, N}, st, s);
}

}  // namespace klst

using namespace klst;

extern "C" int klst_gemm_f64_tc(const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc,
                                int32_t M, int32_t N, int32_t K, klst_stream stream) {
    if (!A || !B || !C || M < 1 || N < 1 || K < 1 || K > OZ_KMAX || lda < M || ldb < K || ldc < M) {
        set_error("invalid arguments to klst_gemm_f64_tc (1 <= K <= %d)", OZ_KMAX);
        return KLST_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    void* ws = nullptr;
    Status* st = nullptr;
    cudaError_t e;
    if ((e = dmalloc(&ws, oz_workspace_bytes(M, N, K), s)) != cudaSuccess) return cuda_fail(e, "cudaMalloc", __FILE__, __LINE__);
    if ((e = dmalloc((void**)&st, sizeof(Status), s)) != cudaSuccess) { dfree(ws, s); return cuda_fail(e, "cudaMalloc", __FILE__, __LINE__); }
    cudaMemsetAsync(st, 0, sizeof(Status), s);
    int rc = oz_gemm_f64(A, lda, B, ldb, C, ldc, M, N, K, ws, st, s);
    Status hst;
    memset(&hst, 0, sizeof(hst));
    if (rc == KLST_OK) {
        if ((e = cudaMemcpyAsync(&hst, st, sizeof(Status), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            rc = cuda_fail(e, "gemm sync", __FILE__, __LINE__);
    }
    dfree(ws, s);
    dfree(st, s);
    if (rc == KLST_OK && (hst.flags & ST_TIMEOUT)) { set_error("tensor-core GEMM: a bounded wait gave up"); return KLST_ETIMEOUT; }
    return rc;
}
