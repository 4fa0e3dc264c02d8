// The float64-accurate slice GEMM of the Ozaki scheme as kernel templates (element sources and
// output sinks are functors), shared by the GEMM entry points, the D_x products and the
// Newton-Schulz steps of the block inverses.
#pragma once
#include "oz.cuh"

namespace klst {

constexpr int OZ_NT = 32;      // output columns per CTA (8 diagonal blocks x 32 = 256 TMEM columns)
constexpr size_t kOzSmemCap = 200 * 1024;  // dynamic shared memory the GEMM may use

// B operand: one warp per column c (a row of B^T) into the stacked slice layout of its N-tile.
// skip (optional): per column group of cols_per_flag columns, a flag that marks the group done.
template <class Src>
__global__ void __launch_bounds__(128) k_oz_split_b(Src src, int N, int Kp, unsigned short* __restrict__ out,
                                                    int* __restrict__ eb, const int* __restrict__ skip, int cols_per_flag) {
    const int c = blockIdx.x * 4 + (threadIdx.x >> 5);
    const int ntile = c / OZ_NT, cc = c % OZ_NT;
    if (ntile >= (N + OZ_NT - 1) / OZ_NT) return;
    if (skip && c < N && skip[c / cols_per_flag]) return;
    const int nkc = Kp / 8;
    auto dst = [&](int sl, int kc) { return out + ((((size_t)ntile * nkc + kc) * OZ_S + sl) * OZ_NT + cc) * 8; };
    oz_split_row(src, c, Kp, dst, eb + c);
}

// One CTA = one 128-row M tile x OZ_NT output columns; four warps.  Thread 0 loads (bulk copies)
// and issues the MMAs; every warp then drains its 32 TMEM lanes.  smem: the N-tile's stacked B
// slices (K x OZ_NT x 16 B) and one A slice (K x 256 B).  Waits are bounded: on a timeout the CTA
// sets ST_TIMEOUT in *st, skips the remaining work, frees its TMEM and returns.
// Dst: operator()(r, c, value) for every output of the tile (called by all 32 lanes of a warp
// together), then done() once per thread.
// batched = 1: grid.y indexes independent products (A tile y times its own B tiles y * grid.x + x);
// the columns passed to dst and the B exponents are then numbered across the whole batch.

template <class Dst>
__global__ void __launch_bounds__(128, 1) k_oz_gemm(const unsigned short* __restrict__ As,
                                                    const unsigned short* __restrict__ Bs,
                                                    const int* __restrict__ ea, const int* __restrict__ eb, int Kp,
                                                    Dst dst, Status* st, const int* __restrict__ skip, int cols_per_flag,
                                                    int N, int batched) {
    {
        // every column of this tile belongs to finished work: nothing to do (before any allocation)
        const int c0 = blockIdx.x * OZ_NT, c1 = min(N, c0 + OZ_NT) - 1;
        if (skip && skip[c0 / cols_per_flag] && skip[c1 / cols_per_flag]) return;
    }
    extern __shared__ __align__(128) unsigned char oz_smem[];
    __shared__ __align__(8) uint64_t bar_ld, bar_ld2, bar_mma;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    const int mtile = blockIdx.y, ntile = batched ? blockIdx.y * gridDim.x + blockIdx.x : blockIdx.x;
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    const int nkc = Kp / 8;
    const uint32_t bytesB = (uint32_t)Kp * OZ_NT * 16;   // nkc x OZ_S x OZ_NT x 16 B
    const uint32_t bytesA = (uint32_t)Kp * 256;          // nkc x 128 x 16 B
    unsigned char* sB = oz_smem;
    unsigned char* sA0 = oz_smem + bytesB;
    // two A buffers when the launch gave room for them (the next slice loads while the current one
    // multiplies); a launch with room for one leaves space for a second CTA on the SM instead
    uint32_t dyn;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    const bool dbuf = bytesB + 2 * bytesA <= dyn;
    unsigned char* sA1 = dbuf ? sA0 + bytesA : sA0;
    constexpr uint32_t kCols = 256;                      // 8 diagonal blocks x OZ_NT
    if (tid == 0) {
        mbar_init(&bar_ld, 1);
        mbar_init(&bar_ld2, 1);
        mbar_init(&bar_mma, 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (wid == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)), "r"(kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tbase = tmem_base;
    if (tid == 0) {
        const unsigned short* gB = Bs + (size_t)ntile * nkc * OZ_S * OZ_NT * 8;
        auto gA = [&](int s) { return As + (((size_t)mtile * OZ_S + s) * nkc) * 128 * 8; };
        // slice s is loaded into buffer s & 1 on barrier bar[s & 1]; with one buffer both are the same
        uint64_t* bars[2] = {&bar_ld, dbuf ? &bar_ld2 : &bar_ld};
        unsigned char* bufs[2] = {sA0, sA1};
        uint32_t ph[2] = {0, 0}, ph_mma = 0;
        bool ok = true;
        mbar_expect_tx(bars[0], bytesA + bytesB);
        bulk_g2s(bufs[0], gA(0), bytesA, bars[0]);
        bulk_g2s(sB, gB, bytesB, bars[0]);
        if (dbuf) {
            mbar_expect_tx(bars[1], bytesA);
            bulk_g2s(bufs[1], gA(1), bytesA, bars[1]);
        }
        for (int s = 0; s < OZ_S && ok; ++s) {
            const int b = dbuf ? (s & 1) : 0;
            ok = mbar_wait(bars[b], ph[b]);
            ph[b] ^= 1;
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // a_s x [b_1 .. b_{8-s}] (N = (8 - s) x OZ_NT) into diagonal blocks s+1 .. 8 (0-based d-2)
            const int nst = OZ_S - s;
            const uint32_t idesc = idesc_bf16(128, nst * OZ_NT);
            const uint32_t dcol = tbase + (uint32_t)(s * OZ_NT);
            const uint32_t aBase = smem_u32(bufs[b]), bBase = smem_u32(sB);
            for (int kk = 0; kk < Kp / 16; ++kk) {
                const uint64_t ad = sdesc(aBase + kk * 2 * 2048, 2048, 128);
                const uint64_t bd = sdesc(bBase + kk * 2 * (OZ_S * OZ_NT * 16), OZ_S * OZ_NT * 16, 128);
                mma_bf16(dcol, ad, bd, idesc, (s > 0 || kk > 0) ? 1u : 0u);
            }
            mma_commit(&bar_mma);
            // the buffer is reused only after the MMAs reading it have completed
            ok = mbar_wait(&bar_mma, ph_mma);
            ph_mma ^= 1;
            if (!ok) break;
            const int nxt = s + (dbuf ? 2 : 1);
            if (nxt < OZ_S) {
                mbar_expect_tx(bars[b], bytesA);
                bulk_g2s(bufs[b], gA(nxt), bytesA, bars[b]);
            }
        }
        if (!ok) {
            s_fail = 1;
            atomicOr(&st->flags, ST_TIMEOUT);
            // give any copy or MMA still in flight one more bounded wait before the TMEM is freed
            mbar_wait(&bar_ld, ph[0]);
            if (dbuf) mbar_wait(&bar_ld2, ph[1]);
            mbar_wait(&bar_mma, ph_mma);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!s_fail) {
        // C[r, c] = 2^(ea + eb) sum_{d=2..9} block_d 2^(-7 d), each block an exact integer below 2^24;
        // the thread's own copy of the sink may keep running state, closed by done() (all lanes)
        Dst out = dst;
        const int r = mtile * 128 + wid * 32 + lane;
        const uint32_t lane_off = (uint32_t)(wid * 32) << 16;
        const int era = ea[r];
        for (int c0 = 0; c0 < OZ_NT; c0 += 8) {
            float blk[OZ_S][8];
#pragma unroll
            for (int d = 0; d < OZ_S; ++d) tmem_ld8(tbase + lane_off + (uint32_t)(d * OZ_NT + c0), blk[d]);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                float col[OZ_S];
#pragma unroll
                for (int d = 0; d < OZ_S; ++d) col[d] = blk[d][q];
                const double v = oz_combine(col);
                const int c = ntile * OZ_NT + c0 + q;
                out(r, c, scale2(v, era + eb[c]));
            }
        }
        out.done();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (wid == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kCols));
}

}  // namespace klst
