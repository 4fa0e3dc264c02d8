// A warp-specialised streaming pipeline for the float64-accurate tensor-core products: a CTA walks
// its units (velocity blocks of the block solves, row tiles of the Krylov basis), and every unit
// streams a few operand loads (integer slices of A) from HBM through shared memory into tcgen05
// MMAs against a small B operand that is split in the CTA.
//
//   warp 0, lane 0   producer: one bulk copy per load into a ring of stages
//   warp 1, lane 0   MMA issuer: waits for a stage, issues the unit's MMAs, frees the stage by
//                    tcgen05.commit; after a unit's last load it signals its TMEM accumulator
//   warps 2..5       B preparation for unit u + 1 (into the other B buffer), then the epilogue of
//                    unit u (TMEM -> registers -> global), so both overlap the MMAs and copies
//
// B buffers and TMEM accumulators are double buffered.  Every wait is bounded (mbar_wait): on a
// timeout the waiting thread sets ST_TIMEOUT and a shared failure flag that every role polls, the
// roles stop, and the producer waits once more for each copy still in flight before the CTA frees
// its TMEM and exits.
#pragma once
#include "oz.cuh"

namespace klst {

constexpr int kTsThreads = 192;  // six warps
constexpr int kTsEpi = 128;      // B preparation / epilogue threads (warps 2..5)

// named barrier 1 among the 128 preparation / epilogue threads
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Policy interface (all device functions, called by the roles named above):
//   int nunits() const                          units of this CTA, in MMA order
//   int nloads(int i) const                     loads of unit i
//   const void* src(int i, int l) const         global source of load l of unit i
//   uint32_t bytes(int i, int l) const          its size (multiple of 16, <= stage_bytes)
//   void mma(int i, int l, uint32_t a, uint32_t b, uint32_t tcol) const
//                                               the MMAs of load l (one thread), A at shared
//                                               address a, the B region at b (buffers at b_off),
//                                               accumulator at TMEM tcol
//   int b_wait_load(int i) const                the first load of unit i that reads its new B
//   int tbuf(int i), tuse(int i) const          unit i's TMEM accumulator (< NT) and how many
//                                               earlier units used it
//   bool needs_b(int i) const                   unit i waits for a freshly prepared B
//   int bbuf(int i), buse(int i) const          its B buffer (< NBB) and that buffer's earlier uses
//                                               (counting the units that prepare B only)
//   uint32_t tcol_off(int tb) const, int b_off(int bb) const   buffer placements
//   int first_prep(), prep_before(int i), prep_after(int i) const
//                                               the unit whose B the B/epilogue threads prepare
//                                               first, before the epilogue of unit i and after it
//                                               (-1: none); epilogues run in unit order
//   void prep(int i, unsigned char* sB, unsigned char* sX, int t)
//                                               B of unit i into sB (t = 0..127); sX is scratch
//   void epilogue(int i, uint32_t tcol, unsigned char* sX, int quarter, int lane)
//                                               TMEM lanes quarter*32 + lane of unit i (may keep
//                                               running sums in the thread's copy of the policy)
//   void finish(unsigned char* sX, int quarter, int lane) after the last epilogue
// and the constants stage_bytes, nstages, b_total, x_bytes, NT, NBB, tmem_alloc.
// The body of a kernel launched with kTsThreads threads and tcstream_smem<P>() bytes of dynamic
// shared memory; p is the thread's own copy of the policy.
template <class P>
__device__ __forceinline__ void tcstream_body(P& p, Status* st) {
    extern __shared__ __align__(128) unsigned char ts_smem[];
    constexpr int NS = P::nstages, NT = P::NT, NBB = P::NBB;
    __shared__ __align__(8) uint64_t full[NS], empty[NS], bfull[NBB], bempty[NBB], tfull[NT], tempty[NT];
    __shared__ uint32_t tmem_base;
    __shared__ volatile int s_fail;
    __shared__ int s_issued, s_consumed;
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    unsigned char* stages = ts_smem;
    unsigned char* sBase = ts_smem + NS * P::stage_bytes;
    unsigned char* sX = sBase + P::b_total;
    constexpr uint32_t kCols = P::tmem_alloc;
    if (tid == 0) {
        for (int q = 0; q < NS; ++q) { mbar_init(&full[q], 1); mbar_init(&empty[q], 1); }
        for (int b = 0; b < NBB; ++b) { mbar_init(&bfull[b], kTsEpi); mbar_init(&bempty[b], 1); }
        for (int b = 0; b < NT; ++b) { mbar_init(&tfull[b], 1); mbar_init(&tempty[b], kTsEpi); }
        s_fail = 0;
        s_issued = 0;
        s_consumed = 0;
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
    const int nu = p.nunits();
    auto fail = [&]() {
        if (!s_fail) {
            s_fail = 1;
            atomicOr(&st->flags, ST_TIMEOUT);
        }
    };
    if (wid == 0) {
        if (lane == 0) {
            // producer
            int q = 0;
            for (int i = 0; i < nu && !s_fail; ++i) {
                const int nl = p.nloads(i);
                for (int l = 0; l < nl && !s_fail; ++l, ++q) {
                    const int stg = q % NS, use = q / NS;
                    if (!mbar_wait(&empty[stg], (uint32_t)((use & 1) ^ 1))) { fail(); break; }
                    const uint32_t nb = p.bytes(i, l);
                    mbar_expect_tx(&full[stg], nb);
                    bulk_g2s(stages + stg * P::stage_bytes, p.src(i, l), nb, &full[stg]);
                    s_issued = q + 1;
                }
            }
        }
    } else if (wid == 1) {
        if (lane == 0) {
            // MMA issuer
            int q = 0;
            for (int i = 0; i < nu && !s_fail; ++i) {
                const int tb = p.tbuf(i), bb = p.bbuf(i);
                const bool nb = p.needs_b(i);
                const int bl = nb ? p.b_wait_load(i) : -1;
                if (!mbar_wait(&tempty[tb], (uint32_t)((p.tuse(i) & 1) ^ 1))) { fail(); break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t tcol = tbase + p.tcol_off(tb);
                const uint32_t bsm = smem_u32(sBase);
                const int nl = p.nloads(i);
                bool ok = true;
                for (int l = 0; l < nl; ++l, ++q) {
                    const int stg = q % NS, su = q / NS;
                    // the unit's new B is waited for only before the first load that reads it
                    if (l == bl && !mbar_wait(&bfull[bb], (uint32_t)(p.buse(i) & 1))) { ok = false; break; }
                    if (!mbar_wait(&full[stg], (uint32_t)(su & 1))) { ok = false; break; }
                    s_consumed = q + 1;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    p.mma(i, l, smem_u32(stages + stg * P::stage_bytes), bsm, tcol);
                    mma_commit(&empty[stg]);
                }
                if (!ok) { fail(); break; }
                mma_commit(&tfull[tb]);
                if (nb) mma_commit(&bempty[bb]);
            }
        }
    } else {
        // B preparation and epilogue (128 threads, TMEM lane quarter = warp % 4)
        const int t = tid - 64, quarter = wid & 3;
        auto prep_unit = [&](int i) {
            const int bb = p.bbuf(i);
            if (!mbar_wait(&bempty[bb], (uint32_t)((p.buse(i) & 1) ^ 1))) fail();
            epi_sync();
            if (s_fail) return;
            p.prep(i, sBase + p.b_off(bb), sX, t);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&bfull[bb]);
        };
        if (nu > 0 && p.first_prep() >= 0) prep_unit(p.first_prep());
        for (int i = 0; i < nu; ++i) {
            epi_sync();
            if (s_fail) break;
            const int pb = p.prep_before(i);
            if (pb >= 0) prep_unit(pb);
            const int tb = p.tbuf(i);
            if (!mbar_wait(&tfull[tb], (uint32_t)(p.tuse(i) & 1))) fail();
            epi_sync();
            if (s_fail) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            p.epilogue(i, tbase + p.tcol_off(tb), sX, quarter, lane);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(&tempty[tb]);
            const int pa = p.prep_after(i);
            if (pa >= 0) prep_unit(pa);
        }
        epi_sync();
        if (!s_fail) p.finish(sX, quarter, lane);
    }
    __syncthreads();
    if (s_fail && tid == 0) {
        // copies still in flight land, and the MMAs committed last complete, before the shared
        // memory and the TMEM are released
        for (int q = s_consumed; q < s_issued; ++q) mbar_wait(&full[q % NS], (uint32_t)((q / NS) & 1));
        if (s_consumed > 0) {
            const int q = s_consumed - 1;
            mbar_wait(&empty[q % NS], (uint32_t)((q / NS) & 1));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (wid == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kCols));
}

template <class P>
size_t tcstream_smem() { return (size_t)P::nstages * P::stage_bytes + (size_t)P::b_total + P::x_bytes; }

}  // namespace klst
