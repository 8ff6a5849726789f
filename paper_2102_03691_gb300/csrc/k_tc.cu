// K2: the modal projections on the 5th-generation tensor cores (sm_103a).
//
// For one block of K steps, with B-operand rows c = 4k + {0: sqrt(m) v, 1..3: W^{a.}/sqrt(m)},
//   R[n][c] = sum_d E[d][n] Bt[c][d]          (Eq. 13 for c = 4k, Eq. 16 bracket otherwise)
// is one dense GEMM of E^T (modes x D) with Bt^T (D x 4K).  Each 128-mode x BN-column tile
// accumulates in TMEM (FP32) from 16-bit hi/lo operands staged by TMA:
//   E B ~= E_hi B_hi + E_hi B_lo + E_lo B_hi        (three tcgen05.mma per 16-wide k slice)
// and the epilogue fuses the rest of the step: J_n^a(k) = R[n][4k] R[n][4k+1+a] (Eq. 16),
// then a segmented warp reduction over modes (stored sorted by frequency bin) leaves one
// partial sum per run of equal bins in each 32-mode group.
//
// Accumulation precision: the tensor core adds each MMA's products into the FP32
// accumulator with truncation, so its error grows linearly with the number of MMAs that
// feed one accumulator.  The d loop is therefore cut into chunks of PROMOTE_D = 128
// elements; each chunk accumulates into a fresh TMEM buffer (two buffers alternate) and
// the epilogue warps promote it into FP32 registers with round-to-nearest adds while the
// next chunk runs.  The per-tile sums never leave registers.  Because the chunk is fixed
// in elements, every pipeline shape (BK, STAGES) gives bitwise the same result.
//
// Warp roles (128 + BN threads, one persistent CTA per SM):
//   warp 0          TMA producer (one lane)
//   warp 1          MMA issuer (one lane)
//   warp 2          TMEM allocator
//   warps 4..4+BN/32  promotion + epilogue: warp w reads TMEM lanes 32*(w%4) .. +31 and
//                  the 128 columns starting at 128*((w-4)/4) of each chunk accumulator
// Every barrier wait is bounded; a wait that runs out raises a CTA-wide abort flag and a
// sticky device status, and the CTA drains its in-flight copies and MMAs, frees TMEM and exits.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace mhc {

namespace {

template <int BN, int BK, int STAGES>
struct TcLayout {
    static constexpr int A_BYTES = TC_BM * BK * 2;
    static constexpr int B_BYTES = BN * BK * 2;
    static constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
    static constexpr int TILE_BYTES = STAGES * STAGE_BYTES;
    static constexpr int BAR_BYTES = 256;
    static constexpr int SMEM_BYTES = TILE_BYTES + BAR_BYTES + 1024;   // + alignment slack
    static constexpr uint32_t TMEM_COLS = 2 * BN;   // two chunk accumulators
    static constexpr uint32_t SWIZZLE_CODE = BK == 64 ? 2u : 4u;        // 128 B or 64 B rows
    static constexpr uint32_t SBO = 8 * BK * 2;                         // 8-row core group
    static_assert(BK == 64 || BK == 32, "BK");
    static constexpr int EPI_WARPS = BN / 32;   // each holds 128 columns of 32 lanes
    static constexpr int THREADS = 128 + 32 * EPI_WARPS;
    static_assert(BN == 128 || BN == 256, "BN");
    static_assert(STAGES * 2 + 5 <= 28, "barrier area");
    static_assert(TMEM_COLS == 256 || TMEM_COLS == 512, "TMEM columns");
};

// A unit of work of a CTA (one-SM tiles) or CTA pair: tile (mt, ct) of problem `prob` over the
// k-blocks [kb_lo, kb_hi).  seg < 0: the whole d axis, so the kernel runs the tile epilogue;
// seg >= 0: a part of the d axis, whose promoted sums go to split_ws[seg] for the finish kernel.
struct Unit {
    int prob, mt, ct, kb_lo, kb_hi, seg;
};

// Balanced split: the tiles below sk_t0 (whole waves of the round-robin over all CTAs or pairs)
// run whole, round-robin; the tile-major chunk space of the remaining tiles (tile = mode tile *
// n_col_tiles + column tile, sk_nch promotion chunks each) is cut into sk_parts contiguous
// ranges of equal length (to one chunk), one for each of the first sk_parts CTAs (pairs): the
// last, partial wave is spread over all of them instead of leaving most idle.  Tail-local chunk
// g; part q starts at chunk floor(q T / sk_parts), T = the tail's chunks.
__device__ __forceinline__ long long sk_tail_chunks(const TcProblem &P) {
    return (long long)(P.n_tiles - P.sk_t0) * P.sk_nch;
}
__device__ __forceinline__ long long sk_begin(const TcProblem &P, int q) {
    return (long long)q * sk_tail_chunks(P) / P.sk_parts;
}
// The part whose range holds tail chunk g: the largest q with sk_begin(q) <= g.
__device__ __forceinline__ int sk_part_of(const TcProblem &P, long long g) {
    const long long T = sk_tail_chunks(P);
    return (int)(((g + 1) * P.sk_parts + T - 1) / T - 1);
}
// Segments of a tile under the balanced split (1: one part holds the whole tile).  Every tail
// part holds at least one chunk (sk_parts <= T), so the segments of a tail tile are the parts
// that touch it, in chunk order.
__device__ __forceinline__ int sk_segments(const TcProblem &P, int tile) {
    if (tile < P.sk_t0) return 1;
    const long long g0 = (long long)(tile - P.sk_t0) * P.sk_nch;
    return 1 + sk_part_of(P, g0 + P.sk_nch - 1) - sk_part_of(P, g0);
}

// The units of CTA (pair) `part` of `nparts`: a scheduled tile list (grouped launches), the
// balanced split's chunk range, or round-robin over the units of a single problem (tiles, or
// tile x range with the uniform split; the column tiles of one (mode tile, range) are
// adjacent, so the CTAs that share an E slice run side by side).  CHUNK_KB: k-blocks a chunk.
template <int NPROB, int CHUNK_KB>
struct UnitIter {
    const TcParams<NPROB> &p;
    int i = 0, end = 0, step = 1;
    long long g = 0, g_end = 0;
    __device__ UnitIter(const TcParams<NPROB> &pp, int part, int nparts) : p(pp) {
        if (p.sched) {
            i = p.cta_begin[part];
            end = p.cta_begin[part + 1];
        } else if (p.prob[0].sk_parts > 0) {
            i = part;                      // whole tiles first
            end = p.prob[0].sk_t0;
            step = nparts;
            if (part < p.prob[0].sk_parts) {   // then this part's range of the tail's chunks
                g = sk_begin(p.prob[0], part);
                g_end = sk_begin(p.prob[0], part + 1);
            }
        } else {
            i = part;
            end = p.prob[0].n_tiles;
            step = nparts;
        }
    }
    __device__ bool next(Unit &u) {
        const TcProblem &P = p.prob[0];
        if (!p.sched && P.sk_parts > 0) {
            if (i < end) {
                u.prob = 0;
                u.mt = i / P.n_col_tiles;
                u.ct = i - u.mt * P.n_col_tiles;
                u.kb_lo = 0;
                u.kb_hi = P.n_kb;
                u.seg = -1;
                i += step;
                return true;
            }
            if (g >= g_end) return false;
            const int tl = (int)(g / P.sk_nch), tile = P.sk_t0 + tl;
            const int c0 = (int)(g - (long long)tl * P.sk_nch);
            const int c1 = (int)min((long long)P.sk_nch, (long long)c0 + (g_end - g));
            u.prob = 0;
            u.mt = tile / P.n_col_tiles;
            u.ct = tile - u.mt * P.n_col_tiles;
            u.kb_lo = c0 * CHUNK_KB;
            u.kb_hi = min(P.n_kb, c1 * CHUNK_KB);
            u.seg = (c0 == 0 && c1 == P.sk_nch) ? -1 : sk_part_of(P, g) - sk_part_of(P, g - c0);
            g += c1 - c0;
            return true;
        }
        if (i >= end) return false;
        if (p.sched) {
            const uint32_t id = p.sched[i];
            u.prob = (int)(id >> 28);
            u.ct = (int)((id >> 20) & 0xFFu);
            u.mt = (int)(id & 0xFFFFFu);
            u.kb_lo = 0;
            u.kb_hi = p.prob[u.prob].n_kb;
            u.seg = -1;
        } else {
            const int S = P.n_split > 1 ? P.n_split : 1;
            const int per_mt = P.n_col_tiles * S;
            u.prob = 0;
            u.mt = i / per_mt;
            const int r = i - u.mt * per_mt;
            const int sp = r / P.n_col_tiles;
            u.ct = r - sp * P.n_col_tiles;
            u.kb_lo = S > 1 ? sp * P.kb_split : 0;
            u.kb_hi = S > 1 ? min(P.n_kb, u.kb_lo + P.kb_split) : P.n_kb;
            u.seg = S > 1 ? sp : -1;
        }
        i += step;
        return true;
    }
};

constexpr int PROMOTE_D = TC_PROMOTE_D;   // d elements per TMEM chunk accumulator

// A split unit's promoted sums (128 columns from col0 of mode n) to the split workspace
// split_ws[sp][col][mode]: each warp stores 128 contiguous bytes per column.
__device__ __forceinline__ void store_split(const float (&acc)[128], const TcProblem &P, int sp,
                                            int n, int col0) {
    float *dst = P.split_ws + ((size_t)sp * P.ws_cols + col0) * P.m_pad + n;
#pragma unroll
    for (int j = 0; j < 128; ++j) __stcg(dst + (size_t)j * P.m_pad, acc[j]);
}

// Direction-resolved split.  The d axis is stored direction-major (segment b holds the dofs
// 3i+b), so every chunk lies inside one segment.  The epilogue keeps Xdot (columns 4s)
// accumulating over all segments; at the end of segment b < 2 it parks the finished bracket
// sums Y^{a b} (columns 4s+1+a of its 32 steps: 96 values a thread) in a per-CTA scratch in
// global memory and restarts them from zero.  Scratch layout [CTA][segment][j][epilogue
// thread] (DIR_PARK_CTA_FLOATS a CTA): each warp stores and reloads 128 contiguous bytes per
// value, and each thread reads back only what it wrote itself (program order), so the
// ~200 KB a CTA holds stays in L2 and no barrier is needed.
__device__ __forceinline__ float *dir_park_base(const TcProblem &P) {
    return P.dir_park + (size_t)blockIdx.x * DIR_PARK_CTA_FLOATS + (threadIdx.x - 128);
}

__device__ __forceinline__ void park_y(float (&acc)[128], float *dst) {
#pragma unroll
    for (int j = 0; j < 96; ++j)   // j = 3 s + a
        __stcg(dst + j * DIR_PARK_THREADS, acc[4 * (j / 3) + 1 + j % 3]);
#pragma unroll
    for (int s = 0; s < 32; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) acc[4 * s + 1 + a] = 0.f;
}

__device__ __forceinline__ void unpark_y(float (&acc)[128], const float *src) {
#pragma unroll
    for (int j = 0; j < 96; ++j) acc[4 * (j / 3) + 1 + j % 3] = __ldcg(src + j * DIR_PARK_THREADS);
}

// After promoting the chunk that ends at k-block kn: park the finished direction segment.
__device__ __forceinline__ void dir_maybe_park(float (&acc)[128], const TcProblem &P, int kn) {
    if (P.dir_seg_kb && kn % P.dir_seg_kb == 0 && kn < P.n_kb)
        park_y(acc, dir_park_base(P) + (size_t)(kn / P.dir_seg_kb - 1) * DIR_PARK_SEG_FLOATS);
}

// Eq. 16 product and bin-run sums of one warp's NS steps kbase .. kbase+NS-1 (those < K), from
// the promoted sums in acc (columns 4s: Xdot, 4s+1+a: the bracket sums): the products
// overwrite the bracket columns, and each run tail stores its sums to
// partials[(k*3 + a) * row + col0 + slot].  `sc` holds lane l's four row scales of step
// kbase + l.  Written to be throughput-bound: the scales come by broadcast shuffles, and the
// 3 NS segmented scans advance level by level so that their shuffles overlap (each value still
// takes the same additions in the same order as a scan on its own, so any NS gives the same
// bits for a step).
template <int NS = 32>
__device__ __forceinline__ void epilogue_steps(float (&acc)[4 * NS], const float4 sc, const TcProblem &P,
                                               int kbase, uint32_t take, int slot, size_t row,
                                               size_t col0) {
#pragma unroll
    for (int s4 = 0; s4 < NS; ++s4) {
        const float x = acc[4 * s4] * __shfl_sync(FULL_MASK, sc.x, s4);
        acc[4 * s4 + 1] = x * (acc[4 * s4 + 1] * __shfl_sync(FULL_MASK, sc.y, s4));
        acc[4 * s4 + 2] = x * (acc[4 * s4 + 2] * __shfl_sync(FULL_MASK, sc.z, s4));
        acc[4 * s4 + 3] = x * (acc[4 * s4 + 3] * __shfl_sync(FULL_MASK, sc.w, s4));
    }
#pragma unroll
    for (int r = 0; r < 5; ++r) {
        const bool add = (take >> r) & 1u;
#pragma unroll
        for (int j = 0; j < 3 * NS; ++j) {
            const int c = 4 * (j / 3) + 1 + j % 3;
            const float o = __shfl_up_sync(FULL_MASK, acc[c], 1u << r);
            if (add) acc[c] += o;
        }
    }
    if (slot < 0) return;
    const int nk = P.K - kbase;   // steps of this warp inside the block
#pragma unroll
    for (int s4 = 0; s4 < NS; ++s4) {
        if (s4 >= nk) break;
        float *dst = P.partials + ((size_t)(kbase + s4) * 3) * row + col0 + (size_t)slot;
        dst[0] = acc[4 * s4 + 1];
        dst[row] = acc[4 * s4 + 2];
        dst[2 * row] = acc[4 * s4 + 3];
    }
}

// Lane l's four row scales of step kbase + l (zero past the block).
__device__ __forceinline__ float4 step_scales(const TcProblem &P, int kbase, int lane) {
    if (kbase + lane >= P.K) return make_float4(0.f, 0.f, 0.f, 0.f);
    return __ldg(reinterpret_cast<const float4 *>(P.col_scale) + (kbase + lane));
}

// The epilogue of one warp's 32 steps: plain, or the direction-resolved split
// J_n^{ab}(k) = Xdot_n(k) Y_n^{ab}(k) (direction 2 from the registers, directions 1 and 0
// from their parked sums) into the slot columns b n_slots + slot of rows of 3 n_slots.
template <bool DIR>
__device__ __forceinline__ void tile_epilogue(float (&acc)[128], const TcProblem &P, int kbase,
                                              uint32_t take, int slot, int lane) {
    const float4 sc = step_scales(P, kbase, lane);
    if constexpr (!DIR) {
        epilogue_steps(acc, sc, P, kbase, take, slot, (size_t)P.n_slots, 0);
    } else {
        const size_t row = 3 * (size_t)P.n_slots;
        for (int b = 2; b >= 0; --b) {
            if (b < 2) unpark_y(acc, dir_park_base(P) + (size_t)b * DIR_PARK_SEG_FLOATS);
            epilogue_steps(acc, sc, P, kbase, take, slot, row, (size_t)b * P.n_slots);
        }
    }
}

// DIR: the direction-resolved epilogue (single problems only); the plain kernels keep their own
// register allocation.
template <int BN, int BK, int STAGES, int NPROB, bool DIR>
__global__ void __launch_bounds__(128 + BN, 1) tc_modal_kernel(const __grid_constant__ TcParams<NPROB> p) {
    using L = TcLayout<BN, BK, STAGES>;
    constexpr int CHUNK_KB = PROMOTE_D / BK;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                ~uintptr_t(1023));
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L::TILE_BYTES);
    uint64_t *full = bars;                   // [STAGES] TMA landed
    uint64_t *empty = bars + STAGES;         // [STAGES] MMAs done reading
    uint64_t *acc_full = bars + 2 * STAGES;  // [2] chunk accumulator ready
    uint64_t *acc_empty = acc_full + 2;      // [2] chunk accumulator promoted
    uint64_t *done_bar = acc_empty + 2;      // final MMA drain
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done_bar + 1);
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    griddep_launch_dependents();   // the next kernel may take the SMs this grid leaves

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 32 * L::EPI_WARPS);
        }
        mbar_init(done_bar, 1);
        *abort = 0;
        fence_mbar_init();
    }
    if (warp == 2) {
        tmem_alloc(tmem_slot, L::TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    griddep_wait();   // the pack's rows and scales (set-up above overlapped its end)

    if (warp == 0 && lane == 0) {
        // ------------------------------------------------------------ TMA producer
        for (int q = 0; q < NPROB && q < p.n_prob; ++q) {
            tma_prefetch_desc(&p.prob[q].tmA_hi);
            tma_prefetch_desc(&p.prob[q].tmA_lo);
            tma_prefetch_desc(&p.prob[q].tmB_hi);
            tma_prefetch_desc(&p.prob[q].tmB_lo);
        }
        const uint64_t pol_b = l2_policy_evict_last();
        const uint64_t pol_e = l2_policy_evict_normal();   // E tiles are shared by the CTAs of other column tiles
        uint32_t issued_phase[STAGES];
        bool issued[STAGES];
        for (int s = 0; s < STAGES; ++s) issued[s] = false;
        int stage = 0;
        uint32_t phase = 0;
        UnitIter<NPROB, CHUNK_KB> it(p, blockIdx.x, gridDim.x);
        Unit u;
        bool ok = true;
        while (ok && it.next(u)) {
            const TcProblem &P = p.prob[u.prob];
            const int mt = u.mt, ct = u.ct, kb_lo = u.kb_lo, kb_hi = u.kb_hi;
            for (int kb = kb_lo; kb < kb_hi; ++kb) {
                if (!mbar_wait(&empty[stage], phase ^ 1u, abort, p.wait_limit)) { ok = false; break; }
                uint8_t *sa = smem + stage * L::STAGE_BYTES;
                // test hook: 16 bytes more than the copies deliver keeps the barrier pending
                mbar_arrive_expect_tx(&full[stage], L::STAGE_BYTES + (p.stall_inject && kb == 0 ? 16 : 0));
                const int x = kb * BK;
                tma_load_2d(sa, &P.tmA_hi, &full[stage], x, mt * TC_BM, pol_e);
                tma_load_2d(sa + L::A_BYTES, &P.tmA_lo, &full[stage], x, mt * TC_BM, pol_e);
                tma_load_2d(sa + 2 * L::A_BYTES, &P.tmB_hi, &full[stage], x, ct * BN, pol_b);
                tma_load_2d(sa + 2 * L::A_BYTES + L::B_BYTES, &P.tmB_lo, &full[stage], x, ct * BN, pol_b);
                issued[stage] = true;
                issued_phase[stage] = phase;
                if (++stage == STAGES) { stage = 0; phase ^= 1u; }
            }
        }
        if (!ok) {
            *abort = 1;
            set_status(p.status, DEV_TIMEOUT);
        }
        // Drain: every copy this CTA issued must have landed before the CTA may exit.
        for (int s = 0; s < STAGES; ++s)
            if (issued[s]) {
                const long long t0 = clock64();
                while (!mbar_try_wait(&full[s], issued_phase[s]) &&
                       clock64() - t0 < p.wait_limit) {
                }
            }
    } else if (warp == 1 && lane == 0) {
        // ------------------------------------------------------------ MMA issuer
        const uint32_t idesc = p.idesc;
        int stage = 0, abuf = 0;
        uint32_t phase = 0, aphase = 0;
        UnitIter<NPROB, CHUNK_KB> it(p, blockIdx.x, gridDim.x);
        Unit u;
        bool ok = true;
        const uint32_t smem0 = smem_u32(smem);
        while (ok && it.next(u)) {
            const TcProblem &P = p.prob[u.prob];
            const int kb_lo = u.kb_lo, kb_hi = u.kb_hi;
            for (int kb0 = kb_lo; ok && kb0 < kb_hi; kb0 += CHUNK_KB) {
                if (!mbar_wait(&acc_empty[abuf], aphase ^ 1u, abort, p.wait_limit)) { ok = false; break; }
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(abuf * BN);
                const int kb1 = min(kb0 + CHUNK_KB, kb_hi);
                for (int kb = kb0; kb < kb1; ++kb) {
                    if (!mbar_wait(&full[stage], phase, abort, p.wait_limit)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t a_hi = smem0 + stage * L::STAGE_BYTES;
                    const uint32_t a_lo = a_hi + L::A_BYTES;
                    const uint32_t b_hi = a_hi + 2 * L::A_BYTES;
                    const uint32_t b_lo = b_hi + L::B_BYTES;
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {
                        const uint32_t off = kk * 32;   // 16 elements of 2 bytes
                        const uint64_t dah = smem_desc_kmajor(a_hi + off, L::SBO, L::SWIZZLE_CODE);
                        const uint64_t dal = smem_desc_kmajor(a_lo + off, L::SBO, L::SWIZZLE_CODE);
                        const uint64_t dbh = smem_desc_kmajor(b_hi + off, L::SBO, L::SWIZZLE_CODE);
                        const uint64_t dbl = smem_desc_kmajor(b_lo + off, L::SBO, L::SWIZZLE_CODE);
                        // small cross terms first, the dominant hi*hi product last
                        umma_f16(d_tmem, dah, dbl, idesc, (kb != kb0 || kk != 0) ? 1u : 0u);
                        umma_f16(d_tmem, dal, dbh, idesc, 1u);
                        umma_f16(d_tmem, dah, dbh, idesc, 1u);
                    }
                    umma_commit(&empty[stage]);
                    if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                }
                if (!ok) break;
                umma_commit(&acc_full[abuf]);
                if (++abuf == 2) { abuf = 0; aphase ^= 1u; }
            }
        }
        if (!ok) {
            *abort = 1;
            set_status(p.status, DEV_TIMEOUT);
        }
        // Drain: all MMAs issued by this thread complete before TMEM is released.
        umma_commit(done_bar);
        const long long t0 = clock64();
        while (!mbar_try_wait(done_bar, 0) && clock64() - t0 < p.wait_limit) {
        }
    } else if (warp >= 4) {
        // ------------------------------------------------------------ promotion + epilogue
        const int qw = warp & 3;          // TMEM lane quarter of this warp
        const int ch = (warp - 4) >> 2;   // which 128-column half of the tile
        int abuf = 0;
        uint32_t aphase = 0;
        UnitIter<NPROB, CHUNK_KB> it(p, blockIdx.x, gridDim.x);
        Unit u;
        bool ok = true;
        while (ok && it.next(u)) {
            const TcProblem &P = p.prob[u.prob];
            const int mt = u.mt, ct = u.ct, kb_lo = u.kb_lo, kb_hi = u.kb_hi;
            const int n = mt * TC_BM + qw * 32 + lane;
            const int bin = P.mode_bin[n];
            const int slot = P.mode_slot[n];
            const uint32_t take = seg_scan_masks(bin, lane);
            float acc[128];
#pragma unroll
            for (int j = 0; j < 128; ++j) acc[j] = 0.f;
            // promotion of every chunk accumulator into FP32 registers
            for (int kb0 = kb_lo; kb0 < kb_hi; kb0 += CHUNK_KB) {
                if (!mbar_wait(&acc_full[abuf], aphase, abort, p.wait_limit)) { ok = false; break; }
                tc_fence_after();
                const uint32_t tbase = tmem_base + ((uint32_t)(qw * 32) << 16) +
                                       (uint32_t)(abuf * BN + ch * 128);
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    uint32_t r[16];
                    tmem_ld_32x32b_x16(tbase + (uint32_t)(c * 16), r);
                    tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < 16; ++j) acc[c * 16 + j] += __uint_as_float(r[j]);
                }
                tc_fence_before();
                mbar_arrive(&acc_empty[abuf]);
                if (++abuf == 2) { abuf = 0; aphase ^= 1u; }
                if constexpr (DIR) dir_maybe_park(acc, P, kb0 + CHUNK_KB);
            }
            if (!ok) break;
            if (u.seg >= 0) {   // the split finish kernel adds the segments and runs the epilogue
                store_split(acc, P, u.seg, n, ct * BN + ch * 128);
                continue;
            }
            // Eq. 16 product and the bin-run sums of this warp's 32 steps
            const int kbase = ct * (BN / 4) + ch * 32;
            tile_epilogue<DIR>(acc, P, kbase, take, slot, lane);
        }
        if (!ok) {
            *abort = 1;
            set_status(p.status, DEV_TIMEOUT);
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 2) tmem_dealloc(tmem_base, L::TMEM_COLS);
}

// =====================================================================================
// CTA-pair variant (tcgen05 cta_group::2).  A cluster of two CTAs on two SMs computes a
// 256-mode x BN-column tile (BN = 256 or 128): each CTA stages its own 128 modes of E and
// its own half (BN/2 columns) of B, the leader CTA (rank 0) issues M=256 MMAs that read both
// CTAs' shared memory, and each CTA's TMEM receives the accumulator of its own 128 modes
// (all BN columns).  Per SM this halves the B bytes per flop against the one-SM tile of the
// same width (BN = 256: 64 KB instead of 96 KB per 64-wide k-block at the same tensor work).
//   - TMA loads of both CTAs complete on the leader's `full` barrier (armed by the
//     leader with both CTAs' bytes);
//   - the leader's commits arrive on `empty`/`acc_full` of both CTAs (multicast);
//   - each epilogue warp of both CTAs arrives on the leader's `acc_empty` after
//     promoting a chunk.
template <int BN_, int BK, int STAGES>
struct TcPairLayout {
    static constexpr int BN = BN_;
    static constexpr int A_BYTES = TC_BM * BK * 2;
    static constexpr int B_BYTES = (BN / 2) * BK * 2;
    static constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
    static constexpr int TILE_BYTES = STAGES * STAGE_BYTES;
    static constexpr int SMEM_BYTES = TILE_BYTES + 256 + 1024;
    static constexpr uint32_t TMEM_COLS = 2 * BN;   // two chunk accumulators of this CTA's modes
    static constexpr uint32_t SWIZZLE_CODE = BK == 64 ? 2u : 4u;
    static constexpr uint32_t SBO = 8 * BK * 2;
    static constexpr int EPI_WARPS = BN / 32;
    static_assert(BN == 128 || BN == 256, "BN");
    static constexpr int THREADS = 128 + 32 * EPI_WARPS;
    static_assert(STAGES * 2 + 5 <= 28, "barrier area");
};

template <int BN, int BK, int STAGES, int NPROB, bool DIR>
__global__ void __launch_bounds__(128 + BN, 1) tc_modal_pair_kernel(const __grid_constant__ TcParams<NPROB> p) {
    using L = TcPairLayout<BN, BK, STAGES>;
    constexpr int CHUNK_KB = PROMOTE_D / BK;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                ~uintptr_t(1023));
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L::TILE_BYTES);
    uint64_t *full = bars;                   // [STAGES] leader: both CTAs' TMA bytes landed
    uint64_t *empty = bars + STAGES;         // [STAGES] this CTA's stage free again
    uint64_t *acc_full = bars + 2 * STAGES;  // [2] chunk accumulator ready (both CTAs)
    uint64_t *acc_empty = acc_full + 2;      // [2] leader: chunk promoted by both CTAs
    uint64_t *done_bar = acc_empty + 2;      // leader: final MMA drain
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done_bar + 1);
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_ctarank();
    const bool leader = rank == 0;
    griddep_launch_dependents();   // the next kernel may take the SMs this grid leaves
    const int pair = (int)cluster_id_x(), npairs = (int)nclusters_x();

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 2 * L::EPI_WARPS);
        }
        mbar_init(done_bar, 1);
        *abort = 0;
        fence_mbar_init();
    }
    if (warp == 2) {
        tmem_alloc_pair(tmem_slot, L::TMEM_COLS);
        tmem_relinquish_pair();
    }
    tc_fence_before();
    __syncwarp();
    cluster_sync_all();   // barriers of both CTAs initialised, TMEM allocated in both
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    griddep_wait();   // the pack's rows and scales (set-up above overlapped its end)

    if (warp == 0 && lane == 0) {
        // ------------------------------------------------------------ TMA producer (both CTAs)
        for (int q = 0; q < NPROB && q < p.n_prob; ++q) {
            tma_prefetch_desc(&p.prob[q].tmA_hi);
            tma_prefetch_desc(&p.prob[q].tmA_lo);
            tma_prefetch_desc(&p.prob[q].tmB_hi);
            tma_prefetch_desc(&p.prob[q].tmB_lo);
        }
        const uint64_t pol_b = l2_policy_evict_last();
        const uint64_t pol_e = l2_policy_evict_normal();   // E tiles are shared by the CTAs of other column tiles
        uint32_t issued_phase[STAGES];
        bool issued[STAGES];
        for (int s = 0; s < STAGES; ++s) issued[s] = false;
        int stage = 0;
        uint32_t phase = 0;
        UnitIter<NPROB, CHUNK_KB> it(p, pair, npairs);
        Unit u;
        bool ok = true;
        while (ok && it.next(u)) {
            const TcProblem &P = p.prob[u.prob];
            const int arow = u.mt * 2 * TC_BM + (int)rank * TC_BM;
            const int brow = u.ct * BN + (int)rank * (BN / 2);
            const int kb_lo = u.kb_lo, kb_hi = u.kb_hi;
            for (int kb = kb_lo; kb < kb_hi; ++kb) {
                if (!mbar_wait(&empty[stage], phase ^ 1u, abort, p.wait_limit)) { ok = false; break; }
                if (leader)   // test hook as in the one-SM kernel
                    mbar_arrive_expect_tx(&full[stage], 2 * L::STAGE_BYTES + (p.stall_inject && kb == 0 ? 16 : 0));
                const uint32_t fb = mapa_shared(smem_u32(&full[stage]), 0);
                uint8_t *sa = smem + stage * L::STAGE_BYTES;
                const int x = kb * BK;
                tma_load_2d_pair(sa, &P.tmA_hi, fb, x, arow, pol_e);
                tma_load_2d_pair(sa + L::A_BYTES, &P.tmA_lo, fb, x, arow, pol_e);
                tma_load_2d_pair(sa + 2 * L::A_BYTES, &P.tmB_hi, fb, x, brow, pol_b);
                tma_load_2d_pair(sa + 2 * L::A_BYTES + L::B_BYTES, &P.tmB_lo, fb, x, brow, pol_b);
                issued[stage] = true;
                issued_phase[stage] = phase;
                if (++stage == STAGES) { stage = 0; phase ^= 1u; }
            }
        }
        if (!ok) {
            *abort = 1;
            set_status(p.status, DEV_TIMEOUT);
        }
        if (leader)   // the leader's barriers count both CTAs' copies
            for (int s = 0; s < STAGES; ++s)
                if (issued[s]) {
                    const long long t0 = clock64();
                    while (!mbar_try_wait(&full[s], issued_phase[s]) &&
                           clock64() - t0 < p.wait_limit) {
                    }
                }
    } else if (warp == 1 && lane == 0 && leader) {
        // ------------------------------------------------------------ MMA issuer (leader)
        const uint32_t idesc = p.idesc;
        int stage = 0, abuf = 0;
        uint32_t phase = 0, aphase = 0;
        UnitIter<NPROB, CHUNK_KB> it(p, pair, npairs);
        Unit u;
        bool ok = true;
        const uint32_t smem0 = smem_u32(smem);
        while (ok && it.next(u)) {
            const int kb_lo = u.kb_lo, kb_hi = u.kb_hi;
            for (int kb0 = kb_lo; ok && kb0 < kb_hi; kb0 += CHUNK_KB) {
                if (!mbar_wait(&acc_empty[abuf], aphase ^ 1u, abort, p.wait_limit)) { ok = false; break; }
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(abuf * BN);
                const int kb1 = min(kb0 + CHUNK_KB, kb_hi);
                for (int kb = kb0; kb < kb1; ++kb) {
                    if (!mbar_wait(&full[stage], phase, abort, p.wait_limit)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t a_hi = smem0 + stage * L::STAGE_BYTES;
                    const uint32_t a_lo = a_hi + L::A_BYTES;
                    const uint32_t b_hi = a_hi + 2 * L::A_BYTES;
                    const uint32_t b_lo = b_hi + L::B_BYTES;
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {
                        const uint32_t off = kk * 32;
                        const uint64_t dah = smem_desc_kmajor(a_hi + off, L::SBO, L::SWIZZLE_CODE);
                        const uint64_t dal = smem_desc_kmajor(a_lo + off, L::SBO, L::SWIZZLE_CODE);
                        const uint64_t dbh = smem_desc_kmajor(b_hi + off, L::SBO, L::SWIZZLE_CODE);
                        const uint64_t dbl = smem_desc_kmajor(b_lo + off, L::SBO, L::SWIZZLE_CODE);
                        umma_f16_pair(d_tmem, dah, dbl, idesc, (kb != kb0 || kk != 0) ? 1u : 0u);
                        umma_f16_pair(d_tmem, dal, dbh, idesc, 1u);
                        umma_f16_pair(d_tmem, dah, dbh, idesc, 1u);
                    }
                    umma_commit_pair(&empty[stage], (uint16_t)0x3);
                    if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                }
                if (!ok) break;
                umma_commit_pair(&acc_full[abuf], (uint16_t)0x3);
                if (++abuf == 2) { abuf = 0; aphase ^= 1u; }
            }
        }
        if (!ok) {
            *abort = 1;
            set_status(p.status, DEV_TIMEOUT);
        }
        umma_commit_pair(done_bar, (uint16_t)0x1);
        const long long t0 = clock64();
        while (!mbar_try_wait(done_bar, 0) && clock64() - t0 < p.wait_limit) {
        }
    } else if (warp >= 4) {
        // ------------------------------------------------------------ promotion + epilogue (both)
        const int qw = warp & 3;
        const int ch = (warp - 4) >> 2;
        int abuf = 0;
        uint32_t aphase = 0;
        const uint32_t empty_leader[2] = {mapa_shared(smem_u32(&acc_empty[0]), 0),
                                          mapa_shared(smem_u32(&acc_empty[1]), 0)};
        UnitIter<NPROB, CHUNK_KB> it(p, pair, npairs);
        Unit u;
        bool ok = true;
        while (ok && it.next(u)) {
            const TcProblem &P = p.prob[u.prob];
            const int mp = u.mt, ct = u.ct, kb_lo = u.kb_lo, kb_hi = u.kb_hi;
            const int n = mp * 2 * TC_BM + (int)rank * TC_BM + qw * 32 + lane;
            const int bin = P.mode_bin[n];
            const int slot = P.mode_slot[n];
            const uint32_t take = seg_scan_masks(bin, lane);
            float acc[128];
#pragma unroll
            for (int j = 0; j < 128; ++j) acc[j] = 0.f;
            for (int kb0 = kb_lo; kb0 < kb_hi; kb0 += CHUNK_KB) {
                if (!mbar_wait(&acc_full[abuf], aphase, abort, p.wait_limit)) { ok = false; break; }
                tc_fence_after();
                const uint32_t tbase = tmem_base + ((uint32_t)(qw * 32) << 16) +
                                       (uint32_t)(abuf * BN + ch * 128);
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    uint32_t r[16];
                    tmem_ld_32x32b_x16(tbase + (uint32_t)(c * 16), r);
                    tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < 16; ++j) acc[c * 16 + j] += __uint_as_float(r[j]);
                }
                tc_fence_before();
                __syncwarp();
                // the chunk's TMEM reads have completed (wait::ld): the leader may reuse it
                if (lane == 0) {
                    if (leader) mbar_arrive(&acc_empty[abuf]);
                    else mbar_arrive_cluster_relaxed(empty_leader[abuf]);
                }
                if (++abuf == 2) { abuf = 0; aphase ^= 1u; }
                if constexpr (DIR) dir_maybe_park(acc, P, kb0 + CHUNK_KB);
            }
            if (!ok) break;
            if (u.seg >= 0) {   // the split finish kernel adds the segments and runs the epilogue
                store_split(acc, P, u.seg, n, ct * BN + ch * 128);
                continue;
            }
            const int kbase = ct * (BN / 4) + ch * 32;
            tile_epilogue<DIR>(acc, P, kbase, take, slot, lane);
        }
        if (!ok) {
            *abort = 1;
            set_status(p.status, DEV_TIMEOUT);
        }
    }

    tc_fence_before();
    __syncwarp();
    cluster_sync_all();   // neither CTA leaves while the pair still shares barriers or TMEM
    tc_fence_after();
    if (warp == 2) tmem_dealloc_pair(tmem_base, L::TMEM_COLS);
}

template <int BN, int BK, int STAGES, int NPROB, bool DIR>
cudaError_t launch_pair_impl(const TcParams<NPROB> &p, int grid, cudaStream_t s, bool pdl) {
    using L = TcPairLayout<BN, BK, STAGES>;
    auto kern = tc_modal_pair_kernel<BN, BK, STAGES, NPROB, DIR>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             L::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    cfg.blockDim = dim3(L::THREADS, 1, 1);
    cfg.dynamicSmemBytes = L::SMEM_BYTES;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;   // after the pack
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, kern, p);
}

template <int BN, int BK, int STAGES, int NPROB>
int max_pairs_impl() {
    using L = TcPairLayout<BN, BK, STAGES>;
    auto kern = tc_modal_pair_kernel<BN, BK, STAGES, NPROB, false>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L::SMEM_BYTES) !=
        cudaSuccess)
        return 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2, 1, 1);
    cfg.blockDim = dim3(L::THREADS, 1, 1);
    cfg.dynamicSmemBytes = L::SMEM_BYTES;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

template <int BN, int BK, int STAGES, int NPROB, bool DIR>
cudaError_t launch_impl(const TcParams<NPROB> &p, int grid, cudaStream_t s, bool pdl) {
    using L = TcLayout<BN, BK, STAGES>;
    auto kern = tc_modal_kernel<BN, BK, STAGES, NPROB, DIR>;
    static bool attr_set = false;   // per process; the attribute is per function
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             L::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    cfg.blockDim = dim3(L::THREADS, 1, 1);
    cfg.dynamicSmemBytes = L::SMEM_BYTES;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;   // after the pack
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, p);
}

template <int NPROB, bool DIR>
cudaError_t dispatch(const TcParams<NPROB> &p, const TcConfig &c, cudaStream_t s, bool pdl) {
    if (c.pair) {
        if (c.bn == 256 && c.bk == 64 && c.stages == 3) return launch_pair_impl<256, 64, 3, NPROB, DIR>(p, c.grid, s, pdl);
        if (c.bn == 256 && c.bk == 32 && c.stages == 6) return launch_pair_impl<256, 32, 6, NPROB, DIR>(p, c.grid, s, pdl);
        if (c.bn == 128 && c.bk == 64 && c.stages == 4) return launch_pair_impl<128, 64, 4, NPROB, DIR>(p, c.grid, s, pdl);
        if (c.bn == 128 && c.bk == 32 && c.stages == 8) return launch_pair_impl<128, 32, 8, NPROB, DIR>(p, c.grid, s, pdl);
        return cudaErrorInvalidValue;
    }
    if (c.bn == 256 && c.bk == 64 && c.stages == 2) return launch_impl<256, 64, 2, NPROB, DIR>(p, c.grid, s, pdl);
    if (c.bn == 256 && c.bk == 32 && c.stages == 4) return launch_impl<256, 32, 4, NPROB, DIR>(p, c.grid, s, pdl);
    if (c.bn == 128 && c.bk == 64 && c.stages == 3) return launch_impl<128, 64, 3, NPROB, DIR>(p, c.grid, s, pdl);
    if (c.bn == 128 && c.bk == 32 && c.stages == 6) return launch_impl<128, 32, 6, NPROB, DIR>(p, c.grid, s, pdl);
    return cudaErrorInvalidValue;
}

// Split finish: one warp per (32 modes, 8 steps), lane = mode.  Adds a tile's segments (the
// uniform split's ranges, or the balanced split's parts that cut it) in order and runs the
// fused kernel's epilogue on the sums; under the balanced split, warps of tiles that one part
// held whole return at once (the projection kernel ran their epilogue).  The segments come
// into shared memory by 16-byte asynchronous copies, FIN_SEGS at a time (up to 16 KB a warp
// in flight without holding registers), and each lane then reads its own mode's values.
constexpr int FIN_STEPS = 8;
constexpr int FIN_SEGS = 4;
constexpr int FIN_COLS = 4 * FIN_STEPS;                          // columns of a warp
constexpr int FIN_SMEM = 4 * FIN_SEGS * FIN_COLS * 32 * 4;       // 4 warps, 64 KB
__global__ void __launch_bounds__(128) tc_split_finish_kernel(const __grid_constant__ TcParams<1> p) {
    extern __shared__ float4 fin_smem4[];
    griddep_launch_dependents();
    griddep_wait();   // the projection's stored segments
    const TcProblem &P = p.prob[0];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x * 4 + warp;   // 32-mode group (warp-uniform)
    if (g * 32 >= P.m_pad) return;
    const int n0 = g * 32;
    const int kbase = blockIdx.y * FIN_STEPS;
    const int c0 = kbase * 4;              // first of the warp's columns
    int nseg = P.n_split;
    if (P.sk_parts > 0) {
        nseg = sk_segments(P, (n0 / P.sk_tm) * P.n_col_tiles + c0 / P.sk_bn);
        if (nseg < 2) return;
    }
    const int bin = P.mode_bin[n0 + lane];
    const int slot = P.mode_slot[n0 + lane];
    const uint32_t take = seg_scan_masks(bin, lane);
    float *st = reinterpret_cast<float *>(fin_smem4) + (size_t)warp * FIN_SEGS * FIN_COLS * 32;
    const size_t sstride = (size_t)P.ws_cols * P.m_pad;
    const float *src = P.split_ws + (size_t)c0 * P.m_pad + n0;
    float acc[FIN_COLS];
#pragma unroll
    for (int j = 0; j < FIN_COLS; ++j) acc[j] = 0.f;
    for (int s0 = 0; s0 < nseg; s0 += FIN_SEGS) {
        const int ns = min(FIN_SEGS, nseg - s0);
        // segment s, column j: 32 modes = 128 contiguous bytes, eight 16-byte copies
        for (int q = lane; q < ns * FIN_COLS * 8; q += 32) {
            const int s = q / (FIN_COLS * 8), r = q - s * (FIN_COLS * 8), j = r >> 3, part = r & 7;
            cp_async16(st + (s * FIN_COLS + j) * 32 + part * 4,
                       src + (size_t)(s0 + s) * sstride + (size_t)j * P.m_pad + part * 4);
        }
        cp_async_wait_all();
        __syncwarp();
        for (int s = 0; s < ns; ++s)   // segment order
#pragma unroll
            for (int j = 0; j < FIN_COLS; ++j) acc[j] += st[(s * FIN_COLS + j) * 32 + lane];
        __syncwarp();                  // the staging area is refilled by the next batch
    }
    epilogue_steps<FIN_STEPS>(acc, step_scales(P, kbase, lane), P, kbase, take, slot,
                              (size_t)P.n_slots, 0);
}

}  // namespace

cudaError_t launch_tc_split_finish(const TcParams<1> &p, cudaStream_t s) {
    const TcProblem &P = p.prob[0];
    if ((P.n_split <= 1 && P.sk_parts <= 0) || !P.split_ws || P.m_pad % 128 || P.ws_cols % FIN_COLS)
        return cudaErrorInvalidValue;
    static const cudaError_t smem_ok = cudaFuncSetAttribute(
        tc_split_finish_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, FIN_SMEM);
    if (smem_ok != cudaSuccess) return smem_ok;
    const dim3 grid((unsigned)(P.m_pad / 128), (unsigned)((P.K + FIN_STEPS - 1) / FIN_STEPS));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(128, 1, 1);
    cfg.dynamicSmemBytes = FIN_SMEM;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;   // after the projection
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, tc_split_finish_kernel, p);
}

const TcConfig TC_CONFIGS[TC_NUM_CONFIGS] = {
    {256, 64, 2, 0, 0}, {256, 32, 4, 0, 0}, {128, 64, 3, 0, 0}, {128, 32, 6, 0, 0},
    {256, 64, 3, 1, 0}, {256, 32, 6, 1, 0}, {128, 64, 4, 1, 0}, {128, 32, 8, 1, 0}};

bool tc_config_supported(const TcConfig &c) {
    for (const TcConfig &k : TC_CONFIGS)
        if (k.bn == c.bn && k.bk == c.bk && k.stages == c.stages && k.pair == c.pair) return true;
    return false;
}

int tc_max_pairs(const TcConfig &c) {
    if (!c.pair) return 0;
    if (c.bn == 256) return c.bk == 64 ? max_pairs_impl<256, 64, 3, 1>() : max_pairs_impl<256, 32, 6, 1>();
    return c.bk == 64 ? max_pairs_impl<128, 64, 4, 1>() : max_pairs_impl<128, 32, 8, 1>();
}

size_t tc_smem_bytes(const TcConfig &c) {   // must match TcLayout / TcPairLayout::SMEM_BYTES
    const int brows = c.pair ? c.bn / 2 : c.bn;
    return (size_t)c.stages * (2 * TC_BM * c.bk * 2 + 2 * brows * c.bk * 2) + 256 + 1024;
}

cudaError_t launch_tc_single(const TcParams<1> &p, const TcConfig &c, cudaStream_t s) {
    const TcProblem &P = p.prob[0];
    if (P.n_split > 1 && (P.dir_seg_kb || !P.split_ws || P.sk_parts > 0 ||
                          P.kb_split % (PROMOTE_D / c.bk)))
        return cudaErrorInvalidValue;
    const int parts = c.grid / (c.pair ? 2 : 1);
    if (P.sk_parts > 0 && (P.dir_seg_kb || !P.split_ws || P.sk_bn != c.bn ||
                           P.sk_nch != (P.n_kb + PROMOTE_D / c.bk - 1) / (PROMOTE_D / c.bk) ||
                           P.sk_tm != (c.pair ? 2 : 1) * TC_BM || P.sk_t0 < 0 ||
                           P.sk_t0 % parts || P.sk_t0 >= P.n_tiles || P.sk_parts > parts ||
                           (long long)P.sk_parts > (long long)(P.n_tiles - P.sk_t0) * P.sk_nch))
        return cudaErrorInvalidValue;
    if (p.prob[0].dir_seg_kb) {
        if (!p.prob[0].dir_park || c.grid > p.dir_park_ctas) return cudaErrorInvalidValue;
        return dispatch<1, true>(p, c, s, true);
    }
    return dispatch<1, false>(p, c, s, true);
}
cudaError_t launch_tc_group(const TcParams<TC_MAX_GROUP> &p, const TcConfig &c, cudaStream_t s) {
    for (int q = 0; q < p.n_prob; ++q)   // direction and d-axis splits run on single problems only
        if (p.prob[q].dir_seg_kb || p.prob[q].n_split > 1 || p.prob[q].sk_parts > 0)
            return cudaErrorInvalidValue;
    return dispatch<TC_MAX_GROUP, false>(p, c, s, false);   // after joined streams: plain order
}

}  // namespace mhc
