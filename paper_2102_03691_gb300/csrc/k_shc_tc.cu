// SHC correlation (Eqs. 20-21) on the 5th-generation tensor cores (sm_103a).
//
// For a block of K samples t = t0 .. t0+K-1 and each velocity component b, the products
//   G_b[(a, tau)][t] = sum_i W_i^{ab}(tau) v_i^b(t)
// are one dense contraction over the atoms, and the correlation sums are its diagonals:
//   Ksum^{ab}(l) += sum_{t in block} G_b[(a, t - l)][t],   0 <= l < nc,  t - l >= 0.
// The (tau, t) plane is cut into 128 x 128 tiles (tau tiles aligned to multiples of 128,
// so that each is a contiguous run of rows of the virial ring); only the tiles that touch
// the band 0 <= t - tau < nc are computed, and the atom axis is split into ranges so that
// the units (pair 3a+b, tile, atom range) fill the SMs.
//
// Operands are 16-bit hi/lo pairs with one power-of-two scale per row (FP16: the row maximum
// is scaled below 2^14); three tcgen05.mma per 16-atom slice (hi*lo, lo*hi, hi*hi) into an
// FP32 TMEM accumulator that is promoted into FP32 registers every 128 atoms (the tensor
// core truncates when it accumulates; see k_tc.cu).  Warp roles as in k_tc.cu: warp 0 TMA,
// warp 1 MMA, warp 2 TMEM, warps 4..7 promotion + epilogue.
//
// Epilogue: thread (warp q, lane r) holds row 32q + r of the tile in registers.  The sums
// along the diagonals c - r = j of the warp's 32 x 128 block use a systolic shuffle: at step u
// every lane adds its column u to the partial it holds, lane 31 emits the finished diagonal
// j = u - 31, and the partials move one lane down.  The four warps' diagonals are combined in
// shared memory in a fixed order and the unit writes its 255 tile diagonals; the reduction
// kernel adds the units of each (ab, l) in a fixed order in FP64 (deterministic).
// Every barrier wait is bounded (sticky status on timeout, as in k_tc.cu).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.h"

namespace mhc {

namespace {

constexpr int ST_BM = SHC_TC_TILE;   // rows: times tau
constexpr int ST_BN = SHC_TC_TILE;   // columns: steps t of the block
constexpr int ST_BK = 64;            // atoms per pipeline stage (128-byte rows)
constexpr int ST_STAGES = 3;
constexpr int ST_A_BYTES = ST_BM * ST_BK * 2;
constexpr int ST_B_BYTES = ST_BN * ST_BK * 2;
constexpr int ST_STAGE_BYTES = 2 * ST_A_BYTES + 2 * ST_B_BYTES;
constexpr int ST_TILE_BYTES = ST_STAGES * ST_STAGE_BYTES;
constexpr int ST_DIAG = 160;                       // per-warp diagonal sums (159 used)
constexpr int ST_DIAG_BYTES = 4 * ST_DIAG * 4;
constexpr int ST_SMEM = ST_TILE_BYTES + ST_DIAG_BYTES + 256 + 1024;
constexpr uint32_t ST_TMEM_COLS = 2 * ST_BN;       // two chunk accumulators
constexpr int ST_CHUNK_KB = 128 / ST_BK;           // 128 atoms per chunk accumulator
constexpr uint32_t ST_SBO = 8 * ST_BK * 2;
constexpr uint32_t ST_SWIZZLE = 2;                 // 128-byte swizzle
constexpr int ST_THREADS = 256;
constexpr int PACK_THREADS = 512;

template <int SPLIT>
__device__ __forceinline__ void put_split(void *hi, void *lo, size_t idx, float x) {
    if (SPLIT == SPLIT_BF16) {
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        static_cast<__nv_bfloat16 *>(hi)[idx] = h;
        static_cast<__nv_bfloat16 *>(lo)[idx] = __float2bfloat16_rn(x - __bfloat162float(h));
    } else {
        const __half h = __float2half_rn(x);
        static_cast<__half *>(hi)[idx] = h;
        static_cast<__half *>(lo)[idx] = __float2half_rn(x - __half2float(h));
    }
}

// One CTA per step k.  Phase 1: row maxima |v^b| and |W^{ab}| over the atoms -> scales.
// Phase 2: scaled hi/lo operands (atoms contiguous; the padding atoms stay zero).
template <int SPLIT>
__global__ void __launch_bounds__(PACK_THREADS) shc_tc_pack_kernel(
    const float *__restrict__ v, const float *__restrict__ W, int N, int N_pad, int Kpad, int R,
    long long t0, void *A_hi, void *A_lo, void *B_hi, void *B_lo, float *scaleA, float *scaleB) {
    const int k = blockIdx.x;
    const float *vk = v + (size_t)k * N * 3;
    const float *Wk = W + (size_t)k * N * 9;
    float mx[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) mx[c] = 0.f;
    for (int i = threadIdx.x; i < N; i += PACK_THREADS) {
#pragma unroll
        for (int b = 0; b < 3; ++b) mx[b] = fmaxf(mx[b], fabsf(vk[(size_t)i * 3 + b]));
#pragma unroll
        for (int c = 0; c < 9; ++c) mx[3 + c] = fmaxf(mx[3 + c], fabsf(Wk[(size_t)i * 9 + c]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int c = 0; c < 12; ++c) mx[c] = fmaxf(mx[c], __shfl_down_sync(FULL_MASK, mx[c], o));
    __shared__ float s_mx[PACK_THREADS / 32][12];
    __shared__ float s_mul[12];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        for (int c = 0; c < 12; ++c) s_mx[warp][c] = mx[c];
    __syncthreads();
    const int slot = (int)((t0 + k) % R);
    if (threadIdx.x < 12) {
        const int c = threadIdx.x;
        float m = 0.f;
        for (int w = 0; w < PACK_THREADS / 32; ++w) m = fmaxf(m, s_mx[w][c]);
        int sc = 0;
        if (SPLIT == SPLIT_FP16 && m > 0.f && isfinite(m)) {
            int e;
            frexpf(m, &e);   // m < 2^e
            sc = 14 - e;     // scaled row maximum below 2^14
        }
        s_mul[c] = ldexpf(1.f, sc);
        if (c < 3) scaleB[(size_t)c * Kpad + k] = ldexpf(1.f, -sc);
        else scaleA[(size_t)(c - 3) * R + slot] = ldexpf(1.f, -sc);   // c - 3 = 3a + b
    }
    __syncthreads();
    float mul[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) mul[c] = s_mul[c];
    for (int i = threadIdx.x; i < N; i += PACK_THREADS) {
#pragma unroll
        for (int b = 0; b < 3; ++b)
            put_split<SPLIT>(B_hi, B_lo, ((size_t)b * Kpad + k) * N_pad + i, vk[(size_t)i * 3 + b] * mul[b]);
#pragma unroll
        for (int c = 0; c < 9; ++c)
            put_split<SPLIT>(A_hi, A_lo, ((size_t)c * R + slot) * N_pad + i, Wk[(size_t)i * 9 + c] * mul[3 + c]);
    }
}

__global__ void __launch_bounds__(ST_THREADS, 1) shc_tc_kernel(const __grid_constant__ ShcTcParams p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                ~uintptr_t(1023));
    float *sd = reinterpret_cast<float *>(smem + ST_TILE_BYTES);   // [4][ST_DIAG]
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + ST_TILE_BYTES + ST_DIAG_BYTES);
    uint64_t *full = bars;                       // [STAGES]
    uint64_t *empty = bars + ST_STAGES;          // [STAGES]
    uint64_t *acc_full = bars + 2 * ST_STAGES;   // [2]
    uint64_t *acc_empty = acc_full + 2;          // [2]
    uint64_t *done_bar = acc_empty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done_bar + 1);
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // unit -> (pair c = 3a+b, tile pair, atom range)
    const int per_c = p.n_pairs * p.splits;
    const int u = blockIdx.x;
    const int cpair = u / per_c, rem = u - cpair * per_c;
    const int tp = rem / p.splits, split = rem - tp * p.splits;
    const int bvel = cpair % 3;
    const int pt = p.p_tile[tp], qt = p.q_tile[tp];
    const int arow = cpair * p.R + (pt % p.nR) * ST_BM;
    const int brow = bvel * p.Kpad + qt * ST_BN;
    const int kb0 = split * p.kb_per_split;
    const int kb1 = min(kb0 + p.kb_per_split, p.n_kb);

    if (threadIdx.x == 0) {
        for (int s = 0; s < ST_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 128);
        }
        mbar_init(done_bar, 1);
        *abort = 0;
        fence_mbar_init();
    }
    if (warp == 2) {
        tmem_alloc(tmem_slot, ST_TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ------------------------------------------------------------ TMA producer
        tma_prefetch_desc(&p.tmA_hi);
        tma_prefetch_desc(&p.tmA_lo);
        tma_prefetch_desc(&p.tmB_hi);
        tma_prefetch_desc(&p.tmB_lo);
        const uint64_t pol = l2_policy_evict_normal();   // rows are shared with other units
        uint32_t issued_phase[ST_STAGES];
        bool issued[ST_STAGES];
        for (int s = 0; s < ST_STAGES; ++s) issued[s] = false;
        int stage = 0;
        uint32_t phase = 0;
        bool ok = true;
        for (int kb = kb0; kb < kb1; ++kb) {
            if (!mbar_wait(&empty[stage], phase ^ 1u, abort, p.wait_limit)) { ok = false; break; }
            uint8_t *sa = smem + stage * ST_STAGE_BYTES;
            mbar_arrive_expect_tx(&full[stage], ST_STAGE_BYTES);
            const int x = kb * ST_BK;
            tma_load_2d(sa, &p.tmA_hi, &full[stage], x, arow, pol);
            tma_load_2d(sa + ST_A_BYTES, &p.tmA_lo, &full[stage], x, arow, pol);
            tma_load_2d(sa + 2 * ST_A_BYTES, &p.tmB_hi, &full[stage], x, brow, pol);
            tma_load_2d(sa + 2 * ST_A_BYTES + ST_B_BYTES, &p.tmB_lo, &full[stage], x, brow, pol);
            issued[stage] = true;
            issued_phase[stage] = phase;
            if (++stage == ST_STAGES) { stage = 0; phase ^= 1u; }
        }
        if (!ok) {
            *abort = 1;
            set_status(p.status, DEV_TIMEOUT);
        }
        for (int s = 0; s < ST_STAGES; ++s)
            if (issued[s]) {
                const long long c0 = clock64();
                while (!mbar_try_wait(&full[s], issued_phase[s]) && clock64() - c0 < p.wait_limit) {
                }
            }
    } else if (warp == 1 && lane == 0) {
        // ------------------------------------------------------------ MMA issuer
        int stage = 0, abuf = 0;
        uint32_t phase = 0, aphase = 0;
        bool ok = true;
        const uint32_t smem0 = smem_u32(smem);
        for (int c0 = kb0; ok && c0 < kb1; c0 += ST_CHUNK_KB) {
            if (!mbar_wait(&acc_empty[abuf], aphase ^ 1u, abort, p.wait_limit)) { ok = false; break; }
            tc_fence_after();
            const uint32_t d_tmem = tmem_base + (uint32_t)(abuf * ST_BN);
            const int c1 = min(c0 + ST_CHUNK_KB, kb1);
            for (int kb = c0; kb < c1; ++kb) {
                if (!mbar_wait(&full[stage], phase, abort, p.wait_limit)) { ok = false; break; }
                tc_fence_after();
                const uint32_t a_hi = smem0 + stage * ST_STAGE_BYTES;
                const uint32_t a_lo = a_hi + ST_A_BYTES;
                const uint32_t b_hi = a_hi + 2 * ST_A_BYTES;
                const uint32_t b_lo = b_hi + ST_B_BYTES;
#pragma unroll
                for (int kk = 0; kk < ST_BK / 16; ++kk) {
                    const uint32_t off = kk * 32;
                    const uint64_t dah = smem_desc_kmajor(a_hi + off, ST_SBO, ST_SWIZZLE);
                    const uint64_t dal = smem_desc_kmajor(a_lo + off, ST_SBO, ST_SWIZZLE);
                    const uint64_t dbh = smem_desc_kmajor(b_hi + off, ST_SBO, ST_SWIZZLE);
                    const uint64_t dbl = smem_desc_kmajor(b_lo + off, ST_SBO, ST_SWIZZLE);
                    umma_f16(d_tmem, dah, dbl, p.idesc, (kb != c0 || kk != 0) ? 1u : 0u);
                    umma_f16(d_tmem, dal, dbh, p.idesc, 1u);
                    umma_f16(d_tmem, dah, dbh, p.idesc, 1u);
                }
                umma_commit(&empty[stage]);
                if (++stage == ST_STAGES) { stage = 0; phase ^= 1u; }
            }
            if (!ok) break;
            umma_commit(&acc_full[abuf]);
            if (++abuf == 2) { abuf = 0; aphase ^= 1u; }
        }
        if (!ok) {
            *abort = 1;
            set_status(p.status, DEV_TIMEOUT);
        }
        umma_commit(done_bar);
        const long long c0 = clock64();
        while (!mbar_try_wait(done_bar, 0) && clock64() - c0 < p.wait_limit) {
        }
    } else if (warp >= 4) {
        // ------------------------------------------------------------ promotion + diagonals
        const int qw = warp & 3;
        float acc[ST_BN];
#pragma unroll
        for (int j = 0; j < ST_BN; ++j) acc[j] = 0.f;
        int abuf = 0;
        uint32_t aphase = 0;
        bool ok = true;
        for (int c0 = kb0; c0 < kb1; c0 += ST_CHUNK_KB) {
            if (!mbar_wait(&acc_full[abuf], aphase, abort, p.wait_limit)) { ok = false; break; }
            tc_fence_after();
            const uint32_t tbase = tmem_base + ((uint32_t)(qw * 32) << 16) + (uint32_t)(abuf * ST_BN);
#pragma unroll
            for (int c = 0; c < ST_BN / 16; ++c) {
                uint32_t r[16];
                tmem_ld_32x32b_x16(tbase + (uint32_t)(c * 16), r);
                tmem_ld_wait();
#pragma unroll
                for (int j = 0; j < 16; ++j) acc[c * 16 + j] += __uint_as_float(r[j]);
            }
            tc_fence_before();
            mbar_arrive(&acc_empty[abuf]);
            if (++abuf == 2) { abuf = 0; aphase ^= 1u; }
        }
        if (!ok) {
            *abort = 1;
            set_status(p.status, DEV_TIMEOUT);
        }
        // undo the row scales; steps past the block's K do not exist (zero)
        const float sa = __ldg(p.scaleA + arow + qw * 32 + lane);
        const float *sb = p.scaleB + brow;
        const int kvalid = p.K - qt * ST_BN;
        float *sdw = sd + qw * ST_DIAG;
        float P = 0.f;
#pragma unroll
        for (int uu = 0; uu < ST_BN + 31; ++uu) {
            if (uu < ST_BN) {
                const float s = uu < kvalid ? sa * __ldg(sb + uu) : 0.f;
                P = fmaf(acc[uu], s, P);   // acc * s is exact (power of two)
            }
            const float e = __shfl_sync(FULL_MASK, P, 31);   // diagonal c - r = uu - 31 done
            if (lane == 0) sdw[uu] = e;
            P = __shfl_up_sync(FULL_MASK, P, 1);
            if (lane == 0) P = 0.f;
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");   // the four epilogue warps
        // tile diagonal m = (c - r) + 127 in [0, 255): the four warps' shifted diagonals
        for (int m = threadIdx.x - 128; m < 2 * ST_BM - 1; m += 128) {
            float s = 0.f;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j = m - (ST_BM - 1) + 32 * q;   // c - r_lane in warp q
                if (j >= -31 && j <= ST_BN - 1) s += sd[q * ST_DIAG + j + 31];
            }
            p.partials[(size_t)u * 256 + m] = ok ? s : 0.f;
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 2) tmem_dealloc(tmem_base, ST_TMEM_COLS);
}

// Ksum[c][l] += sum over tile pairs (in order) and atom ranges (in order) of the unit diagonal
// m = l - (t0 + 128 (q - p)) + 127.
__global__ void __launch_bounds__(128) shc_tc_reduce_kernel(const __grid_constant__ ShcTcParams p,
                                                            double *Ksum) {
    const int c = blockIdx.y;
    const int l = blockIdx.x * 128 + threadIdx.x;
    if (l >= p.nc) return;
    const int per_c = p.n_pairs * p.splits;
    double s = 0.0;
    for (int tp = 0; tp < p.n_pairs; ++tp) {
        const long long off = p.t0 + (long long)ST_BN * p.q_tile[tp] - (long long)ST_BM * p.p_tile[tp] -
                              (ST_BM - 1);
        const long long m = l - off;
        if (m < 0 || m >= 2 * ST_BM - 1) continue;
        for (int sp = 0; sp < p.splits; ++sp)
            s += (double)p.partials[((size_t)c * per_c + (size_t)tp * p.splits + sp) * 256 + m];
    }
    Ksum[(size_t)c * p.nc + l] += s;
}

}  // namespace

void launch_shc_tc_pack(const float *v, const float *W, int N, int N_pad, int K, int Kpad, int R,
                        long long t0, int split, void *A_hi, void *A_lo, void *B_hi, void *B_lo,
                        float *scaleA, float *scaleB, cudaStream_t s) {
    if (K <= 0) return;
    if (split == SPLIT_BF16)
        shc_tc_pack_kernel<SPLIT_BF16><<<K, PACK_THREADS, 0, s>>>(v, W, N, N_pad, Kpad, R, t0, A_hi,
                                                                  A_lo, B_hi, B_lo, scaleA, scaleB);
    else
        shc_tc_pack_kernel<SPLIT_FP16><<<K, PACK_THREADS, 0, s>>>(v, W, N, N_pad, Kpad, R, t0, A_hi,
                                                                  A_lo, B_hi, B_lo, scaleA, scaleB);
}

size_t shc_tc_smem_bytes() { return ST_SMEM; }

cudaError_t launch_shc_tc(const ShcTcParams &p, cudaStream_t s) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(shc_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, ST_SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int units = 9 * p.n_pairs * p.splits;
    shc_tc_kernel<<<units, ST_THREADS, ST_SMEM, s>>>(p);
    return cudaGetLastError();
}

void launch_shc_tc_reduce(const ShcTcParams &p, double *Ksum, cudaStream_t s) {
    dim3 grid((p.nc + 127) / 128, 9);
    shc_tc_reduce_kernel<<<grid, 128, 0, s>>>(p, Ksum);
}

}  // namespace mhc
