// SHC correlation (Eqs. 20-21) on the 5th-generation tensor cores (sm_103a).
//
// For a block of K samples t = t0 .. t0+K-1 and each velocity component b, the products
//   G_b[(a, tau)][t] = sum_i W_i^{ab}(tau) v_i^b(t)
// are one dense contraction over the atoms, and the correlation sums are its diagonals:
//   Ksum^{ab}(l) += sum_{t in block} G_b[(a, t - l)][t],   0 <= l < nc,  t - l >= 0.
// The (tau, t) plane is cut into 128 x 256 tiles (tau tiles aligned to multiples of 128,
// so that each is a contiguous run of rows of the virial ring); only the tiles that touch
// the band 0 <= t - tau < nc are computed, and the atom axis is split into ranges so that
// the units (pair 3a+b, tile, atom range) fill the SMs.  Two units that differ only in
// their tau tile (p, p+1) form a CTA pair (tcgen05 cta_group::2): the leader issues M = 256
// MMAs over both tau tiles, each CTA stages its own 128 ring rows and one half (128 rows) of
// the shared velocity tile, and each CTA's TMEM receives its own 128 x 256 accumulator.  The
// kernel is bound by the bytes that reach each SM: 32 KB per CTA and stage, against 48 KB when
// every CTA held the whole velocity tile.
//
// Operands are 16-bit hi/lo pairs with one power-of-two scale per row (FP16: the row maximum
// is scaled below 2^14); three tcgen05.mma per 16-atom slice (hi*lo, lo*hi, hi*hi) into an
// FP32 TMEM accumulator that is promoted into FP32 registers every 128 atoms (the tensor
// core truncates when it accumulates; see k_tc.cu).  Warp roles as in k_tc.cu's pair kernel:
// warp 0 TMA (both CTAs), warp 1 MMA (leader), warp 2 TMEM, warps 4..11 promotion + epilogue.
//
// Epilogue: thread (warp q + 4h, lane r) holds row 32q + r, columns 128h .. 128h+127 of the
// tile in registers.  The sums along the diagonals c - r = j of the warp's 32 x 128 block use
// a systolic shuffle: at step u every lane adds its column u to the partial it holds, lane 31
// emits the finished diagonal j = u - 31, and the partials move one lane down.  The eight
// warps' diagonals are combined in shared memory in a fixed order and the unit writes its 383
// tile diagonals; the reduction kernel adds the units of each (ab, l) in a fixed order in FP64
// (deterministic).  128 x 256 tiles keep the shared-memory operand reads of each MMA below
// the shared-memory bandwidth (a 128 x 128 MMA reading both operands would sit at it).
// Every barrier wait is bounded (sticky status on timeout, as in k_tc.cu).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.h"

namespace mhc {

namespace {

constexpr int ST_BM = SHC_TC_TILE;       // rows: times tau
constexpr int ST_BN = SHC_TC_STEP_TILE;  // columns: steps t of the block
constexpr int ST_BK = 32;                // atoms per pipeline stage (64-byte rows)
constexpr int ST_STAGES = 6;
constexpr int ST_A_BYTES = ST_BM * ST_BK * 2;
constexpr int ST_B_BYTES = (ST_BN / 2) * ST_BK * 2;   // this CTA's half of the velocity rows
constexpr int ST_STAGE_BYTES = 2 * ST_A_BYTES + 2 * ST_B_BYTES;
constexpr int ST_TILE_BYTES = ST_STAGES * ST_STAGE_BYTES;
constexpr int ST_EPI_WARPS = ST_BN / 32;          // 4 lane quarters x column halves
constexpr int ST_DIAG = 160;                       // per-warp diagonal sums (159 used)
constexpr int ST_DIAG_BYTES = ST_EPI_WARPS * ST_DIAG * 4;
constexpr int ST_NDIAG = ST_BM + ST_BN - 1;        // diagonals of a tile
constexpr int ST_PART = SHC_TC_PART;               // floats per unit in the partials
constexpr int ST_SMEM = ST_TILE_BYTES + ST_DIAG_BYTES + 256 + 1024;
constexpr uint32_t ST_TMEM_COLS = 2 * ST_BN;       // two chunk accumulators
constexpr int ST_CHUNK_KB = 128 / ST_BK;           // 128 atoms per chunk accumulator
constexpr uint32_t ST_SBO = 8 * ST_BK * 2;
constexpr uint32_t ST_SWIZZLE = 4;                 // 64-byte swizzle
constexpr int ST_THREADS = 128 + 32 * ST_EPI_WARPS;
static_assert(ST_PART >= ST_NDIAG, "partials row");
static_assert(ST_SMEM <= 227 * 1024, "shared memory");
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

// Power-of-two scale of a row with maximum m: FP16 keeps the scaled maximum below 2^14
// (the lo parts stay normal); BF16 has the FP32 exponent range and takes 1.
template <int SPLIT>
__device__ __forceinline__ int row_shift(float m) {
    int sc = 0;
    if (SPLIT == SPLIT_FP16 && m > 0.f && isfinite(m)) {
        int e;
        frexpf(m, &e);   // m < 2^e
        sc = 14 - e;
    }
    return sc;
}

// Block maximum of the 12 row values of this CTA into s_out[12] (all threads take part).
__device__ __forceinline__ void block_max12(float (&mx)[12], float (*s_mx)[12], float *s_out) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int c = 0; c < 12; ++c) mx[c] = fmaxf(mx[c], __shfl_down_sync(FULL_MASK, mx[c], o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < 12; ++c) s_mx[warp][c] = mx[c];
    __syncthreads();
    if (threadIdx.x < 12) {
        float m = 0.f;
        for (int w = 0; w < PACK_THREADS / 32; ++w) m = fmaxf(m, s_mx[w][threadIdx.x]);
        s_out[threadIdx.x] = m;
    }
}

// Cluster of C CTAs per step k, CTA r taking atoms r*apc .. (r+1)*apc-1 (apc = 512 AP): the
// step's velocities and virials are read once into registers (thread t holds atoms
// t + 512 j, so every load is coalesced), the 12 row maxima are combined across the cluster
// through distributed shared memory, and the scaled hi/lo operands are written from the
// registers.  Velocity rows b Kpad + k, virial ring rows (3a+b) R + (t0+k) mod R.
template <int SPLIT, int AP>
__global__ void __launch_bounds__(PACK_THREADS, 1) shc_tc_pack_cluster_kernel(
    const float *__restrict__ v, const float *__restrict__ W, int N, int N_pad, int Kpad, int R,
    long long t0, void *A_hi, void *A_lo, void *B_hi, void *B_lo, float *scaleA, float *scaleB) {
    __shared__ float s_mx[PACK_THREADS / 32][12];
    __shared__ float s_loc[12], s_mul[12];
    const uint32_t rank = cluster_ctarank(), nrank = cluster_nctarank();
    const int k = (int)(blockIdx.x / nrank);
    const int apc = PACK_THREADS * AP;
    const int i0 = (int)rank * apc + threadIdx.x;
    const float *vk = v + (size_t)k * N * 3;
    const float *Wk = W + (size_t)k * N * 9;
    float x[AP][12];
    float mx[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) mx[c] = 0.f;
#pragma unroll
    for (int j = 0; j < AP; ++j) {
        const int i = i0 + PACK_THREADS * j;
        const bool in = i < N;
#pragma unroll
        for (int b = 0; b < 3; ++b) x[j][b] = in ? vk[(size_t)i * 3 + b] : 0.f;
#pragma unroll
        for (int c = 0; c < 9; ++c) x[j][3 + c] = in ? Wk[(size_t)i * 9 + c] : 0.f;
#pragma unroll
        for (int c = 0; c < 12; ++c) mx[c] = fmaxf(mx[c], fabsf(x[j][c]));
    }
    block_max12(mx, s_mx, s_loc);
    cluster_sync_all();   // every CTA's s_loc is complete
    const int slot = (int)((t0 + k) % R);
    if (threadIdx.x < 12) {
        const int c = threadIdx.x;
        float m = 0.f;
        for (uint32_t q = 0; q < nrank; ++q) m = fmaxf(m, ld_shared_cluster_f32(mapa_shared(smem_u32(&s_loc[c]), q)));
        const int sc = row_shift<SPLIT>(m);
        s_mul[c] = ldexpf(1.f, sc);
        if (rank == 0) {
            if (c < 3) scaleB[(size_t)c * Kpad + k] = ldexpf(1.f, -sc);
            else scaleA[(size_t)(c - 3) * R + slot] = ldexpf(1.f, -sc);   // c - 3 = 3a + b
        }
    }
    cluster_sync_all();   // peers are done reading s_loc; s_mul is visible to the CTA
    float mul[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) mul[c] = s_mul[c];
#pragma unroll
    for (int j = 0; j < AP; ++j) {
        const int i = i0 + PACK_THREADS * j;
        if (i >= N) break;
#pragma unroll
        for (int b = 0; b < 3; ++b)
            put_split<SPLIT>(B_hi, B_lo, ((size_t)b * Kpad + k) * N_pad + i, x[j][b] * mul[b]);
#pragma unroll
        for (int c = 0; c < 9; ++c)
            put_split<SPLIT>(A_hi, A_lo, ((size_t)c * R + slot) * N_pad + i, x[j][3 + c] * mul[3 + c]);
    }
}

// hi = rn16(x), lo = rn16(x - hi) as 16-bit patterns
template <int SPLIT>
__device__ __forceinline__ void split16(float x, uint32_t &hi, uint32_t &lo) {
    if (SPLIT == SPLIT_BF16) {
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        hi = __bfloat16_as_ushort(h);
        lo = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(h)));
    } else {
        const __half h = __float2half_rn(x);
        hi = __half_as_ushort(h);
        lo = __half_as_ushort(__float2half_rn(x - __half2float(h)));
    }
}

// Four 16-bit patterns -> one 8-byte store each for hi and lo.
template <int SPLIT>
__device__ __forceinline__ void put_split4(void *hi, void *lo, size_t idx, float a, float b, float c,
                                           float d) {
    uint32_t h0, l0, h1, l1, h2, l2, h3, l3;
    split16<SPLIT>(a, h0, l0);
    split16<SPLIT>(b, h1, l1);
    split16<SPLIT>(c, h2, l2);
    split16<SPLIT>(d, h3, l3);
    *reinterpret_cast<uint2 *>(static_cast<uint16_t *>(hi) + idx) = make_uint2(h0 | (h1 << 16), h2 | (h3 << 16));
    *reinterpret_cast<uint2 *>(static_cast<uint16_t *>(lo) + idx) = make_uint2(l0 | (l1 << 16), l2 | (l3 << 16));
}

// Cluster of ceil(N / APC) CTAs per step k; CTA r bulk-copies the contiguous velocities and
// virials of its atoms r*APC .. into shared memory (one TMA bulk copy per 16 KB), so every
// load is asynchronous and registers stay few (four 256-thread CTAs per SM for APC = 1024).
// Thread t then takes the four consecutive atoms 4t .. 4t+3 (16-byte shared-memory reads,
// conflict-free), the 12 row maxima are combined across the cluster in distributed shared
// memory, and each operand row gets one 8-byte store per thread.  Needs N % 4 == 0 and
// 16-byte aligned inputs.  A copy that does not land within the wait limit sets the status
// word; the CTA then writes nothing.
template <int SPLIT, int THREADS>
__global__ void __launch_bounds__(THREADS) shc_tc_pack_bulk_kernel(
    const float *__restrict__ v, const float *__restrict__ W, int N, int N_pad, int Kpad, int R,
    long long t0, void *A_hi, void *A_lo, void *B_hi, void *B_lo, float *scaleA, float *scaleB,
    int *status, long long wait_limit) {
    constexpr int APC = 4 * THREADS;
    extern __shared__ float4 pk_smem4[];
    float *sv = reinterpret_cast<float *>(pk_smem4);   // [APC][3]
    float *sw = sv + APC * 3;                          // [APC][9]
    __shared__ float s_mx[THREADS / 32][12];
    __shared__ float s_loc[12], s_mul[12];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    const uint32_t rank = cluster_ctarank(), nrank = cluster_nctarank();
    const int k = (int)(blockIdx.x / nrank);
    const int a0 = (int)rank * APC;
    const int na = max(0, min(APC, N - a0));   // atoms of this CTA (a multiple of 4)
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && na > 0) {
        const uint32_t vb = (uint32_t)na * 12, wb = (uint32_t)na * 36;
        mbar_arrive_expect_tx(&bar, vb + wb);
        const char *gv = reinterpret_cast<const char *>(v + ((size_t)k * N + a0) * 3);
        const char *gw = reinterpret_cast<const char *>(W + ((size_t)k * N + a0) * 9);
        for (uint32_t o = 0; o < vb; o += 16384)
            bulk_load(reinterpret_cast<char *>(sv) + o, gv + o, min(16384u, vb - o), &bar);
        for (uint32_t o = 0; o < wb; o += 16384)
            bulk_load(reinterpret_cast<char *>(sw) + o, gw + o, min(16384u, wb - o), &bar);
    }
    bool ok = true;
    if (na > 0) ok = mbar_wait(&bar, 0, &abort_flag, wait_limit);
    const int i = 4 * (int)threadIdx.x;   // first of this thread's atoms within the CTA
    const bool in = ok && i < na;
    float mx[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) mx[c] = 0.f;
    if (in) {
        const float4 *pv = reinterpret_cast<const float4 *>(sv + i * 3);
        const float4 *pw = reinterpret_cast<const float4 *>(sw + i * 9);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float4 t = pv[q];
            const float e[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) mx[(4 * q + u) % 3] = fmaxf(mx[(4 * q + u) % 3], fabsf(e[u]));
        }
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const float4 t = pw[q];
            const float e[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) mx[3 + (4 * q + u) % 9] = fmaxf(mx[3 + (4 * q + u) % 9], fabsf(e[u]));
        }
    }
    // block maximum (THREADS-wide version of block_max12)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int c = 0; c < 12; ++c) mx[c] = fmaxf(mx[c], __shfl_down_sync(FULL_MASK, mx[c], o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < 12; ++c) s_mx[warp][c] = mx[c];
    __syncthreads();
    if (threadIdx.x < 12) {
        float m = 0.f;
        for (int w = 0; w < THREADS / 32; ++w) m = fmaxf(m, s_mx[w][threadIdx.x]);
        s_loc[threadIdx.x] = m;
    }
    cluster_sync_all();
    const int slot = (int)((t0 + k) % R);
    if (threadIdx.x < 12) {
        const int c = threadIdx.x;
        float m = 0.f;
        for (uint32_t q = 0; q < nrank; ++q) m = fmaxf(m, ld_shared_cluster_f32(mapa_shared(smem_u32(&s_loc[c]), q)));
        const int sc = row_shift<SPLIT>(m);
        s_mul[c] = ldexpf(1.f, sc);
        if (rank == 0) {
            if (c < 3) scaleB[(size_t)c * Kpad + k] = ldexpf(1.f, -sc);
            else scaleA[(size_t)(c - 3) * R + slot] = ldexpf(1.f, -sc);
        }
    }
    cluster_sync_all();
    if (!ok) {   // the CTA stays alive until its copy has landed (bounded) or given up on
        if (threadIdx.x == 0) {
            set_status(status, DEV_TIMEOUT);
            const long long c0 = clock64();
            while (!mbar_try_wait(&bar, 0) && clock64() - c0 < wait_limit) {
            }
        }
        return;
    }
    if (!in) return;
    const float *xv = sv + i * 3, *xw = sw + i * 9;
    const int g = a0 + i;   // global atom index
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const float m = s_mul[b];
        put_split4<SPLIT>(B_hi, B_lo, ((size_t)b * Kpad + k) * N_pad + g, xv[b] * m, xv[3 + b] * m,
                          xv[6 + b] * m, xv[9 + b] * m);
    }
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        const float m = s_mul[3 + c];
        put_split4<SPLIT>(A_hi, A_lo, ((size_t)c * R + slot) * N_pad + g, xw[c] * m, xw[9 + c] * m,
                          xw[18 + c] * m, xw[27 + c] * m);
    }
}

// Fallback for systems larger than a cluster of 8 CTAs holds: one CTA per step, phase 1 the
// row maxima, phase 2 the operands (the step's inputs are read twice).
template <int SPLIT>
__global__ void __launch_bounds__(PACK_THREADS) shc_tc_pack_kernel(
    const float *__restrict__ v, const float *__restrict__ W, int N, int N_pad, int Kpad, int R,
    long long t0, void *A_hi, void *A_lo, void *B_hi, void *B_lo, float *scaleA, float *scaleB) {
    __shared__ float s_mx[PACK_THREADS / 32][12];
    __shared__ float s_loc[12], s_mul[12];
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
    block_max12(mx, s_mx, s_loc);
    const int slot = (int)((t0 + k) % R);
    if (threadIdx.x < 12) {
        const int c = threadIdx.x;
        const int sc = row_shift<SPLIT>(s_loc[c]);
        s_mul[c] = ldexpf(1.f, sc);
        if (c < 3) scaleB[(size_t)c * Kpad + k] = ldexpf(1.f, -sc);
        else scaleA[(size_t)(c - 3) * R + slot] = ldexpf(1.f, -sc);
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
    float *sd = reinterpret_cast<float *>(smem + ST_TILE_BYTES);   // [EPI_WARPS][ST_DIAG]
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + ST_TILE_BYTES + ST_DIAG_BYTES);
    uint64_t *full = bars;                       // [STAGES]
    uint64_t *empty = bars + ST_STAGES;          // [STAGES]
    uint64_t *acc_full = bars + 2 * ST_STAGES;   // [2]
    uint64_t *acc_empty = acc_full + 2;          // [2]
    uint64_t *done_bar = acc_empty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done_bar + 1);
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // unit u = c per_c + (pp splits + split) 2 + rank -> (pair c = 3a+b, tile pair 2 pp + rank,
    // atom range); the cluster's two CTAs hold tau tiles p, p+1 of the same step tile
    const uint32_t rank = cluster_ctarank();
    const int per_c = p.n_pairs * p.splits;
    const int u = blockIdx.x;
    const int cpair = u / per_c, rem = (u - cpair * per_c) >> 1;
    const int pp = rem / p.splits, split = rem - pp * p.splits;
    const int tp = 2 * pp + (int)rank;
    const int bvel = cpair % 3;
    const int pt = p.p_tile[tp], qt = p.q_tile[tp];
    const int arow = cpair * p.R + (pt % p.nR) * ST_BM;
    const int brow = bvel * p.Kpad + qt * ST_BN;
    const int kb0 = split * p.kb_per_split;
    const int kb1 = min(kb0 + p.kb_per_split, p.n_kb);

    const bool leader = rank == 0;
    if (threadIdx.x == 0) {
        for (int s = 0; s < ST_STAGES; ++s) {
            mbar_init(&full[s], 1);    // leader: both CTAs' bytes landed
            mbar_init(&empty[s], 1);   // the leader's MMAs have read the stage (both CTAs)
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 2 * ST_EPI_WARPS);   // leader: one arrival per epilogue warp
        }
        mbar_init(done_bar, 1);
        *abort = 0;
        fence_mbar_init();
    }
    if (warp == 2) {
        tmem_alloc_pair(tmem_slot, ST_TMEM_COLS);
        tmem_relinquish_pair();
    }
    tc_fence_before();
    __syncwarp();
    cluster_sync_all();   // both CTAs' barriers initialised, TMEM allocated in both
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
        const int bhalf = brow + (int)rank * (ST_BN / 2);   // this CTA's velocity rows
        for (int kb = kb0; kb < kb1; ++kb) {
            if (!mbar_wait(&empty[stage], phase ^ 1u, abort, p.wait_limit)) { ok = false; break; }
            uint8_t *sa = smem + stage * ST_STAGE_BYTES;
            if (leader) mbar_arrive_expect_tx(&full[stage], 2 * ST_STAGE_BYTES);
            const uint32_t fb = mapa_shared(smem_u32(&full[stage]), 0);
            const int x = kb * ST_BK;
            tma_load_2d_pair(sa, &p.tmA_hi, fb, x, arow, pol);
            tma_load_2d_pair(sa + ST_A_BYTES, &p.tmA_lo, fb, x, arow, pol);
            tma_load_2d_pair(sa + 2 * ST_A_BYTES, &p.tmB_hi, fb, x, bhalf, pol);
            tma_load_2d_pair(sa + 2 * ST_A_BYTES + ST_B_BYTES, &p.tmB_lo, fb, x, bhalf, pol);
            issued[stage] = true;
            issued_phase[stage] = phase;
            if (++stage == ST_STAGES) { stage = 0; phase ^= 1u; }
        }
        if (!ok) {
            *abort = 1;
            set_status(p.status, DEV_TIMEOUT);
        }
        if (leader)   // the leader's barriers count both CTAs' copies
            for (int s = 0; s < ST_STAGES; ++s)
                if (issued[s]) {
                    const long long c0 = clock64();
                    while (!mbar_try_wait(&full[s], issued_phase[s]) && clock64() - c0 < p.wait_limit) {
                    }
                }
    } else if (warp == 1 && lane == 0 && leader) {
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
                    umma_f16_pair(d_tmem, dah, dbl, p.idesc, (kb != c0 || kk != 0) ? 1u : 0u);
                    umma_f16_pair(d_tmem, dal, dbh, p.idesc, 1u);
                    umma_f16_pair(d_tmem, dah, dbh, p.idesc, 1u);
                }
                umma_commit_pair(&empty[stage], (uint16_t)0x3);   // the stage is free in both CTAs
                if (++stage == ST_STAGES) { stage = 0; phase ^= 1u; }
            }
            if (!ok) break;
            umma_commit_pair(&acc_full[abuf], (uint16_t)0x3);
            if (++abuf == 2) { abuf = 0; aphase ^= 1u; }
        }
        if (!ok) {
            *abort = 1;
            set_status(p.status, DEV_TIMEOUT);
        }
        umma_commit_pair(done_bar, (uint16_t)0x1);
        const long long c0 = clock64();
        while (!mbar_try_wait(done_bar, 0) && clock64() - c0 < p.wait_limit) {
        }
    } else if (warp >= 4) {
        // ------------------------------------------------------------ promotion + diagonals
        const int qw = warp & 3;          // TMEM lane quarter: rows 32 qw ..
        const int ch = (warp - 4) >> 2;   // column half: columns 128 ch ..
        float acc[128];
#pragma unroll
        for (int j = 0; j < 128; ++j) acc[j] = 0.f;
        int abuf = 0;
        uint32_t aphase = 0;
        bool ok = true;
        const uint32_t empty_leader[2] = {mapa_shared(smem_u32(&acc_empty[0]), 0),
                                          mapa_shared(smem_u32(&acc_empty[1]), 0)};
        for (int c0 = kb0; c0 < kb1; c0 += ST_CHUNK_KB) {
            if (!mbar_wait(&acc_full[abuf], aphase, abort, p.wait_limit)) { ok = false; break; }
            tc_fence_after();
            const uint32_t tbase = tmem_base + ((uint32_t)(qw * 32) << 16) +
                                   (uint32_t)(abuf * ST_BN + ch * 128);
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
        }
        if (!ok) {
            *abort = 1;
            set_status(p.status, DEV_TIMEOUT);
        }
        // undo the row scales; steps past the block's K do not exist (zero)
        const float sa = __ldg(p.scaleA + arow + qw * 32 + lane);
        const float *sb = p.scaleB + brow + ch * 128;
        const int kvalid = p.K - qt * ST_BN - ch * 128;
        float *sdw = sd + (warp - 4) * ST_DIAG;
        float P = 0.f;
#pragma unroll
        for (int uu = 0; uu < 128 + 31; ++uu) {
            if (uu < 128) {
                const float s = uu < kvalid ? sa * __ldg(sb + uu) : 0.f;
                P = fmaf(acc[uu], s, P);   // acc * s is exact (power of two)
            }
            const float e = __shfl_sync(FULL_MASK, P, 31);   // diagonal c - r = uu - 31 done
            if (lane == 0) sdw[uu] = e;
            P = __shfl_up_sync(FULL_MASK, P, 1);
            if (lane == 0) P = 0.f;
        }
        asm volatile("bar.sync 1, %0;" :: "n"(32 * ST_EPI_WARPS) : "memory");   // epilogue warps
        // tile diagonal m = (c - r) + 127 in [0, 383): the warps' shifted diagonals, in order
        for (int m = threadIdx.x - 128; m < ST_NDIAG; m += 32 * ST_EPI_WARPS) {
            float s = 0.f;
#pragma unroll
            for (int w = 0; w < ST_EPI_WARPS; ++w) {
                const int j = m - (ST_BM - 1) - 128 * (w >> 2) + 32 * (w & 3);   // c' - lane in warp w
                if (j >= -31 && j <= 127) s += sd[w * ST_DIAG + j + 31];
            }
            p.partials[(size_t)u * ST_PART + m] = ok ? s : 0.f;
        }
    }

    tc_fence_before();
    __syncwarp();
    cluster_sync_all();   // neither CTA leaves while the pair still shares barriers or TMEM
    tc_fence_after();
    if (warp == 2) tmem_dealloc_pair(tmem_base, ST_TMEM_COLS);
}

// Ksum[c][l] += sum over tile pairs (in order) and atom ranges (in order) of the unit diagonal
// m = l - (t0 + 256 q - 128 p) + 127.
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
        if (m < 0 || m >= ST_NDIAG) continue;
        for (int sp = 0; sp < p.splits; ++sp) {
            const size_t u = (size_t)c * per_c + ((size_t)(tp >> 1) * p.splits + sp) * 2 + (tp & 1);
            s += (double)p.partials[u * ST_PART + m];
        }
    }
    Ksum[(size_t)c * p.nc + l] += s;
}

}  // namespace

template <int SPLIT, int AP>
cudaError_t launch_pack_cluster(int csize, const float *v, const float *W, int N, int N_pad, int K,
                                int Kpad, int R, long long t0, void *A_hi, void *A_lo, void *B_hi,
                                void *B_lo, float *scaleA, float *scaleB, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(K * csize), 1, 1);
    cfg.blockDim = dim3(PACK_THREADS, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, shc_tc_pack_cluster_kernel<SPLIT, AP>, v, W, N, N_pad, Kpad, R, t0,
                              A_hi, A_lo, B_hi, B_lo, scaleA, scaleB);
}

template <int SPLIT, int THREADS>
cudaError_t launch_pack_bulk(const float *v, const float *W, int N, int N_pad, int K, int Kpad, int R,
                             long long t0, void *A_hi, void *A_lo, void *B_hi, void *B_lo,
                             float *scaleA, float *scaleB, int *status, long long wait_limit,
                             cudaStream_t s) {
    constexpr int APC = 4 * THREADS;
    const int smem = APC * 48;
    auto kern = shc_tc_pack_bulk_kernel<SPLIT, THREADS>;
    static cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (attr != cudaSuccess) return attr;
    const int csize = (N + APC - 1) / APC;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(K * csize), 1, 1);
    cfg.blockDim = dim3(THREADS, 1, 1);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = s;
    cudaLaunchAttribute la[1];
    la[0].id = cudaLaunchAttributeClusterDimension;
    la[0].val.clusterDim.x = (unsigned)csize;
    la[0].val.clusterDim.y = 1;
    la[0].val.clusterDim.z = 1;
    cfg.attrs = la;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, v, W, N, N_pad, Kpad, R, t0, A_hi, A_lo, B_hi, B_lo, scaleA,
                              scaleB, status, wait_limit);
}

cudaError_t launch_shc_tc_pack(const float *v, const float *W, int N, int N_pad, int K, int Kpad, int R,
                               long long t0, int split, void *A_hi, void *A_lo, void *B_hi, void *B_lo,
                               float *scaleA, float *scaleB, int *status, long long wait_limit,
                               cudaStream_t s) {
    if (K <= 0) return cudaSuccess;
    const int per4 = PACK_THREADS * 4, per8 = PACK_THREADS * 8;
    const bool bf = split == SPLIT_BF16;
    const bool vec = N % 4 == 0 && ((reinterpret_cast<uintptr_t>(v) | reinterpret_cast<uintptr_t>(W)) & 15) == 0;
    if (vec && N <= 8 * 1024) {   // bulk copies into shared memory, 1024 atoms per CTA
        return bf ? launch_pack_bulk<SPLIT_BF16, 256>(v, W, N, N_pad, K, Kpad, R, t0, A_hi, A_lo, B_hi, B_lo, scaleA, scaleB, status, wait_limit, s)
                  : launch_pack_bulk<SPLIT_FP16, 256>(v, W, N, N_pad, K, Kpad, R, t0, A_hi, A_lo, B_hi, B_lo, scaleA, scaleB, status, wait_limit, s);
    }
    if (vec && N <= 8 * 2048) {   // 2048 atoms per CTA
        return bf ? launch_pack_bulk<SPLIT_BF16, 512>(v, W, N, N_pad, K, Kpad, R, t0, A_hi, A_lo, B_hi, B_lo, scaleA, scaleB, status, wait_limit, s)
                  : launch_pack_bulk<SPLIT_FP16, 512>(v, W, N, N_pad, K, Kpad, R, t0, A_hi, A_lo, B_hi, B_lo, scaleA, scaleB, status, wait_limit, s);
    }
    if (N <= 8 * per4) {   // clusters of up to 8 CTAs, 4 atoms per thread
        const int cs = (N + per4 - 1) / per4;
        return bf ? launch_pack_cluster<SPLIT_BF16, 4>(cs, v, W, N, N_pad, K, Kpad, R, t0, A_hi, A_lo, B_hi, B_lo, scaleA, scaleB, s)
                  : launch_pack_cluster<SPLIT_FP16, 4>(cs, v, W, N, N_pad, K, Kpad, R, t0, A_hi, A_lo, B_hi, B_lo, scaleA, scaleB, s);
    }
    if (N <= 8 * per8) {   // 8 atoms per thread
        const int cs = (N + per8 - 1) / per8;
        return bf ? launch_pack_cluster<SPLIT_BF16, 8>(cs, v, W, N, N_pad, K, Kpad, R, t0, A_hi, A_lo, B_hi, B_lo, scaleA, scaleB, s)
                  : launch_pack_cluster<SPLIT_FP16, 8>(cs, v, W, N, N_pad, K, Kpad, R, t0, A_hi, A_lo, B_hi, B_lo, scaleA, scaleB, s);
    }
    if (bf)
        shc_tc_pack_kernel<SPLIT_BF16><<<K, PACK_THREADS, 0, s>>>(v, W, N, N_pad, Kpad, R, t0, A_hi,
                                                                  A_lo, B_hi, B_lo, scaleA, scaleB);
    else
        shc_tc_pack_kernel<SPLIT_FP16><<<K, PACK_THREADS, 0, s>>>(v, W, N, N_pad, Kpad, R, t0, A_hi,
                                                                  A_lo, B_hi, B_lo, scaleA, scaleB);
    return cudaGetLastError();
}

size_t shc_tc_smem_bytes() { return ST_SMEM; }

cudaLaunchConfig_t shc_tc_config(int grid, cudaLaunchAttribute *attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    cfg.blockDim = dim3(ST_THREADS, 1, 1);
    cfg.dynamicSmemBytes = ST_SMEM;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

cudaError_t shc_tc_set_attr() {
    static cudaError_t e = cudaFuncSetAttribute(shc_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, ST_SMEM);
    return e;
}

cudaError_t launch_shc_tc(const ShcTcParams &p, cudaStream_t s) {
    cudaError_t e = shc_tc_set_attr();
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = shc_tc_config(9 * p.n_pairs * p.splits, attr);   // n_pairs is even
    cfg.stream = s;
    return cudaLaunchKernelEx(&cfg, shc_tc_kernel, p);
}

int shc_tc_max_clusters() {
    if (shc_tc_set_attr() != cudaSuccess) return 0;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = shc_tc_config(2, attr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, shc_tc_kernel, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

void launch_shc_tc_reduce(const ShcTcParams &p, double *Ksum, cudaStream_t s) {
    dim3 grid((p.nc + 127) / 128, 9);
    shc_tc_reduce_kernel<<<grid, 128, 0, s>>>(p, Ksum);
}

}  // namespace mhc
