// Bin-bin cross-correlations of the binned modal heat currents (the mode-mode correlations
// the paper notes GKMA allows; at one bin per mode they are exactly those).  Same lag
// convention as Eq. 17: the first current is lagged, the second sits at the time origin.
//   X[l][j][i] += sum_{k: t0+k-l >= 0} J_i(t0 + k) J_j(t0 + k - l),   i = 3b+mu, j = 3b'+nu
//
// For each lag this is a dense contraction over the block's K steps,
//   X_l = A B_l^T,  A[i][k] = J_i(t0 + k),  B_l[j][k] = J_j(t0 + k - l),
// run on the tensor cores.  Both operands are windows of one array per block,
//   W[j][u] = J_j(t0 - (L - 1) + u),  u in [0, K + L - 1)  (zero before the run starts),
// A = W shifted by L - 1 and B_l = W shifted by L - 1 - l.  A TMA tile must start on a 16-byte
// boundary (8 FP16 elements), so the window kernel writes eight copies, copy c shifted left by
// c elements; a tile at shift m comes from copy m mod 8 at x = m - (m mod 8) + 64 kb.  Each row
// of W gets a power-of-two scale (its scaled maximum below 2^14) and is split into FP16 hi + lo:
//   A B^T ~= A_hi B_lo^T + A_lo B_hi^T + A_hi B_hi^T  (three tcgen05.mma per 16 steps)
// accumulated in TMEM over chunks of 128 steps and promoted into FP32 registers (the
// accumulation-precision scheme of the modal kernel).  The scaled products are added into the
// state as unevaluated float pairs (TwoSum, ~48 bits): GB300's FP64 pipe would spend ~30 us a
// block on the FP64 adds alone.  The state is X[l][j][i] (i fastest) so that the 32 lanes of an
// epilogue warp (32 consecutive rows i) update 256 contiguous bytes.
#include <cuda_fp16.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace mhc {

namespace {

constexpr int XC_BK = 64;                                 // steps per k-block (128-byte rows)
constexpr int XC_CHUNK_KB = 2;                            // k-blocks per promotion chunk
constexpr int XC_STAGES = 2;
constexpr int XC_A_BYTES = 128 * XC_BK * 2;               // 128 rows i
constexpr int XC_B_BYTES = XC_NJ_MAX * XC_BK * 2;         // up to 192 rows j
constexpr int XC_STAGE_BYTES = 2 * XC_A_BYTES + 2 * XC_B_BYTES;
constexpr int XC_TILE_BYTES = XC_STAGES * XC_STAGE_BYTES;
constexpr int XC_SMEM = XC_TILE_BYTES + 256 + 1024;       // barriers + alignment slack
constexpr int XC_EPI_WARPS = 8;                           // two per TMEM lane quarter
constexpr int XC_THREADS = 128 + 32 * XC_EPI_WARPS;
constexpr uint32_t XC_TMEM_COLS = 512;                    // chunk buffers at columns 0 and 256
constexpr uint32_t XC_SBO = 8 * XC_BK * 2;                // 8-row core group of 128-byte rows

// (s, c) += x as an unevaluated float pair (TwoSum; _rn keeps it from being contracted)
__device__ __forceinline__ void xc_pair_add(float &s, float &c, float x) {
    const float t = __fadd_rn(s, x);
    const float bp = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
    s = t;
    c = __fadd_rn(c, e);
}

// ring[(t0 + k) mod R][j] = Jb[k][j]: the block's binned currents join the history ring
__global__ void jb_ring_store_kernel(const float *__restrict__ Jb, int K, int n, float *ring,
                                     int R, long long t0_host, const long long *t0_dev) {
    const long long t0 = t0_dev ? *t0_dev : t0_host;
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= (long long)K * n) return;
    const long long k = q / n, j = q - k * n;
    ring[((t0 + k) % R) * n + j] = Jb[q];
}

// One CTA per row j < n: the row's scale from the maximum of |W[j][u]| over the window, then
// the eight shifted FP16 hi/lo copies, Whi/Wlo[(c rows_pad + j) U_pad + u] = split(W[j][u + c]).
constexpr int XW_THREADS = 256;
__global__ void __launch_bounds__(XW_THREADS) xc_window_kernel(const float *__restrict__ ring, int R,
                                                               int n, int K, int L, int U_pad,
                                                               int rows_pad, long long t0_host,
                                                               const long long *t0_dev,
                                                               uint16_t *Whi, uint16_t *Wlo,
                                                               float *inv_scale) {
    const int j = blockIdx.x;
    const long long t0 = t0_dev ? *t0_dev : t0_host;
    const long long tw0 = t0 - (L - 1);
    const int Uw = K + L - 1;
    const int base = (int)(((tw0 % R) + R) % R);   // ring row of u = 0
    auto value = [&](int u) -> float {             // W[j][u]
        if (u >= Uw || tw0 + u < 0) return 0.f;
        int r = base + u;
        if (r >= R) r -= R;                        // u < Uw <= R
        return ring[(size_t)r * n + j];
    };
    float m = 0.f;
    for (int u = threadIdx.x; u < Uw; u += XW_THREADS) m = fmaxf(m, fabsf(value(u)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(FULL_MASK, m, o));
    __shared__ float s_m[XW_THREADS / 32];
    __shared__ float s_mul;
    if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float mm = 0.f;
        for (int w = 0; w < XW_THREADS / 32; ++w) mm = fmaxf(mm, s_m[w]);
        int sc = 0;
        if (mm > 0.f && isfinite(mm)) {
            int e;
            frexpf(mm, &e);            // mm < 2^e
            sc = min(14 - e, 60);      // scaled maximum < 2^14; products of two inverse scales stay normal
        }
        s_mul = ldexpf(1.f, sc);
        inv_scale[j] = ldexpf(1.f, -sc);
    }
    __syncthreads();
    const float mul = s_mul;
    for (int q = threadIdx.x; q < 8 * U_pad; q += XW_THREADS) {
        const int c = q / U_pad, u = q - c * U_pad;
        const float x = value(u + c) * mul;
        const __half hv = __float2half_rn(x);
        const size_t o = ((size_t)c * rows_pad + j) * U_pad + u;
        Whi[o] = __half_as_ushort(hv);
        Wlo[o] = __half_as_ushort(__float2half_rn(x - __half2float(hv)));
    }
}

// Persistent: CTA c owns row tile it = c / cpt (128 rows i) and the items (column tile jt,
// lag l) numbered c mod cpt, + cpt, ...  Warp roles as in the modal kernel:
//   warp 0      TMA producer (one lane): A (rows i) and B (rows j) tiles of each k-block
//   warp 1      MMA issuer (one lane): three tcgen05.mma per 16 steps into a chunk buffer
//   warp 2      TMEM allocator
//   warps 4..11 promotion + epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (rows i) and
//               the half (w - 4) / 4 of the nj columns j; at the end of an item it scales the
//               sums and adds them into the float-pair state
// Every barrier wait is bounded; a wait that runs out sets DEV_TIMEOUT, raises a CTA-wide
// abort flag, and the CTA drains its copies and MMAs, frees TMEM and exits.
__global__ void __launch_bounds__(XC_THREADS, 1) xc_tc_kernel(const __grid_constant__ XcTcParams p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                ~uintptr_t(1023));
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + XC_TILE_BYTES);
    uint64_t *full = bars;                      // [STAGES] TMA landed
    uint64_t *empty = bars + XC_STAGES;         // [STAGES] MMAs done reading
    uint64_t *acc_full = bars + 2 * XC_STAGES;  // [2] chunk accumulator ready
    uint64_t *acc_empty = acc_full + 2;         // [2] chunk accumulator promoted
    uint64_t *done_bar = acc_empty + 2;         // final MMA drain
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done_bar + 1);
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int it = blockIdx.x / p.cpt, r0 = blockIdx.x % p.cpt;
    const int n_items = p.n_jt * p.L;
    const int cA = (p.L - 1) & 7;   // A = W shifted by L - 1

    if (threadIdx.x == 0) {
        for (int s = 0; s < XC_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], XC_EPI_WARPS);
        }
        mbar_init(done_bar, 1);
        *abort = 0;
        fence_mbar_init();
    }
    if (warp == 2) {
        tmem_alloc(tmem_slot, XC_TMEM_COLS);
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
        const uint64_t pol = l2_policy_evict_last();   // the window copies are re-read by every lag
        const uint32_t bytes = 2 * XC_A_BYTES + 2 * (uint32_t)p.nj * XC_BK * 2;
        uint32_t issued_phase[XC_STAGES];
        bool issued[XC_STAGES];
        for (int s = 0; s < XC_STAGES; ++s) issued[s] = false;
        int stage = 0;
        uint32_t phase = 0;
        bool ok = true;
        const int yA = cA * p.rows_pad + it * 128;
        for (int q = r0; ok && q < n_items; q += p.cpt) {
            const int jt = q / p.L, l = q - jt * p.L;
            const int m = p.L - 1 - l, cB = m & 7;   // B_l = W shifted by m
            const int yB = cB * p.rows_pad + jt * p.nj;
            for (int kb = 0; kb < p.n_kb; ++kb) {
                if (!mbar_wait(&empty[stage], phase ^ 1u, abort, p.wait_limit)) { ok = false; break; }
                uint8_t *sa = smem + stage * XC_STAGE_BYTES;
                mbar_arrive_expect_tx(&full[stage], bytes);
                const int xA = kb * XC_BK + (p.L - 1) - cA, xB = kb * XC_BK + m - cB;
                tma_load_2d(sa, &p.tmA_hi, &full[stage], xA, yA, pol);
                tma_load_2d(sa + XC_A_BYTES, &p.tmA_lo, &full[stage], xA, yA, pol);
                tma_load_2d(sa + 2 * XC_A_BYTES, &p.tmB_hi, &full[stage], xB, yB, pol);
                tma_load_2d(sa + 2 * XC_A_BYTES + XC_B_BYTES, &p.tmB_lo, &full[stage], xB, yB, pol);
                issued[stage] = true;
                issued_phase[stage] = phase;
                if (++stage == XC_STAGES) { stage = 0; phase ^= 1u; }
            }
        }
        if (!ok) {
            *abort = 1;
            set_status(p.status, DEV_TIMEOUT);
        }
        for (int s = 0; s < XC_STAGES; ++s)   // every issued copy lands before the CTA exits
            if (issued[s]) {
                const long long t0 = clock64();
                while (!mbar_try_wait(&full[s], issued_phase[s]) && clock64() - t0 < p.wait_limit) {
                }
            }
    } else if (warp == 1 && lane == 0) {
        // ------------------------------------------------------------ MMA issuer
        int stage = 0, abuf = 0;
        uint32_t phase = 0, aphase = 0;
        bool ok = true;
        const uint32_t smem0 = smem_u32(smem);
        for (int q = r0; ok && q < n_items; q += p.cpt) {
            for (int kb0 = 0; ok && kb0 < p.n_kb; kb0 += XC_CHUNK_KB) {
                if (!mbar_wait(&acc_empty[abuf], aphase ^ 1u, abort, p.wait_limit)) { ok = false; break; }
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(abuf * 256);
                const int kb1 = min(kb0 + XC_CHUNK_KB, p.n_kb);
                for (int kb = kb0; kb < kb1; ++kb) {
                    if (!mbar_wait(&full[stage], phase, abort, p.wait_limit)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t a_hi = smem0 + stage * XC_STAGE_BYTES;
                    const uint32_t a_lo = a_hi + XC_A_BYTES;
                    const uint32_t b_hi = a_hi + 2 * XC_A_BYTES;
                    const uint32_t b_lo = b_hi + XC_B_BYTES;
#pragma unroll
                    for (int kk = 0; kk < XC_BK / 16; ++kk) {
                        const uint32_t off = kk * 32;
                        const uint64_t dah = smem_desc_kmajor(a_hi + off, XC_SBO, 2u);
                        const uint64_t dal = smem_desc_kmajor(a_lo + off, XC_SBO, 2u);
                        const uint64_t dbh = smem_desc_kmajor(b_hi + off, XC_SBO, 2u);
                        const uint64_t dbl = smem_desc_kmajor(b_lo + off, XC_SBO, 2u);
                        umma_f16(d_tmem, dah, dbl, p.idesc, (kb != kb0 || kk != 0) ? 1u : 0u);
                        umma_f16(d_tmem, dal, dbh, p.idesc, 1u);
                        umma_f16(d_tmem, dah, dbh, p.idesc, 1u);
                    }
                    umma_commit(&empty[stage]);
                    if (++stage == XC_STAGES) { stage = 0; phase ^= 1u; }
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
        umma_commit(done_bar);
        const long long t0 = clock64();
        while (!mbar_try_wait(done_bar, 0) && clock64() - t0 < p.wait_limit) {
        }
    } else if (warp >= 4) {
        // ------------------------------------------------------------ promotion + epilogue
        const int e = warp - 4, qw = e & 3, half = e >> 2;
        const int nh = p.nj >> 1;   // columns of this warp: a multiple of 16, <= 96
        const int i = it * 128 + qw * 32 + lane;
        const float si = i < p.n ? p.inv_scale[i] : 0.f;
        int abuf = 0;
        uint32_t aphase = 0;
        bool ok = true;
        for (int q = r0; ok && q < n_items; q += p.cpt) {
            const int jt = q / p.L, l = q - jt * p.L;
            const int j0 = jt * p.nj + half * nh;
            const int jn = min(nh, p.n - j0);   // columns of this warp inside the matrix
            // the item's state columns X[l][j][i0 .. i0+31]: 256 bytes (two L2 lines) a column,
            // prefetched into L2 while the item's MMAs run
            float2 *xcol = p.X + ((size_t)l * p.n + j0) * p.n + (it * 128 + qw * 32 + lane);
            if ((lane & 15) == 0 && it * 128 + qw * 32 + lane < p.n)
                for (int c = 0; c < jn; ++c) asm volatile("prefetch.global.L2 [%0];" ::"l"(xcol + (size_t)c * p.n));
            float acc[XC_NJ_MAX / 2];
#pragma unroll
            for (int c = 0; c < XC_NJ_MAX / 2; ++c) acc[c] = 0.f;
            for (int kb0 = 0; kb0 < p.n_kb; kb0 += XC_CHUNK_KB) {
                if (!mbar_wait(&acc_full[abuf], aphase, abort, p.wait_limit)) { ok = false; break; }
                tc_fence_after();
                const uint32_t tbase = tmem_base + ((uint32_t)(qw * 32) << 16) +
                                       (uint32_t)(abuf * 256 + half * nh);
#pragma unroll
                for (int c16 = 0; c16 < XC_NJ_MAX / 32; ++c16) {
                    if (16 * c16 >= nh) break;   // warp-uniform
                    uint32_t r[16];
                    tmem_ld_32x32b_x16(tbase + (uint32_t)(16 * c16), r);
                    tmem_ld_wait();
#pragma unroll
                    for (int u = 0; u < 16; ++u) acc[16 * c16 + u] += __uint_as_float(r[u]);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acc_empty[abuf]);
                if (++abuf == 2) { abuf = 0; aphase ^= 1u; }
            }
            if (!ok) break;
            if (i >= p.n) continue;
            // read-modify-write in batches of 16 columns, all loads of a batch issued before its
            // stores (one column's store could alias the next column's load for the compiler)
#pragma unroll
            for (int c0 = 0; c0 < XC_NJ_MAX / 2; c0 += 16) {
                if (c0 >= jn) break;   // warp-uniform
                float2 st[16];
#pragma unroll
                for (int u = 0; u < 16; ++u)
                    if (c0 + u < jn) st[u] = __ldcg(xcol + (size_t)(c0 + u) * p.n);
#pragma unroll
                for (int u = 0; u < 16; ++u)
                    if (c0 + u < jn) {
                        const float v = acc[c0 + u] * (si * __ldg(p.inv_scale + j0 + c0 + u));
                        xc_pair_add(st[u].x, st[u].y, v);
                        __stcg(xcol + (size_t)(c0 + u) * p.n, st[u]);
                    }
            }
        }
        if (!ok) {
            *abort = 1;
            set_status(p.status, DEV_TIMEOUT);
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 2) tmem_dealloc(tmem_base, XC_TMEM_COLS);
}

// out[((b nb + b2) 3 + mu) 3 + nu][l] = X[l][3b2+nu][3b+mu] (float pair -> FP64)
__global__ void xcorr_transpose_kernel(const float2 *__restrict__ X, int nb, int L, double *out) {
    const int n = 3 * nb;
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= (long long)n * n * L) return;
    const long long l = q % L, r = q / L;   // r = ((b nb + b2) 3 + mu) 3 + nu
    const int nu = (int)(r % 3), mu = (int)((r / 3) % 3);
    const long long bb = r / 9;
    const int b2 = (int)(bb % nb), b = (int)(bb / nb);
    const float2 v = X[(size_t)l * n * n + (size_t)(3 * b2 + nu) * n + 3 * b + mu];
    out[q] = (double)v.x + (double)v.y;
}

}  // namespace

void xcorr_plan(int nb, int L, int k_max, int nsm, XcPlan &pl) {
    pl.n = 3 * nb;
    pl.nj = pl.n <= XC_NJ_MAX ? (pl.n + 31) / 32 * 32 : XC_NJ_MAX;
    pl.n_jt = (pl.n + pl.nj - 1) / pl.nj;
    pl.n_it = (pl.n + 127) / 128;
    pl.rows_pad = std::max(pl.n_it * 128, pl.n_jt * pl.nj);
    pl.U_pad = (k_max + L - 1 + XC_BK - 1) / XC_BK * XC_BK;
    const long long items = (long long)pl.n_jt * L;
    pl.cpt = (int)std::max(1ll, std::min<long long>(nsm / pl.n_it, items));
    pl.grid = pl.n_it * pl.cpt;
}

int xcorr_make_maps(const XcPlan &pl, const void *Whi, const void *Wlo, XcTcParams &p) {
    const uint64_t rows = 8ull * pl.rows_pad, cols = (uint64_t)pl.U_pad;
    int r = tc_make_tmap(&p.tmA_hi, Whi, rows, cols, cols, 128, XC_BK);
    if (!r) r = tc_make_tmap(&p.tmA_lo, Wlo, rows, cols, cols, 128, XC_BK);
    if (!r) r = tc_make_tmap(&p.tmB_hi, Whi, rows, cols, cols, (uint32_t)pl.nj, XC_BK);
    if (!r) r = tc_make_tmap(&p.tmB_lo, Wlo, rows, cols, cols, (uint32_t)pl.nj, XC_BK);
    p.n = pl.n;
    p.nj = pl.nj;
    p.n_jt = pl.n_jt;
    p.rows_pad = pl.rows_pad;
    p.cpt = pl.cpt;
    p.idesc = idesc_f16(0u, 128u, (uint32_t)pl.nj);
    return r;
}

cudaError_t xcorr_prepare() {
    static cudaError_t e = cudaFuncSetAttribute(xc_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                XC_SMEM);
    return e;
}

void launch_jb_ring_store(const float *Jb, int K, int nb, float *ring, int R, long long t0,
                          const long long *t0_dev, cudaStream_t s) {
    const long long total = (long long)K * nb * 3;
    if (total <= 0) return;
    jb_ring_store_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(Jb, K, 3 * nb, ring, R, t0, t0_dev);
}

cudaError_t launch_bin_xcorr(const XcPlan &pl, XcTcParams p, const float *ring, int R, int K,
                             long long t0, const long long *t0_dev, void *Whi, void *Wlo,
                             cudaStream_t s) {
    if (p.L <= 0 || K <= 0 || pl.n <= 0) return cudaSuccess;
    if (K + p.L - 1 > R || K + p.L - 1 > pl.U_pad) return cudaErrorInvalidValue;
    xc_window_kernel<<<pl.n, XW_THREADS, 0, s>>>(ring, R, pl.n, K, p.L, pl.U_pad, pl.rows_pad, t0,
                                                 t0_dev, static_cast<uint16_t *>(Whi),
                                                 static_cast<uint16_t *>(Wlo),
                                                 const_cast<float *>(p.inv_scale));
    const cudaError_t attr = xcorr_prepare();
    if (attr != cudaSuccess) return attr;
    p.n_kb = (K + XC_BK - 1) / XC_BK;
    xc_tc_kernel<<<pl.grid, XC_THREADS, XC_SMEM, s>>>(p);
    return cudaGetLastError();
}

void launch_xcorr_transpose(const float2 *X, int nb, int L, double *out, cudaStream_t s) {
    const long long total = 9ll * nb * nb * L;
    if (total <= 0) return;
    xcorr_transpose_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(X, nb, L, out);
}

}  // namespace mhc
