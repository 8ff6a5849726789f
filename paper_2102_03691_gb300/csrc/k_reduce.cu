// K3 bin finish + HNEMA sums (Eq. 19), K4 GKMA lag correlation (Eq. 17 integrand),
// K5 running Green-Kubo integral (Eq. 17) and the HNEMA normalisation (Eq. 19).
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace mhc {

namespace {

// ------------------------------------------------------------------ K3
// One CTA per bin, one thread per (step, component) of a 256-step pass: thread t handles
// component a = t % 3 and steps k = t/3 + 256 j.  J_b^a(k) = sum of the bin's partial slots in
// slot order; the HNEMA sums over the block's steps in FP64 with a fixed reduction tree
// (deterministic).  CTA 0 also sums the total current.
constexpr int BF_STEPS = 256;
constexpr int BF_THREADS = 3 * BF_STEPS;
__device__ __forceinline__ void bin_finish_body(const float *__restrict__ partials, int n_slots,
                                                const int *slot_begin, int B, int K, float *Jb,
                                                double *hsum, const double *Jtot, double *Jsum,
                                                int b) {
    const int a = threadIdx.x % 3, k0 = threadIdx.x / 3;
    const int s0 = slot_begin[b], s1 = slot_begin[b + 1];
    double acc = 0.0, acc_tot = 0.0;
    for (int k = k0; k < K; k += BF_STEPS) {
        const float *row = partials + ((size_t)k * 3 + a) * n_slots;
        float s = 0.f;
        for (int q = s0; q < s1; ++q) s += row[q];
        Jb[((size_t)k * B + b) * 3 + a] = s;
        acc += (double)s;
        if (b == 0) acc_tot += Jtot[3 * k + a];
    }
    __shared__ double red[2][BF_THREADS];
    red[0][threadIdx.x] = acc;
    red[1][threadIdx.x] = acc_tot;
    __syncthreads();
    for (int off = BF_STEPS / 2; off > 0; off >>= 1) {   // over k0, per component
        if (k0 < off) {
            red[0][threadIdx.x] += red[0][threadIdx.x + 3 * off];
            if (b == 0) red[1][threadIdx.x] += red[1][threadIdx.x + 3 * off];
        }
        __syncthreads();
    }
    if (threadIdx.x < 3) {
        hsum[b * 3 + threadIdx.x] += red[0][threadIdx.x];
        if (b == 0) Jsum[threadIdx.x] += red[1][threadIdx.x];
    }
}

// steps: the step counter to advance by K here (no later kernel of the push reads it), or null.
__global__ void __launch_bounds__(BF_THREADS) bin_finish_kernel(const float *__restrict__ partials,
                                                                int n_slots, const int *slot_begin,
                                                                int B, int K, float *Jb,
                                                                double *hsum, const double *Jtot,
                                                                double *Jsum, long long *steps) {
    if (steps && blockIdx.x == 0 && threadIdx.x == 0) *steps += K;
    bin_finish_body(partials, n_slots, slot_begin, B, K, Jb, hsum, Jtot, Jsum, blockIdx.x);
}

// All systems of a group in one launch: CTAs cta_begin[j] .. cta_begin[j+1) are system j's bins.
__global__ void __launch_bounds__(BF_THREADS) bin_finish_group_kernel(const __grid_constant__ FinishGroupArgs g) {
    int j = 0;
    while (j + 1 < g.n && (int)blockIdx.x >= g.cta_begin[j + 1]) ++j;
    if (g.advance && (int)blockIdx.x == g.cta_begin[j] && threadIdx.x == 0) *g.steps[j] += g.K[j];
    bin_finish_body(g.partials[j], g.n_slots[j], g.slot_begin[j], g.B[j], g.K[j], g.Jb[j],
                    g.hsum[j], g.Jtot[j], g.Jsum[j], (int)blockIdx.x - g.cta_begin[j]);
}

__global__ void advance_steps_group_kernel(const __grid_constant__ FinishGroupArgs g) {
    const int j = threadIdx.x;
    if (j < g.n) *g.steps[j] += g.K[j];
}

// ------------------------------------------------------------------ K4
// Register-tiled like a GEMM micro-kernel.  A CTA owns 32 consecutive lags (one per lane) and
// LC_ROWS rows (b, mu) of LC_ROWS / 3 bins; its W <= LC_WARPS warps take consecutive ranges of
// ceil(K / W) steps of the block.  Per step a thread loads its lag's total current J(t - l)
// (one 16-byte shared-memory load from the CTA's window of J samples) and the step's LC_ROWS
// binned currents (broadcast 16-byte loads) and does 3 LC_ROWS FMAs into FP32 partial sums over
// the warp's steps.  The warps' partials are then added in step order in an unevaluated float
// pair (TwoSum, ~48 bits; GB300's FP64 pipe is narrow) and each lag sum gets one FP64 add.
// At most 16 warps a CTA, so that two CTAs share an SM: one CTA's staging and final sums then
// overlap the other's FMAs, and a grid a little larger than the SM count (N = 512: 175 CTAs)
// still runs in one wave.
constexpr int LC_ROWS = 12;   // 4 bins x 3 components a thread
constexpr int LC_OUT = 3 * LC_ROWS;
constexpr int LC_WARPS = 16;

// (s, c) += x exactly as an unevaluated float pair (_rn keeps it from being contracted)
__device__ __forceinline__ void lc_pair_add(float &s, float &c, float x) {
    const float t = __fadd_rn(s, x);
    const float bp = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
    s = t;
    c = __fadd_rn(c, e);
}
__global__ void __launch_bounds__(32 * LC_WARPS, 2) lag_corr_kernel(const float *__restrict__ Jb,
                                                                    const double *__restrict__ Jring,
                                                                    int R, double *Csum, int K,
                                                                    int B, int L, long long t0_host,
                                                                    const long long *t0_dev,
                                                                    long long *steps,
                                                                    unsigned *ticket) {
    const long long t0 = t0_dev ? *t0_dev : t0_host;
    // staging: rows [K][LC_ROWS], then the J window [K + 31] as float4 (x, y, z, 0); after the
    // step loop the same space holds the warps' partials [warp][LC_OUT][32]
    extern __shared__ float4 lc_smem4[];
    float *sA = reinterpret_cast<float *>(lc_smem4);
    float4 *sW = lc_smem4 + (K * LC_ROWS) / 4;
    float *sP = reinterpret_cast<float *>(lc_smem4);
    const int l0 = blockIdx.x * 32;
    const int b0 = blockIdx.y * (LC_ROWS / 3);
    const int nthreads = blockDim.x;
    if (B % 4 == 0 && (reinterpret_cast<uintptr_t>(Jb) & 15) == 0) {
        // every bin group is whole and its 12 floats of a step start on a 16-byte boundary:
        // three asynchronous 16-byte copies a step, all in flight at once
        for (int q = threadIdx.x; q < 3 * K; q += nthreads) {
            const int k = q / 3, j = q - 3 * k;
            cp_async16(sA + k * LC_ROWS + 4 * j, Jb + ((size_t)k * B + b0) * 3 + 4 * j);
        }
    } else {
        for (int q = threadIdx.x; q < K * LC_ROWS; q += nthreads) {
            const int k = q / LC_ROWS, r = q % LC_ROWS, b = b0 + r / 3;
            sA[q] = b < B ? Jb[((size_t)k * B + b) * 3 + r % 3] : 0.f;
        }
    }
    // window entry w holds J(tw0 + w), tw0 = t0 - l0 - 31: lane l at step k reads w = k - l + 31.
    // Ring slot of entry w: (tw0 mod R) + w brought into [0, R) with 32-bit arithmetic (one
    // 64-bit remainder a thread instead of one an entry).
    const long long tw0 = t0 - l0 - 31;
    const int m0 = (int)(tw0 % R);   // in (-R, R)
    for (int w = threadIdx.x; w < K + 31; w += nthreads) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (tw0 + w >= 0) {
            int slot = m0 + w;
            if (slot < 0) slot += R;
            if (slot >= R) slot %= R;
            const double *src = Jring + (size_t)slot * 3;
            v = make_float4((float)src[0], (float)src[1], (float)src[2], 0.f);
        }
        sW[w] = v;
    }
    cp_async_wait_all();
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = nthreads >> 5;
    const int ks = (K + nwarps - 1) / nwarps;
    const int k_begin = min(K, ks * warp), k_end = min(K, k_begin + ks);
    float acc[LC_OUT];
#pragma unroll
    for (int o = 0; o < LC_OUT; ++o) acc[o] = 0.f;
    const float4 *wp = sW + (k_begin - lane + 31);
    const float4 *ap = reinterpret_cast<const float4 *>(sA) + k_begin * (LC_ROWS / 4);
#pragma unroll 4
    for (int k = k_begin; k < k_end; ++k) {
        const float4 j = *wp++;
        float x[LC_ROWS];
#pragma unroll
        for (int q = 0; q < LC_ROWS / 4; ++q) {
            const float4 a4 = ap[q];
            x[4 * q] = a4.x;
            x[4 * q + 1] = a4.y;
            x[4 * q + 2] = a4.z;
            x[4 * q + 3] = a4.w;
        }
        ap += LC_ROWS / 4;
#pragma unroll
        for (int r = 0; r < LC_ROWS; ++r) {
            acc[3 * r] = fmaf(x[r], j.x, acc[3 * r]);
            acc[3 * r + 1] = fmaf(x[r], j.y, acc[3 * r + 1]);
            acc[3 * r + 2] = fmaf(x[r], j.z, acc[3 * r + 2]);
        }
    }
    __syncthreads();   // staging no longer read: its space takes the partials
#pragma unroll
    for (int o = 0; o < LC_OUT; ++o) sP[(warp * LC_OUT + o) * 32 + lane] = acc[o];
    __syncthreads();
    for (int q = threadIdx.x; q < LC_OUT * 32; q += nthreads) {
        const int o = q >> 5, ln = q & 31;
        const int l = l0 + ln, r = o / 3, b = b0 + r / 3;
        if (l >= L || b >= B) continue;
        double *dst = Csum + ((size_t)b * 9 + (r % 3) * 3 + o % 3) * L + l;
        const double old = *dst;   // in flight while the partials are added
        float s = 0.f, c = 0.f;
        for (int w = 0; w < nwarps; ++w) lc_pair_add(s, c, sP[(w * LC_OUT + o) * 32 + ln]);
        *dst = old + ((double)s + (double)c);
    }
    if (steps) {   // the last CTA to finish advances the step counter: every CTA has read it
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            if (atomicAdd(ticket, 1u) == gridDim.x * gridDim.y - 1) {
                *steps += K;
                *ticket = 0;
            }
        }
    }
}

int lag_corr_warps(int K) { return std::max(1, std::min(LC_WARPS, (K + 31) / 32)); }

size_t lag_corr_smem(int K) {
    const size_t staging = (size_t)K * LC_ROWS * sizeof(float) + (size_t)(K + 31) * sizeof(float4);
    const size_t partials = (size_t)lag_corr_warps(K) * LC_OUT * 32 * sizeof(float);
    return staging > partials ? staging : partials;
}

// ------------------------------------------------------------------ K5
// inv_count(l) = 1 / (T_s - l) (0 when no origin has lag l), computed once per read so that
// the rows below multiply instead of dividing (an FP64 division is ~8 instructions on a pipe
// GB300 keeps narrow).
__global__ void inv_counts_kernel(long long T_s, int L, double *inv) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l < L) inv[l] = T_s > l ? 1.0 / (double)(T_s - l) : 0.0;
}

// One CTA per (b, mu, nu) row, GK_THREADS threads, each owning per = ceil(L / GK_THREADS)
// consecutive lags.  C(l) = Csum(l) inv_count(l); the running trapezoid sum
// S(l) = sum_{1 <= l' <= l} (C(l'-1) + C(l')) comes from per-thread totals and a block-wide
// exclusive scan (warp shuffles, then the four warp totals: a fixed tree, deterministic);
// kappa(l) = (c dt / 2) S(l).  The window average runs over the lags l_lo .. l_hi (the host
// picks them with the same FP64 test on l dt as the oracle).  The pipe GB300 keeps narrow
// bounds the kernel, so each lag costs a few FP64 operations: C(l) is computed once and kept
// in registers when a thread owns at most GK_CACHE lags.
constexpr int GK_THREADS = 128;
constexpr int GK_CACHE = 8;
__device__ __forceinline__ double gk_block_exclusive_scan(double x, double *s_w) {   // all threads
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(FULL_MASK, v, o);
        if (lane >= o) v += y;
    }
    double ex = __shfl_up_sync(FULL_MASK, v, 1);   // exclusive within the warp
    if (lane == 0) ex = 0.0;
    if (lane == 31) s_w[w] = v;
    __syncthreads();
    double base = 0.0;
    for (int q = 0; q < w; ++q) base += s_w[q];
    __syncthreads();
    return base + ex;
}

__global__ void __launch_bounds__(GK_THREADS) gk_kappa_kernel(const double *Csum, int L,
                                                              const double *__restrict__ inv,
                                                              double coef_half, int l_lo, int l_hi,
                                                              double *kappa_tau, double *kappa_w) {
    __shared__ double s_w[GK_THREADS / 32];
    const int r = blockIdx.x;
    const double *cs = Csum + (size_t)r * L;
    const int per = (L + GK_THREADS - 1) / GK_THREADS;
    const int l0 = min(L, threadIdx.x * per), l1 = min(L, l0 + per);
    const double c_before = (l0 > 0 && l0 < l1) ? cs[l0 - 1] * inv[l0 - 1] : 0.0;
    double cc[GK_CACHE];
    double tot = 0.0, prev = c_before;
    if (per <= GK_CACHE) {
#pragma unroll
        for (int u = 0; u < GK_CACHE; ++u) {
            const int l = l0 + u;
            cc[u] = l < l1 ? cs[l] * inv[l] : 0.0;
            if (l < l1) {
                if (l > 0) tot += prev + cc[u];
                prev = cc[u];
            }
        }
    } else {
        for (int l = l0; l < l1; ++l) {
            const double c = cs[l] * inv[l];
            if (l > 0) tot += prev + c;
            prev = c;
        }
    }
    double acc = gk_block_exclusive_scan(tot, s_w);
    double wsum = 0.0;
    prev = c_before;
    auto emit = [&](int l, double c) {
        if (l > 0) acc += prev + c;
        prev = c;
        const double kap = coef_half * acc;
        if (kappa_tau) kappa_tau[(size_t)r * L + l] = kap;
        if (l >= l_lo && l <= l_hi) wsum += kap;
    };
    if (per <= GK_CACHE) {
#pragma unroll
        for (int u = 0; u < GK_CACHE; ++u)
            if (l0 + u < l1) emit(l0 + u, cc[u]);
    } else {
        for (int l = l0; l < l1; ++l) emit(l, cs[l] * inv[l]);
    }
    // window average: block sum of wsum (fixed tree)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wsum += __shfl_down_sync(FULL_MASK, wsum, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = wsum;
    __syncthreads();
    if (threadIdx.x == 0 && kappa_w) {
        double t = 0.0;
        for (int q = 0; q < GK_THREADS / 32; ++q) t += s_w[q];
        const int n = l_hi >= l_lo ? l_hi - l_lo + 1 : 0;
        kappa_w[r] = n > 0 ? t / n : 0.0;
    }
}

// Window average alone (no kappa(tau) wanted): with S(l) the running trapezoid sum above,
//   sum_{l = l_lo..l_hi} S(l) = sum_m C(m) w(m),  w(m) = [m >= 1] cnt(m) + cnt(m + 1),
// cnt(x) = #{l in [l_lo, l_hi] : l >= x} (C(m) enters S(l) as the right end of the step m-1 -> m
// for l >= m >= 1 and as the left end of the step m -> m+1 for l >= m+1).  The integer weights
// and the reciprocal counts are folded into one table tw(m) = inv(m) w(m), so a row takes one
// FP64 FMA a lag instead of the scan's few FP64 operations a lag on GB300's narrow FP64 pipe.
__device__ __forceinline__ double gk_window_weight(long long T_s, int m, int l_lo, int l_hi) {
    const auto cnt = [&](int x) {
        const int lo = max(x, l_lo);
        return l_hi >= lo ? l_hi - lo + 1 : 0;
    };
    const double inv = T_s > m ? 1.0 / (double)(T_s - m) : 0.0;
    return inv * (double)((m >= 1 ? cnt(m) : 0) + cnt(m + 1));
}

__global__ void gk_window_weights_kernel(long long T_s, int L, int l_lo, int l_hi, double *tw) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < L) tw[m] = gk_window_weight(T_s, m, l_lo, l_hi);
}

// One warp per row, GK_ROWS rows a CTA: kappa_w = scale sum_m Csum(m) tw(m) (lanes stride the
// lags; fixed tree).  tw null: each CTA first builds the table in shared memory (L FP64
// divisions spread over its threads), cheaper than a launch of its own while the grid is about
// one CTA an SM; larger grids (the bin-bin read) take the table from one weights launch.
constexpr int GK_ROWS = 8;
__global__ void __launch_bounds__(32 * GK_ROWS) gk_window_kernel(const double *Csum, int rows, int L,
                                                                 const double *__restrict__ tw,
                                                                 long long T_s, int l_lo, int l_hi,
                                                                 double scale, double *kappa_w) {
    extern __shared__ double gk_tw[];
    if (!tw) {
        for (int m = threadIdx.x; m < L; m += blockDim.x) gk_tw[m] = gk_window_weight(T_s, m, l_lo, l_hi);
        __syncthreads();
        tw = gk_tw;
    }
    const int r = blockIdx.x * GK_ROWS + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (r >= rows) return;
    const double *cs = Csum + (size_t)r * L;
    double acc = 0.0;
    for (int m = lane; m < L; m += 32) acc = fma(cs[m], tw[m], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(FULL_MASK, acc, o);
    if (lane == 0) kappa_w[r] = scale * acc;
}

__global__ void hnema_finalize_kernel(const double *hsum, int n, long long T_s, double coef,
                                      double *mean, double *kappa) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const double m = T_s > 0 ? hsum[q] / (double)T_s : 0.0;
    if (mean) mean[q] = m;
    if (kappa) kappa[q] = m * coef;
}

__global__ void hnema_finalize_group_kernel(const HnemaGroupArgs a, double *mean, double *kappa) {
    const int j = blockIdx.y;
    if (j >= a.n) return;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < a.nb[j]; q += gridDim.x * blockDim.x) {
        const double m = a.T_s[j] > 0 ? a.hsum[j][q] / (double)a.T_s[j] : 0.0;
        if (mean) mean[a.off[j] + q] = m;
        if (kappa) kappa[a.off[j] + q] = m * a.coef[j];
    }
}

__global__ void advance_steps_kernel(long long *steps, int K) { *steps += K; }

__global__ void lag_counts_kernel(long long T_s, int L, long long *count) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l < L) count[l] = T_s > l ? T_s - l : 0;
}

}  // namespace

void launch_bin_finish(const float *partials, int n_slots, const int *slot_begin, int B, int K,
                       float *Jb, double *hsum, const double *Jtot, double *Jsum, long long *steps,
                       cudaStream_t s) {
    if (B <= 0 || K <= 0) return;
    // launched plainly: as a programmatic dependent it cost the N = 512 GKMA step ~5 us
    bin_finish_kernel<<<B, BF_THREADS, 0, s>>>(partials, n_slots, slot_begin, B, K, Jb, hsum, Jtot,
                                               Jsum, steps);
}

namespace {
size_t lc_sm_set = 48 * 1024;   // the largest dynamic shared memory opted into so far
// the per-CTA weight table: up to two CTAs an SM and a table within the default 48 KB
constexpr int GK_TABLE_CTAS = 304;
constexpr int GK_TABLE_LAGS = 6144;
}

cudaError_t lag_corr_prepare(int k_max) {
    const size_t sm = lag_corr_smem(k_max);
    if (sm <= lc_sm_set) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(lag_corr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)sm);
    if (e == cudaSuccess) lc_sm_set = sm;
    return e;
}

void launch_bin_finish_group(FinishGroupArgs g, cudaStream_t s) {
    if (g.n < 1) return;
    g.cta_begin[0] = 0;
    for (int j = 0; j < g.n; ++j) g.cta_begin[j + 1] = g.cta_begin[j] + (g.K[j] > 0 ? g.B[j] : 0);
    if (g.cta_begin[g.n] > 0) bin_finish_group_kernel<<<g.cta_begin[g.n], BF_THREADS, 0, s>>>(g);
}

void launch_advance_steps_group(const FinishGroupArgs &g, cudaStream_t s) {
    if (g.n >= 1) advance_steps_group_kernel<<<1, 32, 0, s>>>(g);
}

void launch_lag_corr(const float *Jb, const double *Jring, int R, double *Csum, int K, int B,
                     int L, long long t0, const long long *t0_dev, long long *steps,
                     unsigned *ticket, cudaStream_t s) {
    if (L <= 0 || K <= 0 || B <= 0) return;
    dim3 grid((L + 31) / 32, (B + LC_ROWS / 3 - 1) / (LC_ROWS / 3));
    const int threads = 32 * lag_corr_warps(K);
    const size_t sm = lag_corr_smem(K);
    if (sm > lc_sm_set && lag_corr_prepare(K) != cudaSuccess)
        return;   // the launch is skipped; the caller's cudaGetLastError reports the failure
    lag_corr_kernel<<<grid, threads, sm, s>>>(Jb, Jring, R, Csum, K, B, L, t0, t0_dev, steps,
                                              ticket);
}

int launch_gk_kappa(const double *Csum, int B, int L, long long T_s, double coef_dt,
                    double tau_lo, double tau_hi, double dt, double *kappa_tau, double *kappa_w,
                    double *inv_scratch, cudaStream_t s) {
    if (L <= 0 || B <= 0) return 0;
    // the window's lags: l dt in [tau_lo, tau_hi], tested in FP64 as the oracle tests it
    int l_lo = L, l_hi = -1;
    for (int l = 0; l < L; ++l) {
        const double tau = l * dt;
        if (tau >= tau_lo && tau <= tau_hi) {
            l_lo = std::min(l_lo, l);
            l_hi = l;
        }
    }
    if (!kappa_tau) {   // the window average alone
        const int n = l_hi >= l_lo ? l_hi - l_lo + 1 : 0;
        const int rows = B * 9;
        const int ctas = (rows + GK_ROWS - 1) / GK_ROWS;
        const double scale = n > 0 ? 0.5 * coef_dt / n : 0.0;
        if (ctas <= GK_TABLE_CTAS && L <= GK_TABLE_LAGS) {   // each CTA builds the table
            gk_window_kernel<<<ctas, 32 * GK_ROWS, sizeof(double) * L, s>>>(
                Csum, rows, L, nullptr, T_s, l_lo, l_hi, scale, kappa_w);
            return 1;
        }
        gk_window_weights_kernel<<<(L + 255) / 256, 256, 0, s>>>(T_s, L, l_lo, l_hi, inv_scratch);
        gk_window_kernel<<<ctas, 32 * GK_ROWS, 0, s>>>(Csum, rows, L, inv_scratch, T_s, l_lo, l_hi,
                                                       scale, kappa_w);
        return 2;
    }
    inv_counts_kernel<<<(L + 255) / 256, 256, 0, s>>>(T_s, L, inv_scratch);
    gk_kappa_kernel<<<B * 9, GK_THREADS, 0, s>>>(Csum, L, inv_scratch, 0.5 * coef_dt, l_lo, l_hi,
                                                 kappa_tau, kappa_w);
    return 2;
}

void launch_hnema_finalize(const double *hsum, int B, long long T_s, double coef, double *mean,
                           double *kappa, cudaStream_t s) {
    const int n = B * 3;
    hnema_finalize_kernel<<<(n + 127) / 128, 128, 0, s>>>(hsum, n, T_s, coef, mean, kappa);
}

void launch_hnema_finalize_group(const HnemaGroupArgs &a, double *mean, double *kappa,
                                 cudaStream_t s) {
    hnema_finalize_group_kernel<<<dim3(4, a.n), 128, 0, s>>>(a, mean, kappa);
}

void launch_advance_steps(long long *steps, int K, cudaStream_t s) {
    advance_steps_kernel<<<1, 1, 0, s>>>(steps, K);
}

void launch_lag_counts(long long T_s, int L, long long *count, cudaStream_t s) {
    if (L <= 0) return;
    lag_counts_kernel<<<(L + 127) / 128, 128, 0, s>>>(T_s, L, count);
}

}  // namespace mhc
