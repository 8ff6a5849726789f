// K3 bin finish + HNEMA sums (Eq. 19), K4 GKMA lag correlation (Eq. 17 integrand),
// K5 running Green-Kubo integral (Eq. 17) and the HNEMA normalisation (Eq. 19).
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
__global__ void __launch_bounds__(BF_THREADS) bin_finish_kernel(const float *__restrict__ partials,
                                                                int n_slots, const int *slot_begin,
                                                                int B, int K, float *Jb,
                                                                double *hsum, const double *Jtot,
                                                                double *Jsum) {
    const int b = blockIdx.x;
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

// ------------------------------------------------------------------ K4
// A CTA covers 128 consecutive lags (four lag warps) of LC_BINS bins, and each lag warp runs
// in LC_SPLIT copies over consecutive quarters of the block's steps, so that 16 warps hide the
// latency of the per-step window shift.  Lane l of a warp holds the total current J(t - l) of
// its current step t in registers; moving to step t+1 shifts that window by one lag with a
// warp shuffle (lane l takes lane l-1's value) and lane 0 takes the one new sample from the
// CTA's copy of the J samples it needs, staged in shared memory from the ring once per launch.
// Products and 32-step partial sums are FP32; the partials are summed over the quarter in an
// unevaluated float pair (TwoSum, ~48 bits; GB300's FP64 pipe is narrow), the quarters' pairs
// are added in quarter order (deterministic), and one FP64 value per lag sum is added to the
// FP64 lag sums.
constexpr int LC_LAGS = 128;   // lags per CTA: four lag warps
constexpr int LC_SPLIT = 4;    // step quarters
constexpr int LC_THREADS = LC_LAGS * LC_SPLIT;
constexpr int LC_BINS = 2;

// (s, c) += x exactly as an unevaluated float pair (_rn keeps it from being contracted)
__device__ __forceinline__ void lc_pair_add(float &s, float &c, float x) {
    const float t = __fadd_rn(s, x);
    const float bp = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
    s = t;
    c = __fadd_rn(c, e);
}
__global__ void __launch_bounds__(LC_THREADS) lag_corr_kernel(const float *__restrict__ Jb,
                                                              const double *__restrict__ Jring,
                                                              int R, double *Csum, int K, int B,
                                                              int L, long long t0_host,
                                                              const long long *t0_dev) {
    const long long t0 = t0_dev ? *t0_dev : t0_host;
    // [K][LC_BINS][3] binned currents, the J window [K + LC_LAGS - 1][3], then the quarters'
    // float pairs [LC_SPLIT - 1][2][LC_BINS * 9][LC_LAGS]
    extern __shared__ float sJ[];
    float *sW = sJ + K * LC_BINS * 3;
    const int nw = K + LC_LAGS - 1;
    float *sQ = sW + nw * 3;
    const int b0 = blockIdx.y * LC_BINS;
    const int nb = min(LC_BINS, B - b0);
    for (int q = threadIdx.x; q < K * LC_BINS * 3; q += LC_THREADS) {
        const int k = q / (LC_BINS * 3), r = q % (LC_BINS * 3), bb = r / 3, mu = r % 3;
        sJ[q] = bb < nb ? Jb[((size_t)k * B + b0 + bb) * 3 + mu] : 0.f;
    }
    // window entry j holds J(tw0 + j), tw0 = t0 - (first lag of the CTA) - (LC_LAGS - 1)
    const int lc0 = blockIdx.x * LC_LAGS;
    const long long tw0 = t0 - lc0 - (LC_LAGS - 1);
    for (int q = threadIdx.x; q < nw * 3; q += LC_THREADS) {
        const long long tt = tw0 + q / 3;
        sW[q] = tt >= 0 ? (float)Jring[(tt % R) * 3 + q % 3] : 0.f;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int lw = (threadIdx.x >> 5) % (LC_LAGS / 32);   // lag warp
    const int quarter = (threadIdx.x >> 5) / (LC_LAGS / 32);
    const int l0 = lc0 + 32 * lw;                          // first lag of this warp
    const int l = l0 + lane;
    const int kq = (K + LC_SPLIT - 1) / LC_SPLIT;
    const int k_begin = min(K, quarter * kq), k_end = min(K, k_begin + kq);
    auto load_j = [&](long long tt, float (&j)[3]) {   // J(tt) from the staged window
        const float *src = sW + (tt - tw0) * 3;
        j[0] = src[0];
        j[1] = src[1];
        j[2] = src[2];
    };
    float j[3];
    load_j(t0 + k_begin - l, j);
    float acc[LC_BINS][9], hs[LC_BINS][9], hc[LC_BINS][9];
#pragma unroll
    for (int bb = 0; bb < LC_BINS; ++bb)
#pragma unroll
        for (int c = 0; c < 9; ++c) acc[bb][c] = hs[bb][c] = hc[bb][c] = 0.f;
    for (int k = k_begin; k < k_end; ++k) {
        if (k > k_begin) {
            float nj[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) nj[c] = __shfl_up_sync(FULL_MASK, j[c], 1);
            if (lane == 0) load_j(t0 + k - l0, nj);
#pragma unroll
            for (int c = 0; c < 3; ++c) j[c] = nj[c];
        }
        const float *jb = sJ + k * LC_BINS * 3;
#pragma unroll
        for (int bb = 0; bb < LC_BINS; ++bb)
#pragma unroll
            for (int mu = 0; mu < 3; ++mu) {
                const float x = jb[bb * 3 + mu];
#pragma unroll
                for (int nu = 0; nu < 3; ++nu) acc[bb][mu * 3 + nu] = fmaf(x, j[nu], acc[bb][mu * 3 + nu]);
            }
        if (((k - k_begin) & 31) == 31 || k == k_end - 1) {
#pragma unroll
            for (int bb = 0; bb < LC_BINS; ++bb)
#pragma unroll
                for (int c = 0; c < 9; ++c) {
                    lc_pair_add(hs[bb][c], hc[bb][c], acc[bb][c]);
                    acc[bb][c] = 0.f;
                }
        }
    }
    const int li = 32 * lw + lane;   // lag index within the CTA
    constexpr int QSTRIDE = 2 * LC_BINS * 9 * LC_LAGS;   // floats of one quarter's pairs
    if (quarter > 0) {
#pragma unroll
        for (int bb = 0; bb < LC_BINS; ++bb)
#pragma unroll
            for (int c = 0; c < 9; ++c) {
                float *q = sQ + (size_t)(quarter - 1) * QSTRIDE + (bb * 9 + c) * LC_LAGS + li;
                q[0] = hs[bb][c];
                q[LC_BINS * 9 * LC_LAGS] = hc[bb][c];
            }
    }
    __syncthreads();
    if (quarter == 0 && l < L) {
        for (int bb = 0; bb < nb; ++bb)
#pragma unroll
            for (int c = 0; c < 9; ++c) {
                float s = hs[bb][c], cc = hc[bb][c];
#pragma unroll
                for (int qq = 0; qq < LC_SPLIT - 1; ++qq) {
                    const float *q = sQ + (size_t)qq * QSTRIDE + (bb * 9 + c) * LC_LAGS + li;
                    lc_pair_add(s, cc, q[0]);
                    cc = __fadd_rn(cc, q[LC_BINS * 9 * LC_LAGS]);
                }
                Csum[((size_t)(b0 + bb) * 9 + c) * L + l] += (double)s + (double)cc;
            }
    }
}

size_t lag_corr_smem(int K) {
    return ((size_t)K * LC_BINS * 3 + (size_t)(K + LC_LAGS - 1) * 3 +
            (size_t)(LC_SPLIT - 1) * 2 * LC_BINS * 9 * LC_LAGS) * sizeof(float);
}

// ------------------------------------------------------------------ K5
// inv_count(l) = 1 / (T_s - l) (0 when no origin has lag l), computed once per read so that
// the rows below multiply instead of dividing (an FP64 division is ~8 instructions on a pipe
// GB300 keeps narrow).
__global__ void inv_counts_kernel(long long T_s, int L, double *inv) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l < L) inv[l] = T_s > l ? 1.0 / (double)(T_s - l) : 0.0;
}

// One CTA per (b, mu, nu) row, GK_THREADS threads, each owning GK_PER consecutive lags.
// C(l) = Csum(l) * inv_count(l); trapezoid increments (C(l-1)+C(l))/2 for l >= 1;
// block-wide exclusive scan of the per-thread totals (fixed tree: deterministic);
// kappa(l) = c dt * prefix(l).  The tau-window average is a block reduction.
constexpr int GK_THREADS = 128;
__global__ void __launch_bounds__(GK_THREADS) gk_kappa_kernel(const double *Csum, int L,
                                                              const double *__restrict__ inv,
                                                              double coef_dt,
                                                              double tau_lo, double tau_hi,
                                                              double dt, double *kappa_tau,
                                                              double *kappa_w) {
    const int r = blockIdx.x;
    const double *cs = Csum + (size_t)r * L;
    const int per = (L + GK_THREADS - 1) / GK_THREADS;
    const int l0 = threadIdx.x * per;
    auto C = [&](int l) -> double { return cs[l] * inv[l]; };
    double prev = (l0 > 0 && l0 <= L) ? C(l0 - 1) : 0.0;
    double tot = 0.0;
    for (int l = l0; l < min(L, l0 + per); ++l) {
        const double c = C(l);
        if (l > 0) tot += 0.5 * (prev + c);
        prev = c;
    }
    __shared__ double sc[GK_THREADS];
    sc[threadIdx.x] = tot;
    __syncthreads();
    for (int off = 1; off < GK_THREADS; off <<= 1) {   // Hillis-Steele inclusive scan
        const double add = threadIdx.x >= off ? sc[threadIdx.x - off] : 0.0;
        __syncthreads();
        sc[threadIdx.x] += add;
        __syncthreads();
    }
    double acc = threadIdx.x > 0 ? sc[threadIdx.x - 1] : 0.0;   // exclusive prefix
    double wsum = 0.0;
    int wn = 0;
    prev = (l0 > 0 && l0 <= L) ? C(l0 - 1) : 0.0;
    for (int l = l0; l < min(L, l0 + per); ++l) {
        const double c = C(l);
        if (l > 0) acc += 0.5 * (prev + c);
        prev = c;
        const double kap = coef_dt * acc;
        if (kappa_tau) kappa_tau[(size_t)r * L + l] = kap;
        const double tau = l * dt;
        if (tau >= tau_lo && tau <= tau_hi) {
            wsum += kap;
            ++wn;
        }
    }
    __syncthreads();
    __shared__ int sn[GK_THREADS];
    sc[threadIdx.x] = wsum;
    sn[threadIdx.x] = wn;
    __syncthreads();
    for (int off = GK_THREADS / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) {
            sc[threadIdx.x] += sc[threadIdx.x + off];
            sn[threadIdx.x] += sn[threadIdx.x + off];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && kappa_w) kappa_w[r] = sn[0] > 0 ? sc[0] / sn[0] : 0.0;
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
                       float *Jb, double *hsum, const double *Jtot, double *Jsum, cudaStream_t s) {
    if (B <= 0 || K <= 0) return;
    bin_finish_kernel<<<B, BF_THREADS, 0, s>>>(partials, n_slots, slot_begin, B, K, Jb, hsum, Jtot, Jsum);
}

void launch_lag_corr(const float *Jb, const double *Jring, int R, double *Csum, int K, int B,
                     int L, long long t0, const long long *t0_dev, cudaStream_t s) {
    if (L <= 0 || K <= 0 || B <= 0) return;
    dim3 grid((L + LC_LAGS - 1) / LC_LAGS, (B + LC_BINS - 1) / LC_BINS);
    const size_t sm = lag_corr_smem(K);
    static size_t sm_set = 48 * 1024;   // the largest dynamic size opted into so far
    if (sm > sm_set) {
        if (cudaFuncSetAttribute(lag_corr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sm) != cudaSuccess)
            return;   // the launch below is skipped; the caller's cudaGetLastError reports it
        sm_set = sm;
    }
    lag_corr_kernel<<<grid, LC_THREADS, sm, s>>>(Jb, Jring, R, Csum, K, B, L, t0, t0_dev);
}

void launch_gk_kappa(const double *Csum, int B, int L, long long T_s, double coef_dt,
                     double tau_lo, double tau_hi, double dt, double *kappa_tau, double *kappa_w,
                     double *inv_scratch, cudaStream_t s) {
    if (L <= 0 || B <= 0) return;
    inv_counts_kernel<<<(L + 255) / 256, 256, 0, s>>>(T_s, L, inv_scratch);
    gk_kappa_kernel<<<B * 9, GK_THREADS, 0, s>>>(Csum, L, inv_scratch, coef_dt, tau_lo, tau_hi, dt,
                                                 kappa_tau, kappa_w);
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
