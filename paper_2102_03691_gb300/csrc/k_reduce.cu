// K3 bin finish + HNEMA sums (Eq. 19), K4 GKMA lag correlation (Eq. 17 integrand),
// K5 running Green-Kubo integral (Eq. 17) and the HNEMA normalisation (Eq. 19).
#include "common.cuh"
#include "kernels.h"

namespace mhc {

namespace {

// ------------------------------------------------------------------ K3
// One CTA per bin.  Thread t handles component a = t % 3 and steps k = t/3 + 64 j.
// J_b^a(k) = sum of the bin's partial slots in slot order; HNEMA sum in FP64 with a
// fixed reduction tree (deterministic).  CTA 0 also sums the total current.
constexpr int BF_THREADS = 192;
__global__ void __launch_bounds__(BF_THREADS) bin_finish_kernel(const float *__restrict__ partials,
                                                                int n_slots, const int *slot_begin,
                                                                int B, int K, float *Jb,
                                                                double *hsum, const double *Jtot,
                                                                double *Jsum) {
    const int b = blockIdx.x;
    const int a = threadIdx.x % 3, k0 = threadIdx.x / 3;
    const int s0 = slot_begin[b], s1 = slot_begin[b + 1];
    double acc = 0.0, acc_tot = 0.0;
    for (int k = k0; k < K; k += BF_THREADS / 3) {
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
    if (threadIdx.x < 3) {
        double t = 0.0, u = 0.0;
        for (int q = threadIdx.x; q < BF_THREADS; q += 3) {
            t += red[0][q];
            u += red[1][q];
        }
        hsum[b * 3 + threadIdx.x] += t;
        if (b == 0) Jsum[threadIdx.x] += u;
    }
}

// ------------------------------------------------------------------ K4
// Each warp owns 32 consecutive lags; lane l holds the total current J(t - l) of the
// current step t in registers.  Moving to step t+1 shifts that window by one lag with a
// warp shuffle (lane l takes lane l-1's value) and lane 0 loads the one new sample, so the
// ring of past J is read once per warp per step.  Products and 32-step partial sums are
// FP32, the lag sums themselves are FP64.
constexpr int LC_THREADS = 128;
constexpr int LC_BINS = 4;
__global__ void __launch_bounds__(LC_THREADS) lag_corr_kernel(const float *__restrict__ Jb,
                                                              const double *__restrict__ Jring,
                                                              int R, double *Csum, int K, int B,
                                                              int L, long long t0) {
    extern __shared__ float sJ[];   // [K][LC_BINS][3]
    const int b0 = blockIdx.y * LC_BINS;
    const int nb = min(LC_BINS, B - b0);
    for (int q = threadIdx.x; q < K * LC_BINS * 3; q += LC_THREADS) {
        const int k = q / (LC_BINS * 3), r = q % (LC_BINS * 3), bb = r / 3, mu = r % 3;
        sJ[q] = bb < nb ? Jb[((size_t)k * B + b0 + bb) * 3 + mu] : 0.f;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int l0 = blockIdx.x * LC_THREADS + (threadIdx.x & ~31);   // first lag of this warp
    const int l = l0 + lane;
    auto load_j = [&](long long tt, float (&j)[3]) {
        if (tt >= 0) {
            const double *src = Jring + (tt % R) * 3;
            j[0] = (float)src[0];
            j[1] = (float)src[1];
            j[2] = (float)src[2];
        } else {
            j[0] = j[1] = j[2] = 0.f;
        }
    };
    float j[3];
    load_j(t0 - l, j);
    float acc[LC_BINS][9];
    double dacc[LC_BINS][9];
#pragma unroll
    for (int bb = 0; bb < LC_BINS; ++bb)
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            acc[bb][c] = 0.f;
            dacc[bb][c] = 0.0;
        }
    for (int k = 0; k < K; ++k) {
        if (k > 0) {
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
        if ((k & 31) == 31 || k == K - 1) {
#pragma unroll
            for (int bb = 0; bb < LC_BINS; ++bb)
#pragma unroll
                for (int c = 0; c < 9; ++c) {
                    dacc[bb][c] += (double)acc[bb][c];
                    acc[bb][c] = 0.f;
                }
        }
    }
    if (l < L) {
        for (int bb = 0; bb < nb; ++bb)
#pragma unroll
            for (int c = 0; c < 9; ++c) Csum[((size_t)(b0 + bb) * 9 + c) * L + l] += dacc[bb][c];
    }
}

// ------------------------------------------------------------------ K5
// Thread per (b, mu, nu): C(l) = Csum(l)/(T_s - l); trapezoid running integral, FP64.
__global__ void gk_kappa_kernel(const double *Csum, int rows, int L, long long T_s, double coef_dt,
                                double tau_lo, double tau_hi, double dt, double *kappa_tau,
                                double *kappa_w) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const double *cs = Csum + (size_t)r * L;
    double acc = 0.0, prev = 0.0, wsum = 0.0;
    int wn = 0;
    for (int l = 0; l < L; ++l) {
        const long long cnt = T_s - l;
        const double C = cnt > 0 ? cs[l] / (double)cnt : 0.0;
        if (l > 0) acc += 0.5 * (prev + C);
        prev = C;
        const double kap = coef_dt * acc;
        if (kappa_tau) kappa_tau[(size_t)r * L + l] = kap;
        const double tau = l * dt;
        if (tau >= tau_lo && tau <= tau_hi) {
            wsum += kap;
            ++wn;
        }
    }
    if (kappa_w) kappa_w[r] = wn > 0 ? wsum / wn : 0.0;
}

__global__ void hnema_finalize_kernel(const double *hsum, int n, long long T_s, double coef,
                                      double *mean, double *kappa) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const double m = T_s > 0 ? hsum[q] / (double)T_s : 0.0;
    if (mean) mean[q] = m;
    if (kappa) kappa[q] = m * coef;
}

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
                     int L, long long t0, cudaStream_t s) {
    if (L <= 0 || K <= 0 || B <= 0) return;
    dim3 grid((L + LC_THREADS - 1) / LC_THREADS, (B + LC_BINS - 1) / LC_BINS);
    const size_t sm = (size_t)K * LC_BINS * 3 * sizeof(float);
    lag_corr_kernel<<<grid, LC_THREADS, sm, s>>>(Jb, Jring, R, Csum, K, B, L, t0);
}

void launch_gk_kappa(const double *Csum, int B, int L, long long T_s, double coef_dt,
                     double tau_lo, double tau_hi, double dt, double *kappa_tau, double *kappa_w,
                     cudaStream_t s) {
    const int rows = B * 9;
    gk_kappa_kernel<<<(rows + 127) / 128, 128, 0, s>>>(Csum, rows, L, T_s, coef_dt, tau_lo, tau_hi,
                                                       dt, kappa_tau, kappa_w);
}

void launch_hnema_finalize(const double *hsum, int B, long long T_s, double coef, double *mean,
                           double *kappa, cudaStream_t s) {
    const int n = B * 3;
    hnema_finalize_kernel<<<(n + 127) / 128, 128, 0, s>>>(hsum, n, T_s, coef, mean, kappa);
}

void launch_lag_counts(long long T_s, int L, long long *count, cudaStream_t s) {
    if (L <= 0) return;
    lag_counts_kernel<<<(L + 127) / 128, 128, 0, s>>>(T_s, L, count);
}

}  // namespace mhc
