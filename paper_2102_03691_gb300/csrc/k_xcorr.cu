// Bin-bin cross-correlations of the binned modal heat currents (the mode-mode correlations
// the paper notes GKMA allows; at one bin per mode they are exactly those).  Same lag
// convention as Eq. 17: the first current is lagged, the second sits at the time origin.
//   X[l][i][j] += sum_{k: t0+k-l >= 0} Jb[k][i] * Jb(t0+k-l)[j],   i = 3b+mu, j = 3b'+nu
// FP32 products and 32-step FP32 partials are summed over the block in a float pair and added
// to the FP64 state once per launch.  The state is lag-major so that one CTA (one lag, a
// 64 x 64 block of (i, j)) writes its sums coalesced; the read-out transposes to
// [b][b'][mu][nu][l].
#include "common.cuh"
#include "kernels.h"

namespace mhc {

namespace {

constexpr int XC_TILE = 64;      // rows / columns of a CTA's block
constexpr int XC_KC = 32;        // steps per FP32 partial (folded into a float pair after each)
constexpr int XC_THREADS = 256;  // 16 x 16 threads, 4 x 4 outputs each

// (s, c) += x exactly as an unevaluated float pair (TwoSum; _rn keeps it from being contracted).
// GB300's FP64 pipe is narrow: folding each 32-step partial into FP64 registers cost more issue
// time than the 512 FMAs of the chunk; the pair carries ~48 bits with FP32 instructions only.
__device__ __forceinline__ void pair_add(float &s, float &c, float x) {
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

__global__ void __launch_bounds__(XC_THREADS) bin_xcorr_kernel(
    const float *__restrict__ Jb, const float *__restrict__ ring, int R, double *X, int K, int n,
    long long t0_host, const long long *t0_dev) {
    __shared__ __align__(16) float sA[XC_KC][XC_TILE];
    __shared__ __align__(16) float sS[XC_KC][XC_TILE];
    const long long t0 = t0_dev ? *t0_dev : t0_host;
    const int l = blockIdx.z;
    const int i0 = blockIdx.y * XC_TILE, j0 = blockIdx.x * XC_TILE;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][4], cmp[4][4], part[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = cmp[a][b] = 0.f;
    // Each thread stages the same 8 (kk, c) slots of both tiles for every chunk; the next
    // chunk's values are loaded into registers while the current one is multiplied.
    constexpr int PER = XC_KC * XC_TILE / XC_THREADS;   // 8
    float ra[PER], rs[PER];
    auto fetch = [&](int k0) {
        // origin of step k0 + kk at lag l: time tb + kk, ring row (rb + kk) mod R
        const long long tb = t0 + k0 - l;
        const int rb = tb >= 0 ? (int)(tb % R) : (int)(((tb % R) + R) % R);
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int q = threadIdx.x + u * XC_THREADS;
            const int kk = q / XC_TILE, c = q - kk * XC_TILE;
            const int k = k0 + kk;
            float a = 0.f, sv = 0.f;
            if (k < K) {
                if (i0 + c < n) a = Jb[(size_t)k * n + i0 + c];
                int row = rb + kk;
                if (row >= R) row -= R;
                if (tb + kk >= 0 && j0 + c < n) sv = ring[(size_t)row * n + j0 + c];
            }
            ra[u] = a;
            rs[u] = sv;
        }
    };
    fetch(0);
    for (int k0 = 0; k0 < K; k0 += XC_KC) {
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int q = threadIdx.x + u * XC_THREADS;
            sA[q / XC_TILE][q % XC_TILE] = ra[u];
            sS[q / XC_TILE][q % XC_TILE] = rs[u];
        }
        __syncthreads();
        if (k0 + XC_KC < K) fetch(k0 + XC_KC);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) part[a][b] = 0.f;
#pragma unroll 8
        for (int kk = 0; kk < XC_KC; ++kk) {
            const float4 av = *reinterpret_cast<const float4 *>(&sA[kk][ty * 4]);
            const float4 sv = *reinterpret_cast<const float4 *>(&sS[kk][tx * 4]);
            const float ar[4] = {av.x, av.y, av.z, av.w}, sr[4] = {sv.x, sv.y, sv.z, sv.w};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) part[a][b] = fmaf(ar[a], sr[b], part[a][b]);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) pair_add(acc[a][b], cmp[a][b], part[a][b]);
        __syncthreads();
    }
    double *Xl = X + (size_t)l * n * n;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int i = i0 + ty * 4 + a;
        if (i >= n) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int j = j0 + tx * 4 + b;
            if (j < n) Xl[(size_t)i * n + j] += (double)acc[a][b] + (double)cmp[a][b];
        }
    }
}

// out[((b B + b2) 3 + mu) 3 + nu][l] = X[l][3b+mu][3b2+nu]
__global__ void xcorr_transpose_kernel(const double *__restrict__ X, int nb, int L, double *out) {
    const int n = 3 * nb;
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= (long long)n * n * L) return;
    const long long l = q % L, r = q / L;   // r = ((b nb + b2) 3 + mu) 3 + nu
    const int nu = (int)(r % 3), mu = (int)((r / 3) % 3);
    const long long bb = r / 9;
    const int b2 = (int)(bb % nb), b = (int)(bb / nb);
    out[q] = X[(size_t)l * n * n + (size_t)(3 * b + mu) * n + 3 * b2 + nu];
}

}  // namespace

void launch_jb_ring_store(const float *Jb, int K, int nb, float *ring, int R, long long t0,
                          const long long *t0_dev, cudaStream_t s) {
    const long long total = (long long)K * nb * 3;
    if (total <= 0) return;
    jb_ring_store_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(Jb, K, 3 * nb, ring, R, t0, t0_dev);
}

void launch_bin_xcorr(const float *Jb, const float *ring, int R, double *X, int K, int nb, int L,
                      long long t0, const long long *t0_dev, cudaStream_t s) {
    const int n = 3 * nb;
    if (L <= 0 || K <= 0 || n <= 0) return;
    dim3 grid((n + XC_TILE - 1) / XC_TILE, (n + XC_TILE - 1) / XC_TILE, L);
    bin_xcorr_kernel<<<grid, XC_THREADS, 0, s>>>(Jb, ring, R, X, K, n, t0, t0_dev);
}

void launch_xcorr_transpose(const double *X, int nb, int L, double *out, cudaStream_t s) {
    const long long total = 9ll * nb * nb * L;
    if (total <= 0) return;
    xcorr_transpose_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(X, nb, L, out);
}

}  // namespace mhc
