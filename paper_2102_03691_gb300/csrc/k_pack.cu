// K1 pack: per-step B-operand rows of the two projections and the FP64 total
// heat current (Eq. 10, Eq. 13, Eq. 16).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.h"

namespace mhc {

namespace {

constexpr int PACK_THREADS = 256;

__device__ __forceinline__ void store_split(const PackArgs &a, size_t idx, float val) {
    if (a.split == SPLIT_BF16) {
        __nv_bfloat16 hi = __float2bfloat16_rn(val);
        __nv_bfloat16 lo = __float2bfloat16_rn(val - __bfloat162float(hi));
        static_cast<__nv_bfloat16 *>(a.Bt_hi)[idx] = hi;
        static_cast<__nv_bfloat16 *>(a.Bt_lo)[idx] = lo;
    } else if (a.split == SPLIT_FP16) {
        __half hi = __float2half_rn(val);
        __half lo = __float2half_rn(val - __half2float(hi));
        static_cast<__half *>(a.Bt_hi)[idx] = hi;
        static_cast<__half *>(a.Bt_lo)[idx] = lo;
    } else {
        a.Bt32[idx] = val;
    }
}

__global__ void __launch_bounds__(PACK_THREADS) pack_kernel(const PackArgs a) {
    const int k = blockIdx.x;
    const int D = 3 * a.N;
    const float *v = a.v + (size_t)k * D;
    const float *W = a.W + (size_t)k * a.N * 9;

    // Phase 1: row maxima (for the power-of-two scales) and Eq. 10.  Each product
    // W^{ab} v^b is split exactly into p + e (TwoProduct via FMA) and summed with
    // TwoSum into an unevaluated (s, c) float pair per thread, so the per-thread sums
    // carry about 48 significant bits using FP32 instructions only; they are combined
    // in FP64 below.  (GB300's FP64 pipe is too narrow for 9 FMAs per atom per step.)
    // Thread-strided over degrees of freedom d = 3i + b.
    float mx[4] = {0.f, 0.f, 0.f, 0.f};
    float js[3] = {0.f, 0.f, 0.f}, jc[3] = {0.f, 0.f, 0.f};
    for (int d = threadIdx.x; d < D; d += PACK_THREADS) {
        const int i = d / 3, b = d - 3 * (d / 3);
        const float vv = v[d];
        const float sm = a.sqm[i], ism = a.isqm[i];
        mx[0] = fmaxf(mx[0], fabsf(sm * vv));
#pragma unroll
        for (int al = 0; al < 3; ++al) {
            const float w = W[(size_t)i * 9 + 3 * al + b];
            mx[1 + al] = fmaxf(mx[1 + al], fabsf(w * ism));
            // explicit _rn intrinsics: the compiler must not contract these into FMAs
            const float pr = __fmul_rn(w, vv);
            const float pe = fmaf(w, vv, -pr);                       // w*vv = pr + pe exactly
            const float t = __fadd_rn(js[al], pr);                   // TwoSum(js, pr)
            const float bp = __fsub_rn(t, js[al]);
            const float er = __fadd_rn(__fsub_rn(js[al], __fsub_rn(t, bp)), __fsub_rn(pr, bp));
            js[al] = t;
            jc[al] = __fadd_rn(jc[al], __fadd_rn(er, pe));
        }
    }
    double j[3];
#pragma unroll
    for (int al = 0; al < 3; ++al) j[al] = (double)js[al] + (double)jc[al];
    __shared__ float s_mx[PACK_THREADS / 32][4];
    __shared__ double s_j[PACK_THREADS / 32][3];
    __shared__ float s_mul[4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int c = 0; c < 4; ++c) mx[c] = fmaxf(mx[c], __shfl_down_sync(FULL_MASK, mx[c], o));
#pragma unroll
        for (int c = 0; c < 3; ++c) j[c] += __shfl_down_sync(FULL_MASK, j[c], o);
    }
    if (lane == 0) {
        for (int c = 0; c < 4; ++c) s_mx[warp][c] = mx[c];
        for (int c = 0; c < 3; ++c) s_j[warp][c] = j[c];
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        const int c = threadIdx.x;
        float m = 0.f;
        for (int w = 0; w < PACK_THREADS / 32; ++w) m = fmaxf(m, s_mx[w][c]);
        int s = 0;
        if (a.split == SPLIT_FP16 && m > 0.f && isfinite(m)) {
            int e;
            frexpf(m, &e);      // m < 2^e
            s = 14 - e;         // scaled row maximum < 2^14 keeps the lo parts normal
        }
        s_mul[c] = ldexpf(1.f, s);
        a.col_scale[4 * k + c] = ldexpf(1.f, -(s + a.e_exp));
    } else if (threadIdx.x < 7) {
        const int c = threadIdx.x - 4;
        double t = 0.0;
        for (int w = 0; w < PACK_THREADS / 32; ++w) t += s_j[w][c];
        a.Jtot[3 * k + c] = t;
        if (a.Jring) a.Jring[((a.t0 + k) % a.R) * 3 + c] = t;
    }
    __syncthreads();

    // Phase 2: scaled rows, split into hi/lo (inputs are re-read from L2).
    const float m0 = s_mul[0], m1 = s_mul[1], m2 = s_mul[2], m3 = s_mul[3];
    const size_t r0 = (size_t)(4 * k) * a.D_ld;
    const size_t ld = (size_t)a.D_ld;
    for (int d = threadIdx.x; d < D; d += PACK_THREADS) {
        const int i = d / 3, b = d - 3 * (d / 3);
        const float sm = a.sqm[i], ism = a.isqm[i];
        store_split(a, r0 + d, (sm * v[d]) * m0);
        store_split(a, r0 + ld + d, (W[(size_t)i * 9 + b] * ism) * m1);
        store_split(a, r0 + 2 * ld + d, (W[(size_t)i * 9 + 3 + b] * ism) * m2);
        store_split(a, r0 + 3 * ld + d, (W[(size_t)i * 9 + 6 + b] * ism) * m3);
    }
}

}  // namespace

void launch_pack(const PackArgs &a, cudaStream_t s) {
    if (a.K <= 0) return;
    pack_kernel<<<a.K, PACK_THREADS, 0, s>>>(a);
}

}  // namespace mhc
