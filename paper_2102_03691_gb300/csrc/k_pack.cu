// K1 pack: per-step B-operand rows of the two projections and the FP64 total
// heat current (Eq. 10, Eq. 13, Eq. 16).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.h"

namespace mhc {

namespace {

constexpr int PACK_THREADS = 512;

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

// TwoProduct + TwoSum: add w*v exactly into the unevaluated float pair (s, c).
// Explicit _rn intrinsics keep the compiler from contracting these into FMAs.
__device__ __forceinline__ void acc_exact(float &s, float &c, float w, float v) {
    const float pr = __fmul_rn(w, v);
    const float pe = fmaf(w, v, -pr);                       // w*v = pr + pe exactly
    const float t = __fadd_rn(s, pr);
    const float bp = __fsub_rn(t, s);
    const float er = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(pr, bp));
    s = t;
    c = __fadd_rn(c, __fadd_rn(er, pe));
}

__global__ void __launch_bounds__(PACK_THREADS) pack_kernel(const PackArgs a) {
    const int k = blockIdx.x;
    const float *v = a.v + (size_t)k * a.N * 3;
    const float *W = a.W + (size_t)k * a.N * 9;

    // Phase 1, one thread per atom: row maxima (for the power-of-two scales) and
    // Eq. 10, J^a = sum_i sum_b W_i^{ab} v_i^b.  Products are added exactly into an
    // unevaluated float pair per thread (about 48 significant bits with FP32
    // instructions only) and the pairs are combined in FP64 below.  (GB300's FP64
    // pipe is too narrow for 9 FP64 FMAs per atom per step.)
    float mx[4] = {0.f, 0.f, 0.f, 0.f};
    float js[3] = {0.f, 0.f, 0.f}, jc[3] = {0.f, 0.f, 0.f};
    for (int i = threadIdx.x; i < a.N; i += PACK_THREADS) {
        float vv[3], ww[9];
#pragma unroll
        for (int b = 0; b < 3; ++b) vv[b] = v[(size_t)i * 3 + b];
#pragma unroll
        for (int q = 0; q < 9; ++q) ww[q] = W[(size_t)i * 9 + q];
        const float sm = a.sqm[i], ism = a.isqm[i];
#pragma unroll
        for (int b = 0; b < 3; ++b) mx[0] = fmaxf(mx[0], fabsf(sm * vv[b]));
#pragma unroll
        for (int al = 0; al < 3; ++al)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                mx[1 + al] = fmaxf(mx[1 + al], fabsf(ww[3 * al + b] * ism));
                acc_exact(js[al], jc[al], ww[3 * al + b], vv[b]);
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
    } else if (threadIdx.x >= 32 && threadIdx.x < 35) {
        const int c = threadIdx.x - 32;
        double t = 0.0;
        for (int w = 0; w < PACK_THREADS / 32; ++w) t += s_j[w][c];
        a.Jtot[3 * k + c] = t;
        if (a.Jring) {
            const long long t0 = a.t0_dev ? *a.t0_dev : a.t0;
            a.Jring[((t0 + k) % a.R) * 3 + c] = t;
        }
    }
    __syncthreads();

    // Phase 2, one thread per atom: the four scaled rows of step k,
    //   Bt[4k][3i+b] = sqrt(m_i) v_i^b,  Bt[4k+1+a][3i+b] = W_i^{ab} / sqrt(m_i),
    // split into hi/lo (inputs re-read from L2).
    // (direction-major columns b*npad + i when npad > 0)
    const float mul[4] = {s_mul[0], s_mul[1], s_mul[2], s_mul[3]};
    const size_t r0 = (size_t)(4 * k) * a.D_ld;
    const size_t ld = (size_t)a.D_ld;
    const size_t cs_i = a.npad ? 1 : 3, cs_b = a.npad ? (size_t)a.npad : 1;
    for (int i = threadIdx.x; i < a.N; i += PACK_THREADS) {
        const float sm = a.sqm[i], ism = a.isqm[i];
#pragma unroll
        for (int b = 0; b < 3; ++b)
            store_split(a, r0 + cs_i * i + cs_b * b, (sm * v[(size_t)i * 3 + b]) * mul[0]);
#pragma unroll
        for (int al = 0; al < 3; ++al)
#pragma unroll
            for (int b = 0; b < 3; ++b)
                store_split(a, r0 + (1 + al) * ld + cs_i * i + cs_b * b,
                            (W[(size_t)i * 9 + 3 * al + b] * ism) * mul[1 + al]);
    }
}

}  // namespace

void launch_pack(const PackArgs &a, cudaStream_t s) {
    if (a.K <= 0) return;
    pack_kernel<<<a.K, PACK_THREADS, 0, s>>>(a);
}

}  // namespace mhc
