// Eigenvector preparation (once per mhc_set_modes): max |E|, gather of the kept
// modes in bin order with transpose to mode-major and hi/lo split, and the FP64
// orthonormality check of the basis (E^T E = I for the eigenvectors of Eq. 13-14).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.h"

namespace mhc {

namespace {

template <typename T>
__device__ __forceinline__ double load_e(const T *E, int layout, int64_t ld, int64_t d, int64_t n) {
    // layout 0: dof-major E[d*ld + n]; layout 1: mode-major E[n*ld + d]
    return (double)(layout == 0 ? E[d * ld + n] : E[n * ld + d]);
}

template <typename T>
__global__ void max_abs_kernel(const T *E, int layout, int64_t ld, int64_t D, int64_t M,
                               unsigned *out) {
    float m = 0.f;
    const int64_t total = D * M;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = q / (layout == 0 ? M : D), b = q % (layout == 0 ? M : D);
        const double x = layout == 0 ? (double)E[a * ld + b] : (double)E[a * ld + b];
        const float f = fabsf((float)x);
        if (f == f) m = fmaxf(m, f);   // NaN is ignored here; it shows up downstream
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(FULL_MASK, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// Source dof of stored column c: c itself, or 3i+b for the direction-major column
// c = b*npad + i (-1 for the zero padding of each direction segment).
__device__ __forceinline__ int64_t source_dof(int64_t c, int64_t D, int64_t npad) {
    if (npad == 0) return c < D ? c : -1;
    const int64_t b = c / npad, i = c - b * npad;
    return (b < 3 && i < D / 3) ? 3 * i + b : -1;
}

template <typename T, int SPLIT>
__global__ void prepare_kernel(const T *E, int layout, int64_t ld, int64_t D, int64_t M_eff,
                               const int *perm, int e_exp, void *Et_hi, void *Et_lo,
                               float *Et32, int64_t D_ld, int64_t npad) {
    __shared__ double tile[32][33];
    const int64_t d0 = (int64_t)blockIdx.x * 32, n0 = (int64_t)blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    const double scale = ldexp(1.0, e_exp);
    if (layout == 0) {
        // rows of E are dofs: read E[d][perm[n]] with n along tx
        for (int r = ty; r < 32; r += 8) {
            const int64_t d = source_dof(d0 + r, D, npad), n = n0 + tx;
            double x = 0.0;
            if (d >= 0 && n < M_eff) x = load_e(E, 0, ld, d, (int64_t)perm[n]);
            tile[tx][r] = x;   // tile[n_local][d_local]
        }
    } else {
        for (int r = ty; r < 32; r += 8) {
            const int64_t n = n0 + r, d = source_dof(d0 + tx, D, npad);
            double x = 0.0;
            if (d >= 0 && n < M_eff) x = load_e(E, 1, ld, d, (int64_t)perm[n]);
            tile[r][tx] = x;
        }
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int64_t n = n0 + r, d = d0 + tx;
        const double x = tile[r][tx] * scale;
        const size_t idx = (size_t)n * D_ld + d;
        if (SPLIT == SPLIT_BF16) {
            __nv_bfloat16 hi = __double2bfloat16(x);
            __nv_bfloat16 lo = __double2bfloat16(x - (double)__bfloat162float(hi));
            static_cast<__nv_bfloat16 *>(Et_hi)[idx] = hi;
            static_cast<__nv_bfloat16 *>(Et_lo)[idx] = lo;
        } else if (SPLIT == SPLIT_FP16) {
            __half hi = __double2half(x);
            __half lo = __double2half(x - (double)__half2float(hi));
            static_cast<__half *>(Et_hi)[idx] = hi;
            static_cast<__half *>(Et_lo)[idx] = lo;
        } else {
            Et32[idx] = (float)x;
        }
    }
}

// G[p][m] = sum_d E[d, probe[p]] E[d, m]; reports max |G - delta| as FP64 bits.
template <typename T>
__global__ void ortho_kernel(const T *E, int layout, int64_t ld, int64_t D, int64_t M,
                             const int *probe, int n_probe, unsigned long long *out) {
    __shared__ double sp[32][33], sm[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    const int64_t p0 = (int64_t)blockIdx.y * 32, m0 = (int64_t)blockIdx.x * 32;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t d0 = 0; d0 < D; d0 += 32) {
        for (int r = ty; r < 32; r += 8) {
            const int64_t d = d0 + r;
            const int64_t p = p0 + tx, m = m0 + tx;
            sp[r][tx] = (d < D && p < n_probe) ? load_e(E, layout, ld, d, (int64_t)probe[p]) : 0.0;
            sm[r][tx] = (d < D && m < M) ? load_e(E, layout, ld, d, m) : 0.0;
        }
        __syncthreads();
        for (int dd = 0; dd < 32; ++dd) {
            const double em = sm[dd][tx];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fma(sp[dd][ty + 8 * q], em, acc[q]);
        }
        __syncthreads();
    }
    double worst = 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int64_t p = p0 + ty + 8 * q, m = m0 + tx;
        if (p < n_probe && m < M) {
            const double r = fabs(acc[q] - ((int64_t)probe[p] == m ? 1.0 : 0.0));
            worst = r > worst ? r : worst;
        }
    }
    if (worst > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(worst));
}

}  // namespace

void launch_max_abs(const void *E, int dtype, int layout, int64_t ld, int64_t D, int64_t M,
                    unsigned *out_bits, cudaStream_t s) {
    const int grid = 1024, block = 256;
    if (dtype == 1)
        max_abs_kernel<double><<<grid, block, 0, s>>>((const double *)E, layout, ld, D, M, out_bits);
    else
        max_abs_kernel<float><<<grid, block, 0, s>>>((const float *)E, layout, ld, D, M, out_bits);
}

void launch_prepare_modes(const void *E, int dtype, int layout, int64_t ld, int64_t D,
                          int64_t M_eff, const int *perm, int e_exp, int split, void *Et_hi,
                          void *Et_lo, float *Et32, int64_t D_ld, int64_t M_pad, int64_t npad,
                          cudaStream_t s) {
    dim3 block(32, 8), grid((unsigned)(D_ld / 32), (unsigned)(M_pad / 32));
#define MHC_PREP(T, S)                                                                         \
    prepare_kernel<T, S><<<grid, block, 0, s>>>((const T *)E, layout, ld, D, M_eff, perm, e_exp, \
                                                Et_hi, Et_lo, Et32, D_ld, npad)
    if (dtype == 1) {
        if (split == SPLIT_BF16) MHC_PREP(double, SPLIT_BF16);
        else if (split == SPLIT_FP16) MHC_PREP(double, SPLIT_FP16);
        else MHC_PREP(double, SPLIT_FP32);
    } else {
        if (split == SPLIT_BF16) MHC_PREP(float, SPLIT_BF16);
        else if (split == SPLIT_FP16) MHC_PREP(float, SPLIT_FP16);
        else MHC_PREP(float, SPLIT_FP32);
    }
#undef MHC_PREP
}

void launch_orthonormality(const void *E, int dtype, int layout, int64_t ld, int64_t D,
                           int64_t M, const int *probe, int n_probe,
                           unsigned long long *out_bits, cudaStream_t s) {
    dim3 block(32, 8), grid((unsigned)((M + 31) / 32), (unsigned)((n_probe + 31) / 32));
    if (dtype == 1)
        ortho_kernel<double><<<grid, block, 0, s>>>((const double *)E, layout, ld, D, M, probe,
                                                    n_probe, out_bits);
    else
        ortho_kernel<float><<<grid, block, 0, s>>>((const float *)E, layout, ld, D, M, probe,
                                                   n_probe, out_bits);
}

}  // namespace mhc
