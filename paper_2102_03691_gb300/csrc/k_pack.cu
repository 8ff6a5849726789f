// K1 pack: per-step B-operand rows of the two projections and the FP64 total
// heat current (Eq. 10, Eq. 13, Eq. 16).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

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

// (s, c) += (s2, c2): the leading parts added error-free (TwoSum), the rounding error and the
// trailing parts into c.  FP32 instructions only: GB300's FP64 pipe is too narrow for a
// warp-wide FP64 reduction per CTA (it cost ~5 us of a 26 us pack).
__device__ __forceinline__ void pair_add(float &s, float &c, float s2, float c2) {
    const float t = __fadd_rn(s, s2);
    const float bp = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(s2, bp));
    s = t;
    c = __fadd_rn(c, __fadd_rn(c2, e));
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

// ------------------------------------------------------------------ cluster / bulk-copy pack
__device__ __forceinline__ double ld_cluster_f64(uint32_t addr) {
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ float ld_cluster_f32(uint32_t addr) {
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
    return v;
}

// Four consecutive values of one row: one 8-byte store each for hi and lo (16-byte for FP32).
__device__ __forceinline__ void store_split4(const PackArgs &a, size_t idx, float x0, float x1,
                                             float x2, float x3) {
    if (a.split == SPLIT_FP32) {
        *reinterpret_cast<float4 *>(a.Bt32 + idx) = make_float4(x0, x1, x2, x3);
        return;
    }
    const float x[4] = {x0, x1, x2, x3};
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (a.split == SPLIT_BF16) {
            const __nv_bfloat16 hv = __float2bfloat16_rn(x[q]);
            h[q] = __bfloat16_as_ushort(hv);
            l[q] = __bfloat16_as_ushort(__float2bfloat16_rn(x[q] - __bfloat162float(hv)));
        } else {
            const __half hv = __float2half_rn(x[q]);
            h[q] = __half_as_ushort(hv);
            l[q] = __half_as_ushort(__float2half_rn(x[q] - __half2float(hv)));
        }
    }
    *reinterpret_cast<uint2 *>(static_cast<uint16_t *>(a.Bt_hi) + idx) = make_uint2(h[0] | (h[1] << 16), h[2] | (h[3] << 16));
    *reinterpret_cast<uint2 *>(static_cast<uint16_t *>(a.Bt_lo) + idx) = make_uint2(l[0] | (l[1] << 16), l[2] | (l[3] << 16));
}

// A cluster of ceil(N / (4 THREADS)) CTAs per step k.  CTA r bulk-copies the contiguous
// velocities and virials of its atoms r*4*THREADS .. into shared memory (TMA, so the loads are
// asynchronous and the inputs are read once).  Phase 1, thread t takes the atoms t, t+THREADS,
// t+2 THREADS, t+3 THREADS (shared-memory strides of 3 and 9 words across a warp: no bank
// conflicts): row maxima and the exact total-current pairs (acc_exact), combined per CTA in a
// fixed order (unevaluated float pairs across the warp, FP64 across the warps); one cluster
// barrier, then every CTA combines all ranks' maxima in rank order through distributed shared
// memory (each computes the same scales) and rank 0 the current (FP64, rank order).
// Phase 1 also replaces each atom's inputs in shared memory by its row values sqrt(m) v and
// W / sqrt(m).  Phase 2 writes the four B rows of the CTA's atoms: each row is one contiguous run of
// 16-bit values (three per atom; three runs of one per atom, one per direction, with the
// direction-major columns), cut into groups of four values that consecutive threads take in
// order, so that every warp store covers 256 contiguous bytes.  A CTA leaves only after the
// second half of the cluster barrier: its peers may still be reading its partial sums.
// The body of one CTA: step k of the system `a`, rank `rank` of its cluster of `nrank` CTAs.
template <int THREADS>
__device__ __forceinline__ void pack_bulk_body(const PackArgs &a, int k, uint32_t rank, uint32_t nrank) {
    constexpr int APC = 4 * THREADS;
    extern __shared__ float4 pk_smem4[];
    float *sv = reinterpret_cast<float *>(pk_smem4);   // [APC][3]
    float *sw = sv + APC * 3;                          // [APC][9]
    __shared__ float s_mx[THREADS / 32][4];
    __shared__ float s_js[THREADS / 32][3], s_jcc[THREADS / 32][3];
    __shared__ float s_loc[4], s_mul[4];
    __shared__ double s_jc[3];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    const int a0 = (int)rank * APC;
    const int na = max(0, min(APC, a.N - a0));   // a multiple of 4 (N % 4 == 0)
    const long long limit = a.wait_limit > 0 ? a.wait_limit : WAIT_LIMIT_CYCLES;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && na > 0) {
        const uint32_t vb = (uint32_t)na * 12, wb = (uint32_t)na * 36;
        mbar_arrive_expect_tx(&bar, vb + wb);
        const char *gv = reinterpret_cast<const char *>(a.v + ((size_t)k * a.N + a0) * 3);
        const char *gw = reinterpret_cast<const char *>(a.W + ((size_t)k * a.N + a0) * 9);
        for (uint32_t o = 0; o < vb; o += 16384)
            bulk_load(reinterpret_cast<char *>(sv) + o, gv + o, min(16384u, vb - o), &bar);
        for (uint32_t o = 0; o < wb; o += 16384)
            bulk_load(reinterpret_cast<char *>(sw) + o, gw + o, min(16384u, wb - o), &bar);
    }
    bool ok = true;
    if (na > 0) ok = mbar_wait(&bar, 0, &abort_flag, limit);
    float mx[4] = {0.f, 0.f, 0.f, 0.f};
    float js[3] = {0.f, 0.f, 0.f}, jc[3] = {0.f, 0.f, 0.f};
    if (ok) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int ia = (int)threadIdx.x + u * THREADS;
            if (ia >= na) break;
            const float sm = __ldg(a.sqm + a0 + ia), ism = __ldg(a.isqm + a0 + ia);
            float *vu = sv + ia * 3, *wu = sw + ia * 9;
            float x[12];   // the atom's row values sqrt(m) v^b and W^{ab} / sqrt(m)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                x[b] = sm * vu[b];
                mx[0] = fmaxf(mx[0], fabsf(x[b]));
            }
#pragma unroll
            for (int al = 0; al < 3; ++al)
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    x[3 + 3 * al + b] = wu[3 * al + b] * ism;
                    mx[1 + al] = fmaxf(mx[1 + al], fabsf(x[3 + 3 * al + b]));
                    acc_exact(js[al], jc[al], wu[3 * al + b], vu[b]);
                }
            // the scaled values replace the inputs in shared memory (this thread's atom alone),
            // so phase 2 reads them without the masses
#pragma unroll
            for (int b = 0; b < 3; ++b) vu[b] = x[b];
#pragma unroll
            for (int q = 0; q < 9; ++q) wu[q] = x[3 + q];
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int c = 0; c < 4; ++c) mx[c] = fmaxf(mx[c], __shfl_down_sync(FULL_MASK, mx[c], o));
#pragma unroll
        for (int c = 0; c < 3; ++c)
            pair_add(js[c], jc[c], __shfl_down_sync(FULL_MASK, js[c], o), __shfl_down_sync(FULL_MASK, jc[c], o));
    }
    if (lane == 0) {
        for (int c = 0; c < 4; ++c) s_mx[warp][c] = mx[c];
        for (int c = 0; c < 3; ++c) {
            s_js[warp][c] = js[c];
            s_jcc[warp][c] = jc[c];
        }
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        float m = 0.f;
        for (int w = 0; w < THREADS / 32; ++w) m = fmaxf(m, s_mx[w][threadIdx.x]);
        s_loc[threadIdx.x] = m;
    } else if (threadIdx.x >= 32 && threadIdx.x < 35) {   // the warps' pairs in FP64, warp order
        const int c = threadIdx.x - 32;
        double t = 0.0;
        for (int w = 0; w < THREADS / 32; ++w) t += (double)s_js[w][c] + (double)s_jcc[w][c];
        s_jc[c] = t;
    }
    cluster_sync_all();   // every CTA's maxima and current partials are complete
    if (threadIdx.x < 4) {
        const int c = threadIdx.x;
        float m = 0.f;
        for (uint32_t q = 0; q < nrank; ++q) m = fmaxf(m, ld_cluster_f32(mapa_shared(smem_u32(&s_loc[c]), q)));
        int sc = 0;
        if (a.split == SPLIT_FP16 && m > 0.f && isfinite(m)) {
            int e;
            frexpf(m, &e);   // m < 2^e
            sc = 14 - e;     // scaled row maximum < 2^14 keeps the lo parts normal
        }
        s_mul[c] = ldexpf(1.f, sc);
        if (rank == 0) a.col_scale[4 * k + c] = ldexpf(1.f, -(sc + a.e_exp));
    } else if (rank == 0 && threadIdx.x >= 32 && threadIdx.x < 35) {
        const int c = threadIdx.x - 32;
        double t = 0.0;
        for (uint32_t q = 0; q < nrank; ++q) t += ld_cluster_f64(mapa_shared(smem_u32(&s_jc[c]), q));
        a.Jtot[3 * k + c] = t;
        if (a.Jring) {
            const long long t0 = a.t0_dev ? *a.t0_dev : a.t0;
            a.Jring[((t0 + k) % a.R) * 3 + c] = t;
        }
    }
    cluster_arrive_release();   // this CTA has read its peers' partials
    __syncthreads();            // s_mul is visible to the CTA
    if (!ok) {   // the CTA stays alive until its copy has landed (bounded) or given up on
        if (threadIdx.x == 0) {
            if (a.status) set_status(a.status, DEV_TIMEOUT);
            const long long c0 = clock64();
            while (!mbar_try_wait(&bar, 0) && clock64() - c0 < limit) {
            }
        }
    } else {
        const size_t ld = (size_t)a.D_ld;
        const size_t r0 = (size_t)(4 * k) * ld;
        const int q4 = na / 4;              // groups of four atoms (direction-major runs)
        const int G = 3 * q4;               // groups of four values a row
#pragma unroll 1
        for (int g = (int)threadIdx.x; g < G; g += THREADS) {
            int ia[4], bb[4];
            size_t col;
            if (a.npad) {   // direction-major: run b holds atoms a0 .. a0+na-1 at columns b*npad + i
                const int b = g / q4, i0 = 4 * (g - b * q4);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    ia[e] = i0 + e;
                    bb[e] = b;
                }
                col = (size_t)b * a.npad + a0 + i0;
            } else {        // column 3i+b: values 4g .. 4g+3 of the CTA's run
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    ia[e] = (4 * g + e) / 3;
                    bb[e] = (4 * g + e) - 3 * ia[e];
                }
                col = 3 * (size_t)a0 + 4 * (size_t)g;
            }
            float x[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) x[e] = sv[3 * ia[e] + bb[e]] * s_mul[0];
            store_split4(a, r0 + col, x[0], x[1], x[2], x[3]);
#pragma unroll
            for (int al = 0; al < 3; ++al) {
#pragma unroll
                for (int e = 0; e < 4; ++e) x[e] = sw[9 * ia[e] + 3 * al + bb[e]] * s_mul[1 + al];
                store_split4(a, r0 + (size_t)(1 + al) * ld + col, x[0], x[1], x[2], x[3]);
            }
        }
    }
    cluster_wait_acquire();   // peers have read this CTA's partials: its shared memory may go
}

// Shared memory (48 B an atom) allows eight CTAs of 128 threads, four of 256 or two of 512 per
// SM; the register cap of the launch bounds lets as many be resident.
template <int THREADS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS) pack_bulk_kernel(const PackArgs a) {
    griddep_launch_dependents();   // the projection may set up on the SMs this grid leaves
    const uint32_t nrank = cluster_nctarank();
    pack_bulk_body<THREADS>(a, (int)(blockIdx.x / nrank), cluster_ctarank(), nrank);
}

// Several systems in one launch: system j owns the CTAs cta_begin[j] .. cta_begin[j+1) (K_j
// clusters of the common cluster size; ranks beyond a system's atoms hold no atoms and only
// take part in the cluster's combination).
template <int THREADS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS) pack_bulk_group_kernel(const __grid_constant__ PackGroupArgs g) {
    griddep_launch_dependents();
    int j = 0;
    while (j + 1 < g.n && (int)blockIdx.x >= g.cta_begin[j + 1]) ++j;
    const uint32_t nrank = cluster_nctarank();
    pack_bulk_body<THREADS>(g.a[j], (int)((blockIdx.x - (uint32_t)g.cta_begin[j]) / nrank),
                            cluster_ctarank(), nrank);
}

template <int THREADS>
cudaError_t launch_pack_bulk(const PackArgs &a, cudaStream_t s) {
    constexpr int APC = 4 * THREADS;
    const int smem = APC * 48;
    static cudaError_t attr = cudaFuncSetAttribute(pack_bulk_kernel<THREADS>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (attr != cudaSuccess) return attr;
    const int csize = (a.N + APC - 1) / APC;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(a.K * csize), 1, 1);
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
    return cudaLaunchKernelEx(&cfg, pack_bulk_kernel<THREADS>, a);
}

}  // namespace

namespace {
// CTA size of the bulk-copy pack of a system of N atoms (four atoms a thread): one CTA a step
// and eight an SM up to 512 atoms, clusters of up to 8 CTAs of 256 (four an SM) up to 8192,
// of 512 beyond.
int pack_threads(int N) { return N <= 4 * 128 ? 128 : N <= 8 * 1024 ? 256 : 512; }

bool bulk_ok(const PackArgs &a) {
    const auto al16 = [](const void *q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
    return a.N % 4 == 0 && al16(a.v) && al16(a.W) && al16(a.sqm) && al16(a.isqm) &&
           (a.split == SPLIT_FP32 ? al16(a.Bt32) : true);
}

template <int THREADS>
cudaError_t launch_pack_bulk_group(PackGroupArgs g, int csize, cudaStream_t s) {
    constexpr int APC = 4 * THREADS;
    const int smem = APC * 48;
    static cudaError_t attr = cudaFuncSetAttribute(pack_bulk_group_kernel<THREADS>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (attr != cudaSuccess) return attr;
    g.cta_begin[0] = 0;
    for (int j = 0; j < g.n; ++j) g.cta_begin[j + 1] = g.cta_begin[j] + g.a[j].K * csize;
    if (g.cta_begin[g.n] == 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)g.cta_begin[g.n], 1, 1);
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
    return cudaLaunchKernelEx(&cfg, pack_bulk_group_kernel<THREADS>, g);
}
}  // namespace

cudaError_t launch_pack_group(const PackGroupArgs &g, const cudaStream_t *streams, int n_streams,
                              int *n_launches) {
    *n_launches = 0;
    if (g.n < 1 || g.n > TC_MAX_GROUP) return cudaErrorInvalidValue;
    int nmax = 0;
    for (int j = 0; j < g.n; ++j) {
        if (!bulk_ok(g.a[j])) return cudaErrorNotSupported;
        nmax = std::max(nmax, g.a[j].N);
    }
    if (nmax > 8 * 2048) return cudaErrorNotSupported;
    // one launch per (CTA size, cluster size): every system is packed by the CTA size it gets
    // alone (so its results are bitwise those of a solo push), and no rank is idle
    for (const int threads : {128, 256, 512}) {
        const int apc = 4 * threads;
        for (int cs = 1; cs <= 8; ++cs) {
            PackGroupArgs sub{};
            for (int j = 0; j < g.n; ++j)
                if (pack_threads(g.a[j].N) == threads &&
                    ((g.a[j].N + apc - 1) / apc == cs || (g.a[j].N == 0 && cs == 1)))
                    sub.a[sub.n++] = g.a[j];
            if (sub.n == 0) continue;
            const cudaStream_t s = streams[*n_launches % n_streams];   // independent systems
            const cudaError_t e = threads == 128 ? launch_pack_bulk_group<128>(sub, cs, s)
                                  : threads == 256 ? launch_pack_bulk_group<256>(sub, cs, s)
                                                   : launch_pack_bulk_group<512>(sub, cs, s);
            if (e != cudaSuccess) return e;
            ++*n_launches;
        }
    }
    return cudaSuccess;
}

cudaError_t launch_pack(const PackArgs &a, cudaStream_t s) {
    if (a.K <= 0) return cudaSuccess;
    if (bulk_ok(a) && a.N <= 8 * 2048) {
        const int threads = pack_threads(a.N);
        return threads == 128 ? launch_pack_bulk<128>(a, s)
               : threads == 256 ? launch_pack_bulk<256>(a, s)
                                : launch_pack_bulk<512>(a, s);
    }
    pack_kernel<<<a.K, PACK_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace mhc
