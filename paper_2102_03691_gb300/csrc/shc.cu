// Spectral heat current (SHC, Eqs. 20-23): the virial-velocity correlation
//   Ksum^{ab}(l) += sum_{t in block} sum_i W_i^{ab}(t - l) v_i^b(t),  t - l >= 0,
// accumulated at run time over blocks of K samples with a ring of past virials, and the
// spectrum kappa(omega) = 2 Ktilde(omega) / (V T |F_e|) on read.
// Two paths: the tensor-core banded contraction of k_shc_tc.cu (FP16x3 / BF16x3, default)
// and the FP32 CUDA-core kernel below (MHC_PREC_FP32).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mhc.h"
#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int SHC_LAGS = 256;      // lags per CTA (lag tile)
constexpr int SHC_ATILE = 2;       // atoms per CTA
constexpr int SHC_THREADS = 256;   // one thread per lag of the tile
constexpr double WMK = 1602.176634;

// One CTA: SHC_ATILE atoms x SHC_LAGS lags [L0, L0 + 256).  Warp w owns lags L0 + 32w + lane
// and walks the shifted time tau = t - l shared by the warp, so W(tau) is a broadcast and
// v(tau + l) is a conflict-free vector load.  Shared memory:
//   sW[a][j][12]  W_i^{ab} of times tw0 + j, tw0 = t0 - L0 - 255 (zero before t = 0)
//   sv[a][k][4]   v_i of block step k - 32 (zero outside the block)
__global__ void __launch_bounds__(SHC_THREADS) shc_corr_kernel(const float *__restrict__ v,
                                                               const float *__restrict__ Wring,
                                                               int R, int N, int K, int nc,
                                                               long long t0, float *partials,
                                                               int nc_pad) {
    extern __shared__ float4 smem4[];
    const int L0 = blockIdx.y * SHC_LAGS;
    const int atom0 = blockIdx.x * SHC_ATILE;
    const int nw = K + SHC_LAGS - 1;    // W window entries
    const int nv = K + 64;              // v entries (32 zeros on each side)
    float4 *sW = smem4;                               // [ATILE][nw][3]
    float4 *sv = smem4 + SHC_ATILE * nw * 3;          // [ATILE][nv]
    const long long tw0 = t0 - L0 - (SHC_LAGS - 1);
    for (int q = threadIdx.x; q < SHC_ATILE * nw; q += SHC_THREADS) {
        const int a = q / nw, j = q - a * nw;
        const int i = atom0 + a;
        const long long tt = tw0 + j;
        float w[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (i < N && tt >= 0) {
            const float *src = Wring + ((tt % R) * (long long)N + i) * 9;
#pragma unroll
            for (int c = 0; c < 9; ++c) w[c] = src[c];
        }
        float4 *d = sW + ((size_t)a * nw + j) * 3;
        d[0] = make_float4(w[0], w[1], w[2], w[3]);
        d[1] = make_float4(w[4], w[5], w[6], w[7]);
        d[2] = make_float4(w[8], 0.f, 0.f, 0.f);
    }
    for (int q = threadIdx.x; q < SHC_ATILE * nv; q += SHC_THREADS) {
        const int a = q / nv, k = q - a * nv - 32;
        const int i = atom0 + a;
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < N && k >= 0 && k < K) {
            const float *src = v + ((long long)k * N + i) * 3;
            x = make_float4(src[0], src[1], src[2], 0.f);
        }
        sv[(size_t)a * nv + k + 32] = x;
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lam = warp * 32 + lane;   // lag within the tile
    float acc[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) acc[c] = 0.f;
    for (int a = 0; a < SHC_ATILE; ++a) {
        const float4 *wa = sW + (size_t)a * nw * 3;
        const float4 *va = sv + (size_t)a * nv;
        // tau_rel = i - 32 warp - 31: step k = tau_rel + lam = i - 31 + lane
        for (int it = 0; it < K + 31; ++it) {
            const int j = it - warp * 32 - 31 + (SHC_LAGS - 1);   // window index of W(tau)
            const float4 w0 = wa[j * 3], w1 = wa[j * 3 + 1], w2 = wa[j * 3 + 2];
            const float4 x = va[it - 31 + lane + 32];
            // W^{ab} v^b, row-major ab: w0 = (xx, xy, xz, yx), w1 = (yy, yz, zx, zy), w2.x = zz
            acc[0] = fmaf(w0.x, x.x, acc[0]);
            acc[1] = fmaf(w0.y, x.y, acc[1]);
            acc[2] = fmaf(w0.z, x.z, acc[2]);
            acc[3] = fmaf(w0.w, x.x, acc[3]);
            acc[4] = fmaf(w1.x, x.y, acc[4]);
            acc[5] = fmaf(w1.y, x.z, acc[5]);
            acc[6] = fmaf(w1.z, x.x, acc[6]);
            acc[7] = fmaf(w1.w, x.y, acc[7]);
            acc[8] = fmaf(w2.x, x.z, acc[8]);
        }
    }
    const int l = L0 + lam;
    if (l < nc) {
#pragma unroll
        for (int c = 0; c < 9; ++c)
            partials[((size_t)blockIdx.x * 9 + c) * nc_pad + l] = acc[c];
    }
}

// Ksum[c][l] += sum over atom tiles of partials (FP64).  One CTA per (pair c, 32 lags):
// warp w sums tiles w, w + 32, ... in order, then warp 0 adds the 32 warp sums in order
// (a fixed tree: deterministic).
constexpr int RED_WARPS = 32;
__global__ void __launch_bounds__(RED_WARPS * 32) shc_reduce_kernel(const float *__restrict__ partials,
                                                                   int n_tiles, int nc, int nc_pad,
                                                                   double *Ksum) {
    __shared__ double part[RED_WARPS][33];
    const int c = blockIdx.y;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int l = blockIdx.x * 32 + lane;
    double s = 0.0;
    if (l < nc)
        for (int t = w; t < n_tiles; t += RED_WARPS)
            s += (double)partials[((size_t)t * 9 + c) * nc_pad + l];
    part[w][lane] = s;
    __syncthreads();
    if (w == 0 && l < nc) {
        double tot = 0.0;
        for (int q = 0; q < RED_WARPS; ++q) tot += part[q][lane];
        Ksum[(size_t)c * nc + l] += tot;
    }
}

// kappa[c][k] = 2 Ktilde_c(2 pi f_k) / (V T |F_e|), Ktilde = 2 dt sum_l trap_l w_l K_l cos(omega_k l dt),
// as a small FP64 product: the per-lag coefficients cl = trap_l w_l K_l (K_l = Ksum / count) of
// pair c times a table C[l][k] = cos(2 pi f_k l dt) that is rebuilt only when the frequencies
// change.  CTA = (16 frequencies, pair c); thread (g, kk) sums lags g, g + 8, ... of frequency kk,
// the eight lag groups are added in order (deterministic).
constexpr int KAPPA_MAX_LAGS = 4096;
constexpr int KAPPA_FREQ = 16, KAPPA_GROUPS = 8;
__global__ void shc_cos_table_kernel(const double *f, int n_freq, int nc, double dt, double *C) {
    const double PI = 3.14159265358979323846;
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= (long long)nc * n_freq) return;
    const int l = (int)(q / n_freq), k = (int)(q % n_freq);
    C[q] = cos(2.0 * PI * f[k] * dt * (double)l);
}

// tw[w][l] = trap_l w_l for window w = 0 (none) and 1 (Hann), once per handle
__global__ void shc_weight_table_kernel(int nc, double *tw) {
    const double PI = 3.14159265358979323846;
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nc) return;
    const double trap = (l == 0 || l == nc - 1) ? 0.5 : 1.0;
    tw[l] = trap;
    tw[nc + l] = trap * (nc > 1 ? 0.5 * (1.0 + cos(PI * l / (double)(nc - 1))) : 1.0);
}

__global__ void __launch_bounds__(KAPPA_FREQ * KAPPA_GROUPS) shc_kappa_kernel(
    const double *Ksum, int nc, long long T_s, double dt, double coef, const double *tw,
    const double *C, int n_freq, double *kappa) {
    __shared__ double cl[KAPPA_MAX_LAGS];
    __shared__ double part[KAPPA_GROUPS][KAPPA_FREQ];
    const int c = blockIdx.y;
    for (int l = threadIdx.x; l < nc; l += blockDim.x) {
        const long long cnt = T_s - l;
        cl[l] = cnt > 0 ? tw[l] * (Ksum[(size_t)c * nc + l] / (double)cnt) : 0.0;
    }
    __syncthreads();
    const int kk = threadIdx.x % KAPPA_FREQ, g = threadIdx.x / KAPPA_FREQ;
    const int k = blockIdx.x * KAPPA_FREQ + kk;
    double s = 0.0;
    if (k < n_freq)
        for (int l = g; l < nc; l += KAPPA_GROUPS) s = fma(cl[l], C[(size_t)l * n_freq + k], s);
    part[g][kk] = s;
    __syncthreads();
    if (g == 0 && k < n_freq) {
        double t = 0.0;
        for (int q = 0; q < KAPPA_GROUPS; ++q) t += part[q][kk];
        kappa[(size_t)c * n_freq + k] = coef * 2.0 * (2.0 * t * dt);
    }
}

}  // namespace

struct mhc_shc {
    int device = 0;
    cudaStream_t stream = nullptr;
    int64_t N = 0;
    int nc = 0, nc_pad = 0, k_max = 0, R = 0, n_tiles = 0, sm_count = 0;
    int precision = MHC_PREC_FP16X3;
    double dt = 0, T = 0, V = 0, Fe = 0;
    long long steps = 0;
    float *Wring = nullptr, *partials = nullptr;
    // host inputs: two staging pairs filled on a copy stream (the upload of one push overlaps
    // the kernels of the previous one; a pair is reused only after the push that read it)
    float *v_stage[2] = {nullptr, nullptr}, *W_stage[2] = {nullptr, nullptr};
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t copy_done[2] = {nullptr, nullptr}, use_done[2] = {nullptr, nullptr};
    bool use_pending[2] = {false, false};
    int stage_next = 0;
    double *Ksum = nullptr, *out = nullptr;
    long long *counts = nullptr;
    size_t out_cap = 0;
    std::string err;
    // tensor-core path: 16-bit virial ring [9 R_tc][N_pad], velocities [3 Kpad][N_pad]
    int64_t N_pad = 0;
    int R_tc = 0, Kpad = 0;
    int cta_slots = 0;   // CTAs of the tensor-core kernel resident at once (clusters of two)
    void *A_hi = nullptr, *A_lo = nullptr, *B_hi = nullptr, *B_lo = nullptr;
    float *scaleA = nullptr, *scaleB = nullptr, *tc_partials = nullptr;
    mhc::ShcTcParams tcp{};
    int *status = nullptr;   // sticky device status (a bounded wait that gave up)
    // frequencies of the last spectrum read, as uploaded (a pageable upload per read would
    // make the host wait for the stream)
    std::vector<double> freq_dev_copy;
    // optional CUDA-event timing of the correlation kernel
    bool profile = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_events;
    size_t prof_used = 0;
};

namespace {
thread_local std::string g_shc_create_error;

mhc_status sfail(mhc_shc *s, mhc_status st, const char *fmt, ...) {
    char msg[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    if (s) s->err = msg;
    else g_shc_create_error = msg;
    return st;
}

#define SHC_CUDA(s, call)                                                                         \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return sfail((s), e_ == cudaErrorMemoryAllocation ? MHC_ERR_OOM : MHC_ERR_CUDA,       \
                         "%s failed: %s", #call, cudaGetErrorString(e_));                        \
    } while (0)

size_t shc_smem(int K) {
    return ((size_t)SHC_ATILE * (K + SHC_LAGS - 1) * 3 + (size_t)SHC_ATILE * (K + 64)) * sizeof(float4);
}

bool shc_is_tc(const mhc_shc *s) { return s->precision != MHC_PREC_FP32; }

void free_path(mhc_shc *s) {
    for (void **q : {(void **)&s->Wring, (void **)&s->partials, &s->A_hi, &s->A_lo, &s->B_hi,
                     &s->B_lo, (void **)&s->scaleA, (void **)&s->scaleB, (void **)&s->tc_partials}) {
        cudaFree(*q);
        *q = nullptr;
    }
}

// Buffers of the selected path (zeroed: the rings start empty, padding atoms stay zero).
cudaError_t alloc_path(mhc_shc *s) {
    free_path(s);
    cudaError_t e;
    auto get = [&](void **q, size_t bytes) {
        if ((e = cudaMalloc(q, bytes)) != cudaSuccess) return false;
        return (e = cudaMemsetAsync(*q, 0, bytes, s->stream)) == cudaSuccess;
    };
    if (!shc_is_tc(s)) {
        if (!get((void **)&s->Wring, sizeof(float) * (size_t)s->R * s->N * 9)) return e;
        if (!get((void **)&s->partials, sizeof(float) * (size_t)s->n_tiles * 9 * s->nc_pad)) return e;
        return cudaFuncSetAttribute(shc_corr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)shc_smem(s->k_max));
    }
    const size_t a = (size_t)9 * s->R_tc * s->N_pad * 2, b = (size_t)3 * s->Kpad * s->N_pad * 2;
    const size_t units = std::max<size_t>((size_t)9 * mhc::SHC_TC_MAX_PAIRS, (size_t)s->sm_count);
    if (!get(&s->A_hi, a) || !get(&s->A_lo, a) || !get(&s->B_hi, b) || !get(&s->B_lo, b) ||
        !get((void **)&s->scaleA, sizeof(float) * 9 * s->R_tc) ||
        !get((void **)&s->scaleB, sizeof(float) * 3 * s->Kpad) ||
        !get((void **)&s->tc_partials, sizeof(float) * units * mhc::SHC_TC_PART))
        return e;
    mhc::ShcTcParams &P = s->tcp;
    const uint32_t T = mhc::SHC_TC_TILE, TS = mhc::SHC_TC_STEP_TILE;
    // boxes of 32 atoms (64-byte rows, 64-byte swizzle) x 128 ring rows / 128 velocity rows
    // (each CTA of a cluster loads one half of the 256 velocity rows of a tile)
    if (mhc::tc_make_tmap(&P.tmA_hi, s->A_hi, (uint64_t)9 * s->R_tc, s->N_pad, s->N_pad, T, 32) ||
        mhc::tc_make_tmap(&P.tmA_lo, s->A_lo, (uint64_t)9 * s->R_tc, s->N_pad, s->N_pad, T, 32) ||
        mhc::tc_make_tmap(&P.tmB_hi, s->B_hi, (uint64_t)3 * s->Kpad, s->N_pad, s->N_pad, TS / 2, 32) ||
        mhc::tc_make_tmap(&P.tmB_lo, s->B_lo, (uint64_t)3 * s->Kpad, s->N_pad, s->N_pad, TS / 2, 32))
        return cudaErrorInvalidValue;
    P.scaleA = s->scaleA;
    P.scaleB = s->scaleB;
    P.partials = s->tc_partials;
    P.R = s->R_tc;
    P.nR = s->R_tc / (int)T;
    P.Kpad = s->Kpad;
    P.nc = s->nc;
    P.n_kb = (int)(s->N_pad / 32);
    P.wait_limit = 2000000000ll;
    P.status = s->status;
    const int clusters = mhc::shc_tc_max_clusters();
    s->cta_slots = clusters > 0 ? 2 * clusters : s->sm_count;
    P.idesc = mhc::idesc_f16(s->precision == MHC_PREC_BF16X3 ? 1u : 0u, 2 * T, TS);   // M = 256 (CTA pair)
    return cudaSuccess;
}

mhc_status shc_check_status(mhc_shc *s) {
    int st = 0;
    if (cudaMemcpyAsync(&st, s->status, sizeof(int), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return sfail(s, MHC_ERR_CUDA, "reading the device status failed");
    if (st == mhc::DEV_TIMEOUT) return sfail(s, MHC_ERR_TIMEOUT, "a tensor-core SHC kernel gave up waiting on a barrier");
    if (st != 0) return sfail(s, MHC_ERR_STATE, "device status word %d", st);
    return MHC_OK;
}

long long floor_div(long long a, long long b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// Tile pairs of the block [t0, t0 + K) that touch the band 0 <= t - tau < nc, tau >= 0,
// and the split of the atom axis that fills the SMs.
bool plan_tiles(mhc_shc *s, int K) {
    mhc::ShcTcParams &P = s->tcp;
    const long long T = mhc::SHC_TC_TILE, TS = mhc::SHC_TC_STEP_TILE, t0 = s->steps;
    int n = 0;
    for (int q = 0; q * TS < K; ++q) {
        const long long tmin = t0 + q * TS, tmax = t0 + std::min<long long>((q + 1) * TS, K) - 1;
        const long long p0 = std::max<long long>(0, floor_div(tmin - s->nc + 1, T));
        long long p1 = tmax / T;
        // tiles go to clusters in pairs (p, p+1); an extra tile past tmax only holds lags < 0
        if ((p1 - p0 + 1) % 2) ++p1;
        for (long long pp = p0; pp <= p1; ++pp) {
            if (n == mhc::SHC_TC_MAX_PAIRS) return false;
            P.p_tile[n] = (int)pp;
            P.q_tile[n] = q;
            ++n;
        }
    }
    P.n_pairs = n;
    P.t0 = t0;
    P.K = K;
    const int chunks = (int)(s->N_pad / 128);
    int splits = std::max(1, s->cta_slots / (9 * n));
    splits = std::min(splits, chunks);
    const int per = (chunks + splits - 1) / splits;   // chunks per split
    P.kb_per_split = per * (128 / 32);
    P.splits = (chunks + per - 1) / per;
    return true;
}
}  // namespace

extern "C" {

mhc_status mhc_shc_create(mhc_shc **out, int32_t device, void *stream, int64_t n_atoms,
                          int32_t n_lags, int32_t k_max, double dt_ps, double T_K, double V_A3,
                          const double *F_e) {
    if (!out) return MHC_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_atoms < 1 || n_lags < 1 || n_lags > KAPPA_MAX_LAGS || k_max < 1 || k_max > 1024 ||
        !(dt_ps > 0) || !(T_K > 0) ||
        !(V_A3 > 0) || !F_e)
        return sfail(nullptr, MHC_ERR_INVALID_ARG,
                     "need n_atoms, n_lags >= 1, 1 <= k_max <= 1024, positive dt, T, V and F_e");
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) return sfail(nullptr, MHC_ERR_CUDA, "no CUDA device %d", device);
    if (!(prop.major == 10 && prop.minor == 3))
        return sfail(nullptr, MHC_ERR_UNSUPPORTED, "built for sm_103a only");
    auto *s = new mhc_shc();
    s->device = device;
    s->stream = static_cast<cudaStream_t>(stream);
    s->N = n_atoms;
    s->nc = n_lags;
    s->nc_pad = (n_lags + SHC_LAGS - 1) / SHC_LAGS * SHC_LAGS;
    s->k_max = k_max;
    s->R = k_max + s->nc_pad;   // holds every time the last lag tile reads
    s->n_tiles = (int)((n_atoms + SHC_ATILE - 1) / SHC_ATILE);
    s->sm_count = prop.multiProcessorCount;
    s->N_pad = (n_atoms + 127) / 128 * 128;
    s->Kpad = (k_max + mhc::SHC_TC_STEP_TILE - 1) / mhc::SHC_TC_STEP_TILE * mhc::SHC_TC_STEP_TILE;
    s->R_tc = (k_max + n_lags + 127) / 128 * 128;   // >= K + nc - 1 live samples, whole tiles
    s->dt = dt_ps;
    s->T = T_K;
    s->V = V_A3;
    s->Fe = std::sqrt(F_e[0] * F_e[0] + F_e[1] * F_e[1] + F_e[2] * F_e[2]);
    auto fail_free = [&](cudaError_t er) {
        mhc_shc_destroy(s);
        return sfail(nullptr, er == cudaErrorMemoryAllocation ? MHC_ERR_OOM : MHC_ERR_CUDA,
                     "allocation: %s", cudaGetErrorString(er));
    };
    if ((e = cudaSetDevice(device)) != cudaSuccess) return fail_free(e);
    if ((e = cudaMalloc(&s->status, sizeof(int))) != cudaSuccess) return fail_free(e);
    if ((e = cudaMemsetAsync(s->status, 0, sizeof(int), s->stream)) != cudaSuccess) return fail_free(e);
    if ((e = alloc_path(s)) != cudaSuccess) return fail_free(e);
    if ((e = cudaMalloc(&s->Ksum, sizeof(double) * 9 * n_lags)) != cudaSuccess) return fail_free(e);
    if ((e = cudaMalloc(&s->counts, sizeof(long long) * n_lags)) != cudaSuccess) return fail_free(e);
    for (int q = 0; q < 2; ++q) {
        if ((e = cudaMalloc(&s->v_stage[q], sizeof(float) * (size_t)k_max * n_atoms * 3)) != cudaSuccess) return fail_free(e);
        if ((e = cudaMalloc(&s->W_stage[q], sizeof(float) * (size_t)k_max * n_atoms * 9)) != cudaSuccess) return fail_free(e);
        if ((e = cudaEventCreateWithFlags(&s->copy_done[q], cudaEventDisableTiming)) != cudaSuccess) return fail_free(e);
        if ((e = cudaEventCreateWithFlags(&s->use_done[q], cudaEventDisableTiming)) != cudaSuccess) return fail_free(e);
    }
    if ((e = cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking)) != cudaSuccess) return fail_free(e);
    if ((e = cudaMemsetAsync(s->Ksum, 0, sizeof(double) * 9 * n_lags, s->stream)) != cudaSuccess) return fail_free(e);
    if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess) return fail_free(e);
    *out = s;
    return MHC_OK;
}

void mhc_shc_destroy(mhc_shc *s) {
    if (!s) return;
    cudaStreamSynchronize(s->stream);
    free_path(s);
    for (auto &e : s->prof_events) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    cudaFree(s->status);
    cudaFree(s->Ksum);
    cudaFree(s->counts);
    if (s->copy_stream) {
        cudaStreamSynchronize(s->copy_stream);
        cudaStreamDestroy(s->copy_stream);
    }
    for (int q = 0; q < 2; ++q) {
        cudaFree(s->v_stage[q]);
        cudaFree(s->W_stage[q]);
        if (s->copy_done[q]) cudaEventDestroy(s->copy_done[q]);
        if (s->use_done[q]) cudaEventDestroy(s->use_done[q]);
    }
    cudaFree(s->out);
    delete s;
}

const char *mhc_shc_last_error(const mhc_shc *s) { return s ? s->err.c_str() : g_shc_create_error.c_str(); }

mhc_status mhc_shc_set_precision(mhc_shc *s, int32_t precision) {
    if (!s) return MHC_ERR_INVALID_ARG;
    if (precision < MHC_PREC_FP32 || precision > MHC_PREC_FP16X3)
        return sfail(s, MHC_ERR_INVALID_ARG, "unknown precision %d", precision);
    if (s->steps != 0) return sfail(s, MHC_ERR_INVALID_ARG, "the precision can only change before the first push");
    if (precision == s->precision) return MHC_OK;
    SHC_CUDA(s, cudaSetDevice(s->device));
    SHC_CUDA(s, cudaStreamSynchronize(s->stream));
    s->precision = precision;
    SHC_CUDA(s, alloc_path(s));
    SHC_CUDA(s, cudaStreamSynchronize(s->stream));
    return MHC_OK;
}

mhc_status mhc_shc_push(mhc_shc *s, const float *v, const float *W, int32_t K, int32_t where) {
    if (!s) return MHC_ERR_INVALID_ARG;
    if (!v || !W || K < 1 || K > s->k_max || (where != MHC_MEM_HOST && where != MHC_MEM_DEVICE))
        return sfail(s, MHC_ERR_INVALID_ARG, "bad inputs or K=%d outside [1, %d]", K, s->k_max);
    SHC_CUDA(s, cudaSetDevice(s->device));
    const size_t nv = (size_t)K * s->N * 3, nwf = (size_t)K * s->N * 9;
    int stage = -1;
    if (where == MHC_MEM_HOST) {   // upload, and return only once the caller's memory is read
        stage = s->stage_next;
        s->stage_next ^= 1;
        if (s->use_pending[stage]) SHC_CUDA(s, cudaStreamWaitEvent(s->copy_stream, s->use_done[stage], 0));
        SHC_CUDA(s, cudaMemcpyAsync(s->v_stage[stage], v, nv * 4, cudaMemcpyHostToDevice, s->copy_stream));
        SHC_CUDA(s, cudaMemcpyAsync(s->W_stage[stage], W, nwf * 4, cudaMemcpyHostToDevice, s->copy_stream));
        SHC_CUDA(s, cudaEventRecord(s->copy_done[stage], s->copy_stream));
        SHC_CUDA(s, cudaEventSynchronize(s->copy_done[stage]));
        v = s->v_stage[stage];
        W = s->W_stage[stage];
    }
    auto release = [&]() -> mhc_status {
        if (stage >= 0) {
            SHC_CUDA(s, cudaEventRecord(s->use_done[stage], s->stream));
            s->use_pending[stage] = true;
        }
        return MHC_OK;
    };
    if (shc_is_tc(s)) {
        if (!plan_tiles(s, K)) return sfail(s, MHC_ERR_UNSUPPORTED, "too many tile pairs for K=%d", K);
        SHC_CUDA(s, mhc::launch_shc_tc_pack(v, W, (int)s->N, (int)s->N_pad, K, s->Kpad, s->R_tc, s->steps,
                                            s->precision == MHC_PREC_BF16X3 ? mhc::SPLIT_BF16 : mhc::SPLIT_FP16,
                                            s->A_hi, s->A_lo, s->B_hi, s->B_lo, s->scaleA, s->scaleB,
                                            s->status, s->tcp.wait_limit, s->stream));
        cudaEvent_t ev1 = nullptr;
        if (s->profile) {
            if (s->prof_used == s->prof_events.size()) {
                cudaEvent_t a0, a1;
                SHC_CUDA(s, cudaEventCreate(&a0));
                SHC_CUDA(s, cudaEventCreate(&a1));
                s->prof_events.emplace_back(a0, a1);
            }
            SHC_CUDA(s, cudaEventRecord(s->prof_events[s->prof_used].first, s->stream));
            ev1 = s->prof_events[s->prof_used++].second;
        }
        SHC_CUDA(s, mhc::launch_shc_tc(s->tcp, s->stream));
        if (ev1) SHC_CUDA(s, cudaEventRecord(ev1, s->stream));
        mhc::launch_shc_tc_reduce(s->tcp, s->Ksum, s->stream);
        SHC_CUDA(s, cudaGetLastError());
        s->steps += K;
        return release();
    }
    // this block's virials into the ring at rows (t0 + k) mod R (at most two segments)
    const size_t row = (size_t)s->N * 9 * sizeof(float);
    const cudaMemcpyKind kind = cudaMemcpyDeviceToDevice;
    const int r0 = (int)(s->steps % s->R);
    const int first = std::min(K, s->R - r0);
    SHC_CUDA(s, cudaMemcpyAsync((char *)s->Wring + r0 * row, W, first * row, kind, s->stream));
    if (first < K)
        SHC_CUDA(s, cudaMemcpyAsync(s->Wring, (const char *)W + first * row, (K - first) * row, kind, s->stream));
    (void)nwf;
    dim3 grid(s->n_tiles, s->nc_pad / SHC_LAGS);
    cudaEvent_t ev1 = nullptr;
    if (s->profile) {
        if (s->prof_used == s->prof_events.size()) {
            cudaEvent_t a0, a1;
            SHC_CUDA(s, cudaEventCreate(&a0));
            SHC_CUDA(s, cudaEventCreate(&a1));
            s->prof_events.emplace_back(a0, a1);
        }
        SHC_CUDA(s, cudaEventRecord(s->prof_events[s->prof_used].first, s->stream));
        ev1 = s->prof_events[s->prof_used++].second;
    }
    shc_corr_kernel<<<grid, SHC_THREADS, shc_smem(K), s->stream>>>(v, s->Wring, s->R, (int)s->N, K,
                                                                   s->nc, s->steps, s->partials,
                                                                   s->nc_pad);
    if (ev1) SHC_CUDA(s, cudaEventRecord(ev1, s->stream));
    shc_reduce_kernel<<<dim3((s->nc + 31) / 32, 9), RED_WARPS * 32, 0, s->stream>>>(
        s->partials, s->n_tiles, s->nc, s->nc_pad, s->Ksum);
    SHC_CUDA(s, cudaGetLastError());
    s->steps += K;
    return release();
}

mhc_status mhc_shc_set_profile(mhc_shc *s, int32_t on) {
    if (!s) return MHC_ERR_INVALID_ARG;
    s->profile = on != 0;
    s->prof_used = 0;
    return MHC_OK;
}

mhc_status mhc_shc_kernel_time(mhc_shc *s, double *ms, int64_t *launches) {
    if (!s) return MHC_ERR_INVALID_ARG;
    if (!s->profile) return sfail(s, MHC_ERR_INVALID_ARG, "profiling is off (mhc_shc_set_profile)");
    SHC_CUDA(s, cudaStreamSynchronize(s->stream));
    double total = 0.0;
    for (size_t q = 0; q < s->prof_used; ++q) {
        float t = 0.f;
        SHC_CUDA(s, cudaEventElapsedTime(&t, s->prof_events[q].first, s->prof_events[q].second));
        total += t;
    }
    if (ms) *ms = total;
    if (launches) *launches = (int64_t)s->prof_used;
    s->prof_used = 0;
    return MHC_OK;
}

mhc_status mhc_shc_read_corr(mhc_shc *s, double *Ksum, int64_t *count, int32_t where) {
    if (!s) return MHC_ERR_INVALID_ARG;
    const cudaMemcpyKind kind = where == MHC_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (Ksum) SHC_CUDA(s, cudaMemcpyAsync(Ksum, s->Ksum, sizeof(double) * 9 * s->nc, kind, s->stream));
    if (count) {
        std::vector<long long> c(s->nc);
        for (int l = 0; l < s->nc; ++l) c[l] = s->steps > l ? s->steps - l : 0;
        if (where == MHC_MEM_HOST) std::memcpy(count, c.data(), sizeof(long long) * s->nc);
        else SHC_CUDA(s, cudaMemcpy(count, c.data(), sizeof(long long) * s->nc, cudaMemcpyHostToDevice));
    }
    if (where == MHC_MEM_HOST) return shc_check_status(s);
    return MHC_OK;
}

mhc_status mhc_shc_read_kappa(mhc_shc *s, const double *f_THz, int32_t n_freq, int32_t window,
                              double *kappa, int32_t where) {
    if (!s) return MHC_ERR_INVALID_ARG;
    if (!f_THz || !kappa || n_freq < 1 || (window != 0 && window != 1))
        return sfail(s, MHC_ERR_INVALID_ARG, "need frequencies, an output, window 0 or 1");
    SHC_CUDA(s, cudaSetDevice(s->device));
    const size_t need = sizeof(double) * ((size_t)n_freq * 10 + (size_t)n_freq * s->nc + 2 * (size_t)s->nc);
    if (s->out_cap < need) {
        cudaStreamSynchronize(s->stream);
        cudaFree(s->out);
        s->out = nullptr;
        s->freq_dev_copy.clear();
        SHC_CUDA(s, cudaMalloc(&s->out, need));
        s->out_cap = need;
    }
    double *df = s->out + (size_t)n_freq * 9;
    double *ctab = df + n_freq;   // [nc][n_freq] cos(2 pi f_k l dt)
    double *tw = ctab + (size_t)n_freq * s->nc;   // [2][nc] trapezoid x window weights
    if (s->freq_dev_copy.size() != (size_t)n_freq ||
        std::memcmp(s->freq_dev_copy.data(), f_THz, sizeof(double) * n_freq) != 0) {
        s->freq_dev_copy.assign(f_THz, f_THz + n_freq);
        SHC_CUDA(s, cudaMemcpyAsync(df, s->freq_dev_copy.data(), sizeof(double) * n_freq,
                                    cudaMemcpyHostToDevice, s->stream));
        const long long n = (long long)s->nc * n_freq;
        shc_cos_table_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s->stream>>>(df, n_freq, s->nc, s->dt, ctab);
        shc_weight_table_kernel<<<(s->nc + 255) / 256, 256, 0, s->stream>>>(s->nc, tw);
        SHC_CUDA(s, cudaGetLastError());
        SHC_CUDA(s, cudaStreamSynchronize(s->stream));   // the host copy may change before the copy runs
    }
    const double coef = s->Fe > 0 ? WMK / (s->V * s->T * s->Fe) : 0.0;
    shc_kappa_kernel<<<dim3((n_freq + KAPPA_FREQ - 1) / KAPPA_FREQ, 9), KAPPA_FREQ * KAPPA_GROUPS, 0,
                       s->stream>>>(s->Ksum, s->nc, s->steps, s->dt, coef, tw + (size_t)window * s->nc,
                                    ctab, n_freq, s->out);
    SHC_CUDA(s, cudaGetLastError());
    const cudaMemcpyKind kind = where == MHC_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    SHC_CUDA(s, cudaMemcpyAsync(kappa, s->out, sizeof(double) * 9 * n_freq, kind, s->stream));
    if (where == MHC_MEM_HOST) return shc_check_status(s);
    return MHC_OK;
}

}  // extern "C"
