// mhc_binned_current_noalloc: the binned modal current of one block for callers that
// cannot allocate device memory.
//
// Who needs this: an MD engine that calls the analysis from inside its time-step loop,
// where a cudaMalloc would synchronise the whole device and stall the integrator, or a host
// application that hands out device memory only from a pool it reserved at start-up and
// forbids libraries to allocate behind its back.  Those callers can still pass their own
// input and output buffers, so this entry point computes into them and keeps every
// intermediate array in one fixed, file-scope device buffer instead of allocating.
//
// The buffer is a static __device__ array of MHC_NOALLOC_SCRATCH_BYTES: every GPU that
// loads this library holds it until the process exits.  Its name in host code is only a
// host-side stand-in, so its device address is looked up once per device with
// cudaGetSymbolAddress (on the first call on that device) and passed to the kernels.
// All calls share the buffer and it keeps the previous call's contents; whatever must
// start at zero is cleared on every call.  Calls whose work overlaps on the GPU (two host
// threads, or two streams) race on the buffer.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/mhc.h"
#include "common.cuh"
#include "kernels.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[MHC_NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
void *g_scratch_addr[MAX_DEVICES] = {};
std::mutex g_scratch_mutex;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Per-device address of the static buffer; looked up on the first call on each device.
cudaError_t scratch_address(int device, void **out) {
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[device] = p;
    }
    *out = g_scratch_addr[device];
    return cudaSuccess;
}

// Identity mode order, per-mode bin/slot tables and per-atom mass weights.  One CTA;
// bins must be in [0, B) and non-decreasing (modes already ordered by bin).  A slot is
// the last mode of a run of equal bins inside a 32-mode group; slot_begin[b] is the
// first slot of bin b.  A violated precondition sets *status.  Every slot entry is reset
// first, so that no entry left by an earlier call survives a call that stops early.
__global__ void noalloc_tables_kernel(const int32_t *bin_of_mode, int M, int M_pad, int B,
                                      const double *mass, int N, int *perm, int *mode_bin,
                                      int *mode_slot, int *slot_begin, float *sqm, float *isqm,
                                      int *status) {
    for (int n = threadIdx.x; n < M_pad; n += blockDim.x) {
        if (n < M) perm[n] = n;
        mode_bin[n] = n < M ? bin_of_mode[n] : -1;
        mode_slot[n] = -1;
    }
    for (int b = threadIdx.x; b <= B; b += blockDim.x) slot_begin[b] = 0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const double m = mass[i];
        if (!(m > 0.0)) atomicCAS(status, 0, 1);
        sqm[i] = (float)sqrt(m);
        isqm[i] = (float)(1.0 / sqrt(m));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0, b_next = 0;
        for (int n = 0; n < M; ++n) {
            const int b = mode_bin[n];
            if (b < 0 || b >= B || (n > 0 && b < mode_bin[n - 1])) {
                atomicCAS(status, 0, 1);
                b_next = B;
                break;
            }
            while (b_next <= b) slot_begin[b_next++] = s;
            const bool tail = (n % 32) == 31 || n + 1 == M || mode_bin[n + 1] != b;
            mode_slot[n] = tail ? s++ : -1;
        }
        while (b_next <= B) slot_begin[b_next++] = s;
        for (int n = M; n < M_pad; ++n) mode_slot[n] = -1;
    }
}

}  // namespace

extern "C" mhc_status mhc_binned_current_noalloc(int32_t n_atoms, int32_t n_modes, const float *E,
                                                 int64_t ld, const int32_t *bin_of_mode,
                                                 int32_t n_bins, const double *mass_amu,
                                                 const float *v, const float *W, int32_t K,
                                                 float *Jb, double *J, int32_t device,
                                                 void *stream) {
    using namespace mhc;
    if (n_atoms < 1 || n_modes < 1 || n_modes > 3 * (int64_t)n_atoms || n_bins < 1 || K < 1 ||
        ld < 3 * (int64_t)n_atoms || !E || !bin_of_mode || !mass_amu || !v || !W || !Jb || !J ||
        device < 0 || device >= MAX_DEVICES)
        return MHC_ERR_INVALID_ARG;
    const int64_t N = n_atoms, D = 3 * N, M = n_modes;
    const int64_t D_ld = (D + 63) / 64 * 64, M_pad = (M + 127) / 128 * 128;
    const int64_t B_rows = (4 * (int64_t)K + 127) / 128 * 128;
    // scratch layout: every region 256-byte aligned
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align256(off + bytes);
        return at;
    };
    const size_t o_status = take(sizeof(int));
    const size_t o_perm = take(sizeof(int) * M_pad);
    const size_t o_bin = take(sizeof(int) * M_pad);
    const size_t o_slot = take(sizeof(int) * M_pad);
    const size_t o_sbeg = take(sizeof(int) * (n_bins + 1));
    const size_t o_sqm = take(sizeof(float) * N);
    const size_t o_isqm = take(sizeof(float) * N);
    const size_t o_E = take(sizeof(float) * M_pad * D_ld);
    const size_t o_Bt = take(sizeof(float) * B_rows * D_ld);
    const size_t o_R = take(sizeof(float) * B_rows * M_pad);
    const size_t o_cs = take(sizeof(float) * 4 * K);
    const size_t o_part = take(sizeof(float) * K * 3 * M_pad);   // slot stride M_pad >= n_slots
    const size_t o_hsum = take(sizeof(double) * n_bins * 3);
    const size_t o_jsum = take(sizeof(double) * 3);
    if (off > MHC_NOALLOC_SCRATCH_BYTES) return MHC_ERR_INVALID_ARG;   // problem too large

    cudaError_t e = cudaSetDevice(device);
    void *base = nullptr;
    if (e == cudaSuccess) e = scratch_address(device, &base);
    if (e != cudaSuccess) return MHC_ERR_CUDA;
    char *s = static_cast<char *>(base);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int *status = reinterpret_cast<int *>(s + o_status);
    int *perm = reinterpret_cast<int *>(s + o_perm);
    int *mode_bin = reinterpret_cast<int *>(s + o_bin);
    int *mode_slot = reinterpret_cast<int *>(s + o_slot);
    int *slot_begin = reinterpret_cast<int *>(s + o_sbeg);
    float *Et32 = reinterpret_cast<float *>(s + o_E);
    float *Bt32 = reinterpret_cast<float *>(s + o_Bt);
    float *partials = reinterpret_cast<float *>(s + o_part);
    double *hsum = reinterpret_cast<double *>(s + o_hsum);
    double *jsum = reinterpret_cast<double *>(s + o_jsum);

    // cleared every call: status word, B-operand padding columns, HNEMA sums
    e = cudaMemsetAsync(status, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(Bt32, 0, sizeof(float) * B_rows * D_ld, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(hsum, 0, o_jsum + sizeof(double) * 3 - o_hsum, st);
    if (e != cudaSuccess) return MHC_ERR_CUDA;
    noalloc_tables_kernel<<<1, 256, 0, st>>>(bin_of_mode, (int)M, (int)M_pad, n_bins, mass_amu,
                                            (int)N, perm, mode_bin, mode_slot, slot_begin,
                                            reinterpret_cast<float *>(s + o_sqm),
                                            reinterpret_cast<float *>(s + o_isqm), status);
    // Bins and masses are checked on the device; nothing else runs (and no output is
    // written) unless they passed.
    int h_status = 0;
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return MHC_ERR_CUDA;
    if (h_status) return MHC_ERR_INVALID_ARG;
    launch_prepare_modes(E, MHC_F32, MHC_MODE_MAJOR, ld, D, M, perm, 0, SPLIT_FP32, nullptr,
                         nullptr, Et32, D_ld, M_pad, 0, st);
    PackArgs a{};
    a.v = v;
    a.W = W;
    a.sqm = reinterpret_cast<float *>(s + o_sqm);
    a.isqm = reinterpret_cast<float *>(s + o_isqm);
    a.N = (int)N;
    a.K = K;
    a.D_ld = (int)D_ld;
    a.split = SPLIT_FP32;
    a.Bt32 = Bt32;
    a.col_scale = reinterpret_cast<float *>(s + o_cs);
    a.Jtot = J;
    launch_pack(a, st);
    launch_sgemm(Et32, Bt32, reinterpret_cast<float *>(s + o_R), (int)D_ld, (int)D_ld, (int)M_pad,
                 4 * K, st);
    launch_fp32_bin_epilogue(reinterpret_cast<float *>(s + o_R), (int)M_pad, K, mode_bin, mode_slot,
                             partials, (int)M_pad, st);
    launch_bin_finish(partials, (int)M_pad, slot_begin, n_bins, K, Jb, hsum, J, jsum, nullptr, st);
    if ((e = cudaGetLastError()) != cudaSuccess) return MHC_ERR_CUDA;
    if ((e = cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return MHC_ERR_CUDA;
    return h_status ? MHC_ERR_INVALID_ARG : MHC_OK;
}
