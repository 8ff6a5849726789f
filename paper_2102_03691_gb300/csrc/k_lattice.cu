// Gamma-point lattice dynamics on the GPU (Sec. II.B: the eigenvectors e_{i,n} and frequencies
// of the modal analysis come from the harmonic eigenmodes of the whole cell).
//
// Dyn[3i+a][3j+b] = Phi[3i+a][3j+b] / sqrt(m_i m_j); Dyn e_n = w_n^2 e_n, by parallel cyclic
// Jacobi in FP64.  A sweep is n - 1 rounds (n = 3N rounded up to even) of the round-robin
// tournament: in round r the n indices form n/2 disjoint pairs (p, q), and every pair's
// rotation J_pq (the one that zeroes a_pq) is applied at once -- the rotations of disjoint pairs
// commute, and a pair's own 2x2 block (a_pp, a_qq, a_pq) is untouched by the others, so the
// round computes J^T A J and V J for the product J of all of them:
//   lat_angles:  (c, s) of every pair from the current A
//   lat_cols:    A <- A J and V <- V J   (one CTA per row; a row's pairs are disjoint)
//   lat_rows:    A <- J^T A              (one CTA per pair; rows p and q, coalesced)
// and sets a_pq = a_qp = 0.  After each sweep a two-stage deterministic reduction gives the
// off-diagonal and total Frobenius norms; the host stops once off <= tol * total.  One sweep's
// launches are captured once into a CUDA graph and replayed.  The eigenvalues are sorted on the
// host (stable, ascending) and a gather kernel writes the eigenvectors in that order, each with
// the sign that makes its first component of largest magnitude positive.
//
// Cost on GB300: each round streams A and V (2 x 8 D^2 bytes, L2-resident up to D ~ 2500)
// with 3 FP64 operations per element, and a sweep has n - 1 rounds: about 9 D^3 FP64 flops and
// 24 D^3 bytes per sweep, and ~10 sweeps.  GB300's FP64 rate is low, so this is meant for the
// basis of systems up to a few thousand atoms; larger bases come from elsewhere (mhc_set_modes).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/mhc.h"
#include "kernels.h"

namespace mhc {
namespace {

constexpr int LAT_THREADS = 256;
constexpr int LAT_RED_BLOCKS = 256;

__device__ __forceinline__ int rr_pos(int idx, int r, int n) {
    return idx == 0 ? 0 : 1 + (idx - 1 + r) % (n - 1);
}

// Pair k of round r: indices p < q (either may be the padding index D when D is odd).
__device__ __forceinline__ void rr_pair(int k, int r, int n, int &p, int &q) {
    const int a = rr_pos(k, r, n), b = rr_pos(n - 1 - k, r, n);
    p = min(a, b);
    q = max(a, b);
}

__global__ void lat_init_kernel(const double *__restrict__ Phi, const double *__restrict__ isq, int D,
                                double *__restrict__ A, double *__restrict__ V) {
    const size_t n2 = (size_t)D * D;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n2; e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / D), c = (int)(e - (size_t)r * D);
        A[e] = Phi[e] * isq[r / 3] * isq[c / 3];
        V[e] = r == c ? 1.0 : 0.0;
    }
}

__global__ void lat_angles_kernel(const double *__restrict__ A, int D, int n, int r,
                                  double2 *__restrict__ cs, int2 *__restrict__ pq) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n / 2) return;
    int p, q;
    rr_pair(k, r, n, p, q);
    double c = 1.0, s = 0.0;
    if (q < D) {
        const double apq = A[(size_t)p * D + q];
        if (apq != 0.0) {
            const double theta = (A[(size_t)q * D + q] - A[(size_t)p * D + p]) / (2.0 * apq);
            const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            s = t * c;
        }
    }
    cs[k] = make_double2(c, s);
    pq[k] = make_int2(p, q);
}

// A <- A J, V <- V J: row `blockIdx.x` of both, every pair of the round.
__global__ void __launch_bounds__(LAT_THREADS) lat_cols_kernel(double *__restrict__ A, double *__restrict__ V,
                                                              int D, int npairs,
                                                              const double2 *__restrict__ cs,
                                                              const int2 *__restrict__ pq) {
    const size_t row = (size_t)blockIdx.x * D;
    for (int k = threadIdx.x; k < npairs; k += blockDim.x) {
        const int2 ij = pq[k];
        if (ij.y >= D) continue;
        const double2 t = cs[k];
        double *a = A + row, *v = V + row;
        const double ap = a[ij.x], aq = a[ij.y];
        a[ij.x] = t.x * ap - t.y * aq;
        a[ij.y] = t.y * ap + t.x * aq;
        const double vp = v[ij.x], vq = v[ij.y];
        v[ij.x] = t.x * vp - t.y * vq;
        v[ij.y] = t.y * vp + t.x * vq;
    }
}

// A <- J^T A: rows p and q of pair `blockIdx.x`; the pair's off-diagonal entries become 0.
__global__ void __launch_bounds__(LAT_THREADS) lat_rows_kernel(double *__restrict__ A, int D,
                                                              const double2 *__restrict__ cs,
                                                              const int2 *__restrict__ pq) {
    const int2 ij = pq[blockIdx.x];
    if (ij.y >= D) return;
    const double2 t = cs[blockIdx.x];
    double *ap = A + (size_t)ij.x * D, *aq = A + (size_t)ij.y * D;
    for (int j = threadIdx.x; j < D; j += blockDim.x) {
        const double x = ap[j], y = aq[j];
        ap[j] = j == ij.y ? 0.0 : t.x * x - t.y * y;
        aq[j] = j == ij.x ? 0.0 : t.y * x + t.x * y;
    }
}

// Per-block partial sums of the squared off-diagonal and of all squared entries (fixed order).
__global__ void __launch_bounds__(LAT_THREADS) lat_norm_kernel(const double *__restrict__ A, int D,
                                                              double2 *__restrict__ part) {
    const size_t n2 = (size_t)D * D;
    double off = 0.0, tot = 0.0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n2; e += (size_t)gridDim.x * blockDim.x) {
        const double x = A[e] * A[e];
        tot += x;
        if (e / D != e % D) off += x;
    }
    __shared__ double s_off[LAT_THREADS], s_tot[LAT_THREADS];
    s_off[threadIdx.x] = off;
    s_tot[threadIdx.x] = tot;
    __syncthreads();
    for (int w = LAT_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            s_off[threadIdx.x] += s_off[threadIdx.x + w];
            s_tot[threadIdx.x] += s_tot[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = make_double2(s_off[0], s_tot[0]);
}

__global__ void lat_norm_final_kernel(const double2 *__restrict__ part, int nb, double2 *__restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double off = 0.0, tot = 0.0;
    for (int b = 0; b < nb; ++b) {
        off += part[b].x;
        tot += part[b].y;
    }
    *out = make_double2(off, tot);
}

__global__ void lat_diag_kernel(const double *__restrict__ A, int D, double *__restrict__ diag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < D) diag[i] = A[(size_t)i * D + i];
}

// Sign of eigenvector column `blockIdx.x` of V: + where its first largest-magnitude component
// is positive.
__global__ void __launch_bounds__(LAT_THREADS) lat_sign_kernel(const double *__restrict__ V, int D,
                                                              double *__restrict__ sign) {
    const int col = blockIdx.x;
    double best = -1.0;
    int arg = 0;
    for (int d = threadIdx.x; d < D; d += blockDim.x) {
        const double x = fabs(V[(size_t)d * D + col]);
        if (x > best) {
            best = x;
            arg = d;
        }
    }
    __shared__ double s_b[LAT_THREADS];
    __shared__ int s_a[LAT_THREADS];
    s_b[threadIdx.x] = best;
    s_a[threadIdx.x] = arg;
    __syncthreads();
    for (int w = LAT_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            const double ob = s_b[threadIdx.x + w];
            const int oa = s_a[threadIdx.x + w];
            if (ob > s_b[threadIdx.x] || (ob == s_b[threadIdx.x] && oa < s_a[threadIdx.x])) {
                s_b[threadIdx.x] = ob;
                s_a[threadIdx.x] = oa;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) sign[col] = V[(size_t)s_a[0] * D + col] < 0.0 ? -1.0 : 1.0;
}

// E[d][n] = sign[perm[n]] V[d][perm[n]]
__global__ void lat_gather_kernel(const double *__restrict__ V, int D, const int *__restrict__ perm,
                                  const double *__restrict__ sign, double *__restrict__ E) {
    const size_t n2 = (size_t)D * D;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n2; e += (size_t)gridDim.x * blockDim.x) {
        const int d = (int)(e / D), n = (int)(e - (size_t)d * D);
        const int src = perm[n];
        E[e] = sign[src] * V[(size_t)d * D + src];
    }
}

struct DevMem {
    std::vector<void *> ptrs;
    ~DevMem() {
        for (void *p : ptrs) cudaFree(p);
    }
    template <typename T>
    cudaError_t get(T **p, size_t count) {
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, sizeof(T) * std::max<size_t>(count, 1));
        if (e == cudaSuccess) ptrs.push_back(q);
        *p = static_cast<T *>(q);
        return e;
    }
};

}  // namespace
}  // namespace mhc

using namespace mhc;

extern "C" mhc_status mhc_lattice_modes(int32_t device, void *stream, int64_t n_atoms,
                                        const double *Phi, const double *mass_amu, int32_t where_in,
                                        double tol, int32_t max_sweeps, double *w2, double *freq_THz,
                                        double *E, int32_t where_out, int32_t *sweeps) {
    auto fail = [](mhc_status s, const std::string &m) {
        set_handleless_error(m.c_str());
        return s;
    };
    set_handleless_error("");
    if (n_atoms < 1 || n_atoms > 10000 || !Phi || !mass_amu || !(tol > 0) || max_sweeps < 1 ||
        (where_in != MHC_MEM_HOST && where_in != MHC_MEM_DEVICE) ||
        (where_out != MHC_MEM_HOST && where_out != MHC_MEM_DEVICE))
        return fail(MHC_ERR_INVALID_ARG, "mhc_lattice_modes: bad size, pointer, tolerance or memory space");
    const int D = (int)(3 * n_atoms);
    const int n = D + (D & 1);            // round-robin over an even number of indices
    const int npairs = n / 2;
    std::vector<double> isq((size_t)n_atoms);
    for (int64_t i = 0; i < n_atoms; ++i) {
        if (!(mass_amu[i] > 0) || !std::isfinite(mass_amu[i]))
            return fail(MHC_ERR_INVALID_ARG, "mhc_lattice_modes: masses must be positive");
        isq[(size_t)i] = 1.0 / std::sqrt(mass_amu[i]);
    }
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return fail(MHC_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t n2 = (size_t)D * D;
    DevMem mem;
    double *dPhi = nullptr, *dA = nullptr, *dV = nullptr, *disq = nullptr, *ddiag = nullptr, *dsign = nullptr;
    double *dE = nullptr;
    double2 *dcs = nullptr, *dpart = nullptr, *dnorm = nullptr;
    int2 *dpq = nullptr;
    int *dperm = nullptr;
    if ((e = mem.get(&dA, n2)) != cudaSuccess || (e = mem.get(&dV, n2)) != cudaSuccess ||
        (e = mem.get(&disq, (size_t)n_atoms)) != cudaSuccess || (e = mem.get(&ddiag, (size_t)D)) != cudaSuccess ||
        (e = mem.get(&dsign, (size_t)D)) != cudaSuccess || (e = mem.get(&dcs, (size_t)npairs)) != cudaSuccess ||
        (e = mem.get(&dpq, (size_t)npairs)) != cudaSuccess || (e = mem.get(&dpart, LAT_RED_BLOCKS)) != cudaSuccess ||
        (e = mem.get(&dnorm, 1)) != cudaSuccess || (e = mem.get(&dperm, (size_t)D)) != cudaSuccess)
        return fail(MHC_ERR_OOM, std::string("mhc_lattice_modes: cudaMalloc: ") + cudaGetErrorString(e));
    const double *phi = Phi;
    if (where_in == MHC_MEM_HOST) {
        if ((e = mem.get(&dPhi, n2)) != cudaSuccess)
            return fail(MHC_ERR_OOM, std::string("mhc_lattice_modes: cudaMalloc: ") + cudaGetErrorString(e));
        if ((e = cudaMemcpyAsync(dPhi, Phi, sizeof(double) * n2, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return fail(MHC_ERR_CUDA, std::string("copy of Phi: ") + cudaGetErrorString(e));
        phi = dPhi;
    }
    if (E && where_out == MHC_MEM_DEVICE) {
        dE = E;
    } else if ((e = mem.get(&dE, n2)) != cudaSuccess) {
        return fail(MHC_ERR_OOM, std::string("mhc_lattice_modes: cudaMalloc: ") + cudaGetErrorString(e));
    }
    if ((e = cudaMemcpyAsync(disq, isq.data(), sizeof(double) * isq.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return fail(MHC_ERR_CUDA, std::string("copy of masses: ") + cudaGetErrorString(e));
    const int gs = (int)std::min<size_t>((n2 + 255) / 256, 152 * 16);
    lat_init_kernel<<<gs, 256, 0, st>>>(phi, disq, D, dA, dV);

    // one sweep captured into a graph (a private stream: capture of the caller's legacy stream
    // is not allowed), replayed until convergence
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess)
        return fail(MHC_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int r = 0; r < n - 1; ++r) {
            lat_angles_kernel<<<(npairs + 127) / 128, 128, 0, cap>>>(dA, D, n, r, dcs, dpq);
            lat_cols_kernel<<<D, LAT_THREADS, 0, cap>>>(dA, dV, D, npairs, dcs, dpq);
            lat_rows_kernel<<<npairs, LAT_THREADS, 0, cap>>>(dA, D, dcs, dpq);
        }
        lat_norm_kernel<<<LAT_RED_BLOCKS, LAT_THREADS, 0, cap>>>(dA, D, dpart);
        lat_norm_final_kernel<<<1, 32, 0, cap>>>(dpart, LAT_RED_BLOCKS, dnorm);
        cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
        if (e2 != cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    auto cleanup = [&]() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cap) cudaStreamDestroy(cap);
    };
    if (e != cudaSuccess) {
        cleanup();
        return fail(MHC_ERR_CUDA, std::string("mhc_lattice_modes: graph of a sweep: ") + cudaGetErrorString(e));
    }
    // the initial norms (zero sweeps), then sweeps
    lat_norm_kernel<<<LAT_RED_BLOCKS, LAT_THREADS, 0, st>>>(dA, D, dpart);
    lat_norm_final_kernel<<<1, 32, 0, st>>>(dpart, LAT_RED_BLOCKS, dnorm);
    cudaEvent_t ev = nullptr;
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) {
        cleanup();
        return fail(MHC_ERR_CUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(e));
    }
    int done = -1;
    for (int sw = 0; sw <= max_sweeps && e == cudaSuccess; ++sw) {
        double2 nrm;
        if ((e = cudaMemcpyAsync(&nrm, dnorm, sizeof nrm, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            break;
        if (std::sqrt(nrm.x) <= tol * std::sqrt(nrm.y)) {
            done = sw;
            break;
        }
        if (sw == max_sweeps) break;
        // the sweep runs on the capture stream, ordered after the caller's stream and before it
        if ((e = cudaEventRecord(ev, st)) != cudaSuccess || (e = cudaStreamWaitEvent(cap, ev, 0)) != cudaSuccess ||
            (e = cudaGraphLaunch(exec, cap)) != cudaSuccess || (e = cudaEventRecord(ev, cap)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(st, ev, 0)) != cudaSuccess)
            break;
    }
    cudaEventDestroy(ev);
    cleanup();
    if (e != cudaSuccess) return fail(MHC_ERR_CUDA, std::string("mhc_lattice_modes: ") + cudaGetErrorString(e));
    if (sweeps) *sweeps = done;
    if (done < 0) return fail(MHC_ERR_STATE, "mhc_lattice_modes: not converged within max_sweeps");

    // eigenvalues in ascending order (stable), signed eigenvectors gathered in that order
    std::vector<double> diag((size_t)D);
    lat_diag_kernel<<<(D + 255) / 256, 256, 0, st>>>(dA, D, ddiag);
    if ((e = cudaMemcpyAsync(diag.data(), ddiag, sizeof(double) * D, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return fail(MHC_ERR_CUDA, std::string("mhc_lattice_modes: ") + cudaGetErrorString(e));
    std::vector<int> perm((size_t)D);
    std::iota(perm.begin(), perm.end(), 0);
    std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return diag[(size_t)a] < diag[(size_t)b]; });
    const double two_pi = 6.283185307179586476925;
    for (int q = 0; q < D; ++q) {
        const double lam = diag[(size_t)perm[(size_t)q]];
        if (w2) w2[q] = lam;
        if (freq_THz) {
            const double w = std::sqrt(std::fabs(lam) * A2_PS2_PER_EV_AMU);
            freq_THz[q] = (lam < 0 ? -w : w) / two_pi;
        }
    }
    if (E) {
        if ((e = cudaMemcpyAsync(dperm, perm.data(), sizeof(int) * D, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return fail(MHC_ERR_CUDA, std::string("mhc_lattice_modes: ") + cudaGetErrorString(e));
        lat_sign_kernel<<<D, LAT_THREADS, 0, st>>>(dV, D, dsign);
        lat_gather_kernel<<<gs, 256, 0, st>>>(dV, D, dperm, dsign, dE);
        if (where_out == MHC_MEM_HOST &&
            (e = cudaMemcpyAsync(E, dE, sizeof(double) * n2, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return fail(MHC_ERR_CUDA, std::string("mhc_lattice_modes: ") + cudaGetErrorString(e));
    }
    if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return fail(MHC_ERR_CUDA, std::string("mhc_lattice_modes: ") + cudaGetErrorString(e));
    return MHC_OK;
}
