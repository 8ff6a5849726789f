// C-ABI layer of the modal heat-current library (declarations and semantics: include/mhc.h).
// Owns the device buffers of a handle, turns frequencies into the bin-sorted mode order
// the fused epilogue needs, and issues the kernels of one push on the handle's stream.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <queue>
#include <tuple>
#include <string>
#include <vector>

#include "../../include/mhc.h"
#include "kernels.h"

using namespace mhc;

namespace {
thread_local std::string g_create_error;
}  // namespace

void mhc::set_handleless_error(const char *msg) { g_create_error = msg; }

namespace {

constexpr double KB_EV_PER_K = 8.617333262145179e-5;   // k_B / e (SI exact ratio)
constexpr double WMK_PER_EV_PS_A_K = 1602.176634;      // 1 eV/(ps A K) in W/(m K)
constexpr int K_MAX_LIMIT = 1024;
constexpr uint32_t STATE_MAGIC = 0x4d484331u;         // "MHC1"

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

PFN_cuTensorMapEncodeTiled_v12000 tmap_encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

}  // namespace

int mhc::tc_make_tmap(CUtensorMap *m, const void *base, uint64_t rows, uint64_t cols, uint64_t ld,
                      uint32_t box_rows, uint32_t box_cols) {
    auto fn = tmap_encode_fn();
    if (!fn) return -1;
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {ld * 2};
    cuuint32_t box[2] = {box_cols, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUtensorMapSwizzle sw = box_cols * 2 == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, const_cast<void *>(base), dims, strides,
                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : (int)r;
}

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct mhc_handle;
using Handle = mhc_handle;

struct mhc_handle {
    mhc_params prm{};
    cudaStream_t stream = nullptr;
    int sm_count = 0, cc_major = 0, cc_minor = 0;
    std::string device_name;
    int split = SPLIT_BF16;
    std::string err;

    // modes
    bool modes_ready = false, bins_ready = false;
    int64_t N = 0, D = 0, M_in = 0, M_eff = 0, D_ld = 0, M_pad = 0;
    // direction-resolved split (MHC_FLAG_DIRECTION): d stored direction-major in three
    // segments of N_pad columns; every per-bin output has 3 B rows, row = b * B + bin
    bool dir = false;
    int64_t N_pad = 0;
    std::vector<double> freq, mass;
    std::vector<int> perm;          // stored (bin-sorted) mode -> input mode
    int e_exp = 0;
    double ortho_err = -1.0;

    // bins
    int32_t B = 0;
    int64_t n_slots = 0;
    int64_t B_rows = 0;             // rows of the B operand (>= 4 k_max, multiple of 256)
    int R_ring = 0;

    // accumulators / counters
    int64_t steps = 0, pushes = 0, launches = 0;
    int K_last = 0;

    // device buffers
    std::map<std::string, DevBuf> buf;
    int *status = nullptr;

    // CUDA graphs of whole pushes, keyed by (K, v, W, tile shape); replayable because the
    // kernels read the block's first step from a device counter
    struct GraphEntry {
        cudaGraphExec_t exec = nullptr;
        uint64_t last_use = 0;
        int64_t nodes = 0;
    };
    std::map<std::tuple<int, const void *, const void *, int>, GraphEntry> graphs;
    uint64_t graph_clock = 0;
    int64_t graph_replays = 0;
    cudaStream_t cap_stream = nullptr;

    // host-input staging: two buffer pairs filled on a copy stream, so that the upload of one
    // push overlaps the kernels of the previous one (each buffer is reused only after the
    // push that read it has finished)
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t copy_done[2] = {nullptr, nullptr}, use_done[2] = {nullptr, nullptr};
    bool use_pending[2] = {false, false};
    int stage_next = 0, stage_used = -1;
    int async_stage = -1;   // staging pair of an MHC_MEM_HOST_ASYNC upload not yet waited for

    // optional CUDA-event timing of the projection kernel (MHC_FLAG_PROFILE)
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_events;
    size_t prof_used = 0;

    // tensor-core state
    TcConfig tc{256, 64, 2, 0, 0};
    std::map<int, TcConfig> tuned;  // K -> config
    TcParams<1> tcp{};
    XcPlan xc_plan{};     // cross-correlations (MHC_FLAG_XCORR): tensor-core plan and parameters
    XcTcParams xcp{};
};

struct GroupSchedule {
    DevBuf sched, cta_begin;   // device copies (owned by the group)
    int grid = 0;
};

struct mhc_group {
    std::vector<mhc_handle *> hs;
    TcConfig tc{256, 64, 2, 0, 0};
    std::map<std::vector<int>, TcConfig> tuned;   // autotuned tile shape of each block-length vector
    TcParams<TC_MAX_GROUP> tcp{};
    std::map<std::pair<int, std::vector<int>>, GroupSchedule> sched_cache;   // (bn, Ks)
    // graphs of whole group pushes keyed by (Ks, input pointers, tile shape)
    struct GraphEntry {
        cudaGraphExec_t exec = nullptr;
        uint64_t last_use = 0;
        int64_t nodes = 0;
    };
    std::map<std::tuple<std::vector<int>, std::vector<const void *>, int>, GraphEntry> graphs;
    uint64_t graph_clock = 0;
    cudaStream_t cap_stream = nullptr;
    // side streams for the grouped packs (fork after the main stream, join before it goes on)
    static constexpr int PACK_SIDE = 3;
    cudaStream_t pack_side[PACK_SIDE] = {};
    cudaEvent_t pack_fork = nullptr, pack_join[PACK_SIDE] = {};
};

namespace {

mhc_status fail(mhc_handle *h, mhc_status s, const char *fmt, ...) {
    char msg[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    if (h) h->err = msg;
    else g_create_error = msg;
    return s;
}

#define MHC_CUDA(h, call)                                                                        \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return fail((h), e_ == cudaErrorMemoryAllocation ? MHC_ERR_OOM : MHC_ERR_CUDA,       \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

mhc_status dev_alloc(mhc_handle *h, const char *name, size_t bytes, bool zero = true) {
    DevBuf &b = h->buf[name];
    if (b.p && b.bytes >= bytes) {
        if (zero) MHC_CUDA(h, cudaMemsetAsync(b.p, 0, b.bytes, h->stream));
        return MHC_OK;
    }
    if (b.p) {
        cudaStreamSynchronize(h->stream);
        cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
    }
    if (bytes == 0) return MHC_OK;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        b.p = nullptr;
        cudaGetLastError();
        return fail(h, MHC_ERR_OOM, "cudaMalloc of %zu bytes for %s failed: %s", bytes, name,
                    cudaGetErrorString(e));
    }
    b.bytes = bytes;
    if (zero) MHC_CUDA(h, cudaMemsetAsync(b.p, 0, bytes, h->stream));
    return MHC_OK;
}

template <typename T>
T *dptr(mhc_handle *h, const char *name) {
    auto it = h->buf.find(name);
    return it == h->buf.end() ? nullptr : static_cast<T *>(it->second.p);
}

void dev_free(mhc_handle *h, const char *name) {
    auto it = h->buf.find(name);
    if (it == h->buf.end()) return;
    if (it->second.p) cudaFree(it->second.p);
    h->buf.erase(it);
}

bool is_tc(const mhc_handle *h) { return h->split != SPLIT_FP32; }

// Rows of the per-bin outputs: B, or 3 B (direction b, bin) with the direction split.
int64_t n_out_bins(const mhc_handle *h) { return (int64_t)h->B * (h->dir ? 3 : 1); }

// Partial-sum slots per step component (one set per direction with the split).
int64_t slot_stride(const mhc_handle *h) { return h->n_slots * (h->dir ? 3 : 1); }

bool has_xcorr(const mhc_handle *h) { return (h->prm.flags & MHC_FLAG_XCORR) != 0; }

void drop_graphs(mhc_handle *h) {
    for (auto &kv : h->graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    h->graphs.clear();
}

mhc_status check_device_status(mhc_handle *h) {
    int st = 0;
    MHC_CUDA(h, cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    MHC_CUDA(h, cudaStreamSynchronize(h->stream));
    if (st == DEV_TIMEOUT)
        return fail(h, MHC_ERR_TIMEOUT, "a tensor-core kernel gave up waiting on a barrier");
    if (st != 0) return fail(h, MHC_ERR_STATE, "device status word %d", st);
    return MHC_OK;
}

mhc_status reset_accumulators(mhc_handle *h) {
    h->steps = 0;
    h->K_last = 0;
    const int64_t B = std::max<int64_t>(n_out_bins(h), 1), L = std::max<int32_t>(h->prm.n_lags, 0);
    mhc_status s;
    if ((s = dev_alloc(h, "hsum", sizeof(double) * B * 3)) != MHC_OK) return s;
    if ((s = dev_alloc(h, "Jsum", sizeof(double) * 3)) != MHC_OK) return s;
    if ((s = dev_alloc(h, "steps_dev", sizeof(long long))) != MHC_OK) return s;
    if (h->prm.flags & MHC_FLAG_GKMA) {
        if ((s = dev_alloc(h, "Csum", sizeof(double) * B * 9 * L)) != MHC_OK) return s;
        if ((s = dev_alloc(h, "Jring", sizeof(double) * h->R_ring * 3)) != MHC_OK) return s;
        if ((s = dev_alloc(h, "lc_ticket", sizeof(unsigned))) != MHC_OK) return s;
        MHC_CUDA(h, lag_corr_prepare(h->prm.k_max));
    }
    if (has_xcorr(h)) {   // lag-major [L][3R][3R] float-pair sums, the ring of past binned
                          // currents, and the tensor-core kernel's window copies
        if ((s = dev_alloc(h, "Xsum", sizeof(float2) * L * 9 * B * B)) != MHC_OK) return s;
        if ((s = dev_alloc(h, "Jbring", sizeof(float) * h->R_ring * 3 * B)) != MHC_OK) return s;
        XcPlan &pl = h->xc_plan;
        xcorr_plan((int)B, (int)L, h->prm.k_max, h->sm_count, pl);
        const size_t wbytes = sizeof(uint16_t) * 8 * (size_t)pl.rows_pad * pl.U_pad;
        if ((s = dev_alloc(h, "Xwin_hi", wbytes)) != MHC_OK) return s;
        if ((s = dev_alloc(h, "Xwin_lo", wbytes)) != MHC_OK) return s;
        if ((s = dev_alloc(h, "Xinv", sizeof(float) * pl.rows_pad)) != MHC_OK) return s;
        XcTcParams &xp = h->xcp;
        if (xcorr_make_maps(pl, dptr<void>(h, "Xwin_hi"), dptr<void>(h, "Xwin_lo"), xp))
            return fail(h, MHC_ERR_CUDA, "cuTensorMapEncodeTiled failed (cross-correlation windows)");
        xp.inv_scale = dptr<float>(h, "Xinv");
        xp.X = dptr<float2>(h, "Xsum");
        xp.L = (int)L;
        xp.status = h->status;
        xp.wait_limit = 2000000000ll;
        MHC_CUDA(h, xcorr_prepare());
    }
    return MHC_OK;
}

// Host binning of Sec. III.A: floor((f - f_min)/w) in double, last bin closed.
void bins_uniform_host(const std::vector<double> &f, double f_min, double f_max, int B,
                       std::vector<int> &out) {
    const double w = (f_max - f_min) / (double)B;
    out.resize(f.size());
    for (size_t n = 0; n < f.size(); ++n) {
        const double x = f[n];
        if (!std::isfinite(x) || x < f_min || x > f_max) {
            out[n] = -1;
            continue;
        }
        int64_t b = (int64_t)std::floor((x - f_min) / w);
        if (b >= B) b = B - 1;
        if (b < 0) b = 0;
        out[n] = (int)b;
    }
}

// Tensor maps of one system for tile configuration c: E hi/lo boxes of 128 modes, B hi/lo
// boxes of the CTA's columns (all BN columns, or half of them for a two-SM tile).
int encode_maps(mhc_handle *h, const TcConfig &c, TcProblem &P) {
    const uint32_t brows = c.pair ? c.bn / 2 : c.bn;
    int r = tc_make_tmap(&P.tmA_hi, dptr<void>(h, "Et_hi"), h->M_pad, h->D_ld, h->D_ld, TC_BM, c.bk);
    if (!r) r = tc_make_tmap(&P.tmA_lo, dptr<void>(h, "Et_lo"), h->M_pad, h->D_ld, h->D_ld, TC_BM, c.bk);
    if (!r) r = tc_make_tmap(&P.tmB_hi, dptr<void>(h, "Bt_hi"), h->B_rows, h->D_ld, h->D_ld, brows, c.bk);
    if (!r) r = tc_make_tmap(&P.tmB_lo, dptr<void>(h, "Bt_lo"), h->B_rows, h->D_ld, h->D_ld, brows, c.bk);
    return r;
}

// Mode tiles of a system for configuration c (128 modes, or 256 for a CTA pair).
int mode_tiles(const mhc_handle *h, const TcConfig &c) {
    const int64_t per = (c.pair ? 2 : 1) * TC_BM;
    return (int)((h->M_eff + per - 1) / per);
}

// Persistent scheduling units that can run at once: SMs, or resident CTA pairs.
int sched_units(const mhc_handle *h, const TcConfig &c) {
    if (!c.pair) return h->sm_count;
    static int pairs[TC_NUM_CONFIGS] = {};
    for (int q = 0; q < TC_NUM_CONFIGS; ++q)
        if (TC_CONFIGS[q].bk == c.bk && TC_CONFIGS[q].pair == c.pair && TC_CONFIGS[q].stages == c.stages) {
            if (!pairs[q]) pairs[q] = tc_max_pairs(c);
            return std::max(1, std::min(pairs[q], h->sm_count / 2));
        }
    return std::max(1, h->sm_count / 2);
}

// Sort kept modes by bin (stable), build the per-mode bin/slot tables of the fused
// epilogue, gather+split E into the stored order and set up the tensor maps.
mhc_status apply_bins(mhc_handle *h, const std::vector<int> &bin_of_mode, int32_t B) {
    if (B < 1) return fail(h, MHC_ERR_INVALID_ARG, "number of bins must be >= 1");
    cudaStreamSynchronize(h->stream);
    drop_graphs(h);
    for (int b : bin_of_mode)
        if (b < -1 || b >= B) return fail(h, MHC_ERR_INVALID_ARG, "bin id %d outside [-1, %d)", b, B);
    h->B = B;
    // counting sort, stable in the input mode index
    std::vector<int64_t> cnt(B + 1, 0);
    for (int b : bin_of_mode)
        if (b >= 0) cnt[b + 1]++;
    for (int b = 0; b < B; ++b) cnt[b + 1] += cnt[b];
    h->M_eff = cnt[B];
    h->perm.assign(h->M_eff, 0);
    {
        std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
        for (int64_t n = 0; n < (int64_t)bin_of_mode.size(); ++n)
            if (bin_of_mode[n] >= 0) h->perm[pos[bin_of_mode[n]]++] = (int)n;
    }
    // a multiple of 256 so that two-SM tiles (256 modes per CTA pair) need no bounds checks
    h->M_pad = round_up(std::max<int64_t>(h->M_eff, 1), is_tc(h) ? 2 * TC_BM : TC_BM);
    std::vector<int> mbin(h->M_pad, -1), mslot(h->M_pad, -1), sbeg(B + 1, 0);
    for (int64_t q = 0; q < h->M_eff; ++q) mbin[q] = bin_of_mode[h->perm[q]];
    // a slot for the last mode of every run of equal bins inside each 32-mode group
    int64_t ns = 0;
    std::vector<int> slot_bin;
    for (int64_t q = 0; q < h->M_eff; ++q) {
        const bool group_end = (q % 32) == 31 || q + 1 == h->M_eff;
        if (group_end || mbin[q + 1] != mbin[q]) {
            mslot[q] = (int)ns++;
            slot_bin.push_back(mbin[q]);
        }
    }
    h->n_slots = std::max<int64_t>(ns, 1);
    for (int b = 0, s = 0; b <= B; ++b) {
        while (s < (int)slot_bin.size() && slot_bin[s] < b) ++s;
        sbeg[b] = s;
    }
    sbeg[B] = (int)slot_bin.size();
    if (h->dir) {
        // output row b*B + bin reads slots b*n_slots + [sbeg[bin], sbeg[bin+1])
        std::vector<int> sd(3 * (size_t)B + 1);
        for (int b = 0; b < 3; ++b)
            for (int q = 0; q < B; ++q) sd[(size_t)b * B + q] = b * (int)h->n_slots + sbeg[q];
        sd[3 * (size_t)B] = 2 * (int)h->n_slots + sbeg[B];
        sbeg.swap(sd);
    }
    const int64_t nbo = n_out_bins(h);

    mhc_status s;
    const int K = h->prm.k_max;
    if ((s = dev_alloc(h, "mode_bin", sizeof(int) * h->M_pad, false)) != MHC_OK) return s;
    if ((s = dev_alloc(h, "mode_slot", sizeof(int) * h->M_pad, false)) != MHC_OK) return s;
    if ((s = dev_alloc(h, "slot_begin", sizeof(int) * (nbo + 1), false)) != MHC_OK) return s;
    if ((s = dev_alloc(h, "perm", sizeof(int) * std::max<int64_t>(h->M_eff, 1), false)) != MHC_OK) return s;
    if ((s = dev_alloc(h, "partials", sizeof(float) * K * 3 * slot_stride(h))) != MHC_OK) return s;
    if ((s = dev_alloc(h, "Jb", sizeof(float) * K * nbo * 3)) != MHC_OK) return s;
    MHC_CUDA(h, cudaMemcpyAsync(dptr<int>(h, "mode_bin"), mbin.data(), sizeof(int) * h->M_pad,
                                cudaMemcpyHostToDevice, h->stream));
    MHC_CUDA(h, cudaMemcpyAsync(dptr<int>(h, "mode_slot"), mslot.data(), sizeof(int) * h->M_pad,
                                cudaMemcpyHostToDevice, h->stream));
    MHC_CUDA(h, cudaMemcpyAsync(dptr<int>(h, "slot_begin"), sbeg.data(), sizeof(int) * (nbo + 1),
                                cudaMemcpyHostToDevice, h->stream));
    if (h->M_eff > 0)
        MHC_CUDA(h, cudaMemcpyAsync(dptr<int>(h, "perm"), h->perm.data(), sizeof(int) * h->M_eff,
                                    cudaMemcpyHostToDevice, h->stream));

    // stored eigenvectors
    const size_t ecount = (size_t)h->M_pad * h->D_ld;
    if (is_tc(h)) {
        dev_free(h, "Et32");
        if ((s = dev_alloc(h, "Et_hi", ecount * 2, false)) != MHC_OK) return s;
        if ((s = dev_alloc(h, "Et_lo", ecount * 2, false)) != MHC_OK) return s;
        if (h->dir && (s = dev_alloc(h, "dir_park", sizeof(float) * DIR_PARK_CTA_FLOATS * h->sm_count,
                                     false)) != MHC_OK)
            return s;
    } else {
        if ((s = dev_alloc(h, "Et32", ecount * 4, false)) != MHC_OK) return s;
        if ((s = dev_alloc(h, "R", sizeof(float) * h->B_rows * h->M_pad * (h->dir ? 3 : 1), false)) != MHC_OK)
            return s;
    }
    // Eraw is already in the stored column order (direction-major with the split)
    launch_prepare_modes(dptr<float>(h, "Eraw"), MHC_F32, MHC_MODE_MAJOR, h->D_ld,
                         h->dir ? h->D_ld : h->D, h->M_eff, dptr<int>(h, "perm"), h->e_exp,
                         h->split, dptr<void>(h, "Et_hi"), dptr<void>(h, "Et_lo"),
                         dptr<float>(h, "Et32"), h->D_ld, h->M_pad, 0, h->stream);
    h->launches++;
    MHC_CUDA(h, cudaGetLastError());

    if (is_tc(h)) {
        TcProblem &P = h->tcp.prob[0];
        const TcConfig &c = h->tc;
        if (encode_maps(h, c, P)) return fail(h, MHC_ERR_CUDA, "cuTensorMapEncodeTiled failed");
        P.mode_bin = dptr<int>(h, "mode_bin");
        P.mode_slot = dptr<int>(h, "mode_slot");
        P.col_scale = dptr<float>(h, "col_scale");
        P.partials = dptr<float>(h, "partials");
        P.n_slots = (int)h->n_slots;
        P.n_kb = (int)(h->D_ld / c.bk);
        P.dir_seg_kb = h->dir ? (int)(h->N_pad / c.bk) : 0;
        P.dir_park = h->dir ? dptr<float>(h, "dir_park") : nullptr;
        h->tcp.dir_park_ctas = h->dir ? h->sm_count : 0;
        h->tcp.sched = nullptr;
        h->tcp.cta_begin = nullptr;
        h->tcp.n_prob = 1;
        h->tcp.status = h->status;
        h->tcp.wait_limit = 2000000000ll;
        h->tcp.idesc = idesc_f16(h->split == SPLIT_BF16 ? 1u : 0u, (c.pair ? 2 : 1) * TC_BM, (uint32_t)c.bn);
    }
    h->bins_ready = true;
    return reset_accumulators(h);
}

// Balanced split, host side (the kernels' arithmetic): the part holding tail chunk g when T
// chunks are cut into `parts` ranges, and the plan of one block: whole waves of tiles first
// (t0 tiles on all `parts_all` CTAs or pairs), then the remaining tiles' chunks over
// `parts` <= parts_all ranges; max_seg is the largest number of segments a tail tile is cut into.
int sk_part_of_host(long long g, long long T, int parts) {
    return (int)(((g + 1) * parts + T - 1) / T - 1);
}

struct SkPlan {
    int nch = 0, tiles = 0, parts_all = 0, t0 = 0, parts = 0, max_seg = 1;
};

SkPlan sk_plan(const mhc_handle *h, const TcConfig &c, int n_col_tiles) {
    SkPlan q;
    const int chunk_kb = TC_PROMOTE_D / c.bk;
    q.nch = (int)((h->D_ld / c.bk + chunk_kb - 1) / chunk_kb);
    q.tiles = mode_tiles(h, c) * n_col_tiles;
    q.parts_all = std::max(1, sched_units(h, c));
    q.t0 = q.tiles / q.parts_all * q.parts_all;
    if (q.t0 == q.tiles) return q;   // whole waves only: no tail, nothing to split
    const long long T = (long long)(q.tiles - q.t0) * q.nch;
    q.parts = (int)std::min<long long>(q.parts_all, T);
    for (int t = q.t0; t < q.tiles; ++t) {
        const long long g0 = (long long)(t - q.t0) * q.nch;
        q.max_seg = std::max(q.max_seg, 1 + sk_part_of_host(g0 + q.nch - 1, T, q.parts) -
                                            sk_part_of_host(g0, T, q.parts));
    }
    return q;
}

// Bytes of the d-axis split workspace of configuration c: [segment][columns][M_pad], for the
// largest block (the uniform split), or the largest segments x columns of any block length up
// to k_max (the balanced split: short blocks have fewer tiles, cut into more segments).
size_t split_ws_bytes(const mhc_handle *h, const TcConfig &c) {
    if (c.split == TC_SPLIT_BALANCED) {
        size_t worst = 0;
        const int nct_max = (4 * h->prm.k_max + c.bn - 1) / c.bn;
        for (int nct = 1; nct <= nct_max; ++nct)
            worst = std::max(worst, (size_t)sk_plan(h, c, nct).max_seg * nct * c.bn);
        return sizeof(float) * worst * (size_t)h->M_pad;
    }
    if (c.split <= 1) return 0;
    const size_t cols = (size_t)((4 * h->prm.k_max + c.bn - 1) / c.bn) * c.bn;
    return sizeof(float) * (size_t)c.split * cols * (size_t)h->M_pad;
}

// The split workspace of configuration c, grown if needed (outside any stream capture: a
// larger workspace replaces the old one, so the graphs captured with its address are dropped).
mhc_status ensure_split_ws(mhc_handle *h, const TcConfig &c) {
    const size_t need = split_ws_bytes(h, c);
    if (!need) return MHC_OK;
    auto it = h->buf.find("split_ws");
    if (it != h->buf.end() && it->second.bytes >= need) return MHC_OK;
    cudaStreamSynchronize(h->stream);
    drop_graphs(h);
    return dev_alloc(h, "split_ws", need, false);
}

mhc_status set_tc_config(mhc_handle *h, const TcConfig &c) {
    if (!tc_config_supported(c)) return fail(h, MHC_ERR_INVALID_ARG, "unsupported tile configuration");
    if ((c.split > 1 || c.split == TC_SPLIT_BALANCED) && (h->dir || c.split > TC_MAX_SPLIT))
        return fail(h, MHC_ERR_INVALID_ARG, "d-axis split %d not available here", c.split);
    if (c.split < 1 && c.split != TC_SPLIT_BALANCED)
        return fail(h, MHC_ERR_INVALID_ARG, "d-axis split %d not available here", c.split);
    if (mhc_status s = ensure_split_ws(h, c); s != MHC_OK) return s;
    const bool remap = h->bins_ready && (c.bn != h->tc.bn || c.bk != h->tc.bk || c.pair != h->tc.pair);
    h->tc = c;
    if (remap) {
        TcProblem &P = h->tcp.prob[0];
        if (encode_maps(h, c, P)) return fail(h, MHC_ERR_CUDA, "cuTensorMapEncodeTiled failed");
        P.n_kb = (int)(h->D_ld / c.bk);
        P.dir_seg_kb = h->dir ? (int)(h->N_pad / c.bk) : 0;
        h->tcp.idesc = idesc_f16(h->split == SPLIT_BF16 ? 1u : 0u, (c.pair ? 2 : 1) * TC_BM, (uint32_t)c.bn);
    }
    return MHC_OK;
}

// The projections + fused epilogue of one block of K steps (after pack).
mhc_status run_projection(mhc_handle *h, int K) {
    if (h->M_eff == 0) {
        MHC_CUDA(h, cudaMemsetAsync(dptr<float>(h, "partials"), 0,
                                    sizeof(float) * K * 3 * slot_stride(h), h->stream));
        return MHC_OK;
    }
    if (!is_tc(h) && h->dir) {
        // one product per direction segment of d, then Xdot = sum over segments
        const size_t rstride = (size_t)h->B_rows * h->M_pad;
        for (int b = 0; b < 3; ++b)
            launch_sgemm(dptr<float>(h, "Et32") + b * h->N_pad, dptr<float>(h, "Bt32") + b * h->N_pad,
                         dptr<float>(h, "R") + b * rstride, (int)h->N_pad, (int)h->D_ld,
                         (int)h->M_pad, 4 * K, h->stream);
        launch_fp32_dir_epilogue(dptr<float>(h, "R"), rstride, (int)h->M_pad, K,
                                 dptr<int>(h, "mode_bin"), dptr<int>(h, "mode_slot"),
                                 dptr<float>(h, "partials"), (int)h->n_slots, h->stream);
        h->launches += 4;
        MHC_CUDA(h, cudaGetLastError());
        return MHC_OK;
    }
    if (!is_tc(h)) {
        launch_sgemm(dptr<float>(h, "Et32"), dptr<float>(h, "Bt32"), dptr<float>(h, "R"),
                     (int)h->D_ld, (int)h->D_ld, (int)h->M_pad, 4 * K, h->stream);
        launch_fp32_bin_epilogue(dptr<float>(h, "R"), (int)h->M_pad, K, dptr<int>(h, "mode_bin"),
                                 dptr<int>(h, "mode_slot"), dptr<float>(h, "partials"),
                                 (int)h->n_slots, h->stream);
        h->launches += 2;
        MHC_CUDA(h, cudaGetLastError());
        return MHC_OK;
    }
    TcConfig c = h->tc;
    TcProblem &P = h->tcp.prob[0];
    const bool stall = (h->prm.flags & MHC_FLAG_TEST_STALL) != 0;
    h->tcp.stall_inject = stall ? 1 : 0;
    h->tcp.wait_limit = stall ? 200000000ll : 2000000000ll;   // 0.1 s when testing the timeout
    P.K = K;
    P.n_col_tiles = (int)((4 * K + c.bn - 1) / c.bn);
    P.sk_parts = 0;
    P.ws_cols = P.n_col_tiles * c.bn;
    P.m_pad = (int)h->M_pad;
    const SkPlan skq = c.split == TC_SPLIT_BALANCED ? sk_plan(h, c, P.n_col_tiles) : SkPlan{};
    if (c.split == TC_SPLIT_BALANCED && skq.parts > 0) {
        // balanced split: whole waves of tiles, then one range of the tail's chunks per CTA
        // (pair); tiles cut by a range boundary are finished by the split finish kernel
        const SkPlan &q = skq;
        const size_t need = sizeof(float) * (size_t)q.max_seg * P.ws_cols * (size_t)h->M_pad;
        auto it = h->buf.find("split_ws");
        if (it == h->buf.end() || it->second.bytes < need)
            return fail(h, MHC_ERR_STATE, "balanced split workspace too small (%zu bytes needed)", need);
        P.n_split = 1;
        P.kb_split = P.n_kb;
        P.sk_parts = q.parts;
        P.sk_nch = q.nch;
        P.sk_tm = (c.pair ? 2 : 1) * TC_BM;
        P.sk_bn = c.bn;
        P.sk_t0 = q.t0;
        P.split_ws = dptr<float>(h, "split_ws");
        P.n_tiles = q.tiles;
        c.grid = q.parts_all * (c.pair ? 2 : 1);
        cudaError_t e = launch_tc_single(h->tcp, c, h->stream);
        h->launches++;
        if (e == cudaSuccess && q.max_seg > 1) {
            e = launch_tc_split_finish(h->tcp, h->stream);
            h->launches++;
        }
        if (e != cudaSuccess)
            return fail(h, MHC_ERR_CUDA, "tensor-core kernel launch failed: %s", cudaGetErrorString(e));
        return MHC_OK;
    }
    // d-axis split: whole promotion chunks per split, no empty split (a balanced split whose
    // tiles fill whole waves runs unsplit)
    const int chunk_kb = TC_PROMOTE_D / c.bk;
    int kb_split = P.n_kb, S = 1;
    if (c.split > 1) {
        kb_split = ((P.n_kb + c.split - 1) / c.split + chunk_kb - 1) / chunk_kb * chunk_kb;
        S = (P.n_kb + kb_split - 1) / kb_split;
    }
    P.n_split = S;
    P.kb_split = kb_split;
    P.split_ws = S > 1 ? dptr<float>(h, "split_ws") : nullptr;
    P.n_tiles = mode_tiles(h, c) * P.n_col_tiles * S;
    c.grid = std::min(sched_units(h, c), P.n_tiles) * (c.pair ? 2 : 1);
    cudaError_t e = launch_tc_single(h->tcp, c, h->stream);
    h->launches++;
    if (e == cudaSuccess && S > 1) {
        e = launch_tc_split_finish(h->tcp, h->stream);
        h->launches++;
    }
    if (e != cudaSuccess)
        return fail(h, MHC_ERR_CUDA, "tensor-core kernel launch failed: %s", cudaGetErrorString(e));
    return MHC_OK;
}

// ---- autotuning of the tile shape and the d-axis split count
// Results are kept per process (every handle of the same device, precision, shape and block
// length reuses them) and, when the environment variable MHC_TUNE_CACHE names a file, in that
// file across processes.
struct TuneKey {
    std::string device;
    int sm, prec, dir, K, split_req;
    int64_t D_ld, M_eff;
    bool operator<(const TuneKey &o) const {
        return std::tie(device, sm, prec, dir, K, split_req, D_ld, M_eff) <
               std::tie(o.device, o.sm, o.prec, o.dir, o.K, o.split_req, o.D_ld, o.M_eff);
    }
};
std::mutex g_tune_mutex;
std::map<TuneKey, TcConfig> g_tune_cache;
bool g_tune_file_read = false;

TuneKey tune_key(const mhc_handle *h, int K) {
    return TuneKey{h->device_name, h->sm_count, (int)h->split, h->dir ? 1 : 0, K,
                   (int)h->prm.split_d, h->D_ld, h->M_eff};
}

// Cache file lines: sm prec dir K split_req D_ld M_eff bn bk stages pair split <device name>
void tune_file_read_locked() {
    if (g_tune_file_read) return;
    g_tune_file_read = true;
    const char *path = std::getenv("MHC_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    char line[512];
    while (std::fgets(line, sizeof line, f)) {
        TuneKey k;
        TcConfig c{};
        long long D = 0, M = 0;
        int used = 0;
        if (std::sscanf(line, "%d %d %d %d %d %lld %lld %d %d %d %d %d %n", &k.sm, &k.prec, &k.dir, &k.K,
                        &k.split_req, &D, &M, &c.bn, &c.bk, &c.stages, &c.pair, &c.split, &used) < 12)
            continue;
        std::string name(line + used);
        while (!name.empty() && (name.back() == '\n' || name.back() == '\r')) name.pop_back();
        k.device = name;
        k.D_ld = D;
        k.M_eff = M;
        if (tc_config_supported(c) && ((c.split >= 1 && c.split <= TC_MAX_SPLIT) || c.split == TC_SPLIT_BALANCED))
            g_tune_cache[k] = c;
    }
    std::fclose(f);
}

void tune_file_append_locked(const TuneKey &k, const TcConfig &c) {
    const char *path = std::getenv("MHC_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%d %d %d %d %d %lld %lld %d %d %d %d %d %s\n", k.sm, k.prec, k.dir, k.K,
                 k.split_req, (long long)k.D_ld, (long long)k.M_eff, c.bn, c.bk, c.stages, c.pair,
                 c.split, k.device.c_str());
    std::fclose(f);
}

// Time candidate configurations in interleaved rounds (one warm-up launch each, then
// `rounds` rounds of one timed launch of every candidate) and keep each candidate's fastest
// launch: the candidates see the same clock and power state, where timing them one after the
// other let the power cap, reached during the first candidates' launches, slow the last ones.
mhc_status time_candidates(mhc_handle *h, int K, std::vector<std::pair<float, TcConfig>> &cands,
                           int rounds = 3) {
    cudaEvent_t e0, e1;
    MHC_CUDA(h, cudaEventCreate(&e0));
    MHC_CUDA(h, cudaEventCreate(&e1));
    mhc_status s = MHC_OK;
    for (auto &x : cands) {
        x.first = 1e30f;
        if ((s = set_tc_config(h, x.second)) != MHC_OK || (s = run_projection(h, K)) != MHC_OK) break;
    }
    for (int r = 0; r < rounds && s == MHC_OK; ++r)
        for (auto &x : cands) {
            float ms = 0.f;
            if ((s = set_tc_config(h, x.second)) != MHC_OK) break;
            if (cudaEventRecord(e0, h->stream) != cudaSuccess) { s = fail(h, MHC_ERR_CUDA, "event record"); break; }
            if ((s = run_projection(h, K)) != MHC_OK) break;
            if (cudaEventRecord(e1, h->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                s = fail(h, MHC_ERR_CUDA, "autotune timing failed");
                break;
            }
            x.first = std::min(x.first, ms);
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return s;
}

// Autotune on the block just packed: time every tile shape unsplit (or with the fixed split of
// mhc_params.split_d), then, for the two fastest shapes, the balanced split when the last wave
// of tiles is partial and the uniform d-axis splits 2..8 when one block gives fewer than three
// waves.  The winner is cached.
mhc_status autotune(mhc_handle *h, int K) {
    const TuneKey key = tune_key(h, K);
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        tune_file_read_locked();
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            h->tuned[K] = it->second;
            return set_tc_config(h, it->second);
        }
    }
    std::vector<std::pair<float, TcConfig>> res;
    const int fixed =
        h->prm.split_d == TC_SPLIT_BALANCED ? TC_SPLIT_BALANCED : std::max(1, (int)h->prm.split_d);
    for (TcConfig c : TC_CONFIGS) {
        c.split = fixed;
        res.emplace_back(0.f, c);
    }
    mhc_status s = time_candidates(h, K, res);
    if (s == MHC_OK && h->prm.split_d == 0 && !h->dir) {
        std::sort(res.begin(), res.end(),
                  [](const std::pair<float, TcConfig> &a, const std::pair<float, TcConfig> &b) {
                      return a.first < b.first;
                  });
        // the two fastest shapes again, unsplit, beside their splits (timed in the same rounds)
        std::vector<std::pair<float, TcConfig>> sp;
        const size_t n_shapes = std::min<size_t>(2, res.size());
        const size_t budget = (size_t)512 << 20;   // largest split workspace tried
        for (size_t q = 0; q < n_shapes; ++q) {
            TcConfig c = res[q].second;
            sp.emplace_back(0.f, c);
            const int n_kb = (int)(h->D_ld / c.bk), chunk_kb = TC_PROMOTE_D / c.bk;
            const int64_t units = (int64_t)mode_tiles(h, c) * ((4 * K + c.bn - 1) / c.bn);
            const int64_t su = sched_units(h, c);
            c.split = TC_SPLIT_BALANCED;   // whenever the last wave is partial
            if (units % su && split_ws_bytes(h, c) <= budget) sp.emplace_back(0.f, c);
            if (units >= 3 * su) continue;
            for (int S : {2, 3, 4, 6, 8}) {
                if (n_kb < S * chunk_kb) break;
                c.split = S;
                if (split_ws_bytes(h, c) > budget) break;
                sp.emplace_back(0.f, c);
            }
        }
        if (sp.size() > n_shapes) {
            s = time_candidates(h, K, sp);
            res = sp;
        }
    }
    if (s != MHC_OK) return s;
    TcConfig best_c = h->tc;
    float best = 1e30f;
    for (auto &r : res)
        if (r.first < best) {
            best = r.first;
            best_c = r.second;
        }
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        if (!g_tune_cache.count(key)) {
            g_tune_cache[key] = best_c;
            tune_file_append_locked(key, best_c);
        }
    }
    h->tuned[K] = best_c;
    return set_tc_config(h, best_c);
}

// Host inputs: copy into the next staging pair on the copy stream once the push that last
// read that pair is done (stage_issue); the push's kernels wait for the copy on the device
// (stage_order) and are queued before the host waits for it (stage_wait_on: host inputs are
// read before the call returns), so the previous push's kernels keep running meanwhile and the
// launches of this one overlap its upload.
mhc_status stage_issue(mhc_handle *h, const float *&v, const float *&W, int K, int where) {
    if (where == MHC_MEM_DEVICE) return MHC_OK;
    if (!h->copy_stream) {
        MHC_CUDA(h, cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
        for (int q = 0; q < 2; ++q) {
            MHC_CUDA(h, cudaEventCreateWithFlags(&h->copy_done[q], cudaEventDisableTiming));
            MHC_CUDA(h, cudaEventCreateWithFlags(&h->use_done[q], cudaEventDisableTiming));
        }
    }
    const int b = h->stage_next;
    const size_t nv = (size_t)K * h->N * 3, nw = (size_t)K * h->N * 9;
    float *dv = dptr<float>(h, b ? "v_stage1" : "v_stage"), *dw = dptr<float>(h, b ? "W_stage1" : "W_stage");
    if (h->use_pending[b]) MHC_CUDA(h, cudaStreamWaitEvent(h->copy_stream, h->use_done[b], 0));
    MHC_CUDA(h, cudaMemcpyAsync(dv, v, nv * 4, cudaMemcpyHostToDevice, h->copy_stream));
    MHC_CUDA(h, cudaMemcpyAsync(dw, W, nw * 4, cudaMemcpyHostToDevice, h->copy_stream));
    MHC_CUDA(h, cudaEventRecord(h->copy_done[b], h->copy_stream));
    h->stage_used = b;
    h->stage_next ^= 1;
    v = dv;
    W = dw;
    return MHC_OK;
}

mhc_status stage_order(mhc_handle *h, cudaStream_t s) {
    if (h->stage_used >= 0) MHC_CUDA(h, cudaStreamWaitEvent(s, h->copy_done[h->stage_used], 0));
    return MHC_OK;
}

// Host wait for staging pair b (b < 0: nothing was staged); keeps an earlier failure status.
mhc_status stage_wait_on(mhc_handle *h, int b, mhc_status prior) {
    if (b < 0) return prior;
    const cudaError_t e = cudaEventSynchronize(h->copy_done[b]);
    if (prior != MHC_OK) return prior;
    if (e != cudaSuccess) return fail(h, MHC_ERR_CUDA, "upload of host inputs failed: %s", cudaGetErrorString(e));
    return MHC_OK;
}

// After the kernels of a push that read a staging pair: mark when the pair is free again.
mhc_status release_stage(mhc_handle *h) {
    if (h->stage_used < 0) return MHC_OK;
    MHC_CUDA(h, cudaEventRecord(h->use_done[h->stage_used], h->stream));
    h->use_pending[h->stage_used] = true;
    h->stage_used = -1;
    return MHC_OK;
}

PackArgs pack_args(mhc_handle *h, const float *v, const float *W, int K) {
    PackArgs a{};
    a.v = v;
    a.W = W;
    a.sqm = dptr<float>(h, "sqm");
    a.isqm = dptr<float>(h, "isqm");
    a.N = (int)h->N;
    a.K = K;
    a.D_ld = (int)h->D_ld;
    a.split = h->split;
    a.e_exp = h->e_exp;
    a.t0 = h->steps;
    a.t0_dev = dptr<long long>(h, "steps_dev");
    a.Bt_hi = dptr<void>(h, "Bt_hi");
    a.Bt_lo = dptr<void>(h, "Bt_lo");
    a.Bt32 = dptr<float>(h, "Bt32");
    a.col_scale = dptr<float>(h, "col_scale");
    a.Jtot = dptr<double>(h, "Jtot");
    a.Jring = (h->prm.flags & MHC_FLAG_GKMA) ? dptr<double>(h, "Jring") : nullptr;
    a.R = h->R_ring;
    a.npad = h->dir ? (int)h->N_pad : 0;
    a.status = h->status;
    a.wait_limit = 0;
    return a;
}

mhc_status pack_block(mhc_handle *h, const float *v, const float *W, int K) {
    MHC_CUDA(h, launch_pack(pack_args(h, v, W, K), h->stream));
    h->launches++;
    MHC_CUDA(h, cudaGetLastError());
    return MHC_OK;
}

// The correlation kernels of a push (after its bin finish): GKMA lag correlation and the
// cross-correlations.
// advance: the lag correlation, when no cross-correlation kernel follows it, also advances the
// device step counter (*advanced is set then).
mhc_status correlate_block(mhc_handle *h, int K, bool advance = false, bool *advanced = nullptr) {
    if (advanced) *advanced = false;
    if (h->prm.flags & MHC_FLAG_GKMA) {
        const bool adv = advance && !has_xcorr(h);
        launch_lag_corr(dptr<float>(h, "Jb"), dptr<double>(h, "Jring"), h->R_ring,
                        dptr<double>(h, "Csum"), K, (int)n_out_bins(h), h->prm.n_lags, h->steps,
                        dptr<long long>(h, "steps_dev"),
                        adv ? dptr<long long>(h, "steps_dev") : nullptr,
                        dptr<unsigned>(h, "lc_ticket"), h->stream);
        if (advanced) *advanced = adv;
        h->launches++;
    }
    if (has_xcorr(h)) {
        launch_jb_ring_store(dptr<float>(h, "Jb"), K, (int)n_out_bins(h), dptr<float>(h, "Jbring"),
                             h->R_ring, h->steps, dptr<long long>(h, "steps_dev"), h->stream);
        MHC_CUDA(h, launch_bin_xcorr(h->xc_plan, h->xcp, dptr<float>(h, "Jbring"), h->R_ring, K,
                                     h->steps, dptr<long long>(h, "steps_dev"),
                                     dptr<void>(h, "Xwin_hi"), dptr<void>(h, "Xwin_lo"), h->stream));
        h->launches += 3;
    }
    MHC_CUDA(h, cudaGetLastError());
    return MHC_OK;
}

// Kernels that close a push: bin finish + HNEMA sums, correlations, step counter.
mhc_status finish_kernels(mhc_handle *h, int K) {
    // without correlation kernels (which read the step counter) the bin finish advances it, and
    // with the lag correlation alone that kernel does
    const bool corr = (h->prm.flags & MHC_FLAG_GKMA) || has_xcorr(h);
    launch_bin_finish(dptr<float>(h, "partials"), (int)slot_stride(h), dptr<int>(h, "slot_begin"),
                      (int)n_out_bins(h), K, dptr<float>(h, "Jb"), dptr<double>(h, "hsum"),
                      dptr<double>(h, "Jtot"), dptr<double>(h, "Jsum"),
                      corr ? nullptr : dptr<long long>(h, "steps_dev"), h->stream);
    h->launches++;
    if (corr) {
        bool advanced = false;
        mhc_status s = correlate_block(h, K, true, &advanced);
        if (s != MHC_OK) return s;
        if (!advanced) {
            launch_advance_steps(dptr<long long>(h, "steps_dev"), K, h->stream);
            h->launches++;
        }
    }
    MHC_CUDA(h, cudaGetLastError());
    return MHC_OK;
}

void count_push(mhc_handle *h, int K) {
    h->steps += K;
    h->pushes++;
    h->K_last = K;
}

mhc_status finish_block(mhc_handle *h, int K) {
    mhc_status s = finish_kernels(h, K);
    if (s == MHC_OK) count_push(h, K);
    return s;
}

int config_index(const mhc_handle *h) {
    for (int q = 0; q < TC_NUM_CONFIGS; ++q)
        if (TC_CONFIGS[q].bn == h->tc.bn && TC_CONFIGS[q].bk == h->tc.bk &&
            TC_CONFIGS[q].stages == h->tc.stages && TC_CONFIGS[q].pair == h->tc.pair)
            return q;
    return -1;
}

// Capture pack -> projection -> finish of one push into a graph (on a private stream) and
// replay it on the handle's stream.  Inputs must already be in device memory.
mhc_status push_graph(mhc_handle *h, const float *v, const float *W, int K) {
    const int split_code = h->tc.split == TC_SPLIT_BALANCED ? 63 : std::max(1, h->tc.split);
    auto key = std::make_tuple(K, (const void *)v, (const void *)W,
                               is_tc(h) ? config_index(h) * 64 + split_code : -1);
    auto it = h->graphs.find(key);
    if (it == h->graphs.end()) {
        if (h->graphs.size() >= 32) {   // evict the least recently used graph
            auto lru = h->graphs.begin();
            for (auto g = h->graphs.begin(); g != h->graphs.end(); ++g)
                if (g->second.last_use < lru->second.last_use) lru = g;
            cudaGraphExecDestroy(lru->second.exec);
            h->graphs.erase(lru);
        }
        if (!h->cap_stream) MHC_CUDA(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
        cudaStream_t user = h->stream;
        const int64_t launches0 = h->launches;
        MHC_CUDA(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
        h->stream = h->cap_stream;
        mhc_status s = pack_block(h, v, W, K);
        if (s == MHC_OK) s = run_projection(h, K);
        if (s == MHC_OK) s = finish_kernels(h, K);
        h->stream = user;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(h->cap_stream, &graph);
        if (s != MHC_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        if (e != cudaSuccess) return fail(h, MHC_ERR_CUDA, "stream capture of a push failed: %s", cudaGetErrorString(e));
        Handle::GraphEntry ge;
        e = cudaGraphInstantiate(&ge.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return fail(h, MHC_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
        ge.nodes = h->launches - launches0;
        h->launches = launches0;
        it = h->graphs.emplace(key, ge).first;
    }
    it->second.last_use = ++h->graph_clock;
    MHC_CUDA(h, cudaGraphLaunch(it->second.exec, h->stream));
    h->launches += it->second.nodes;
    h->graph_replays++;
    count_push(h, K);
    return MHC_OK;
}

mhc_status copy_out(mhc_handle *h, void *dst, const void *src, size_t bytes, int where) {
    if (where == MHC_MEM_DEVICE) {
        MHC_CUDA(h, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, h->stream));
        return MHC_OK;
    }
    MHC_CUDA(h, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, h->stream));
    MHC_CUDA(h, cudaStreamSynchronize(h->stream));
    return check_device_status(h);
}

// The kernels of a push whose inputs are in device memory (or staged there, ordered on the
// handle's stream): a graph replay once the tile is tuned, else direct launches.
mhc_status push_staged(mhc_handle *h, const float *v, const float *W, int K) {
    mhc_status s;
    const bool tuned = !is_tc(h) || h->prm.tile_config != 0 || h->tuned.count(K);
    if (tuned && !(h->prm.flags & (MHC_FLAG_NO_GRAPH | MHC_FLAG_PROFILE | MHC_FLAG_TEST_STALL))) {
        if (is_tc(h) && h->prm.tile_config == 0 && (s = set_tc_config(h, h->tuned[K])) != MHC_OK) return s;
        if ((s = push_graph(h, v, W, K)) != MHC_OK) return s;
        return release_stage(h);
    }
    if ((s = pack_block(h, v, W, K)) != MHC_OK) return s;
    if (is_tc(h) && h->prm.tile_config == 0) {
        auto it = h->tuned.find(K);
        if (it == h->tuned.end()) {
            if ((s = autotune(h, K)) != MHC_OK) return s;
        } else if ((s = set_tc_config(h, it->second)) != MHC_OK) {
            return s;
        }
    }
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (h->prm.flags & MHC_FLAG_PROFILE) {
        if (h->prof_used == h->prof_events.size()) {
            cudaEvent_t a0, a1;
            MHC_CUDA(h, cudaEventCreate(&a0));
            MHC_CUDA(h, cudaEventCreate(&a1));
            h->prof_events.emplace_back(a0, a1);
        }
        ev0 = h->prof_events[h->prof_used].first;
        ev1 = h->prof_events[h->prof_used].second;
        ++h->prof_used;
        MHC_CUDA(h, cudaEventRecord(ev0, h->stream));
    }
    if ((s = run_projection(h, K)) != MHC_OK) return s;
    if (ev1) MHC_CUDA(h, cudaEventRecord(ev1, h->stream));
    if ((s = finish_block(h, K)) != MHC_OK) return s;
    return release_stage(h);
}

}  // namespace

// =====================================================================================
extern "C" {

void mhc_default_params(mhc_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->device = 0;
    p->stream = nullptr;
    p->k_max = 256;
    p->n_lags = 0;
    p->precision = MHC_PREC_BF16X3;
    p->flags = 0;
    p->tile_config = 0;
    p->split_d = 0;
    p->ortho_probe = -1;
    p->dt_ps = 0.01;
    p->T_K = 300.0;
    p->V_A3 = 1.0;
    p->F_e[0] = 1e-5;
}

const char *mhc_status_string(mhc_status s) {
    switch (s) {
    case MHC_OK: return "ok";
    case MHC_ERR_INVALID_ARG: return "invalid argument";
    case MHC_ERR_OOM: return "out of memory";
    case MHC_ERR_CUDA: return "CUDA error";
    case MHC_ERR_TIMEOUT: return "device wait timed out";
    case MHC_ERR_STATE: return "invalid state";
    case MHC_ERR_UNSUPPORTED: return "unsupported";
    case MHC_WARN_NOT_ORTHONORMAL: return "basis not orthonormal";
    }
    return "unknown status";
}

const char *mhc_last_error(const mhc_handle *h) {
    return h ? h->err.c_str() : g_create_error.c_str();
}

mhc_status mhc_measure_fp32_fma(int32_t device, void *stream, double *tflops) {
    set_handleless_error("");
    if (!tflops) {
        set_handleless_error("mhc_measure_fp32_fma: null output");
        return MHC_ERR_INVALID_ARG;
    }
    int sms = 0;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = measure_fp32_fma(static_cast<cudaStream_t>(stream), sms, tflops);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_handleless_error(cudaGetErrorString(e));
        return MHC_ERR_CUDA;
    }
    return MHC_OK;
}

mhc_status mhc_create(mhc_handle **out, const mhc_params *p) {
    if (!out || !p) return fail(nullptr, MHC_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    g_create_error.clear();
    if (p->k_max < 1 || p->k_max > K_MAX_LIMIT)
        return fail(nullptr, MHC_ERR_INVALID_ARG, "k_max must be in [1, %d]", K_MAX_LIMIT);
    if (p->n_lags < 0) return fail(nullptr, MHC_ERR_INVALID_ARG, "n_lags must be >= 0");
    if ((p->flags & MHC_FLAG_GKMA) && p->n_lags < 1)
        return fail(nullptr, MHC_ERR_INVALID_ARG, "GKMA needs n_lags >= 1");
    if ((p->flags & MHC_FLAG_XCORR) && !(p->flags & MHC_FLAG_GKMA))
        return fail(nullptr, MHC_ERR_INVALID_ARG, "MHC_FLAG_XCORR needs MHC_FLAG_GKMA");
    if (p->precision < MHC_PREC_FP32 || p->precision > MHC_PREC_FP16X3)
        return fail(nullptr, MHC_ERR_INVALID_ARG, "unknown precision %d", p->precision);
    if (p->tile_config < 0 || p->tile_config > TC_NUM_CONFIGS)
        return fail(nullptr, MHC_ERR_INVALID_ARG, "tile_config must be in [0, %d]", TC_NUM_CONFIGS);
    if (p->split_d < TC_SPLIT_BALANCED || p->split_d > TC_MAX_SPLIT)
        return fail(nullptr, MHC_ERR_INVALID_ARG, "split_d must be in [-1, %d]", TC_MAX_SPLIT);
    if ((p->flags & MHC_FLAG_DIRECTION) && (p->split_d > 1 || p->split_d == TC_SPLIT_BALANCED))
        return fail(nullptr, MHC_ERR_INVALID_ARG, "the direction split runs without d-axis splits");
    if (!(p->dt_ps > 0) || !(p->T_K > 0) || !(p->V_A3 > 0))
        return fail(nullptr, MHC_ERR_INVALID_ARG, "dt_ps, T_K and V_A3 must be positive");
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || p->device < 0 || p->device >= ndev)
        return fail(nullptr, MHC_ERR_CUDA, "no CUDA device %d (%s)", p->device,
                    e == cudaSuccess ? "out of range" : cudaGetErrorString(e));
    cudaDeviceProp prop;
    if ((e = cudaGetDeviceProperties(&prop, p->device)) != cudaSuccess)
        return fail(nullptr, MHC_ERR_CUDA, "cudaGetDeviceProperties: %s", cudaGetErrorString(e));
    const bool sm103 = prop.major == 10 && prop.minor == 3;
    if (!sm103)
        return fail(nullptr, MHC_ERR_UNSUPPORTED,
                    "device %d is sm_%d%d; this library is built for sm_103a only", p->device,
                    prop.major, prop.minor);
    auto *h = new mhc_handle();
    h->prm = *p;
    h->stream = static_cast<cudaStream_t>(p->stream);
    h->sm_count = prop.multiProcessorCount;
    h->device_name = prop.name;
    h->cc_major = prop.major;
    h->cc_minor = prop.minor;
    h->split = p->precision == MHC_PREC_FP32 ? SPLIT_FP32
               : p->precision == MHC_PREC_BF16X3 ? SPLIT_BF16 : SPLIT_FP16;
    h->dir = (p->flags & MHC_FLAG_DIRECTION) != 0;
    if (p->tile_config > 0) h->tc = TC_CONFIGS[p->tile_config - 1];
    else if (h->dir) h->tc = TC_CONFIGS[2];
    h->tc.split = p->split_d == TC_SPLIT_BALANCED ? TC_SPLIT_BALANCED : std::max(1, (int)p->split_d);
    if ((e = cudaSetDevice(p->device)) != cudaSuccess) {
        delete h;
        return fail(nullptr, MHC_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    }
    if ((e = cudaMalloc(&h->status, sizeof(int))) != cudaSuccess ||
        (e = cudaMemsetAsync(h->status, 0, sizeof(int), h->stream)) != cudaSuccess) {
        if (h->status) cudaFree(h->status);
        delete h;
        return fail(nullptr, MHC_ERR_OOM, "status word: %s", cudaGetErrorString(e));
    }
    *out = h;
    return MHC_OK;
}

void mhc_destroy(mhc_handle *h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    for (auto &e : h->prof_events) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    drop_graphs(h);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->copy_stream) {
        cudaStreamSynchronize(h->copy_stream);
        cudaStreamDestroy(h->copy_stream);
        for (int q = 0; q < 2; ++q) {
            cudaEventDestroy(h->copy_done[q]);
            cudaEventDestroy(h->use_done[q]);
        }
    }
    for (auto &kv : h->buf)
        if (kv.second.p) cudaFree(kv.second.p);
    if (h->status) cudaFree(h->status);
    delete h;
}

mhc_status mhc_set_modes(mhc_handle *h, int64_t n_atoms, int64_t n_modes, const void *E,
                         int32_t dtype, int32_t layout, int64_t ld, int32_t where,
                         const double *freq_THz, const double *mass_amu) {
    if (!h) return MHC_ERR_INVALID_ARG;
    if (!E || !mass_amu) return fail(h, MHC_ERR_INVALID_ARG, "E and mass_amu are required");
    if (n_atoms < 1 || n_modes < 1 || n_modes > 3 * n_atoms)
        return fail(h, MHC_ERR_INVALID_ARG, "need 1 <= M <= 3N (N=%lld, M=%lld)", (long long)n_atoms,
                    (long long)n_modes);
    if (dtype != MHC_F32 && dtype != MHC_F64) return fail(h, MHC_ERR_INVALID_ARG, "dtype");
    if (layout != MHC_DOF_MAJOR && layout != MHC_MODE_MAJOR) return fail(h, MHC_ERR_INVALID_ARG, "layout");
    if (where != MHC_MEM_HOST && where != MHC_MEM_DEVICE) return fail(h, MHC_ERR_INVALID_ARG, "where");
    const int64_t D = 3 * n_atoms;
    if (ld < (layout == MHC_DOF_MAJOR ? n_modes : D))
        return fail(h, MHC_ERR_INVALID_ARG, "ld %lld too small", (long long)ld);
    for (int64_t i = 0; i < n_atoms; ++i)
        if (!(mass_amu[i] > 0) || !std::isfinite(mass_amu[i]))
            return fail(h, MHC_ERR_INVALID_ARG, "mass of atom %lld must be positive", (long long)i);
    MHC_CUDA(h, cudaSetDevice(h->prm.device));
    MHC_CUDA(h, cudaStreamSynchronize(h->stream));
    drop_graphs(h);
    h->modes_ready = h->bins_ready = false;
    h->N = n_atoms;
    h->D = D;
    h->M_in = n_modes;
    // direction split: three segments of N_pad columns, N_pad a multiple of the 128-element
    // promotion chunk so that no chunk straddles two directions
    h->N_pad = h->dir ? round_up(n_atoms, 128) : 0;
    h->D_ld = h->dir ? 3 * h->N_pad : round_up(D, 64);
    h->mass.assign(mass_amu, mass_amu + n_atoms);
    if (freq_THz) h->freq.assign(freq_THz, freq_THz + n_modes);
    else h->freq.clear();
    h->B_rows = round_up(4 * (int64_t)h->prm.k_max, 256);
    h->R_ring = h->prm.k_max + std::max(h->prm.n_lags, 1);

    mhc_status s;
    // input eigenvectors on the device, as given
    const size_t esz = dtype == MHC_F64 ? 8 : 4;
    const int64_t rows = layout == MHC_DOF_MAJOR ? D : n_modes;
    const void *Edev = E;
    if (where == MHC_MEM_HOST) {
        if ((s = dev_alloc(h, "Ein", esz * rows * ld, false)) != MHC_OK) return s;
        MHC_CUDA(h, cudaMemcpyAsync(dptr<void>(h, "Ein"), E, esz * rows * ld, cudaMemcpyHostToDevice,
                                    h->stream));
        Edev = dptr<void>(h, "Ein");
    }
    // power-of-two scale of E for the FP16 split: max |E 2^e| < 2^14
    h->e_exp = 0;
    if (h->split == SPLIT_FP16) {
        if ((s = dev_alloc(h, "maxbits", sizeof(unsigned))) != MHC_OK) return s;
        launch_max_abs(Edev, dtype, layout, ld, D, n_modes, dptr<unsigned>(h, "maxbits"), h->stream);
        h->launches++;
        unsigned bits = 0;
        MHC_CUDA(h, cudaMemcpyAsync(&bits, dptr<unsigned>(h, "maxbits"), 4, cudaMemcpyDeviceToHost, h->stream));
        MHC_CUDA(h, cudaStreamSynchronize(h->stream));
        float mx;
        std::memcpy(&mx, &bits, 4);
        if (!(mx > 0) || !std::isfinite(mx)) return fail(h, MHC_ERR_INVALID_ARG, "E is zero or not finite");
        int ex;
        std::frexp(mx, &ex);
        h->e_exp = 14 - ex;
    }
    // optional FP64 basis check on the input (E^T E = I, Eq. 13-14)
    mhc_status warn = MHC_OK;
    h->ortho_err = -1.0;
    if (h->prm.ortho_probe >= 0) {
        const int64_t P = h->prm.ortho_probe == 0 ? n_modes : std::min<int64_t>(h->prm.ortho_probe, n_modes);
        std::vector<int> probe(P);
        for (int64_t q = 0; q < P; ++q) probe[q] = (int)((q * n_modes) / P);
        if ((s = dev_alloc(h, "probe", sizeof(int) * P, false)) != MHC_OK) return s;
        if ((s = dev_alloc(h, "orthobits", sizeof(unsigned long long))) != MHC_OK) return s;
        MHC_CUDA(h, cudaMemcpyAsync(dptr<int>(h, "probe"), probe.data(), sizeof(int) * P,
                                    cudaMemcpyHostToDevice, h->stream));
        launch_orthonormality(Edev, dtype, layout, ld, D, n_modes, dptr<int>(h, "probe"), (int)P,
                              dptr<unsigned long long>(h, "orthobits"), h->stream);
        h->launches++;
        unsigned long long bits = 0;
        MHC_CUDA(h, cudaMemcpyAsync(&bits, dptr<unsigned long long>(h, "orthobits"), 8,
                                    cudaMemcpyDeviceToHost, h->stream));
        MHC_CUDA(h, cudaStreamSynchronize(h->stream));
        std::memcpy(&h->ortho_err, &bits, 8);
        dev_free(h, "probe");
        dev_free(h, "orthobits");
        if (h->ortho_err > 1e-6) warn = MHC_WARN_NOT_ORTHONORMAL;
    }
    // resident FP32 copy in input mode order, mode-major (re-gathered on every re-binning)
    std::vector<int> ident(n_modes);
    for (int64_t q = 0; q < n_modes; ++q) ident[q] = (int)q;
    if ((s = dev_alloc(h, "perm", sizeof(int) * n_modes, false)) != MHC_OK) return s;
    MHC_CUDA(h, cudaMemcpyAsync(dptr<int>(h, "perm"), ident.data(), sizeof(int) * n_modes,
                                cudaMemcpyHostToDevice, h->stream));
    const int64_t Mraw = round_up(n_modes, 32);
    if ((s = dev_alloc(h, "Eraw", sizeof(float) * Mraw * h->D_ld, false)) != MHC_OK) return s;
    launch_prepare_modes(Edev, dtype, layout, ld, D, n_modes, dptr<int>(h, "perm"), 0, SPLIT_FP32,
                         nullptr, nullptr, dptr<float>(h, "Eraw"), h->D_ld, Mraw, h->N_pad, h->stream);
    h->launches++;
    MHC_CUDA(h, cudaGetLastError());
    MHC_CUDA(h, cudaStreamSynchronize(h->stream));
    dev_free(h, "Ein");

    // per-atom weights and per-block buffers
    std::vector<float> sq(n_atoms), isq(n_atoms);
    for (int64_t i = 0; i < n_atoms; ++i) {
        sq[i] = (float)std::sqrt(h->mass[i]);
        isq[i] = (float)(1.0 / std::sqrt(h->mass[i]));
    }
    const int K = h->prm.k_max;
    if ((s = dev_alloc(h, "sqm", sizeof(float) * n_atoms, false)) != MHC_OK) return s;
    if ((s = dev_alloc(h, "isqm", sizeof(float) * n_atoms, false)) != MHC_OK) return s;
    MHC_CUDA(h, cudaMemcpyAsync(dptr<float>(h, "sqm"), sq.data(), 4 * n_atoms, cudaMemcpyHostToDevice, h->stream));
    MHC_CUDA(h, cudaMemcpyAsync(dptr<float>(h, "isqm"), isq.data(), 4 * n_atoms, cudaMemcpyHostToDevice, h->stream));
    const size_t bcount = (size_t)h->B_rows * h->D_ld;
    if (is_tc(h)) {
        dev_free(h, "Bt32");
        if ((s = dev_alloc(h, "Bt_hi", bcount * 2)) != MHC_OK) return s;
        if ((s = dev_alloc(h, "Bt_lo", bcount * 2)) != MHC_OK) return s;
    } else {
        if ((s = dev_alloc(h, "Bt32", bcount * 4)) != MHC_OK) return s;
    }
    if ((s = dev_alloc(h, "col_scale", sizeof(float) * 4 * K)) != MHC_OK) return s;
    if ((s = dev_alloc(h, "Jtot", sizeof(double) * 3 * K)) != MHC_OK) return s;
    for (const char *nm : {"v_stage", "v_stage1"})
        if ((s = dev_alloc(h, nm, sizeof(float) * K * n_atoms * 3, false)) != MHC_OK) return s;
    for (const char *nm : {"W_stage", "W_stage1"})
        if ((s = dev_alloc(h, nm, sizeof(float) * K * n_atoms * 9, false)) != MHC_OK) return s;
    MHC_CUDA(h, cudaStreamSynchronize(h->stream));
    h->modes_ready = true;
    h->tuned.clear();
    return warn;
}

mhc_status mhc_set_bins_uniform(mhc_handle *h, double f_min, double f_max, int32_t n_bins) {
    if (!h) return MHC_ERR_INVALID_ARG;
    if (!h->modes_ready) return fail(h, MHC_ERR_INVALID_ARG, "mhc_set_modes must come first");
    if (h->freq.empty()) return fail(h, MHC_ERR_INVALID_ARG, "no frequencies were given");
    if (n_bins < 1 || !(f_max > f_min) || !std::isfinite(f_min) || !std::isfinite(f_max))
        return fail(h, MHC_ERR_INVALID_ARG, "need n_bins >= 1 and f_min < f_max");
    std::vector<int> bins;
    bins_uniform_host(h->freq, f_min, f_max, n_bins, bins);
    MHC_CUDA(h, cudaSetDevice(h->prm.device));
    mhc_status s = apply_bins(h, bins, n_bins);
    if (s == MHC_OK) MHC_CUDA(h, cudaStreamSynchronize(h->stream));
    return s;
}

mhc_status mhc_set_bin_ids(mhc_handle *h, const int32_t *bin_of_mode, int32_t n_bins) {
    if (!h) return MHC_ERR_INVALID_ARG;
    if (!h->modes_ready) return fail(h, MHC_ERR_INVALID_ARG, "mhc_set_modes must come first");
    if (!bin_of_mode) return fail(h, MHC_ERR_INVALID_ARG, "bin_of_mode is null");
    std::vector<int> bins(bin_of_mode, bin_of_mode + h->M_in);
    MHC_CUDA(h, cudaSetDevice(h->prm.device));
    mhc_status s = apply_bins(h, bins, n_bins);
    if (s == MHC_OK) MHC_CUDA(h, cudaStreamSynchronize(h->stream));
    return s;
}

mhc_status mhc_push(mhc_handle *h, const float *v, const float *W, int32_t K, int32_t where) {
    if (!h) return MHC_ERR_INVALID_ARG;
    if (!h->bins_ready) return fail(h, MHC_ERR_INVALID_ARG, "modes and bins must be set before pushing");
    if (!v || !W) return fail(h, MHC_ERR_INVALID_ARG, "v and W are required");
    if (K < 1 || K > h->prm.k_max) return fail(h, MHC_ERR_INVALID_ARG, "K=%d outside [1, %d]", K, h->prm.k_max);
    if (where != MHC_MEM_HOST && where != MHC_MEM_DEVICE && where != MHC_MEM_HOST_ASYNC)
        return fail(h, MHC_ERR_INVALID_ARG, "where");
    MHC_CUDA(h, cudaSetDevice(h->prm.device));
    mhc_status s;
    if (is_tc(h) && (s = ensure_split_ws(h, h->tc)) != MHC_OK) return s;
    if ((s = stage_issue(h, v, W, K, where)) != MHC_OK) return s;
    const int staged = h->stage_used;
    s = stage_order(h, h->stream);
    if (s == MHC_OK) s = push_staged(h, v, W, K);
    // the previous asynchronous upload was queued before this one's
    const int pending = h->async_stage;
    h->async_stage = -1;
    s = stage_wait_on(h, pending, s);
    if (where == MHC_MEM_HOST_ASYNC && s == MHC_OK) {
        h->async_stage = staged;
        return MHC_OK;
    }
    return stage_wait_on(h, staged, s);
}

mhc_status mhc_autotune_k(mhc_handle *h, const int32_t *candidates, int32_t n, int32_t *best_K,
                          double *steps_per_s) {
    if (!h) return MHC_ERR_INVALID_ARG;
    if (!candidates || n < 1 || !best_K) return fail(h, MHC_ERR_INVALID_ARG, "need candidates and best_K");
    if (!h->bins_ready) return fail(h, MHC_ERR_INVALID_ARG, "modes and bins must be set first");
    for (int32_t q = 0; q < n; ++q)
        if (candidates[q] < 1 || candidates[q] > h->prm.k_max)
            return fail(h, MHC_ERR_INVALID_ARG, "candidate K=%d outside [1, %d]", candidates[q], h->prm.k_max);
    MHC_CUDA(h, cudaSetDevice(h->prm.device));
    // a block of the largest K of constant, finite samples in the first staging pair, after the
    // pushes that may still read that pair
    MHC_CUDA(h, cudaStreamSynchronize(h->stream));
    if (h->copy_stream) MHC_CUDA(h, cudaStreamSynchronize(h->copy_stream));
    float *v = dptr<float>(h, "v_stage"), *W = dptr<float>(h, "W_stage");
    MHC_CUDA(h, cudaMemsetAsync(v, 0x3f, sizeof(float) * h->prm.k_max * h->N * 3, h->stream));
    MHC_CUDA(h, cudaMemsetAsync(W, 0x3f, sizeof(float) * h->prm.k_max * h->N * 9, h->stream));
    cudaEvent_t e0, e1;
    MHC_CUDA(h, cudaEventCreate(&e0));
    MHC_CUDA(h, cudaEventCreate(&e1));
    mhc_status s = MHC_OK;
    double best = -1.0;
    int32_t bestK = candidates[0];
    for (int32_t q = 0; q < n && s == MHC_OK; ++q) {
        const int K = candidates[q];
        if ((s = pack_block(h, v, W, K)) != MHC_OK) break;
        if (is_tc(h) && h->prm.tile_config == 0) {
            auto it = h->tuned.find(K);
            s = it == h->tuned.end() ? autotune(h, K) : set_tc_config(h, it->second);
            if (s != MHC_OK) break;
        }
        const int reps = 3;
        cudaError_t e = cudaEventRecord(e0, h->stream);
        for (int r = 0; r < reps && s == MHC_OK; ++r)
            if ((s = pack_block(h, v, W, K)) == MHC_OK) s = run_projection(h, K);
        if (s != MHC_OK) break;
        if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            s = fail(h, MHC_ERR_CUDA, "timing of K=%d failed: %s", K, cudaGetErrorString(e));
            break;
        }
        const double rate = ms > 0 ? reps * (double)K / (ms * 1e-3) : 0.0;
        if (rate > best) {
            best = rate;
            bestK = K;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != MHC_OK) return s;
    h->K_last = 0;   // the packed operands no longer belong to the last pushed block
    *best_K = bestK;
    if (steps_per_s) *steps_per_s = best;
    return MHC_OK;
}

mhc_status mhc_sync(mhc_handle *h) {
    if (!h) return MHC_ERR_INVALID_ARG;
    MHC_CUDA(h, cudaStreamSynchronize(h->stream));
    const int pending = h->async_stage;
    h->async_stage = -1;
    const mhc_status s = stage_wait_on(h, pending, MHC_OK);
    return s != MHC_OK ? s : check_device_status(h);
}

mhc_status mhc_read_binned_current(mhc_handle *h, float *out, int32_t where) {
    if (!h || !out) return h ? fail(h, MHC_ERR_INVALID_ARG, "null output") : MHC_ERR_INVALID_ARG;
    if (h->K_last == 0) return fail(h, MHC_ERR_INVALID_ARG, "nothing pushed yet");
    return copy_out(h, out, dptr<float>(h, "Jb"), sizeof(float) * h->K_last * n_out_bins(h) * 3, where);
}

mhc_status mhc_read_total_current(mhc_handle *h, double *out, int32_t where) {
    if (!h || !out) return h ? fail(h, MHC_ERR_INVALID_ARG, "null output") : MHC_ERR_INVALID_ARG;
    if (h->K_last == 0) return fail(h, MHC_ERR_INVALID_ARG, "nothing pushed yet");
    return copy_out(h, out, dptr<double>(h, "Jtot"), sizeof(double) * h->K_last * 3, where);
}

mhc_status mhc_read_hnema(mhc_handle *h, double *kappa, double *mean_J, int32_t where) {
    if (!h) return MHC_ERR_INVALID_ARG;
    if (!h->bins_ready) return fail(h, MHC_ERR_INVALID_ARG, "no bins");
    mhc_status s;
    const size_t n = (size_t)n_out_bins(h) * 3;
    if ((s = dev_alloc(h, "hn_out", sizeof(double) * 2 * n, false)) != MHC_OK) return s;
    const double fe = std::sqrt(h->prm.F_e[0] * h->prm.F_e[0] + h->prm.F_e[1] * h->prm.F_e[1] +
                                h->prm.F_e[2] * h->prm.F_e[2]);
    const double coef = fe > 0 ? WMK_PER_EV_PS_A_K / (h->prm.T_K * h->prm.V_A3 * fe) : 0.0;
    double *dm = dptr<double>(h, "hn_out"), *dk = dm + n;
    launch_hnema_finalize(dptr<double>(h, "hsum"), (int)n_out_bins(h), h->steps, coef, dm, dk, h->stream);
    h->launches++;
    MHC_CUDA(h, cudaGetLastError());
    if (kappa && (s = copy_out(h, kappa, dk, sizeof(double) * n, where)) != MHC_OK) return s;
    if (mean_J && (s = copy_out(h, mean_J, dm, sizeof(double) * n, where)) != MHC_OK) return s;
    return MHC_OK;
}

mhc_status mhc_read_corr(mhc_handle *h, double *corr_sum, int64_t *count, int32_t where) {
    if (!h) return MHC_ERR_INVALID_ARG;
    if (!(h->prm.flags & MHC_FLAG_GKMA) || !h->bins_ready)
        return fail(h, MHC_ERR_INVALID_ARG, "GKMA is not enabled or no bins");
    const int L = h->prm.n_lags;
    mhc_status s;
    if (corr_sum && (s = copy_out(h, corr_sum, dptr<double>(h, "Csum"),
                                  sizeof(double) * n_out_bins(h) * 9 * L, where)) != MHC_OK)
        return s;
    if (count) {
        if ((s = dev_alloc(h, "counts", sizeof(long long) * L, false)) != MHC_OK) return s;
        launch_lag_counts(h->steps, L, dptr<long long>(h, "counts"), h->stream);
        h->launches++;
        if ((s = copy_out(h, count, dptr<long long>(h, "counts"), sizeof(long long) * L, where)) != MHC_OK)
            return s;
    }
    return MHC_OK;
}

mhc_status mhc_read_kappa_gk(mhc_handle *h, double *kappa_tau, double tau_lo, double tau_hi,
                             double *kappa_w, int32_t where) {
    if (!h) return MHC_ERR_INVALID_ARG;
    if (!(h->prm.flags & MHC_FLAG_GKMA) || !h->bins_ready)
        return fail(h, MHC_ERR_INVALID_ARG, "GKMA is not enabled or no bins");
    const int L = h->prm.n_lags;
    const size_t rows = (size_t)n_out_bins(h) * 9;
    mhc_status s;
    if ((s = dev_alloc(h, "gk_out", sizeof(double) * (rows * (L + 1) + L), false)) != MHC_OK) return s;
    double *dk = dptr<double>(h, "gk_out"), *dw = dk + rows * L;
    const double coef = WMK_PER_EV_PS_A_K / (KB_EV_PER_K * h->prm.T_K * h->prm.T_K * h->prm.V_A3);
    // without a kappa(tau) output only the window average is computed (one FMA a lag)
    h->launches += launch_gk_kappa(dptr<double>(h, "Csum"), (int)n_out_bins(h), L, h->steps,
                                   coef * h->prm.dt_ps, tau_lo, tau_hi, h->prm.dt_ps,
                                   kappa_tau ? dk : nullptr, dw, dw + rows, h->stream);
    MHC_CUDA(h, cudaGetLastError());
    if (kappa_tau && (s = copy_out(h, kappa_tau, dk, sizeof(double) * rows * L, where)) != MHC_OK) return s;
    if (kappa_w && (s = copy_out(h, kappa_w, dw, sizeof(double) * rows, where)) != MHC_OK) return s;
    return MHC_OK;
}

mhc_status mhc_read_xcorr(mhc_handle *h, double *xsum, int64_t *count, int32_t where) {
    if (!h) return MHC_ERR_INVALID_ARG;
    if (!has_xcorr(h) || !h->bins_ready)
        return fail(h, MHC_ERR_INVALID_ARG, "MHC_FLAG_XCORR is not set or no bins");
    const int L = h->prm.n_lags;
    const int nb = (int)n_out_bins(h);
    const size_t n = (size_t)9 * nb * nb * L;
    mhc_status s;
    if (xsum) {
        if ((s = dev_alloc(h, "xc_out", sizeof(double) * n, false)) != MHC_OK) return s;
        launch_xcorr_transpose(dptr<float2>(h, "Xsum"), nb, L, dptr<double>(h, "xc_out"), h->stream);
        h->launches++;
        MHC_CUDA(h, cudaGetLastError());
        if ((s = copy_out(h, xsum, dptr<double>(h, "xc_out"), sizeof(double) * n, where)) != MHC_OK) return s;
    }
    if (count) {
        if ((s = dev_alloc(h, "counts", sizeof(long long) * L, false)) != MHC_OK) return s;
        launch_lag_counts(h->steps, L, dptr<long long>(h, "counts"), h->stream);
        h->launches++;
        if ((s = copy_out(h, count, dptr<long long>(h, "counts"), sizeof(long long) * L, where)) != MHC_OK)
            return s;
    }
    return MHC_OK;
}

mhc_status mhc_read_kappa_xcorr(mhc_handle *h, double *kappa_tau, double tau_lo, double tau_hi,
                                double *kappa_w, int32_t where) {
    if (!h) return MHC_ERR_INVALID_ARG;
    if (!has_xcorr(h) || !h->bins_ready)
        return fail(h, MHC_ERR_INVALID_ARG, "MHC_FLAG_XCORR is not set or no bins");
    const int L = h->prm.n_lags;
    const int nb = (int)n_out_bins(h);
    const size_t rows = (size_t)9 * nb * nb;
    mhc_status s;
    if ((s = dev_alloc(h, "xc_out", sizeof(double) * rows * L, false)) != MHC_OK) return s;
    if ((s = dev_alloc(h, "xk_out", sizeof(double) * (rows * (L + 1) + L), false)) != MHC_OK) return s;
    launch_xcorr_transpose(dptr<float2>(h, "Xsum"), nb, L, dptr<double>(h, "xc_out"), h->stream);
    double *dk = dptr<double>(h, "xk_out"), *dw = dk + rows * L;
    const double coef = WMK_PER_EV_PS_A_K / (KB_EV_PER_K * h->prm.T_K * h->prm.T_K * h->prm.V_A3);
    h->launches += 1 + launch_gk_kappa(dptr<double>(h, "xc_out"), nb * nb, L, h->steps,
                                       coef * h->prm.dt_ps, tau_lo, tau_hi, h->prm.dt_ps,
                                       kappa_tau ? dk : nullptr, dw, dw + rows, h->stream);
    MHC_CUDA(h, cudaGetLastError());
    if (kappa_tau && (s = copy_out(h, kappa_tau, dk, sizeof(double) * rows * L, where)) != MHC_OK) return s;
    if (kappa_w && (s = copy_out(h, kappa_w, dw, sizeof(double) * rows, where)) != MHC_OK) return s;
    return MHC_OK;
}

mhc_status mhc_check_orthonormality(mhc_handle *h, double tol, double *max_abs_err) {
    if (!h) return MHC_ERR_INVALID_ARG;
    if (h->ortho_err < 0) return fail(h, MHC_ERR_INVALID_ARG, "no basis check was run (ortho_probe < 0)");
    if (max_abs_err) *max_abs_err = h->ortho_err;
    return h->ortho_err > tol ? MHC_WARN_NOT_ORTHONORMAL : MHC_OK;
}

mhc_status mhc_get_info(mhc_handle *h, mhc_info *info) {
    if (!h || !info) return MHC_ERR_INVALID_ARG;
    std::memset(info, 0, sizeof *info);
    info->n_atoms = h->N;
    info->n_dof = h->D;
    info->n_modes_in = h->M_in;
    info->n_modes_kept = h->M_eff;
    info->n_bins = h->B;
    info->n_lags = h->prm.n_lags;
    info->k_max = h->prm.k_max;
    info->precision = h->prm.precision;
    info->steps_pushed = h->steps;
    info->pushes = h->pushes;
    info->n_slots = h->n_slots;
    info->tile_n = is_tc(h) ? h->tc.bn : 128;
    info->tile_pair = is_tc(h) ? h->tc.pair : 0;
    info->tile_k = is_tc(h) ? h->tc.bk : 16;
    info->stages = is_tc(h) ? h->tc.stages : 0;
    info->tile_split = !is_tc(h) ? 1 : h->tc.split == TC_SPLIT_BALANCED ? TC_SPLIT_BALANCED
                                                                        : std::max(1, h->tc.split);
    info->grid = h->sm_count;
    info->e_exp = h->e_exp;
    info->ortho_err = h->ortho_err;
    int64_t bytes = 0;
    for (auto &kv : h->buf) bytes += (int64_t)kv.second.bytes;
    info->device_bytes = bytes;
    info->kernel_launches = h->launches;
    info->graph_replays = h->graph_replays;
    return MHC_OK;
}

mhc_status mhc_set_flags(mhc_handle *h, int32_t flags) {
    if (!h) return MHC_ERR_INVALID_ARG;
    const int32_t mutable_bits = MHC_FLAG_NO_GRAPH | MHC_FLAG_PROFILE | MHC_FLAG_TEST_STALL;
    if ((flags & ~mutable_bits) != (h->prm.flags & ~mutable_bits))
        return fail(h, MHC_ERR_INVALID_ARG, "only the NO_GRAPH, PROFILE and TEST_STALL flags can change");
    h->prm.flags = flags;
    return MHC_OK;
}

mhc_status mhc_kernel_time(mhc_handle *h, double *ms, int64_t *launches) {
    if (!h) return MHC_ERR_INVALID_ARG;
    if (!(h->prm.flags & MHC_FLAG_PROFILE)) return fail(h, MHC_ERR_INVALID_ARG, "MHC_FLAG_PROFILE is not set");
    MHC_CUDA(h, cudaStreamSynchronize(h->stream));
    double total = 0.0;
    for (size_t q = 0; q < h->prof_used; ++q) {
        float t = 0.f;
        MHC_CUDA(h, cudaEventElapsedTime(&t, h->prof_events[q].first, h->prof_events[q].second));
        total += t;
    }
    if (ms) *ms = total;
    if (launches) *launches = (int64_t)h->prof_used;
    h->prof_used = 0;
    return MHC_OK;
}

mhc_status mhc_reset(mhc_handle *h) {
    if (!h) return MHC_ERR_INVALID_ARG;
    if (!h->bins_ready) return fail(h, MHC_ERR_INVALID_ARG, "no bins");
    MHC_CUDA(h, cudaSetDevice(h->prm.device));
    mhc_status s = reset_accumulators(h);
    if (s == MHC_OK) MHC_CUDA(h, cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
    if (s == MHC_OK) MHC_CUDA(h, cudaStreamSynchronize(h->stream));
    return s;
}

// Blob: header {magic, rows, L, k_max, R_ring, kind, steps, M_eff} then hsum[rows*3], Jsum[3],
// Csum[rows*9*L], Jring[R*3]; rows = B (3 B with the direction split), kind = GKMA bit 0,
// direction split bit 1.
struct StateHeader {
    uint32_t magic;
    int32_t B, L, k_max, R_ring, kind;
    int64_t steps, M_eff;
};

mhc_status mhc_state_size(mhc_handle *h, size_t *bytes) {
    if (!h || !bytes) return MHC_ERR_INVALID_ARG;
    if (!h->bins_ready) return fail(h, MHC_ERR_INVALID_ARG, "no bins");
    const bool g = h->prm.flags & MHC_FLAG_GKMA;
    const size_t nb = (size_t)n_out_bins(h);
    *bytes = sizeof(StateHeader) + sizeof(double) * (nb * 3 + 3) +
             (g ? sizeof(double) * (nb * 9 * h->prm.n_lags + (size_t)h->R_ring * 3) : 0) +
             (has_xcorr(h) ? sizeof(double) * 9 * nb * nb * h->prm.n_lags +
                                 sizeof(float) * (size_t)h->R_ring * 3 * nb
                           : 0);
    return MHC_OK;
}

mhc_status mhc_get_state(mhc_handle *h, void *blob, size_t bytes) {
    size_t need = 0;
    mhc_status s = mhc_state_size(h, &need);
    if (s != MHC_OK) return s;
    if (!blob || bytes < need) return fail(h, MHC_ERR_INVALID_ARG, "state buffer too small (%zu < %zu)", bytes, need);
    if ((s = mhc_sync(h)) != MHC_OK) return s;
    auto *hd = static_cast<StateHeader *>(blob);
    const bool g = h->prm.flags & MHC_FLAG_GKMA;
    const size_t nb = (size_t)n_out_bins(h);
    *hd = StateHeader{STATE_MAGIC, (int32_t)nb, h->prm.n_lags, h->prm.k_max, h->R_ring,
                      (g ? 1 : 0) | (h->dir ? 2 : 0) | (has_xcorr(h) ? 4 : 0), h->steps, h->M_eff};
    char *p = static_cast<char *>(blob) + sizeof(StateHeader);
    MHC_CUDA(h, cudaMemcpy(p, dptr<double>(h, "hsum"), sizeof(double) * nb * 3, cudaMemcpyDeviceToHost));
    p += sizeof(double) * nb * 3;
    MHC_CUDA(h, cudaMemcpy(p, dptr<double>(h, "Jsum"), sizeof(double) * 3, cudaMemcpyDeviceToHost));
    p += sizeof(double) * 3;
    if (g) {
        const size_t nc = nb * 9 * h->prm.n_lags;
        MHC_CUDA(h, cudaMemcpy(p, dptr<double>(h, "Csum"), sizeof(double) * nc, cudaMemcpyDeviceToHost));
        p += sizeof(double) * nc;
        MHC_CUDA(h, cudaMemcpy(p, dptr<double>(h, "Jring"), sizeof(double) * h->R_ring * 3, cudaMemcpyDeviceToHost));
        p += sizeof(double) * h->R_ring * 3;
    }
    if (has_xcorr(h)) {
        const size_t nx = 9 * nb * nb * h->prm.n_lags, nr = (size_t)h->R_ring * 3 * nb;
        MHC_CUDA(h, cudaMemcpy(p, dptr<double>(h, "Xsum"), sizeof(double) * nx, cudaMemcpyDeviceToHost));
        p += sizeof(double) * nx;
        MHC_CUDA(h, cudaMemcpy(p, dptr<float>(h, "Jbring"), sizeof(float) * nr, cudaMemcpyDeviceToHost));
    }
    return MHC_OK;
}

mhc_status mhc_set_state(mhc_handle *h, const void *blob, size_t bytes) {
    size_t need = 0;
    mhc_status s = mhc_state_size(h, &need);
    if (s != MHC_OK) return s;
    if (!blob || bytes < need) return fail(h, MHC_ERR_STATE, "state blob too small");
    const auto *hd = static_cast<const StateHeader *>(blob);
    const bool g = h->prm.flags & MHC_FLAG_GKMA;
    const size_t nb = (size_t)n_out_bins(h);
    if (hd->magic != STATE_MAGIC || hd->B != (int32_t)nb || hd->L != h->prm.n_lags ||
        hd->k_max != h->prm.k_max || hd->R_ring != h->R_ring ||
        hd->kind != ((g ? 1 : 0) | (h->dir ? 2 : 0) | (has_xcorr(h) ? 4 : 0)) || hd->M_eff != h->M_eff ||
        hd->steps < 0)
        return fail(h, MHC_ERR_STATE, "state blob does not match this handle's modes/bins/lags/k_max");
    MHC_CUDA(h, cudaStreamSynchronize(h->stream));
    const char *p = static_cast<const char *>(blob) + sizeof(StateHeader);
    MHC_CUDA(h, cudaMemcpy(dptr<double>(h, "hsum"), p, sizeof(double) * nb * 3, cudaMemcpyHostToDevice));
    p += sizeof(double) * nb * 3;
    MHC_CUDA(h, cudaMemcpy(dptr<double>(h, "Jsum"), p, sizeof(double) * 3, cudaMemcpyHostToDevice));
    p += sizeof(double) * 3;
    if (g) {
        const size_t nc = nb * 9 * h->prm.n_lags;
        MHC_CUDA(h, cudaMemcpy(dptr<double>(h, "Csum"), p, sizeof(double) * nc, cudaMemcpyHostToDevice));
        p += sizeof(double) * nc;
        MHC_CUDA(h, cudaMemcpy(dptr<double>(h, "Jring"), p, sizeof(double) * h->R_ring * 3, cudaMemcpyHostToDevice));
        p += sizeof(double) * h->R_ring * 3;
    }
    if (has_xcorr(h)) {
        const size_t nx = 9 * nb * nb * h->prm.n_lags, nr = (size_t)h->R_ring * 3 * nb;
        MHC_CUDA(h, cudaMemcpy(dptr<double>(h, "Xsum"), p, sizeof(double) * nx, cudaMemcpyHostToDevice));
        p += sizeof(double) * nx;
        MHC_CUDA(h, cudaMemcpy(dptr<float>(h, "Jbring"), p, sizeof(float) * nr, cudaMemcpyHostToDevice));
    }
    h->steps = hd->steps;
    h->K_last = 0;
    const long long st = hd->steps;
    MHC_CUDA(h, cudaMemcpy(dptr<long long>(h, "steps_dev"), &st, sizeof st, cudaMemcpyHostToDevice));
    return MHC_OK;
}

}  // extern "C"

// ----------------------------------------------------------------------------- groups
namespace {

mhc_status group_encode(mhc_group *g) {
    mhc_handle *h0 = g->hs[0];
    const TcConfig &c = g->tc;
    for (size_t j = 0; j < g->hs.size(); ++j) {
        mhc_handle *h = g->hs[j];
        TcProblem &P = g->tcp.prob[j];
        P = h->tcp.prob[0];
        P.n_split = 1;   // grouped launches run every system unsplit
        P.sk_parts = 0;
        P.split_ws = nullptr;
        if (encode_maps(h, c, P))
            return fail(h0, MHC_ERR_CUDA, "cuTensorMapEncodeTiled failed (group member %zu)", j);
        P.n_kb = (int)(h->D_ld / c.bk);
    }
    g->tcp.status = h0->status;
    g->tcp.wait_limit = 2000000000ll;
    g->tcp.stall_inject = 0;
    g->tcp.n_prob = (int)g->hs.size();
    g->tcp.idesc = idesc_f16(h0->split == SPLIT_BF16 ? 1u : 0u, (c.pair ? 2 : 1) * TC_BM, (uint32_t)c.bn);
    return MHC_OK;
}

// Longest-processing-time assignment of every tile of every system to the persistent
// CTAs.  A tile's cost is its number of k-blocks (proportional to 3N).  Tiles of one
// system are taken in mode-tile-major order, so the column tiles that share an
// eigenvector tile land on different CTAs at about the same time (shared through L2).
mhc_status group_schedule(mhc_group *g, const std::vector<int> &Ks, GroupSchedule *&out) {
    mhc_handle *h0 = g->hs[0];
    const TcConfig &c = g->tc;
    auto key = std::make_pair(c.bn * 2 + c.pair, Ks);
    auto it = g->sched_cache.find(key);
    if (it != g->sched_cache.end()) {
        out = &it->second;
        return MHC_OK;
    }
    struct Tile { int cost; uint32_t id; };
    std::vector<Tile> tiles;
    std::vector<int> order(g->hs.size());
    for (size_t j = 0; j < order.size(); ++j) order[j] = (int)j;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return g->hs[a]->D_ld > g->hs[b]->D_ld;
    });
    for (int j : order) {
        mhc_handle *h = g->hs[j];
        const int n_mt = mode_tiles(h, c);
        const int n_ct = (4 * Ks[j] + c.bn - 1) / c.bn;
        for (int mt = 0; mt < n_mt; ++mt)
            for (int ct = 0; ct < n_ct; ++ct)
                tiles.push_back({(int)(h->D_ld / c.bk), tc_tile_id(j, mt, ct)});
    }
    const int grid = std::max(1, std::min<int>(sched_units(h0, c), (int)tiles.size()));
    std::vector<std::vector<uint32_t>> per(grid);
    using Load = std::pair<long long, int>;
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> pq;
    for (int b = 0; b < grid; ++b) pq.push({0, b});
    for (const Tile &t : tiles) {
        Load l = pq.top();
        pq.pop();
        per[l.second].push_back(t.id);
        pq.push({l.first + t.cost, l.second});
    }
    std::vector<uint32_t> flat;
    std::vector<int> begin(grid + 1, 0);
    for (int b = 0; b < grid; ++b) {
        begin[b] = (int)flat.size();
        flat.insert(flat.end(), per[b].begin(), per[b].end());
    }
    begin[grid] = (int)flat.size();
    GroupSchedule &gs = g->sched_cache[key];
    gs.grid = grid;
    cudaError_t e = cudaMalloc(&gs.sched.p, sizeof(uint32_t) * std::max<size_t>(flat.size(), 1));
    if (e == cudaSuccess) e = cudaMalloc(&gs.cta_begin.p, sizeof(int) * (grid + 1));
    if (e != cudaSuccess) {
        g->sched_cache.erase(key);
        return fail(h0, MHC_ERR_OOM, "group schedule allocation: %s", cudaGetErrorString(e));
    }
    gs.sched.bytes = sizeof(uint32_t) * flat.size();
    gs.cta_begin.bytes = sizeof(int) * (grid + 1);
    MHC_CUDA(h0, cudaMemcpyAsync(gs.sched.p, flat.data(), sizeof(uint32_t) * flat.size(),
                                 cudaMemcpyHostToDevice, h0->stream));
    MHC_CUDA(h0, cudaMemcpyAsync(gs.cta_begin.p, begin.data(), sizeof(int) * (grid + 1),
                                 cudaMemcpyHostToDevice, h0->stream));
    MHC_CUDA(h0, cudaStreamSynchronize(h0->stream));   // host vectors die on return
    out = &gs;
    return MHC_OK;
}

// The packs of all systems in one launch (clusters of a common size), or one by one when a
// system does not qualify for the bulk-copy pack.  All handles of a group share one stream.
mhc_status group_pack(mhc_group *g, const std::vector<const float *> &vs,
                      const std::vector<const float *> &ws, const std::vector<int> &Ks) {
    mhc_handle *h0 = g->hs[0];
    PackGroupArgs pg{};
    pg.n = (int)g->hs.size();
    for (int j = 0; j < pg.n; ++j) pg.a[j] = pack_args(g->hs[j], vs[j], ws[j], Ks[j]);
    if (!g->pack_fork) {
        MHC_CUDA(h0, cudaEventCreateWithFlags(&g->pack_fork, cudaEventDisableTiming));
        for (int q = 0; q < mhc_group::PACK_SIDE; ++q) {
            MHC_CUDA(h0, cudaStreamCreateWithFlags(&g->pack_side[q], cudaStreamNonBlocking));
            MHC_CUDA(h0, cudaEventCreateWithFlags(&g->pack_join[q], cudaEventDisableTiming));
        }
    }
    cudaStream_t streams[1 + mhc_group::PACK_SIDE] = {h0->stream};
    MHC_CUDA(h0, cudaEventRecord(g->pack_fork, h0->stream));
    for (int q = 0; q < mhc_group::PACK_SIDE; ++q) {
        streams[1 + q] = g->pack_side[q];
        MHC_CUDA(h0, cudaStreamWaitEvent(g->pack_side[q], g->pack_fork, 0));
    }
    int nl = 0;
    const cudaError_t e = launch_pack_group(pg, streams, 1 + mhc_group::PACK_SIDE, &nl);
    for (int q = 0; q < mhc_group::PACK_SIDE; ++q) {   // join every side stream (also on error)
        MHC_CUDA(h0, cudaEventRecord(g->pack_join[q], g->pack_side[q]));
        MHC_CUDA(h0, cudaStreamWaitEvent(h0->stream, g->pack_join[q], 0));
    }
    if (e == cudaErrorNotSupported) {
        for (int j = 0; j < pg.n; ++j) {
            const mhc_status s = pack_block(g->hs[j], vs[j], ws[j], Ks[j]);
            if (s != MHC_OK) return s;
        }
        return MHC_OK;
    }
    MHC_CUDA(h0, e);
    h0->launches += nl;
    return MHC_OK;
}

// The kernels that close a group push: one bin-finish launch for all systems, each system's
// correlation kernels, one launch for all step counters.
mhc_status group_finish(mhc_group *g, const std::vector<int> &Ks) {
    mhc_handle *h0 = g->hs[0];
    FinishGroupArgs fg{};
    fg.n = (int)g->hs.size();
    for (int j = 0; j < fg.n; ++j) {
        mhc_handle *h = g->hs[j];
        fg.partials[j] = dptr<float>(h, "partials");
        fg.n_slots[j] = (int)slot_stride(h);
        fg.slot_begin[j] = dptr<int>(h, "slot_begin");
        fg.B[j] = (int)n_out_bins(h);
        fg.K[j] = Ks[j];
        fg.Jb[j] = dptr<float>(h, "Jb");
        fg.hsum[j] = dptr<double>(h, "hsum");
        fg.Jtot[j] = dptr<double>(h, "Jtot");
        fg.Jsum[j] = dptr<double>(h, "Jsum");
        fg.steps[j] = dptr<long long>(h, "steps_dev");
    }
    // without correlation kernels (which read the step counters) the bin finish advances them
    bool corr = false;
    for (mhc_handle *h : g->hs) corr = corr || (h->prm.flags & MHC_FLAG_GKMA) || has_xcorr(h);
    fg.advance = corr ? 0 : 1;
    launch_bin_finish_group(fg, h0->stream);
    h0->launches++;
    MHC_CUDA(h0, cudaGetLastError());
    if (!corr) return MHC_OK;
    for (int j = 0; j < fg.n; ++j) {
        const mhc_status s = correlate_block(g->hs[j], Ks[j]);
        if (s != MHC_OK) return s;
    }
    launch_advance_steps_group(fg, h0->stream);
    h0->launches++;
    MHC_CUDA(h0, cudaGetLastError());
    return MHC_OK;
}

mhc_status group_launch(mhc_group *g, const std::vector<int> &Ks) {
    mhc_handle *h0 = g->hs[0];
    GroupSchedule *gs = nullptr;
    mhc_status s = group_schedule(g, Ks, gs);
    if (s != MHC_OK) return s;
    for (size_t j = 0; j < g->hs.size(); ++j) {
        TcProblem &P = g->tcp.prob[j];
        P.K = Ks[j];
        P.n_col_tiles = (4 * Ks[j] + g->tc.bn - 1) / g->tc.bn;
        P.n_tiles = mode_tiles(g->hs[j], g->tc) * P.n_col_tiles;
    }
    g->tcp.sched = static_cast<const uint32_t *>(gs->sched.p);
    g->tcp.cta_begin = static_cast<const int *>(gs->cta_begin.p);
    TcConfig c = g->tc;
    c.grid = gs->grid * (c.pair ? 2 : 1);
    cudaError_t e = launch_tc_group(g->tcp, c, h0->stream);
    h0->launches++;
    if (e != cudaSuccess)
        return fail(h0, MHC_ERR_CUDA, "grouped tensor-core launch failed: %s", cudaGetErrorString(e));
    return MHC_OK;
}

mhc_status group_autotune(mhc_group *g, const std::vector<int> &Ks) {
    // interleaved rounds over the shapes, each shape's fastest launch (as time_candidates)
    mhc_handle *h0 = g->hs[0];
    cudaEvent_t e0, e1;
    MHC_CUDA(h0, cudaEventCreate(&e0));
    MHC_CUDA(h0, cudaEventCreate(&e1));
    float best_ms[TC_NUM_CONFIGS];
    mhc_status s = MHC_OK;
    for (int q = 0; q < TC_NUM_CONFIGS && s == MHC_OK; ++q) {   // warm-up (and schedules)
        best_ms[q] = 1e30f;
        g->tc = TC_CONFIGS[q];
        if ((s = group_encode(g)) == MHC_OK) s = group_launch(g, Ks);
    }
    for (int r = 0; r < 3 && s == MHC_OK; ++r)
        for (int q = 0; q < TC_NUM_CONFIGS && s == MHC_OK; ++q) {
            g->tc = TC_CONFIGS[q];
            if ((s = group_encode(g)) != MHC_OK) break;
            float ms = 0.f;
            if (cudaEventRecord(e0, h0->stream) != cudaSuccess) { s = fail(h0, MHC_ERR_CUDA, "event record"); break; }
            if ((s = group_launch(g, Ks)) != MHC_OK || (s = group_launch(g, Ks)) != MHC_OK) break;
            if (cudaEventRecord(e1, h0->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                s = fail(h0, MHC_ERR_CUDA, "group autotune timing failed");
                break;
            }
            best_ms[q] = std::min(best_ms[q], ms);   // two launches back to back, as in a run
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != MHC_OK) return s;
    int best = 0;
    for (int q = 1; q < TC_NUM_CONFIGS; ++q)
        if (best_ms[q] < best_ms[best]) best = q;
    g->tc = TC_CONFIGS[best];
    g->tuned[Ks] = g->tc;
    return group_encode(g);
}

// The tile shape for block lengths Ks: fixed (tile_config), cached, or autotuned now (on the
// blocks just packed).  Re-encodes the tensor maps when the shape changes.
mhc_status group_select(mhc_group *g, const std::vector<int> &Ks) {
    if (g->hs[0]->prm.tile_config != 0) return MHC_OK;
    auto it = g->tuned.find(Ks);
    if (it == g->tuned.end()) return group_autotune(g, Ks);
    const TcConfig &c = it->second;
    if (c.bn == g->tc.bn && c.bk == g->tc.bk && c.stages == g->tc.stages && c.pair == g->tc.pair)
        return MHC_OK;
    g->tc = c;
    return group_encode(g);
}

}  // namespace

namespace {
mhc_status group_push_staged(mhc_group *g, const std::vector<const float *> &vs,
                             const std::vector<const float *> &ws, const std::vector<int> &Ks);
}  // namespace

extern "C" {

mhc_status mhc_group_create(mhc_group **out, mhc_handle *const *handles, int32_t n) {
    if (!out || !handles || n < 1) return MHC_ERR_INVALID_ARG;
    *out = nullptr;
    mhc_handle *h0 = handles[0];
    if (!h0) return MHC_ERR_INVALID_ARG;
    if (n > TC_MAX_GROUP) return fail(h0, MHC_ERR_INVALID_ARG, "at most %d systems per group", TC_MAX_GROUP);
    for (int j = 0; j < n; ++j) {
        mhc_handle *h = handles[j];
        if (!h) return fail(h0, MHC_ERR_INVALID_ARG, "handle %d is null", j);
        if (!h->bins_ready) return fail(h0, MHC_ERR_INVALID_ARG, "handle %d has no modes/bins", j);
        if (!is_tc(h)) return fail(h0, MHC_ERR_UNSUPPORTED, "grouped launches need a tensor-core precision");
        if (h->dir) return fail(h0, MHC_ERR_UNSUPPORTED, "grouped launches do not take the direction split");
        if (h->prm.device != h0->prm.device || h->stream != h0->stream || h->split != h0->split)
            return fail(h0, MHC_ERR_INVALID_ARG, "handle %d differs in device, stream or precision", j);
        for (int q = 0; q < j; ++q)
            if (handles[q] == h) return fail(h0, MHC_ERR_INVALID_ARG, "handle %d appears twice", j);
    }
    auto *g = new mhc_group();
    g->hs.assign(handles, handles + n);
    g->tc = h0->tc;
    g->tc.split = 1;   // grouped launches run unsplit
    mhc_status s = group_encode(g);
    if (s != MHC_OK) {
        delete g;
        return s;
    }
    *out = g;
    return MHC_OK;
}

void mhc_group_destroy(mhc_group *g) {
    if (!g) return;
    cudaStreamSynchronize(g->hs[0]->stream);
    for (auto &kv : g->graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    for (int q = 0; q < mhc_group::PACK_SIDE; ++q) {
        if (g->pack_side[q]) cudaStreamDestroy(g->pack_side[q]);
        if (g->pack_join[q]) cudaEventDestroy(g->pack_join[q]);
    }
    if (g->pack_fork) cudaEventDestroy(g->pack_fork);
    for (auto &kv : g->sched_cache) {
        if (kv.second.sched.p) cudaFree(kv.second.sched.p);
        if (kv.second.cta_begin.p) cudaFree(kv.second.cta_begin.p);
    }
    delete g;
}

mhc_status mhc_group_read_hnema(mhc_group *g, double *kappa, double *mean_J, int32_t where) {
    if (!g) return MHC_ERR_INVALID_ARG;
    mhc_handle *h0 = g->hs[0];
    if (where != MHC_MEM_HOST && where != MHC_MEM_DEVICE) return fail(h0, MHC_ERR_INVALID_ARG, "where");
    MHC_CUDA(h0, cudaSetDevice(h0->prm.device));
    HnemaGroupArgs a{};
    a.n = (int)g->hs.size();
    int total = 0;
    for (int j = 0; j < a.n; ++j) {
        mhc_handle *h = g->hs[j];
        const double fe = std::sqrt(h->prm.F_e[0] * h->prm.F_e[0] + h->prm.F_e[1] * h->prm.F_e[1] +
                                    h->prm.F_e[2] * h->prm.F_e[2]);
        a.hsum[j] = dptr<double>(h, "hsum");
        a.T_s[j] = h->steps;
        a.coef[j] = fe > 0 ? WMK_PER_EV_PS_A_K / (h->prm.T_K * h->prm.V_A3 * fe) : 0.0;
        a.nb[j] = h->B * 3;
        a.off[j] = total;
        total += h->B * 3;
    }
    double *dk = kappa, *dm = mean_J;
    if (where == MHC_MEM_HOST) {   // one staging buffer, one copy, one synchronisation
        mhc_status s;
        if ((s = dev_alloc(h0, "group_hn", sizeof(double) * 2 * total, false)) != MHC_OK) return s;
        dm = mean_J ? dptr<double>(h0, "group_hn") : nullptr;
        dk = kappa ? dptr<double>(h0, "group_hn") + total : nullptr;
    }
    launch_hnema_finalize_group(a, dm, dk, h0->stream);
    h0->launches++;
    MHC_CUDA(h0, cudaGetLastError());
    if (where == MHC_MEM_HOST) {
        if (kappa) MHC_CUDA(h0, cudaMemcpyAsync(kappa, dk, sizeof(double) * total, cudaMemcpyDeviceToHost, h0->stream));
        if (mean_J) MHC_CUDA(h0, cudaMemcpyAsync(mean_J, dm, sizeof(double) * total, cudaMemcpyDeviceToHost, h0->stream));
        MHC_CUDA(h0, cudaStreamSynchronize(h0->stream));
        return check_device_status(h0);
    }
    return MHC_OK;
}

mhc_status mhc_group_autotune_k(mhc_group *g, const int32_t *candidates, int32_t n, int32_t *best_K,
                                double *units_per_s) {
    if (!g) return MHC_ERR_INVALID_ARG;
    mhc_handle *h0 = g->hs[0];
    if (!candidates || n < 1 || !best_K) return fail(h0, MHC_ERR_INVALID_ARG, "need candidates and best_K");
    const size_t m = g->hs.size();
    for (int32_t q = 0; q < n; ++q)
        for (size_t j = 0; j < m; ++j)
            if (candidates[q] < 1 || candidates[q] > g->hs[j]->prm.k_max)
                return fail(h0, MHC_ERR_INVALID_ARG, "candidate K=%d outside [1, k_max] of system %zu",
                            candidates[q], j);
    MHC_CUDA(h0, cudaSetDevice(h0->prm.device));
    // constant, finite samples of the largest K in every member's first staging pair, after
    // whatever may still read those pairs
    std::vector<const float *> vs(m), ws(m);
    for (size_t j = 0; j < m; ++j) {
        mhc_handle *h = g->hs[j];
        MHC_CUDA(h0, cudaStreamSynchronize(h->stream));
        if (h->copy_stream) MHC_CUDA(h0, cudaStreamSynchronize(h->copy_stream));
        float *v = dptr<float>(h, "v_stage"), *W = dptr<float>(h, "W_stage");
        MHC_CUDA(h0, cudaMemsetAsync(v, 0x3f, sizeof(float) * h->prm.k_max * h->N * 3, h0->stream));
        MHC_CUDA(h0, cudaMemsetAsync(W, 0x3f, sizeof(float) * h->prm.k_max * h->N * 9, h0->stream));
        vs[j] = v;
        ws[j] = W;
    }
    double units_per_step = 0.0;   // mode * atom per step summed over the members
    for (size_t j = 0; j < m; ++j) units_per_step += (double)g->hs[j]->M_eff * (double)g->hs[j]->N;
    cudaEvent_t e0, e1;
    MHC_CUDA(h0, cudaEventCreate(&e0));
    MHC_CUDA(h0, cudaEventCreate(&e1));
    mhc_status s = MHC_OK;
    double best = -1.0;
    int32_t bestK = candidates[0];
    for (int32_t q = 0; q < n && s == MHC_OK; ++q) {
        const std::vector<int> Ks(m, candidates[q]);
        if ((s = group_pack(g, vs, ws, Ks)) != MHC_OK) break;
        if ((s = group_select(g, Ks)) != MHC_OK) break;   // each K with its own tile shape
        const int reps = 3;
        cudaError_t e = cudaEventRecord(e0, h0->stream);
        for (int r = 0; r < reps && s == MHC_OK; ++r)
            if ((s = group_pack(g, vs, ws, Ks)) == MHC_OK) s = group_launch(g, Ks);
        if (s != MHC_OK) break;
        if (e == cudaSuccess) e = cudaEventRecord(e1, h0->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            s = fail(h0, MHC_ERR_CUDA, "timing of K=%d failed: %s", candidates[q], cudaGetErrorString(e));
            break;
        }
        const double rate = ms > 0 ? reps * units_per_step * candidates[q] / (ms * 1e-3) : 0.0;
        if (rate > best) {
            best = rate;
            bestK = candidates[q];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != MHC_OK) return s;
    for (size_t j = 0; j < m; ++j) g->hs[j]->K_last = 0;   // operands overwritten
    if ((s = group_select(g, std::vector<int>(m, bestK))) != MHC_OK) return s;
    *best_K = bestK;
    if (units_per_s) *units_per_s = best;
    return MHC_OK;
}

mhc_status mhc_group_push(mhc_group *g, const float *const *v, const float *const *W,
                          const int32_t *K, int32_t where) {
    if (!g || !v || !W || !K) return MHC_ERR_INVALID_ARG;
    mhc_handle *h0 = g->hs[0];
    if (where != MHC_MEM_HOST && where != MHC_MEM_DEVICE && where != MHC_MEM_HOST_ASYNC)
        return fail(h0, MHC_ERR_INVALID_ARG, "where");
    const size_t n = g->hs.size();
    std::vector<int> Ks(n);
    for (size_t j = 0; j < n; ++j) {
        if (!v[j] || !W[j]) return fail(h0, MHC_ERR_INVALID_ARG, "inputs of system %zu are null", j);
        if (K[j] < 1 || K[j] > g->hs[j]->prm.k_max)
            return fail(h0, MHC_ERR_INVALID_ARG, "K[%zu]=%d outside [1, %d]", j, K[j], g->hs[j]->prm.k_max);
        if (!g->hs[j]->bins_ready) return fail(h0, MHC_ERR_INVALID_ARG, "system %zu lost its bins", j);
        Ks[j] = K[j];
    }
    MHC_CUDA(h0, cudaSetDevice(h0->prm.device));
    mhc_status s = MHC_OK;
    std::vector<const float *> vs(v, v + n), ws(W, W + n);
    // all systems' uploads first, ordered before the group's kernels on the device; the host
    // waits for them after the push is queued
    std::vector<int> staged(n, -1);
    for (size_t j = 0; j < n && s == MHC_OK; ++j) {
        s = stage_issue(g->hs[j], vs[j], ws[j], Ks[j], where);
        if (s == MHC_OK) {
            staged[j] = g->hs[j]->stage_used;
            s = stage_order(g->hs[j], h0->stream);
        }
    }
    if (s == MHC_OK) s = group_push_staged(g, vs, ws, Ks);
    for (size_t j = 0; j < n; ++j) {   // earlier asynchronous uploads, queued before these
        const int pending = g->hs[j]->async_stage;
        g->hs[j]->async_stage = -1;
        s = stage_wait_on(g->hs[j], pending, s);
    }
    const bool keep = where == MHC_MEM_HOST_ASYNC && s == MHC_OK;
    for (size_t j = 0; j < n; ++j) {
        if (keep) g->hs[j]->async_stage = staged[j];
        else s = stage_wait_on(g->hs[j], staged[j], s);
    }
    return s;
}

}  // extern "C"

namespace {

mhc_status group_push_staged(mhc_group *g, const std::vector<const float *> &vs,
                             const std::vector<const float *> &ws, const std::vector<int> &Ks) {
    mhc_handle *h0 = g->hs[0];
    const size_t n = g->hs.size();
    mhc_status s;
    const bool tuned = h0->prm.tile_config != 0 || g->tuned.count(Ks);
    if (tuned && (s = group_select(g, Ks)) != MHC_OK) return s;
    const bool profile = (h0->prm.flags & MHC_FLAG_PROFILE) != 0;
    if (tuned && !(h0->prm.flags & (MHC_FLAG_NO_GRAPH | MHC_FLAG_PROFILE | MHC_FLAG_TEST_STALL))) {
        // replay (or capture once) the whole group push as one CUDA graph
        std::vector<const void *> ptrs;
        for (size_t j = 0; j < n; ++j) {
            ptrs.push_back(vs[j]);
            ptrs.push_back(ws[j]);
        }
        int cfg = -1;
        for (int q = 0; q < TC_NUM_CONFIGS; ++q)
            if (TC_CONFIGS[q].bn == g->tc.bn && TC_CONFIGS[q].bk == g->tc.bk &&
                TC_CONFIGS[q].stages == g->tc.stages && TC_CONFIGS[q].pair == g->tc.pair)
                cfg = q;
        auto key = std::make_tuple(Ks, ptrs, cfg);
        auto it = g->graphs.find(key);
        if (it == g->graphs.end()) {
            if (g->graphs.size() >= 16) {
                auto lru = g->graphs.begin();
                for (auto q = g->graphs.begin(); q != g->graphs.end(); ++q)
                    if (q->second.last_use < lru->second.last_use) lru = q;
                cudaGraphExecDestroy(lru->second.exec);
                g->graphs.erase(lru);
            }
            GroupSchedule *gs = nullptr;   // build (and upload) the schedule outside the capture
            if ((s = group_schedule(g, Ks, gs)) != MHC_OK) return s;
            if (!g->cap_stream) MHC_CUDA(h0, cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking));
            std::vector<int64_t> l0(n);
            for (size_t j = 0; j < n; ++j) l0[j] = g->hs[j]->launches;
            cudaStream_t user = h0->stream;
            // graph: grouped pack -> grouped projection -> grouped bin finish -> correlations
            //        -> step counters
            MHC_CUDA(h0, cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal));
            for (size_t j = 0; j < n; ++j) g->hs[j]->stream = g->cap_stream;
            s = group_pack(g, vs, ws, Ks);
            if (s == MHC_OK) s = group_launch(g, Ks);
            if (s == MHC_OK) s = group_finish(g, Ks);
            for (size_t j = 0; j < n; ++j) g->hs[j]->stream = user;
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamEndCapture(g->cap_stream, &graph);
            if (s != MHC_OK) {
                if (graph) cudaGraphDestroy(graph);
                return s;
            }
            if (e != cudaSuccess) return fail(h0, MHC_ERR_CUDA, "capture of a group push failed: %s", cudaGetErrorString(e));
            mhc_group::GraphEntry ge;
            e = cudaGraphInstantiate(&ge.exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return fail(h0, MHC_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
            for (size_t j = 0; j < n; ++j) {
                ge.nodes += g->hs[j]->launches - l0[j];
                g->hs[j]->launches = l0[j];
            }
            it = g->graphs.emplace(key, ge).first;
        }
        it->second.last_use = ++g->graph_clock;
        MHC_CUDA(h0, cudaGraphLaunch(it->second.exec, h0->stream));
        h0->launches += it->second.nodes;
        h0->graph_replays++;
        for (size_t j = 0; j < n; ++j) {
            count_push(g->hs[j], Ks[j]);
            if ((s = release_stage(g->hs[j])) != MHC_OK) return s;
        }
        return MHC_OK;
    }
    if ((s = group_pack(g, vs, ws, Ks)) != MHC_OK) return s;
    if ((s = group_select(g, Ks)) != MHC_OK) return s;
    cudaEvent_t ev1 = nullptr;
    if (profile) {   // time the grouped launch with the first handle's event pairs
        if (h0->prof_used == h0->prof_events.size()) {
            cudaEvent_t a0, a1;
            MHC_CUDA(h0, cudaEventCreate(&a0));
            MHC_CUDA(h0, cudaEventCreate(&a1));
            h0->prof_events.emplace_back(a0, a1);
        }
        MHC_CUDA(h0, cudaEventRecord(h0->prof_events[h0->prof_used].first, h0->stream));
        ev1 = h0->prof_events[h0->prof_used].second;
        ++h0->prof_used;
    }
    if ((s = group_launch(g, Ks)) != MHC_OK) return s;
    if (ev1) MHC_CUDA(h0, cudaEventRecord(ev1, h0->stream));
    if ((s = group_finish(g, Ks)) != MHC_OK) return s;
    for (size_t j = 0; j < n; ++j) {
        count_push(g->hs[j], Ks[j]);
        if ((s = release_stage(g->hs[j])) != MHC_OK) return s;
    }
    return MHC_OK;
}

}  // namespace
