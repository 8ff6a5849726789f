// Internal launch interface between the C-ABI layer (mhc_api.cu) and the kernels.
// Not part of the public ABI.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mhc {

enum Split { SPLIT_FP32 = 0, SPLIT_BF16 = 1, SPLIT_FP16 = 2 };

constexpr int TC_MAX_GROUP = 16;  // systems per grouped launch
constexpr int TC_MAX_SPLIT = 16;  // d-axis splits of one projection
constexpr double A2_PS2_PER_EV_AMU = 9648.533212331;   // 1 eV/amu in A^2/ps^2

// Sticky device status codes (same values as mhc_status).
constexpr int DEV_OK = 0, DEV_TIMEOUT = 4, DEV_STATE = 5;

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator, A and B of
// the same 16-bit type (ab_fmt 0 = f16, 1 = bf16), both K-major, M x N tile.
__host__ __device__ constexpr uint32_t idesc_f16(uint32_t ab_fmt, uint32_t M, uint32_t N) {
    return (1u << 4) | (ab_fmt << 7) | (ab_fmt << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

// ---------------------------------------------------------------- K1 pack
// One CTA per step k of the block.  Builds the four B-operand rows of step k,
//   Bt[4k][d]       = sqrt(m_i) v_i^b            (Eq. 13 weights)
//   Bt[4k+1+a][d]   = W_i^{ab} / sqrt(m_i)       (Eq. 16 bracket weights)
// (d = 3i+b), split into hi/lo 16-bit parts after a per-row power-of-two scale
// 2^s (FP16), and the FP64 total current J(t0+k) of Eq. 10.
// With npad > 0 the d axis is stored direction-major: column b*npad + i holds dof 3i+b
// (columns npad*b + [N, npad) stay zero), the layout of the direction-resolved split.
struct PackArgs {
    const float *v;        // [K][N][3]
    const float *W;        // [K][N][9]
    const float *sqm;      // [N] sqrt(m_i)
    const float *isqm;     // [N] 1/sqrt(m_i)
    int N, K, D_ld, split, e_exp;
    long long t0;          // global index of the block's first step (if t0_dev is null)
    const long long *t0_dev;   // device step counter read at run time (graph replay)
    void *Bt_hi, *Bt_lo;   // [rows][D_ld] 16-bit (split != FP32)
    float *Bt32;           // [rows][D_ld] (split == FP32)
    float *col_scale;      // [4K] 2^-(s_row + e_exp): undoes both power-of-two scales
    double *Jtot;          // [K][3]
    double *Jring;         // [R][3] ring of past J (GKMA) or null
    int R;
    int npad;              // 0: column 3i+b; > 0: column b*npad + i
    int *status;           // sticky status for a bounded wait that runs out (may be null)
    long long wait_limit;  // SM cycles (0: a default of about a second)
};
// Systems with N % 4 == 0 (up to 16384 atoms) and 16-byte aligned inputs are packed by a
// cluster of CTAs per step that bulk-copies its atoms into shared memory (the inputs are read
// once); other shapes by one CTA per step that reads them twice.
cudaError_t launch_pack(const PackArgs &a, cudaStream_t s);
// The packs of up to TC_MAX_GROUP systems in one launch per cluster size (systems needing the
// same number of CTAs a step go together; cta_begin is filled by the launcher).
// cudaErrorNotSupported when a system does not qualify for the bulk-copy pack (the caller then
// packs the systems one by one).
struct PackGroupArgs {
    PackArgs a[TC_MAX_GROUP];
    int cta_begin[TC_MAX_GROUP + 1];
    int n;
};
// The launches go round-robin to streams[0 .. n_streams) (the systems of different launches are
// independent); the caller orders the other streams after streams[0] before the call and
// streams[0] after them afterwards.
cudaError_t launch_pack_group(const PackGroupArgs &g, const cudaStream_t *streams, int n_streams,
                              int *n_launches);

// ---------------------------------------------------------------- E preparation
// max |E| over the valid D x M region (bit pattern of a non-negative float)
void launch_max_abs(const void *E, int dtype, int layout, int64_t ld, int64_t D, int64_t M,
                    unsigned *out_bits, cudaStream_t s);
// Gather the kept modes in bin order (perm), transpose to mode-major and split:
//   Et[n'][c] = E[d(c), perm[n']] * 2^e_exp   (zero for n' >= M_eff or d(c) >= D)
// with d(c) = c (npad == 0) or, direction-major, d(b*npad + i) = 3i+b for i < D/3.
void launch_prepare_modes(const void *E, int dtype, int layout, int64_t ld, int64_t D,
                          int64_t M_eff, const int *perm, int e_exp, int split, void *Et_hi,
                          void *Et_lo, float *Et32, int64_t D_ld, int64_t M_pad, int64_t npad,
                          cudaStream_t s);
// FP64 basis check: max over probe modes p and all modes m of |sum_d E[d,p]E[d,m] - delta|
void launch_orthonormality(const void *E, int dtype, int layout, int64_t ld, int64_t D,
                           int64_t M, const int *probe, int n_probe,
                           unsigned long long *out_bits, cudaStream_t s);

// ---------------------------------------------------------------- FP32 path
// R[c][n] = sum_{d < Dk} Bt32[c][d] Et32[n][d] for c < C (rows of the block), n < Mp;
// both operands have row pitch ld (Dk a multiple of 16).
// Measured FP32 FMA throughput of the device (the comparison path's peak), TFLOP/s.
cudaError_t measure_fp32_fma(cudaStream_t s, int sm_count, double *tflops);
void launch_sgemm(const float *Et32, const float *Bt32, float *R, int Dk, int ld, int Mp, int C,
                  cudaStream_t s);
// J_n^a(k) = R[4k][n] R[4k+1+a][n]; segmented bin sums into partials[k][a][slot].
void launch_fp32_bin_epilogue(const float *R, int Mp, int K, const int *mode_bin,
                              const int *mode_slot, float *partials, int n_slots, cudaStream_t s);
// Direction-resolved epilogue over the three per-direction products R_b = R + b*rstride:
// Xdot = sum_b R_b[4k][n], J_n^{ab}(k) = Xdot R_b[4k+1+a][n]; bin-run sums into
// partials[k][a][b*n_slots + slot].
void launch_fp32_dir_epilogue(const float *R, size_t rstride, int Mp, int K, const int *mode_bin,
                              const int *mode_slot, float *partials, int n_slots, cudaStream_t s);

// ---------------------------------------------------------------- tensor-core path
constexpr int TC_BM = 128;        // modes per tile = TMEM lanes

struct TcProblem {   // 128-byte aligned through CUtensorMap
    CUtensorMap tmA_hi, tmA_lo;   // Et hi/lo [M_pad][D_ld]
    CUtensorMap tmB_hi, tmB_lo;   // Bt hi/lo [rows][D_ld]
    const int *mode_bin;          // [M_pad] bin of each stored mode, -1 for padding
    const int *mode_slot;         // [M_pad] partial-sum slot of run tails, else -1
    const float *col_scale;       // [4K]
    float *partials;              // [K][3][n_slots] ([K][3][3 n_slots] with the direction split)
    int n_slots, n_kb, K, n_col_tiles, n_tiles;
    // Direction-resolved split: k-blocks per direction segment of the direction-major d axis
    // (0 when off), and the scratch where each CTA parks the bracket sums of the finished
    // segments ([grid][2][96][DIR_PARK_THREADS] floats, grid <= the SM count).
    int dir_seg_kb;
    float *dir_park;
    // Split of the d axis (n_split > 1, single problems only): unit (mode tile, column tile,
    // split s) accumulates the k-blocks [s kb_split, (s+1) kb_split) and stores its promoted
    // FP32 sums to split_ws[s][column][mode] (ws_cols columns, m_pad modes); the finish kernel
    // adds the splits in order and runs the tile epilogue.  n_split <= 1: one unit per tile.
    int n_split, kb_split, ws_cols, m_pad;
    float *split_ws;
    // Balanced split (sk_parts > 0, single problems only; n_tiles then counts tiles): the tiles
    // below sk_t0 (whole waves: a multiple of the launch's CTAs or pairs) run whole,
    // round-robin; the sk_nch promotion chunks of each remaining tile, tile-major (tile = mode
    // tile x n_col_tiles + column tile), are cut into sk_parts contiguous ranges of equal
    // length, one for each of the first sk_parts CTAs (pairs).  A tile cut by range boundaries
    // stores segment s (the s-th range that touches it, in chunk order) to split_ws[s]; the
    // finish kernel adds its segments in order.  sk_tm: modes per tile (128, or 256 for CTA
    // pairs); sk_bn: columns per tile.
    int sk_parts, sk_nch, sk_tm, sk_bn, sk_t0;
};
constexpr int DIR_PARK_THREADS = 256;                        // epilogue threads of the widest tile
constexpr int DIR_PARK_SEG_FLOATS = 96 * DIR_PARK_THREADS;   // one parked segment of a CTA
constexpr int DIR_PARK_CTA_FLOATS = 2 * DIR_PARK_SEG_FLOATS;

template <int NPROB>
struct TcParams {
    TcProblem prob[NPROB];
    const uint32_t *sched;   // packed tile list (null: round-robin over prob[0])
    const int *cta_begin;    // [grid+1] offsets into sched
    int n_prob;              // problems in use (prob[0..n_prob-1])
    long long wait_limit;    // SM cycles a barrier wait may take before the CTA gives up
    int stall_inject;        // test hook: arm the first stage barrier for 16 bytes more than its copies deliver
    int *status;
    uint32_t idesc;
    int dir_park_ctas;       // CTAs the direction-split scratch has room for
};

struct TcConfig {
    int bn;       // columns per tile (MMA N): 128 or 256
    int bk;       // K elements per stage: 64 (128-byte swizzle) or 32 (64-byte swizzle)
    int stages;   // shared-memory pipeline depth
    int pair;     // 1: two-SM tile (cta_group::2, 256 modes per CTA pair, bn columns shared)
    int grid;
    int split;    // d-axis splits of a single problem (0 or 1: none; TC_SPLIT_BALANCED: one
                  // range of equal chunk count per CTA or pair over all tiles)
};
constexpr int TC_SPLIT_BALANCED = -1;
// Pipeline shapes the autotuner chooses from (index + 1 = mhc_params.tile_config).
constexpr int TC_NUM_CONFIGS = 8;
extern const TcConfig TC_CONFIGS[TC_NUM_CONFIGS];
// Clusters of two CTAs of a two-SM configuration that can be resident at once (0 on error).
int tc_max_pairs(const TcConfig &c);
size_t tc_smem_bytes(const TcConfig &c);
bool tc_config_supported(const TcConfig &c);
// Encode a 2D 16-bit tensor map: rows x cols (cols innermost, row pitch ld elements).
int tc_make_tmap(CUtensorMap *m, const void *base, uint64_t rows, uint64_t cols, uint64_t ld,
                 uint32_t box_rows, uint32_t box_cols);
cudaError_t launch_tc_single(const TcParams<1> &p, const TcConfig &c, cudaStream_t s);
// With prob[0].n_split > 1: sum the splits' partial projections of the block (in split order)
// and run the tile epilogue (Eq. 16 product, bin-run sums into partials).
cudaError_t launch_tc_split_finish(const TcParams<1> &p, cudaStream_t s);
// d elements per promotion chunk of the tensor-core kernels (splits are whole chunks)
constexpr int TC_PROMOTE_D = 128;
cudaError_t launch_tc_group(const TcParams<TC_MAX_GROUP> &p, const TcConfig &c, cudaStream_t s);
// Pack a tile id for the scheduler.
__host__ __device__ inline uint32_t tc_tile_id(int prob, int mt, int ct) {
    return ((uint32_t)prob << 28) | ((uint32_t)ct << 20) | (uint32_t)mt;
}

// ---------------------------------------------------------------- SHC on the tensor cores
// Tile pairs (tau tile p, step tile q) of one block, 128 x 256 each; see k_shc_tc.cu.
constexpr int SHC_TC_MAX_PAIRS = 288;
constexpr int SHC_TC_TILE = 128;        // times tau per tile (ring rows)
constexpr int SHC_TC_STEP_TILE = 256;   // steps t per tile
constexpr int SHC_TC_PART = 384;        // floats per unit: the 383 diagonals of a tile
struct ShcTcParams {
    CUtensorMap tmA_hi, tmA_lo;   // virial ring [9 R][N_pad]: row (3a+b) R + slot, 16-bit hi/lo
    CUtensorMap tmB_hi, tmB_lo;   // velocities [3 Kpad][N_pad]: row b Kpad + k
    const float *scaleA;          // [9 R] 2^-s of each virial row
    const float *scaleB;          // [3 Kpad] 2^-s of each velocity row
    float *partials;              // [units][SHC_TC_PART] diagonal sums of each unit's tile
    long long t0;                 // first sample of the block
    int R, nR, Kpad, K, nc;
    int n_pairs, splits, kb_per_split, n_kb;
    long long wait_limit;
    int *status;
    uint32_t idesc;
    int p_tile[SHC_TC_MAX_PAIRS]; // tau tile index (tau0 = 128 p, p >= 0)
    int q_tile[SHC_TC_MAX_PAIRS]; // step tile index in the block (k0 = 256 q)
};
// Split/scale one block into the operands: velocities of step k to rows b Kpad + k and the
// virials to ring rows (3a+b) R + (t0+k) mod R, with one power-of-two scale per row.
// A bounded wait that runs out sets DEV_TIMEOUT in *status.
cudaError_t launch_shc_tc_pack(const float *v, const float *W, int N, int N_pad, int K, int Kpad, int R,
                               long long t0, int split, void *A_hi, void *A_lo, void *B_hi, void *B_lo,
                               float *scaleA, float *scaleB, int *status, long long wait_limit,
                               cudaStream_t s);
// One CTA per unit (pair c = 3a+b, tile pair, atom split): 9 n_pairs splits CTAs in clusters
// of two (tile pairs 2j, 2j+1 share their step tile; n_pairs must be even).
cudaError_t launch_shc_tc(const ShcTcParams &p, cudaStream_t s);
// Clusters of two that can be resident at once (0 on error).
int shc_tc_max_clusters();
size_t shc_tc_smem_bytes();
// Ksum[c][l] += sum over the units of pair c, in order, of their diagonal sums at lag l (FP64).
void launch_shc_tc_reduce(const ShcTcParams &p, double *Ksum, cudaStream_t s);

// ---------------------------------------------------------------- K3 .. K5
// Jb[k][b][a] = sum of partial slots of bin b; HNEMA sums += sum_k Jb (FP64);
// Jsum[a] += sum_k Jtot[k][a].
// steps (or null): the device step counter, advanced by K by the same launch when no later
// kernel of the push reads it.
void launch_bin_finish(const float *partials, int n_slots, const int *slot_begin, int B, int K,
                       float *Jb, double *hsum, const double *Jtot, double *Jsum, long long *steps,
                       cudaStream_t s);
// The bin finish (as launch_bin_finish) and the step counters (*steps += K) of up to
// TC_MAX_GROUP systems, one launch each; cta_begin is filled by the launcher.
struct FinishGroupArgs {
    const float *partials[TC_MAX_GROUP];
    int n_slots[TC_MAX_GROUP];
    const int *slot_begin[TC_MAX_GROUP];
    int B[TC_MAX_GROUP], K[TC_MAX_GROUP];
    float *Jb[TC_MAX_GROUP];
    double *hsum[TC_MAX_GROUP];
    const double *Jtot[TC_MAX_GROUP];
    double *Jsum[TC_MAX_GROUP];
    long long *steps[TC_MAX_GROUP];
    int cta_begin[TC_MAX_GROUP + 1];
    int n;
    int advance;   // 1: the bin finish also advances the step counters (no correlation kernels)
};
void launch_bin_finish_group(FinishGroupArgs g, cudaStream_t s);
void launch_advance_steps_group(const FinishGroupArgs &g, cudaStream_t s);
// Csum[b][mu][nu][l] += sum_k Jb[k][b][mu] J(t0+k-l)^nu over t0+k-l >= 0.
// lag_corr_prepare(k_max): opt into the shared memory of blocks up to k_max steps (call outside
// any stream capture).
cudaError_t lag_corr_prepare(int k_max);
// steps, ticket: when steps is not null, the last CTA to finish adds K to *steps (the push's
// last reader of the counter) and resets *ticket, a device counter that starts at 0.
void launch_lag_corr(const float *Jb, const double *Jring, int R, double *Csum, int K, int B,
                     int L, long long t0, const long long *t0_dev, long long *steps,
                     unsigned *ticket, cudaStream_t s);
// *steps += K (one thread; last kernel of a push)
void launch_advance_steps(long long *steps, int K, cudaStream_t s);
// kappa_tau[r][l] (r = b*9+mu*3+nu) and window averages kappa_w[r], FP64; kappa_tau null:
// the window averages alone, as one weighted sum of C(l) a row.
// inv_scratch: [L] doubles of device scratch (the reciprocal lag counts of this read).
// Returns the number of kernels launched.
int launch_gk_kappa(const double *Csum, int B, int L, long long T_s, double coef_dt,
                    double tau_lo, double tau_hi, double dt, double *kappa_tau,
                    double *kappa_w, double *inv_scratch, cudaStream_t s);
// mean[b][a] = hsum/T_s; kappa[b][a] = mean * coef
void launch_hnema_finalize(const double *hsum, int B, long long T_s, double coef, double *mean,
                           double *kappa, cudaStream_t s);
// HNEMA read-out of up to TC_MAX_GROUP systems in one launch, written one after another.
struct HnemaGroupArgs {
    const double *hsum[TC_MAX_GROUP];
    long long T_s[TC_MAX_GROUP];
    double coef[TC_MAX_GROUP];
    int nb[TC_MAX_GROUP];     // B_j * 3
    int off[TC_MAX_GROUP];    // offset of system j in the outputs
    int n;
};
void launch_hnema_finalize_group(const HnemaGroupArgs &a, double *mean, double *kappa, cudaStream_t s);
// ---------------------------------------------------------------- bin-bin cross-correlations
// ring[(t0 + k) mod R][3b+mu] = Jb[k][b][mu] (nb output rows of 3 components)
void launch_jb_ring_store(const float *Jb, int K, int nb, float *ring, int R, long long t0,
                          const long long *t0_dev, cudaStream_t s);
// Tensor-core cross-correlation (k_xcorr.cu): n = 3 nb rows; column tiles of nj <= XC_NJ_MAX
// rows j; row tiles of 128 rows i; the window copies hold 8 x rows_pad rows of U_pad steps.
constexpr int XC_NJ_MAX = 192;
struct XcPlan {
    int n, nj, n_jt, n_it, rows_pad, U_pad, cpt, grid;
};
struct XcTcParams {
    CUtensorMap tmA_hi, tmA_lo;   // window copies [8 rows_pad][U_pad] FP16 hi/lo, 128-row boxes
    CUtensorMap tmB_hi, tmB_lo;   // the same arrays, nj-row boxes
    const float *inv_scale;       // [rows_pad] 2^-s of each window row (written per block)
    float2 *X;                    // [L][n][n] float-pair sums, X[l][j][i]
    int n, L, n_kb, nj, n_jt, rows_pad, cpt;
    long long wait_limit;
    int *status;
    uint32_t idesc;
};
void xcorr_plan(int nb, int L, int k_max, int nsm, XcPlan &pl);
// Opt the tensor-core kernel into its shared memory (once; outside any stream capture).
cudaError_t xcorr_prepare();
// Encode the four tensor maps over the window copies and fill the plan's fields of p.
int xcorr_make_maps(const XcPlan &pl, const void *Whi, const void *Wlo, XcTcParams &p);
// X[l][3b'+nu][3b+mu] += sum_k Jb[k][b][mu] Jb(t0+k-l)[b'][nu] over t0+k-l >= 0, the block
// already in the ring: the window kernel (scales + eight shifted FP16 hi/lo copies of
// [t0 - L + 1, t0 + K)) then the tensor-core kernel.  Needs K + L - 1 <= min(R, U_pad).
cudaError_t launch_bin_xcorr(const XcPlan &pl, XcTcParams p, const float *ring, int R, int K,
                             long long t0, const long long *t0_dev, void *Whi, void *Wlo,
                             cudaStream_t s);
// out[b][b'][mu][nu][l] = X[l][3b'+nu][3b+mu] (float pair -> FP64)
void launch_xcorr_transpose(const float2 *X, int nb, int L, double *out, cudaStream_t s);
// count[l] = max(T_s - l, 0)
void launch_lag_counts(long long T_s, int L, long long *count, cudaStream_t s);

// Message of the last failed call without a handle (read through mhc_last_error(NULL)).
void set_handleless_error(const char *msg);

}  // namespace mhc
