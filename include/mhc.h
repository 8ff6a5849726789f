/*
 * mhc.h -- C ABI of the GB300 (sm_103a) modal heat-current library.
 *
 * The library computes, for a stream of molecular-dynamics samples, the
 * modal heat current of the velocity-decomposition methods GKMA and HNEMA
 * (Gabourie, Fan, Ala-Nissila, Pop, arXiv:2102.03691, Sec. II.B):
 *
 *   Eq. 10  J^a(t)       = sum_i sum_b W_i^{ab}(t) v_i^b(t)           total current
 *   Eq. 13  Xdot_n(t)    = sum_i sqrt(m_i) e_{i,n} . v_i(t)           modal velocity
 *   Eq. 16  J_n^a(t)     = (sum_i m_i^{-1/2} (W_i(t) e_{i,n})^a) Xdot_n(t)
 *           J_b^a(t)     = sum_{n in bin b} J_n^a(t)                  (Sec. III.A binning)
 *   Eq. 17  kappa_b^{mu nu}(tau) = (k_B T^2 V)^{-1} int_0^tau <J_b^mu(t') J^nu(0)> dt'
 *   Eq. 19  kappa_b^mu   = <J_b^mu> / (T V |F_e|)
 *
 * Conventions shared by every call:
 *   - N atoms, D = 3N degrees of freedom indexed d = 3 i + b, M modes kept.
 *   - e is real (Gamma point).  The eigenvector matrix E has E[d, n] = e^b_{i,n}.
 *   - v is [K][N][3] float32 (A/ps); W is [K][N][9] float32 (eV) with
 *     W[k][i][3 a + b] = W_i^{ab} (row-major, full non-symmetric tensor, Eq. 8).
 *   - Units: m in amu, frequencies in THz, dt in ps, T in K, V in A^3, F_e in 1/A;
 *     currents in eV*A/ps, kappa in W/(m K).
 *   - Every call returns an mhc_status; nothing throws across the ABI.  On an
 *     error the handle keeps a message readable through mhc_last_error().
 *   - All device work is issued on the stream given in mhc_params, in order.
 *     Calls that return data to the host synchronise that stream first.
 *   - Device kernels never trap: a kernel that finds a broken invariant or
 *     waits too long on a barrier writes a sticky status word and returns;
 *     the next mhc_sync / read call reports it as MHC_ERR_TIMEOUT or
 *     MHC_ERR_STATE.
 *   - A handle is not thread-safe; use one handle per host thread.
 */
#ifndef MHC_H
#define MHC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mhc_handle mhc_handle;
typedef struct mhc_group mhc_group;

typedef enum {
    MHC_OK = 0,
    MHC_ERR_INVALID_ARG = 1,   /* bad pointer, size, layout or order of calls */
    MHC_ERR_OOM = 2,           /* a device or host allocation failed */
    MHC_ERR_CUDA = 3,          /* a CUDA runtime call failed (message has the name) */
    MHC_ERR_TIMEOUT = 4,       /* a kernel gave up waiting on a barrier */
    MHC_ERR_STATE = 5,         /* corrupt state blob or device invariant broken */
    MHC_ERR_UNSUPPORTED = 6,   /* precision/feature not available on this device */
    MHC_WARN_NOT_ORTHONORMAL = 100 /* basis check above tolerance (not fatal) */
} mhc_status;

/* Arithmetic of the two projections (Eq. 13 and the bracket of Eq. 16). */
typedef enum {
    MHC_PREC_FP32 = 0,   /* CUDA-core FP32 FMA GEMM, FP32 accumulation */
    MHC_PREC_BF16X3 = 1, /* tensor cores: hi/lo bfloat16 split, 3 products, FP32 accum */
    MHC_PREC_FP16X3 = 2  /* tensor cores: hi/lo float16 split with power-of-two
                            scaling, 3 products, FP32 accumulation */
} mhc_precision;

/* MHC_MEM_HOST_ASYNC (mhc_push / mhc_group_push inputs only): host memory read after the call
 * returns; the caller keeps it unchanged until the next mhc_push / mhc_group_push of that
 * handle or mhc_sync on it returns MHC_OK. */
typedef enum { MHC_MEM_HOST = 0, MHC_MEM_DEVICE = 1, MHC_MEM_HOST_ASYNC = 2 } mhc_mem;
typedef enum { MHC_F32 = 0, MHC_F64 = 1 } mhc_dtype;
/* DOF_MAJOR: E[d * ld + n] (rows are degrees of freedom, as printed in Eq. 13).
 * MODE_MAJOR: E[n * ld + d] (each eigenvector contiguous). */
typedef enum { MHC_DOF_MAJOR = 0, MHC_MODE_MAJOR = 1 } mhc_layout;

/* Flags for mhc_params.flags */
#define MHC_FLAG_GKMA 0x1          /* accumulate Eq. 17 lag correlations (needs n_lags > 0) */
#define MHC_FLAG_NO_GRAPH 0x2      /* launch kernels directly instead of replaying a CUDA graph.
                                      By default each push after the first of a given K (the
                                      autotuning push) replays a graph captured per (K, input
                                      pointers, tile shape); host inputs are first copied to
                                      fixed staging buffers.  Up to 32 graphs are cached. */
#define MHC_FLAG_PROFILE 0x4       /* time each projection launch with CUDA events (mhc_kernel_time);
                                      implies direct launches */
#define MHC_FLAG_TEST_STALL 0x8    /* fault injection for tests of the failure path: the tensor-core
                                      kernel arms its first stage barrier to expect 16 bytes more
                                      than its copies deliver, so its bounded waits (0.1 s with this flag)
                                      give up and the next sync/read returns MHC_ERR_TIMEOUT; no
                                      memory is touched out of bounds.  Implies direct launches. */
#define MHC_FLAG_DIRECTION 0x10    /* direction-resolved split (Sec. II.A: the current along a is the
                                      sum of the contributions of the atoms' motion along each
                                      direction b; Sec. II.C applies the split to every method's
                                      spectral result).  Per mode, with the modal velocity of Eq. 14,
                                        J_n^{ab} = Xdot_n sum_i m_i^{-1/2} W_i^{ab} e^b_{i,n},
                                      sum_b J_n^{ab} = J_n^a of Eq. 16.  Every per-bin output then
                                      has 3 B rows, row b * B + bin (b = direction of the motion):
                                      binned current [K][3][B][3], HNEMA [3][B][3], GKMA sums
                                      [3][B][3][3][L], each correlated with the total J (Eq. 17).
                                      Same tensor work as without the split, on every tile
                                      configuration; each running CTA keeps the finished bracket
                                      sums of two directions in a device scratch of 192 KB (about
                                      30 MB on a 152-SM GPU, allocated with the bins).  Set at
                                      mhc_create, not with mhc_set_flags; not for groups. */
#define MHC_FLAG_XCORR 0x20        /* with MHC_FLAG_GKMA: also accumulate the cross-correlations of
                                      the binned currents, X_{b b'}^{mu nu}(l) = sum over origins of
                                      J_b^mu(t) J_{b'}^nu(t - l) (the mode-mode correlations that the
                                      modal currents of GKMA allow, at bin resolution; one bin per
                                      mode gives them per mode).  Summed over b' they equal the
                                      Eq. 17 sums when every mode is binned.  Computed on the tensor
                                      cores (FP16x3 operands, per-lag contractions over each block);
                                      state: R^2 * 9 * L sums kept as float pairs (~48 bits, 8 bytes
                                      each; R = output rows, B or 3B) plus ~7 MB of window copies;
                                      read as FP64 with mhc_read_xcorr / mhc_read_kappa_xcorr.  Set
                                      at mhc_create. */

typedef struct {
    int32_t device;      /* CUDA device ordinal */
    void *stream;        /* cudaStream_t to issue on; NULL = the legacy default stream */
    int32_t k_max;       /* largest K accepted by mhc_push (steps per block) */
    int32_t n_lags;      /* L: lags 0..L-1 of the Eq. 17 correlation (GKMA) */
    int32_t precision;   /* mhc_precision */
    int32_t flags;       /* MHC_FLAG_* */
    int32_t tile_config; /* tensor-core tile: 0 = autotune on the first push of each K (the
                            shape and, see split_d, the d-axis split; the choice is kept for
                            every handle of the process with the same device, precision, D, M
                            and K, and in the file named by the environment variable
                            MHC_TUNE_CACHE when it is set);
                            1..4 = one-SM tiles of 128 modes x (columns, k per stage, stages)
                            (256,64,2), (256,32,4), (128,64,3), (128,32,6); 5..8 = two-SM tiles
                            (CTA pair, 256 modes x columns) with (256,64,3), (256,32,6),
                            (128,64,4), (128,32,8). */
    int32_t ortho_probe; /* -1: no basis check in set_modes; 0: full E^T E; P>0: P probe modes */
    double dt_ps;        /* sampling interval between pushed steps (Eq. 17 dt') */
    double T_K;          /* temperature T (Eq. 17, 19) */
    double V_A3;         /* cell volume V (Eq. 17, 19) */
    double F_e[3];       /* HNEMD driving-force parameter F_e (Eq. 12, 19), 1/A */
    int32_t split_d;     /* d-axis splits of the tensor-core projection (the GEMM's reduction
                            over the 3N degrees of freedom cut into split_d ranges of whole
                            128-element chunks, run as separate units and added in a fixed order
                            by a finish kernel; it fills the SMs when one block has few tiles):
                            0 = autotuned with the tile shape (tile_config 0) or 1 (tile_config
                            > 0); 1..16 = fixed; -1 = balanced: the chunks of all tiles, tile
                            after tile, cut into one range of equal length per CTA (or CTA
                            pair), a tile cut by a range boundary finished by the same kernel.
                            Not with MHC_FLAG_DIRECTION (must be 0 or 1); grouped launches run
                            unsplit. */
} mhc_params;

/* Counters and derived sizes of a handle. */
typedef struct {
    int64_t n_atoms, n_dof, n_modes_in, n_modes_kept; /* N, 3N, M given, M after excluding bin -1 */
    int32_t n_bins, n_lags, k_max, precision;
    int64_t steps_pushed;        /* T_s so far */
    int64_t pushes;              /* number of mhc_push calls */
    int64_t n_slots;             /* per-step partial-sum slots of the bin reduction */
    int32_t tile_n, tile_k;      /* tensor-core tile: columns per tile, d elements per stage */
    int32_t tile_pair;           /* 1 if the tile spans a CTA pair on two SMs */
    int32_t stages, grid;        /* pipeline depth, SM count */
    int32_t e_exp;               /* power-of-two scale applied to E before the split */
    double ortho_err;            /* last basis check result, -1 if none */
    int64_t device_bytes;        /* device memory owned by the handle */
    int64_t kernel_launches;     /* kernels launched by the handle so far (graph nodes included) */
    int64_t graph_replays;       /* pushes executed by replaying a captured CUDA graph */
    int32_t tile_split;          /* d-axis splits of the current tile configuration (1: none,
                                    -1: balanced) */
} mhc_info;

/* Fill *p with defaults: device 0, default stream, k_max 256, no GKMA,
 * BF16X3, dt 0.01 ps, T 300 K, V 1 A^3, F_e = (1e-5, 0, 0), autotune, no check. */
void mhc_default_params(mhc_params *p);

/* Create a handle.  Allocates nothing large until mhc_set_modes.
 * Errors: INVALID_ARG (null, k_max < 1, n_lags < 0, GKMA without lags),
 * UNSUPPORTED (tensor-core precision on a device other than sm_103),
 * CUDA.  On error *h is NULL. */
mhc_status mhc_create(mhc_handle **h, const mhc_params *p);

/* Release every device buffer and the handle.  Synchronises the stream. NULL is ignored. */
void mhc_destroy(mhc_handle *h);

/* Message of the last error on h (empty string if none); valid until the next call on h.
 * With h == NULL, the last error of a failed mhc_create or mhc_lattice_modes on this thread. */
const char *mhc_last_error(const mhc_handle *h);
const char *mhc_status_string(mhc_status s);

/*
 * Load the eigenvectors e_{i,n} (Eq. 13, 14; Sec. II.B), mode frequencies and
 * atomic masses.
 *   n_atoms  N (D = 3N rows of E)
 *   n_modes  M columns of E (M <= 3N; a mode subset is allowed, Sec. III.C.i)
 *   E        eigenvectors, dtype MHC_F32/MHC_F64, layout MHC_DOF_MAJOR/MODE_MAJOR,
 *            leading dimension ld (>= M for DOF_MAJOR, >= D for MODE_MAJOR),
 *            host or device memory according to `where`
 *   freq_THz [M] host, may be NULL if bins are given by mhc_set_bin_ids
 *   mass_amu [N] host, every m_i > 0
 * The library copies everything; the caller may free its buffers on return.
 * Resets all accumulators.  Binning must be (re)applied afterwards with
 * mhc_set_bins_uniform or mhc_set_bin_ids.
 * Errors: INVALID_ARG, OOM, CUDA; WARN_NOT_ORTHONORMAL if ortho_probe >= 0 and
 * max |E^T E - I| > 1e-6 (the modes are still loaded).
 */
mhc_status mhc_set_modes(mhc_handle *h, int64_t n_atoms, int64_t n_modes, const void *E,
                         int32_t dtype, int32_t layout, int64_t ld, int32_t where,
                         const double *freq_THz, const double *mass_amu);

/*
 * Frequency bins of fixed width (Sec. III.A: 1 THz for CNT/graphene, 0.25 THz
 * for Si).  Bin b covers [f_min + b w, f_min + (b+1) w), w = (f_max - f_min)/B,
 * the last bin also takes f_max; modes outside [f_min, f_max] are excluded.
 * The bin index is floor((f - f_min) / w) in double precision.
 * Requires frequencies from mhc_set_modes.  Resets the accumulators.
 */
mhc_status mhc_set_bins_uniform(mhc_handle *h, double f_min, double f_max, int32_t n_bins);

/*
 * Explicit bin of every mode (host array [M], values in [0, B) or -1 to exclude),
 * e.g. mode-count bins (Sec. III.C.ii uses 27 modes per bin).  Resets the accumulators.
 */
mhc_status mhc_set_bin_ids(mhc_handle *h, const int32_t *bin_of_mode, int32_t n_bins);

/*
 * Push one block of K consecutive samples (1 <= K <= k_max):
 *   v [K][N][3] float32, W [K][N][9] float32, in host or device memory (`where`).
 * Computes J(t) (Eq. 10), the binned modal currents J_b(t) (Eq. 13, 16), adds
 * them to the HNEMA sums (Eq. 19) and, with MHC_FLAG_GKMA, to the lag
 * correlation sums (Eq. 17).  Asynchronous: device inputs must stay valid until
 * the stream reaches the push; host inputs are copied before the call returns (into one of
 * two device staging buffers, on an internal copy stream, so that the upload overlaps the
 * kernels of the previous push; page-locked host memory uploads fastest).  With
 * MHC_MEM_HOST_ASYNC the call returns once the upload and the kernels are queued and waits
 * instead, before it returns, for the upload of the previous asynchronous push: uploads then
 * follow each other on the copy stream without a host round trip between them.
 * Errors: INVALID_ARG (no modes/bins yet, K out of range, null), CUDA.
 */
mhc_status mhc_push(mhc_handle *h, const float *v, const float *W, int32_t K, int32_t where);

/*
 * Autotune the block length K (steps per push): for each of the n candidates (1 <= K <= k_max)
 * times three pushes' pack and projection kernels (with the tile shape and split autotuned for
 * that K, as on a first push) on a synthetic block of constant samples, and returns in *best_K
 * the candidate with the most steps per second (the rate in *steps_per_s, may be NULL).  No
 * accumulator changes; the operands of the last pushed block are overwritten, so
 * mhc_read_binned_current / mhc_read_total_current return INVALID_ARG until the next push.
 * Synchronises the stream.  Errors: INVALID_ARG (no modes/bins, candidate out of range), CUDA.
 */
mhc_status mhc_autotune_k(mhc_handle *h, const int32_t *candidates, int32_t n, int32_t *best_K,
                          double *steps_per_s);

/* Wait for the stream (and an asynchronous upload of host inputs) and report a sticky device
 * status (TIMEOUT/STATE). */
mhc_status mhc_sync(mhc_handle *h);

/* Binned modal current of the last pushed block, out [K_last][B][3] float32. */
mhc_status mhc_read_binned_current(mhc_handle *h, float *out, int32_t where);

/* Total current (Eq. 10) of the last pushed block, out [K_last][3] float64. */
mhc_status mhc_read_total_current(mhc_handle *h, double *out, int32_t where);

/*
 * HNEMA (Eq. 19): mean_J [B][3] = <J_b^mu> over all pushed steps (eV A/ps) and
 * kappa [B][3] = <J_b^mu> / (T V |F_e|) in W/(m K).  Either pointer may be NULL.
 */
mhc_status mhc_read_hnema(mhc_handle *h, double *kappa, double *mean_J, int32_t where);

/*
 * GKMA raw correlation sums (Eq. 17 integrand before averaging):
 *   corr_sum [B][3][3][L] = sum_{t >= l} J_b^mu(t) J^nu(t - l), float64
 *   count    [L]          = number of time origins of each lag (int64), may be NULL.
 * Requires MHC_FLAG_GKMA.
 */
mhc_status mhc_read_corr(mhc_handle *h, double *corr_sum, int64_t *count, int32_t where);

/*
 * GKMA modal thermal conductivity (Eq. 17), trapezoid rule, kappa(0) = 0:
 *   kappa_tau [B][3][3][L]  running integral kappa_b^{mu nu}(l dt), W/(m K); may be NULL
 *   kappa_w   [B][3][3]     its average over lags with tau_lo <= l dt <= tau_hi
 *                           (the tau window of Sec. III.A), may be NULL.
 * With kappa_tau NULL the window average is evaluated directly as a weighted sum of the
 * correlation over the lags (the same value up to FP64 rounding order, and faster).
 */
mhc_status mhc_read_kappa_gk(mhc_handle *h, double *kappa_tau, double tau_lo, double tau_hi,
                             double *kappa_w, int32_t where);

/*
 * Bin-bin cross-correlation sums (MHC_FLAG_XCORR): xsum [R][R][3][3][L] float64 with
 * xsum[b][b'][mu][nu][l] = sum_{t=l}^{T_s-1} J_b^mu(t) J_{b'}^nu(t-l), R = B (3B with the
 * direction split, rows b*B + bin), and the origin counts [L] as for mhc_read_corr.
 * mhc_read_kappa_xcorr applies the Eq. 17 running integral of mhc_read_kappa_gk to every
 * pair: kappa_tau [R][R][3][3][L], kappa_w [R][R][3][3], W/(m K).  Either pointer may be NULL.
 * Errors: INVALID_ARG without MHC_FLAG_XCORR.
 */
mhc_status mhc_read_xcorr(mhc_handle *h, double *xsum, int64_t *count, int32_t where);
mhc_status mhc_read_kappa_xcorr(mhc_handle *h, double *kappa_tau, double tau_lo, double tau_hi,
                                double *kappa_w, int32_t where);

/*
 * Orthonormality of the loaded eigenvectors, the property that makes Eq. 14 the inverse of
 * Eq. 13 (sum_n e_{i,n} e_{j,n} = delta_ij for the full basis, and e_n . e_m = delta_nm for
 * the kept modes, Sec. II.B).  Reports the last basis check of mhc_set_modes (run in FP64 on
 * the GPU when mhc_params.ortho_probe >= 0: over all mode pairs, or P probe modes against
 * all): *max_abs_err = max |E^T E - I|.  Returns WARN_NOT_ORTHONORMAL above tol,
 * INVALID_ARG if no check was run.
 */
mhc_status mhc_check_orthonormality(mhc_handle *h, double tol, double *max_abs_err);

/* Counters and sizes. */
mhc_status mhc_get_info(mhc_handle *h, mhc_info *info);

/* Change the run-time flags MHC_FLAG_NO_GRAPH, MHC_FLAG_PROFILE and MHC_FLAG_TEST_STALL of a
 * handle (the other bits of `flags` must equal the handle's).  Takes effect at the next push. */
mhc_status mhc_set_flags(mhc_handle *h, int32_t flags);

/* With MHC_FLAG_PROFILE: total device time (ms) of the projection launches (the
 * tensor-core or FP32 GEMM with its fused epilogue) since the previous call, measured
 * with CUDA events recorded on the handle's stream around each launch, and their count.
 * Synchronises the stream; resets the totals. */
mhc_status mhc_kernel_time(mhc_handle *h, double *ms, int64_t *launches);

/* Zero the HNEMA and GKMA accumulators, the step counter and the sticky device status
 * (modes and bins stay). */
mhc_status mhc_reset(mhc_handle *h);

/*
 * Checkpoint / resume of the accumulators (step count, HNEMA sums, GKMA sums
 * and the ring of recent total currents).  mhc_state_size gives the blob size;
 * the blob is only valid for a handle with the same modes, bins, L and k_max.
 * A run split by get/set_state gives bitwise the same results as an unsplit run.
 */
mhc_status mhc_state_size(mhc_handle *h, size_t *bytes);
mhc_status mhc_get_state(mhc_handle *h, void *blob, size_t bytes);
mhc_status mhc_set_state(mhc_handle *h, const void *blob, size_t bytes);

/*
 * Grouped execution of up to 16 independent systems of uneven size (e.g. the
 * replicas or the nanotube batch of Sec. III.A): one persistent tensor-core launch
 * covers the tiles of all handles, assigned to the SMs by a longest-processing-time
 * schedule (a tile's cost is proportional to its 3N).  All handles must be on the
 * same device and stream, use the same tensor-core precision, and have modes and
 * bins loaded; the group does not own them and must be destroyed before them.  The
 * tile shape is autotuned on the first group push (tile_config of the first handle
 * 0) and gives the same results as pushing each handle on its own.  Errors of group
 * calls are reported through mhc_last_error of the first handle.
 */
mhc_status mhc_group_create(mhc_group **g, mhc_handle *const *handles, int32_t n);
void mhc_group_destroy(mhc_group *g);
/* v[j], W[j] are the inputs of handle j with K[j] steps (same rules as mhc_push).  After the
 * first (autotuning) push, group pushes replay a CUDA graph captured per (K vector, input
 * pointers, tile shape) unless the first handle has MHC_FLAG_NO_GRAPH, MHC_FLAG_PROFILE or
 * MHC_FLAG_TEST_STALL set; with MHC_FLAG_PROFILE on the first handle, mhc_kernel_time of that
 * handle times the grouped tensor-core launches. */
mhc_status mhc_group_push(mhc_group *g, const float *const *v, const float *const *W,
                          const int32_t *K, int32_t where);
/* Block length of the group (every member pushes K steps): for each of the n candidates times
 * three grouped pushes' packs and grouped projection (the group's tile shape autotuned on the
 * first candidate if it was not yet) on constant synthetic blocks, and returns in *best_K the
 * candidate with the most mode*atom*steps per second (summed over the members; the rate in
 * *units_per_s, may be NULL).  No accumulator changes; the members' last-block operands are
 * overwritten (their binned and total currents are unreadable until the next push).
 * Synchronises the stream.  Errors: INVALID_ARG (a candidate above a member's k_max), CUDA. */
mhc_status mhc_group_autotune_k(mhc_group *g, const int32_t *candidates, int32_t n, int32_t *best_K,
                                double *units_per_s);
/* HNEMA read-out (as mhc_read_hnema) of every member in one call: kappa and mean_J receive
 * the members' [B_j][3] arrays one after another (either may be NULL); host outputs cost one
 * synchronisation for the whole group. */
mhc_status mhc_group_read_hnema(mhc_group *g, double *kappa, double *mean_J, int32_t where);

/*
 * Spectral heat current (SHC, Sec. II.C): the virial-velocity correlation of Eq. 20-21,
 *   Ksum[3a+b][l] = sum_{t >= l} sum_i W_i^{ab}(t - l) v_i^b(t),   count[l] = T_s - l,
 * accumulated at run time (no eigenvectors needed), and the spectrum of Eq. 22-23,
 *   kappa[3a+b][k] = 2 Ktilde(2 pi f_k) / (V T |F_e|)   in W/(m K) per THz,
 *   Ktilde(omega) = 2 dt sum_l c_l w_l K(l) cos(omega l dt)  (K extended evenly to t < 0,
 *   trapezoid weights c_l, window w = 1 or Hann (1 + cos(pi l / (L-1))) / 2).
 * Summing a tensor pair over b gives the a component of Eq. 21 / 23; at lag 0 it is the
 * time average of the total heat current (Eq. 10).  v, W as for mhc_push.
 *   n_lags  L correlation lags, L <= 4096 (the paper uses 250 lags of 2 fs); k_max <= 1024.
 * Arithmetic (mhc_shc_set_precision, default MHC_PREC_FP16X3): the tensor-core precisions
 * compute each block as a banded contraction over the atoms, G_b[(a,tau)][t] =
 * sum_i W_i^{ab}(tau) v_i^b(t), in 128 x 256 tiles (two per CTA pair) with split 16-bit
 * operands (one power-of-two scale per row) and FP32 accumulation, whose diagonals
 * t - tau = l are the lag sums; MHC_PREC_FP32 runs FP32 FMAs on the CUDA cores.  Lag sums
 * are FP64 in both.
 * Errors as for the modal handle; messages through mhc_shc_last_error.  A kernel that waited
 * too long on a barrier is reported as MHC_ERR_TIMEOUT by the next host read.
 */
typedef struct mhc_shc mhc_shc;
mhc_status mhc_shc_create(mhc_shc **s, int32_t device, void *stream, int64_t n_atoms,
                          int32_t n_lags, int32_t k_max, double dt_ps, double T_K, double V_A3,
                          const double *F_e);
void mhc_shc_destroy(mhc_shc *s);
const char *mhc_shc_last_error(const mhc_shc *s);
/* Select the arithmetic (mhc_precision) before the first push; INVALID_ARG afterwards.
 * Reallocates the handle's ring buffers. */
mhc_status mhc_shc_set_precision(mhc_shc *s, int32_t precision);
/* CUDA-event timing of the correlation kernel of each push while on != 0 (restarts the
 * count); mhc_shc_kernel_time returns the total ms and launches since the last call and
 * resets them.  INVALID_ARG when profiling is off. */
mhc_status mhc_shc_set_profile(mhc_shc *s, int32_t on);
mhc_status mhc_shc_kernel_time(mhc_shc *s, double *ms, int64_t *launches);
/* One block of K samples (host or device memory).  Device inputs must stay valid until the
 * stream reaches the push; host inputs are copied before the call returns (two staging
 * buffers on an internal copy stream: the upload overlaps the previous push's kernels). */
mhc_status mhc_shc_push(mhc_shc *s, const float *v, const float *W, int32_t K, int32_t where);
/* Raw sums Ksum [9][L] (float64) and origin counts [L] (int64); either may be NULL. */
mhc_status mhc_shc_read_corr(mhc_shc *s, double *Ksum, int64_t *count, int32_t where);
/* kappa [9][n_freq] for the host array of frequencies f_THz; window 0 (none) or 1 (Hann). */
mhc_status mhc_shc_read_kappa(mhc_shc *s, const double *f_THz, int32_t n_freq, int32_t window,
                              double *kappa, int32_t where);

/*
 * Gamma-point lattice dynamics on the GPU (Sec. II.B: the modal analysis projects onto the
 * 3N eigenmodes of the harmonic solid, found by lattice dynamics with the whole cell as the
 * unit cell; Sec. III.C: O(N^3) time, O(N^2) memory).  With the force constants Phi and masses
 * m_i, the dynamical matrix Dyn[3i+a][3j+b] = Phi[3i+a][3j+b] / sqrt(m_i m_j) is diagonalised,
 * Dyn e_n = w_n^2 e_n, by parallel cyclic Jacobi rotations in FP64 until the off-diagonal
 * Frobenius norm is at most tol times the total.
 *   n_atoms    N (at most 10000; the cost grows as (3N)^3 and GB300's FP64 rate is low)
 *   Phi        [3N][3N] float64, row-major, eV/A^2, symmetric; host or device (where_in)
 *   mass_amu   [N] host, every m_i > 0
 *   w2         [3N] host or NULL: w_n^2 in eV/(A^2 amu), ascending
 *   freq_THz   [3N] host or NULL: f_n = w_n / (2 pi) with w in rad/ps (negative for w^2 < 0)
 *   E          [3N][3N] float64 or NULL: eigenvectors dof-major, E[d * 3N + n] = component d
 *              of mode n (the layout mhc_set_modes takes as MHC_DOF_MAJOR), each signed so its
 *              first component of largest magnitude is positive; host or device (where_out)
 *   sweeps     number of sweeps taken (may be NULL)
 * Allocates its own work space (about 3 (3N)^2 doubles) and synchronises `stream`.  With E on
 * the device the basis goes from the force constants to mhc_set_modes without leaving the GPU.
 * Errors (message through mhc_last_error(NULL)): INVALID_ARG, OOM, CUDA, STATE (not converged
 * within max_sweeps).
 */
mhc_status mhc_lattice_modes(int32_t device, void *stream, int64_t n_atoms, const double *Phi,
                             const double *mass_amu, int32_t where_in, double tol,
                             int32_t max_sweeps, double *w2, double *freq_THz, double *E,
                             int32_t where_out, int32_t *sweeps);

/*
 * Measured FP32 FMA throughput of `device` (TFLOP/s, 2 flops an FMA), the peak of the FP32
 * comparison path: the best of three launches of a kernel in which every thread runs 16
 * independent FMA chains (one warm-up launch first), on `stream` (cudaStream_t or NULL;
 * synchronised).  Allocates and frees a small device buffer.  Errors: INVALID_ARG for a null
 * output, CUDA for runtime errors (message in mhc_last_error(NULL)).
 */
mhc_status mhc_measure_fp32_fma(int32_t device, void *stream, double *tflops);

/*
 * No-allocation variant of one block's binned modal current.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate device memory,
 * e.g. an MD engine calling from inside its time-step loop (where cudaMalloc would
 * synchronise the device) or an application that owns all device memory through a pool
 * reserved at start-up.  It computes what mhc_push + mhc_read_binned_current /
 * mhc_read_total_current give with MHC_PREC_FP32, for one block, with no handle.
 *
 *   E            device, FP32, mode-major E[n * ld + 3i + b] = e^b_{i,n}, ld >= 3N
 *   bin_of_mode  device [M]: bin of each mode, in [0, B) and non-decreasing (order the
 *                modes by bin and drop excluded ones before the call)
 *   mass_amu     device [N] float64, every m_i > 0
 *   v, W         device [K][N][3] and [K][N][9] float32 (layouts as for mhc_push)
 *   Jb           device output [K][B][3] float32 (binned modal current)
 *   J            device output [K][3] float64 (total heat current sum_i W_i v_i)
 *   stream       cudaStream_t or NULL
 * Every intermediate array lives in one static device buffer of
 * MHC_NOALLOC_SCRATCH_BYTES that every GPU loading this library holds until exit; no
 * call allocates.  The first call on a device looks up the buffer's device address
 * (cudaGetSymbolAddress).  No call can be captured into a CUDA graph (each reads a status
 * word back and synchronises `stream`).  Calls share
 * the buffer and keep the last call's contents (what must start at zero is cleared each
 * call); calls whose work overlaps on the GPU race.  Every call synchronises `stream`
 * twice: once after the bins and masses are checked on the device, once at the end.
 * Errors: INVALID_ARG for bad sizes or pointers, bins that are out of range or
 * decreasing, non-positive masses (then nothing is computed and Jb, J are not written),
 * or a problem whose intermediates exceed the buffer (roughly
 * 4 (M_pad + 4K) D_pad + 16 K M_pad bytes with M_pad = M rounded up to 128 and
 * D_pad = 3N rounded up to 64); CUDA for runtime errors.
 */
#define MHC_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
mhc_status mhc_binned_current_noalloc(int32_t n_atoms, int32_t n_modes, const float *E, int64_t ld,
                                      const int32_t *bin_of_mode, int32_t n_bins,
                                      const double *mass_amu, const float *v, const float *W,
                                      int32_t K, float *Jb, double *J, int32_t device,
                                      void *stream);

#ifdef __cplusplus
}
#endif
#endif /* MHC_H */
