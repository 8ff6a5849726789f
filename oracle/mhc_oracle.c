/*
 * FP64 CPU oracle for the modal heat current (GKMA / HNEMA).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code:
 * only the tests, the smoke check and the benchmark's CPU-baseline leg load it.
 * It shares no code with the CUDA library.
 *
 * Every routine is the plain definition from the paper, written out as straight
 * FP64 loops in the paper's notation.  Inputs v and W arrive as float32 (the
 * precision an MD engine hands over) and are widened to double exactly.
 *
 *   Eq. 10   J^a       = sum_i sum_b W_i^{ab} v_i^b               (total current)
 *   Eq. 13   Xdot_n    = sum_i sqrt(m_i) e_{i,n} . v_i            (modal velocity)
 *   Eq. 16   J_n^a     = (sum_i m_i^{-1/2} (W_i e_{i,n})^a) Xdot_n (modal current)
 *   binning  J_b^a     = sum_{n in b} J_n^a   (frequency bins, Sec. III.A)
 *   Eq. 17   kappa_n^{mu nu}(tau) = (k_B T^2 V)^{-1} int_0^tau <J_n^mu(t') J^nu(0)> dt'
 *   Eq. 19   <J_n^mu>/(T V) = sum_nu kappa_n^{mu nu} F_e^nu
 *   Eq. 21   K(t) = sum_i <W_i(0) . v_i(t)>                     (SHC correlation)
 *   Eq. 22   Ktilde(omega) = int K(t) e^{i omega t} dt
 *   Eq. 23   kappa(omega) = 2 Ktilde(omega) / (V T F_e)
 *
 * Readings where the paper is silent (each stated where it is used):
 *   - e is real (Gamma point), so e* = e in Eq. 13.
 *   - W is stored row-major [alpha][beta]; (W e)^a = sum_b W^{ab} e^b (Eq. 10).
 *   - correlation average over all origins t with t - lag >= 0, divided by the
 *     number of origins; trapezoid rule with kappa(0) = 0.
 *
 * Layouts: E is passed mode-major, Et[n * D + (3 i + b)] = e^b_{i,n} (column n of
 * the dof-major eigenvector matrix stored contiguously).  v is [T][N][3],
 * W is [T][N][9] with W[t][i][3 a + b] = W_i^{ab}.
 *
 * Parity pins for every function live in tests/test_oracle_pins.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_KB_EV_PER_K 8.617333262145179e-5 /* k_B = 1.380649e-23 J/K over e = 1.602176634e-19 C (SI exact) */
#define ORC_WMK_PER_EV_PS_A_K 1602.176634 /* 1 eV/(ps A K) in W/(m K) */

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/*
 * Frequency binning (Sec. III.A: bins of fixed width in THz).
 * Bin b covers [f_min + b*w, f_min + (b+1)*w) with w = (f_max - f_min)/B; the
 * last bin also takes f == f_max.  Frequencies outside [f_min, f_max] (or not
 * finite) get -1 (mode excluded).  The bin index is floor((f - f_min) / w)
 * evaluated in double precision.
 */
void orc_bins_uniform(int64_t M, const double *f_THz, double f_min, double f_max,
                      int32_t B, int32_t *bin_of_mode)
{
    double w = (f_max - f_min) / (double)B;
    for (int64_t n = 0; n < M; ++n) {
        double f = f_THz[n];
        if (!isfinite(f) || f < f_min || f > f_max) {
            bin_of_mode[n] = -1;
            continue;
        }
        int64_t b = (int64_t)floor((f - f_min) / w);
        if (b >= B) b = B - 1;
        if (b < 0) b = 0;
        bin_of_mode[n] = (int32_t)b;
    }
}

/* Eq. 10: total potential heat current of one step, J^a = sum_i sum_b W_i^{ab} v_i^b. */
static void total_current(int64_t N, const float *v, const float *W, double J[3])
{
    for (int a = 0; a < 3; ++a) {
        double s = 0.0;
        for (int64_t i = 0; i < N; ++i)
            for (int b = 0; b < 3; ++b)
                s += (double)W[i * 9 + 3 * a + b] * (double)v[i * 3 + b];
        J[a] = s;
    }
}

/*
 * Modal heat current for T steps (Eqs. 10, 13, 16 and frequency binning).
 *   Jb    [T][B][3]  binned modal current, sum over modes in ascending n
 *   J     [T][3]     total current (Eq. 10)
 *   xdot  [T][M]     modal velocities (optional, may be NULL)
 *   Jn    [T][M][3]  per-mode currents (optional, may be NULL)
 * Modes with bin -1 are excluded from Jb (their Jn/xdot are still produced).
 */
void orc_modal_current(int64_t N, int64_t M, const double *Et, const double *mass,
                       int64_t T, const float *v, const float *W,
                       const int32_t *bin_of_mode, int32_t B,
                       double *Jb, double *J, double *xdot, double *Jn)
{
    const int64_t D = 3 * N;
    double *sqm = (double *)malloc(sizeof(double) * (size_t)N);
    double *isqm = (double *)malloc(sizeof(double) * (size_t)N);
    double *jn = (double *)malloc(sizeof(double) * (size_t)M * 3);
    for (int64_t i = 0; i < N; ++i) {
        sqm[i] = sqrt(mass[i]);
        isqm[i] = 1.0 / sqrt(mass[i]);
    }
    for (int64_t t = 0; t < T; ++t) {
        const float *vt = v + t * N * 3;
        const float *Wt = W + t * N * 9;
        total_current(N, vt, Wt, J + t * 3);

#pragma omp parallel for schedule(static)
        for (int64_t n = 0; n < M; ++n) {
            const double *e = Et + n * D;
            /* Eq. 13 with real e: Xdot_n = sum_i sqrt(m_i) sum_b e^b_{i,n} v_i^b */
            double x = 0.0;
            for (int64_t i = 0; i < N; ++i) {
                double ev = 0.0;
                for (int b = 0; b < 3; ++b) ev += e[3 * i + b] * (double)vt[i * 3 + b];
                x += sqm[i] * ev;
            }
            /* Eq. 16 bracket: y^a = sum_i m_i^{-1/2} sum_b W_i^{ab} e^b_{i,n} */
            double y[3] = {0.0, 0.0, 0.0};
            for (int64_t i = 0; i < N; ++i) {
                for (int a = 0; a < 3; ++a) {
                    double we = 0.0;
                    for (int b = 0; b < 3; ++b)
                        we += (double)Wt[i * 9 + 3 * a + b] * e[3 * i + b];
                    y[a] += isqm[i] * we;
                }
            }
            for (int a = 0; a < 3; ++a) jn[n * 3 + a] = y[a] * x;
            if (xdot) xdot[t * M + n] = x;
        }
        if (Jn) memcpy(Jn + t * M * 3, jn, sizeof(double) * (size_t)M * 3);
        /* binning: modes in ascending order within each bin */
        double *jb = Jb + t * (int64_t)B * 3;
        for (int64_t k = 0; k < (int64_t)B * 3; ++k) jb[k] = 0.0;
        for (int64_t n = 0; n < M; ++n) {
            int32_t b = bin_of_mode[n];
            if (b < 0 || b >= B) continue;
            for (int a = 0; a < 3; ++a) jb[b * 3 + a] += jn[n * 3 + a];
        }
    }
    free(sqm);
    free(isqm);
    free(jn);
}

/*
 * Direction-resolved modal heat current (Sec. II.A: the heat current along a splits
 * into the contributions of the atoms' motion along each Cartesian direction b; the
 * closing paragraph of Sec. II.C applies this split to every method's spectral result).
 * With the modal atomic velocity of Eq. 14, v_{i,n} = Xdot_n e_{i,n} / sqrt(m_i):
 *   J_n^{ab}(t) = Xdot_n(t) sum_i m_i^{-1/2} W_i^{ab}(t) e^b_{i,n}        (no sum over b)
 * so that sum_b J_n^{ab} is the J_n^a of Eq. 16.
 *   Jbd  [T][3 (b)][B][3 (a)]   binned, modes in ascending n within each bin
 *   Jd   [T][3 (b)][3 (a)]      J^{ab} = sum_i W_i^{ab} v_i^b (optional, may be NULL)
 *   Jnd  [T][M][3 (b)][3 (a)]   per mode (optional, may be NULL)
 */
void orc_modal_current_dir(int64_t N, int64_t M, const double *Et, const double *mass,
                           int64_t T, const float *v, const float *W,
                           const int32_t *bin_of_mode, int32_t B,
                           double *Jbd, double *Jd, double *Jnd)
{
    const int64_t D = 3 * N;
    double *jn = (double *)malloc(sizeof(double) * (size_t)M * 9);
    for (int64_t t = 0; t < T; ++t) {
        const float *vt = v + t * N * 3;
        const float *Wt = W + t * N * 9;
        if (Jd) {
            for (int b = 0; b < 3; ++b)
                for (int a = 0; a < 3; ++a) {
                    double s = 0.0;
                    for (int64_t i = 0; i < N; ++i)
                        s += (double)Wt[i * 9 + 3 * a + b] * (double)vt[i * 3 + b];
                    Jd[t * 9 + 3 * b + a] = s;
                }
        }
#pragma omp parallel for schedule(static)
        for (int64_t n = 0; n < M; ++n) {
            const double *e = Et + n * D;
            double x = 0.0;   /* Eq. 13 */
            for (int64_t i = 0; i < N; ++i) {
                double ev = 0.0;
                for (int b = 0; b < 3; ++b) ev += e[3 * i + b] * (double)vt[i * 3 + b];
                x += sqrt(mass[i]) * ev;
            }
            for (int b = 0; b < 3; ++b)
                for (int a = 0; a < 3; ++a) {
                    double y = 0.0;   /* only the b-th velocity component of the modal motion */
                    for (int64_t i = 0; i < N; ++i)
                        y += (double)Wt[i * 9 + 3 * a + b] * e[3 * i + b] / sqrt(mass[i]);
                    jn[n * 9 + 3 * b + a] = x * y;
                }
        }
        if (Jnd) memcpy(Jnd + t * M * 9, jn, sizeof(double) * (size_t)M * 9);
        double *jb = Jbd + t * 3 * (int64_t)B * 3;
        for (int64_t k = 0; k < 9 * (int64_t)B; ++k) jb[k] = 0.0;
        for (int64_t n = 0; n < M; ++n) {
            const int32_t bn = bin_of_mode[n];
            if (bn < 0 || bn >= B) continue;
            for (int b = 0; b < 3; ++b)
                for (int a = 0; a < 3; ++a) jb[((int64_t)b * B + bn) * 3 + a] += jn[n * 9 + 3 * b + a];
        }
    }
    free(jn);
}

/*
 * GKMA correlation sums (Eq. 17 integrand, reading: the modal current is lagged,
 * the total current sits at the time origin, all origins with t - lag >= 0):
 *   Csum[b][mu][nu][l] = sum_{t=l}^{T-1} Jb[t][b][mu] * J[t-l][nu]
 *   count[l]           = max(T - l, 0)
 */
void orc_gkma_corr(int64_t T, int32_t B, const double *Jb, const double *J, int32_t L,
                   double *Csum, int64_t *count)
{
    for (int32_t l = 0; l < L; ++l) count[l] = T > l ? T - l : 0;
#pragma omp parallel for schedule(static)
    for (int32_t b = 0; b < B; ++b)
        for (int mu = 0; mu < 3; ++mu)
            for (int nu = 0; nu < 3; ++nu)
                for (int32_t l = 0; l < L; ++l) {
                    double s = 0.0;
                    for (int64_t t = l; t < T; ++t)
                        s += Jb[(t * B + b) * 3 + mu] * J[(t - l) * 3 + nu];
                    Csum[(((int64_t)b * 3 + mu) * 3 + nu) * L + l] = s;
                }
}

/*
 * Cross-correlations of binned modal heat currents (the mode-mode correlations the paper
 * notes GKMA allows, Sec. II.B after Eq. 17 and Sec. III.C.i; with one bin per mode they are
 * the mode-mode correlations themselves).  Same lag convention as Eq. 17: the first current
 * is lagged, the second sits at the time origin; all origins with t - l >= 0:
 *   Xsum[b][b2][mu][nu][l] = sum_{t=l}^{T-1} Jb[t][b][mu] * Jb[t-l][b2][nu]
 * With every mode binned, sum_b2 Jb[t][b2] = J[t] (Eq. 15), so sum_b2 Xsum = Csum of Eq. 17.
 */
void orc_gkma_xcorr(int64_t T, int32_t B, const double *Jb, int32_t L, double *Xsum)
{
#pragma omp parallel for schedule(static)
    for (int32_t b = 0; b < B; ++b)
        for (int32_t b2 = 0; b2 < B; ++b2)
            for (int mu = 0; mu < 3; ++mu)
                for (int nu = 0; nu < 3; ++nu)
                    for (int32_t l = 0; l < L; ++l) {
                        double s = 0.0;
                        for (int64_t t = l; t < T; ++t)
                            s += Jb[(t * B + b) * 3 + mu] * Jb[((t - l) * B + b2) * 3 + nu];
                        Xsum[((((int64_t)b * B + b2) * 3 + mu) * 3 + nu) * L + l] = s;
                    }
}

/*
 * Eq. 17 running integral by the trapezoid rule, kappa(0) = 0:
 *   C(l)      = Csum(l) / count(l)          (0 where count is 0)
 *   kappa(l)  = c * dt * sum_{j=1}^{l} (C(j-1) + C(j)) / 2
 *   c         = 1 / (k_B T^2 V), converted to W/(m K)
 * Output kappa[b][mu][nu][l] in W/(m K) for dt in ps, T in K, V in A^3.
 */
void orc_gk_kappa(int32_t B, int32_t L, const double *Csum, const int64_t *count,
                  double dt_ps, double T_K, double V_A3, double *kappa)
{
    double c = ORC_WMK_PER_EV_PS_A_K / (ORC_KB_EV_PER_K * T_K * T_K * V_A3);
    for (int64_t r = 0; r < (int64_t)B * 9; ++r) {
        const double *cs = Csum + r * L;
        double *kp = kappa + r * L;
        double acc = 0.0, prev = 0.0;
        for (int32_t l = 0; l < L; ++l) {
            double C = count[l] > 0 ? cs[l] / (double)count[l] : 0.0;
            if (l > 0) acc += 0.5 * (prev + C) * dt_ps;
            kp[l] = c * acc;
            prev = C;
        }
    }
}

/*
 * kappa(omega) for GKMA: the running integral averaged over the lags whose
 * correlation time l*dt lies in [tau_lo, tau_hi] (the paper averages kappa_n(tau)
 * over a tau window, Sec. III.A.i-iii).  Returns the number of lags averaged.
 */
int32_t orc_kappa_window(int32_t B, int32_t L, const double *kappa, double dt_ps,
                         double tau_lo, double tau_hi, double *kappa_w)
{
    int32_t n = 0;
    for (int64_t r = 0; r < (int64_t)B * 9; ++r) {
        double s = 0.0;
        n = 0;
        for (int32_t l = 0; l < L; ++l) {
            double tau = l * dt_ps;
            if (tau >= tau_lo && tau <= tau_hi) {
                s += kappa[r * L + l];
                ++n;
            }
        }
        kappa_w[r] = n > 0 ? s / n : 0.0;
    }
    return n;
}

/*
 * HNEMA (Eq. 19): time average of the binned modal current and
 *   kappa_b^mu = <J_b^mu> / (T V |F_e|)   in W/(m K)
 * i.e. sum_nu kappa_b^{mu nu} Fhat^nu; for F_e along x this is kappa_b^{mu x}.
 */
void orc_hnema(int64_t T, int32_t B, const double *Jb, double T_K, double V_A3,
               const double Fe[3], double *meanJ, double *kappa)
{
    double fe = sqrt(Fe[0] * Fe[0] + Fe[1] * Fe[1] + Fe[2] * Fe[2]);
    for (int64_t k = 0; k < (int64_t)B * 3; ++k) {
        double s = 0.0;
        for (int64_t t = 0; t < T; ++t) s += Jb[t * B * 3 + k];
        meanJ[k] = T > 0 ? s / (double)T : 0.0;
        kappa[k] = fe > 0 ? meanJ[k] / (T_K * V_A3 * fe) * ORC_WMK_PER_EV_PS_A_K : 0.0;
    }
}

/* Orthonormality residual of the mode-major eigenvectors: max |E^T E - I|. */
double orc_orthonormality(int64_t D, int64_t M, const double *Et)
{
    double worst = 0.0;
#pragma omp parallel for schedule(dynamic) reduction(max : worst)
    for (int64_t n = 0; n < M; ++n)
        for (int64_t m = n; m < M; ++m) {
            double s = 0.0;
            for (int64_t d = 0; d < D; ++d) s += Et[n * D + d] * Et[m * D + d];
            double r = fabs(s - (n == m ? 1.0 : 0.0));
            if (r > worst) worst = r;
        }
    return worst;
}

/*
 * SHC correlation sums (Eq. 20-21), resolved by the tensor pair (a, b):
 *   Ksum[3a+b][l] = sum_{t=l}^{T-1} sum_i W_i^{ab}(t - l) v_i^b(t)
 *   count[l]      = max(T - l, 0)
 * K^a(l) of Eq. 21 is sum_b Ksum[3a+b][l] / count[l]; at l = 0 it is the time average
 * of the total heat current of Eq. 10.  v is [T][N][3], W is [T][N][9].
 */
void orc_shc_corr(int64_t N, int64_t T, const float *v, const float *W, int32_t nc,
                  double *Ksum, int64_t *count)
{
    for (int32_t l = 0; l < nc; ++l) count[l] = T > l ? T - l : 0;
#pragma omp parallel for schedule(static)
    for (int32_t l = 0; l < nc; ++l)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double s = 0.0;
                for (int64_t t = l; t < T; ++t)
                    for (int64_t i = 0; i < N; ++i)
                        s += (double)W[((t - l) * N + i) * 9 + 3 * a + b] *
                             (double)v[(t * N + i) * 3 + b];
                Ksum[(int64_t)(3 * a + b) * nc + l] = s;
            }
}

/*
 * SHC spectrum (Eq. 22-23).  Reading: K is computed for t >= 0 only and extended
 * evenly, K(-t) = K(t), so Ktilde(omega) = 2 int_0^{t_c} w(t) K(t) cos(omega t) dt with
 * t_c = (nc - 1) dt, the trapezoid rule on the lags, and w = 1 (window 0) or the Hann
 * window w = (1 + cos(pi t / t_c)) / 2 (window 1).  omega = 2 pi f with f in THz.
 *   kappa[c][k] = 2 Ktilde_c(2 pi f_k) / (V T |F_e|)   in W/(m K) per THz
 * for every tensor pair c = 3a+b (sum over b gives the a component of Eq. 23).
 */
void orc_shc_kappa(int32_t nc, const double *Ksum, const int64_t *count, double dt_ps,
                   double T_K, double V_A3, double Fe, int32_t window, int32_t n_freq,
                   const double *f_THz, double *kappa)
{
    const double PI = 3.14159265358979323846;
    const double tc = (nc - 1) * dt_ps;
    for (int c = 0; c < 9; ++c)
        for (int32_t k = 0; k < n_freq; ++k) {
            const double omega = 2.0 * PI * f_THz[k];
            double s = 0.0;
            for (int32_t l = 0; l < nc; ++l) {
                const double K = count[l] > 0 ? Ksum[(int64_t)c * nc + l] / (double)count[l] : 0.0;
                const double t = l * dt_ps;
                double w = 1.0;
                if (window == 1 && tc > 0) w = 0.5 * (1.0 + cos(PI * t / tc));
                const double trap = (l == 0 || l == nc - 1) ? 0.5 : 1.0;
                s += trap * w * K * cos(omega * t);
            }
            const double Kt = 2.0 * s * dt_ps;   /* eV A */
            kappa[(int64_t)c * n_freq + k] =
                Fe > 0 ? 2.0 * Kt / (V_A3 * T_K * Fe) * ORC_WMK_PER_EV_PS_A_K : 0.0;
        }
}

/*
 * Gamma-point lattice dynamics (Sec. II.B: the 3N eigenmodes of the harmonic solid whose
 * eigenvectors e_{i,n} and frequencies the modal analysis uses; Sec. III.C: O(N^3) time,
 * O(N^2) memory).  With force constants Phi[3i+a][3j+b] (eV/A^2, symmetric) and masses m_i
 * (amu), the dynamical matrix
 *   Dyn[3i+a][3j+b] = Phi[3i+a][3j+b] / sqrt(m_i m_j)
 * has the eigenpairs Dyn e_n = w_n^2 e_n.  w^2 comes out in eV/(A^2 amu); times
 * 9648.533212331 (1 eV/amu in A^2/ps^2) it is in rad^2/ps^2, and f_n = w_n / (2 pi) in THz
 * (a negative w^2 gives a negative frequency).
 * Method: cyclic Jacobi rotations over the pairs p < q in row order; each rotation J in the
 * (p, q) plane (J_pp = J_qq = c, J_pq = s, J_qp = -s, t = s/c the smaller root of
 * t^2 + 2 theta t - 1 = 0 with theta = (a_qq - a_pp) / (2 a_pq)) replaces A by J^T A J, which
 * zeroes a_pq, and the eigenvector matrix V by V J.  Sweeps stop once the off-diagonal
 * Frobenius norm is at most tol times the Frobenius norm of A.
 * Output: w2[n], f_THz[n] in ascending order of w2 (stable), E[d * D + n] = component d of
 * eigenvector n (dof-major), each eigenvector's sign chosen so that its first component of
 * largest magnitude is positive.  Returns the number of sweeps, -1 if max_sweeps was reached.
 */
int32_t orc_lattice_modes(int64_t N, const double *Phi, const double *mass, int32_t max_sweeps,
                          double tol, double *w2, double *f_THz, double *E)
{
    const int64_t D = 3 * N;
    double *A = (double *)malloc(sizeof(double) * (size_t)(D * D));
    double *V = (double *)malloc(sizeof(double) * (size_t)(D * D));
    for (int64_t r = 0; r < D; ++r)
        for (int64_t c = 0; c < D; ++c) {
            A[r * D + c] = Phi[r * D + c] / sqrt(mass[r / 3] * mass[c / 3]);
            V[r * D + c] = r == c ? 1.0 : 0.0;
        }
    int32_t sweeps = -1;
    for (int32_t sw = 0; sw <= max_sweeps; ++sw) {
        double off = 0.0, tot = 0.0;
        for (int64_t r = 0; r < D; ++r)
            for (int64_t c = 0; c < D; ++c) {
                const double x = A[r * D + c] * A[r * D + c];
                tot += x;
                if (r != c) off += x;
            }
        if (sqrt(off) <= tol * sqrt(tot)) {
            sweeps = sw;
            break;
        }
        if (sw == max_sweeps) break;
        for (int64_t p = 0; p < D - 1; ++p)
            for (int64_t q = p + 1; q < D; ++q) {
                const double apq = A[p * D + q];
                if (apq == 0.0) continue;
                const double theta = (A[q * D + q] - A[p * D + p]) / (2.0 * apq);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int64_t k = 0; k < D; ++k) {   /* columns: A J */
                    const double akp = A[k * D + p], akq = A[k * D + q];
                    A[k * D + p] = c * akp - s * akq;
                    A[k * D + q] = s * akp + c * akq;
                }
                for (int64_t k = 0; k < D; ++k) {   /* rows: J^T (A J) */
                    const double apk = A[p * D + k], aqk = A[q * D + k];
                    A[p * D + k] = c * apk - s * aqk;
                    A[q * D + k] = s * apk + c * aqk;
                }
                A[p * D + q] = 0.0;
                A[q * D + p] = 0.0;
                for (int64_t k = 0; k < D; ++k) {   /* eigenvectors: V J */
                    const double vkp = V[k * D + p], vkq = V[k * D + q];
                    V[k * D + p] = c * vkp - s * vkq;
                    V[k * D + q] = s * vkp + c * vkq;
                }
            }
    }
    /* ascending order of the eigenvalues (stable insertion sort of an index array) */
    int64_t *ord = (int64_t *)malloc(sizeof(int64_t) * (size_t)D);
    for (int64_t n = 0; n < D; ++n) {
        int64_t j = n;
        while (j > 0 && A[ord[j - 1] * D + ord[j - 1]] > A[n * D + n]) {
            ord[j] = ord[j - 1];
            --j;
        }
        ord[j] = n;
    }
    const double PI = 3.14159265358979323846;
    for (int64_t n = 0; n < D; ++n) {
        const int64_t src = ord[n];
        const double lam = A[src * D + src];
        w2[n] = lam;
        const double w = sqrt(fabs(lam) * 9648.533212331);
        f_THz[n] = (lam < 0.0 ? -w : w) / (2.0 * PI);
        int64_t big = 0;
        for (int64_t d = 1; d < D; ++d)
            if (fabs(V[d * D + src]) > fabs(V[big * D + src])) big = d;
        const double sg = V[big * D + src] < 0.0 ? -1.0 : 1.0;
        for (int64_t d = 0; d < D; ++d) E[d * D + n] = sg * V[d * D + src];
    }
    free(ord);
    free(A);
    free(V);
    return sweeps;
}
