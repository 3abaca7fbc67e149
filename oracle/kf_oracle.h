/*
 * kf_oracle.h -- plain FP64 CPU oracle for the multi-scale shape-filter bank of
 * Kennedy, "Digital filters with vanishing moments for shape analysis"
 * (arXiv:1912.07133).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path links, loads or calls
 * this code: only tests/, the smoke check and the CPU-baseline leg of the bench
 * use it. It shares no source, header, table or helper with the CUDA library.
 *
 * Every routine follows the paper's steps in the paper's order, in FP64, with no
 * blocking, fusion or reordering beyond what the cited passage states.
 */
#ifndef KF_ORACLE_H
#define KF_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define KO_MAXK 8 /* largest recursive order handled by the IIR designs */

/* A Laurent polynomial sum_{m=-K..K} c[m+K] z^m is stored as 2K+1 doubles. */

/* ---- building blocks (exported for the pins in tests/) ------------------ */

/* Eulerian number <n,k>: permutations of n with k ascents. */
double ko_eulerian(int n, int k);

/* sum_{m>=1} m^n z^m for |z|<1 (polylogarithm of order -n), via the Eulerian
 * closed form z A_n(z) / (1-z)^(n+1). */
double ko_li_neg(int n, double z);

/* Dense solve A x = b (n x n, row-major), Gaussian elimination with partial
 * pivoting after row/column equilibration. A and b are overwritten; x is
 * returned in b. Returns 0 on success, -1 if singular. */
int ko_solve(int n, double *A, double *b);

/* Roots of the real polynomial sum_{i=0..d} c[i] x^i (Durand-Kerner, Newton
 * polish). re/im receive d roots. Returns 0 on success. */
int ko_poly_roots(int d, const double *c, double *re, double *im);

/* Appendix eqs (A13)-(A19): three-part decomposition of H(z) = B(z)/A(z).
 * b, a: Laurent coefficients (2K+1) of B and A.  aplus: K+1 coefficients of
 * A+(z) = 1 + sum a+_m z^-m (aplus[0] = 1).  Builds the (2K+1)^2 matrix of
 * eq (A17), solves b = Atilde btilde and returns:
 *   btilde[2K+1]      the raw solution vector of eq (A17)
 *   a0circ            a0 / a0^{+-} (eq A19 text)
 *   bplus[K+1]        DE forward numerator, bplus[0] = 0, bplus[m] = btilde/a0circ
 *   bminus[K+1]       DE backward numerator
 *   b0                DE centre coefficient, btilde_centre / a0circ
 * Returns 0 on success. */
int ko_a17(int K, const double *b, const double *a, const double *aplus,
           double *btilde, double *a0circ, double *bplus, double *bminus,
           double *b0);

/* ---- filter designs (Sec. 4) ------------------------------------------- */

/* Filter D, repeated-pole IIR blur (Sec. 4.3, eqs 12-15, 23-24), d = 0.
 * (L_D, Lpi) -> K = L_D + Lpi; p = exp(-1/sigma).  Outputs the DE of eq (A10):
 * b0, bplus[0..K] (bplus[0]=0), aplus[0..K] (aplus[0]=1), and the basis
 * weights c[0..K] of eq (12a).  Returns K, or -1 on failure. */
int ko_design_repeated_pole(int L_D, int Lpi, double sigma, double *b0,
                            double *bplus, double *aplus, double *c);

/* Filter E, discrete Butterworth IIR blur (Sec. 4.4, eq 25, A17-A19).
 * L_B = 2(L_D+1), omega_c = sqrt(2 ln 2)/sigma, bilinear s = 2(z-1)/(z+1),
 * no pre-warp.  Returns K = L_D + 1, or -1. omega_c_out may be NULL. */
int ko_design_butterworth(int L_D, double sigma, double *b0, double *bplus,
                          double *aplus, double *omega_c_out);

/* Filter C, colored Savitzky-Golay FIR blur (Sec. 4.2, eqs 16, 20-22).
 * K = ceil(5 sigma) for L_D = 1, ceil(7 sigma) for L_D = 2, then capped at
 * Kmax (Kmax <= 0: no cap).  omega_c = 3/sigma.  Writes h[0..K] (h(-m)=h(m)).
 * Returns K, or -1 (omega_c >= pi, or singular). */
int ko_design_colored_sg(int L_D, double sigma, int Kmax, double *h);

/* Filter A (Sec. 3.1, eqs 9 and 11 with d = 0): the Gaussian g0(x) =
 * exp(-x^2 / 2 sigma^2) / (sigma sqrt(2 pi)) sampled at the integers |m| <= K
 * and renormalised to unit gain at dc (eq 11: c_g = 1 / sum_m g0(m)), so
 * h(m) = c_g g0(m).  K = ceil(5 sigma) (the half-length of the paper's
 * timing comparison), capped at fir_kmax when fir_kmax > 0.  Writes h[0..K]
 * (the symmetric half); returns K, or -1 for sigma <= 0. */
int ko_design_gaussian(double sigma, int fir_kmax, double *h);

/* The same KKT design with an explicit half-length K and cut-off omega_c;
 * omega_c = 0 gives the classic (white-noise) Savitzky-Golay smoother. */
int ko_design_colored_sg_raw(int L_D, int K, double omega_c, double *h);

/* ---- 1-D realisations (Appendix A4-A10, A32) ---------------------------- */

#define KO_BOUNDARY_HOLD 0 /* edge pixels held to +-infinity (IIR init A32) */
#define KO_BOUNDARY_ZERO 1 /* zeros outside the frame (FIR init, Sec. 5) */

/* Three-term recursive DE, eqs (A6), (A10a-c); x and y strided, length n.
 * bminus = sym * bplus (sym = +1 for even IRs), a- = a+. */
void ko_iir1d(const double *x, long n, long sx, double *y, long sy, int K,
              double b0, const double *bplus, const double *aplus, double sym,
              int boundary);

/* Non-recursive symmetric FIR, eq (A5), taps h[0..K] with h(-m) = h(m). */
void ko_fir1d(const double *x, long n, long sx, double *y, long sy, int K,
              const double *h, int boundary);

/* ---- the filter bank and detector (Sec. 5) ----------------------------- */

#define KO_IIR_REPEATED_POLE 0 /* Filter D */
#define KO_IIR_BUTTERWORTH 1   /* Filter E */
#define KO_FIR_COLORED_SG 2    /* Filter C */
#define KO_FIR_GAUSSIAN 3      /* Filter A */

#define KO_RESP_LAPLACIAN 0 /* R_L = -sigma^2 (D20 + D02) */
#define KO_RESP_HESSIAN 1   /* R_H = sigma^4 (D20 D02 - D11^2), eq (26) */

/* One frame (H x W, row-major, pitch = W), nscales blob scales lambda_s
 * (sigma_s = lambda_s / 2).  For each scale: separable blur of the frame
 * extended by the boundary rule (rows, then columns), derivative bank of
 * Table I / Sec. 5, response.  R receives nscales*H*W values.  If D is not
 * NULL it receives 5*nscales*H*W values, ordered (scale, which, y, x) with
 * which = D10, D01, D20, D02, D11.  fir_kmax caps the colored-SG length.
 * For the colored SG, taps (nscales rows of tap_stride doubles, h[0..tapK[s]])
 * may be given by the caller (the high-precision design of oracle.py);
 * NULL designs them here in FP64.  Returns 0, or -1 if a design fails. */
int ko_bank(const double *img, int H, int W, int nscales, const double *lambdas,
            int type, int order, int resp, int boundary, int fir_kmax,
            const double *taps, const int *tapK, int tap_stride, double *R,
            double *D);

/* Threads the oracle's parallel loops use (OpenMP; 1 without it). */
int ko_threads(void);

/* Offsets of eq (27) and |H| of eq (26) from the five derivatives. */
void ko_eq27(double d10, double d01, double d20, double d02, double d11,
             double *dx, double *dy, double *det);

/* Blob record of the detector. */
typedef struct {
  int frame, x, y, scale;
  int polarity;      /* +1 bright (maximum), -1 dark (minimum) */
  double response;   /* R at the pixel */
  double dx, dy;     /* eq (27) offsets (0 when D is not given) */
  double det;        /* |H| of eq (26) (0 when D is not given) */
} ko_blob;

#define KO_NEIGH_ALL_SCALES 0 /* 3 x 3 x S */
#define KO_NEIGH_ADJACENT 1   /* 3 x 3 x 3 */

/* Scale-space extremum detector over the R stack (nscales x H x W).
 * Bright: R > T and R beats every in-frame neighbour; dark (Laplacian
 * response only): R < -T and R is beaten by every neighbour.  A neighbour
 * earlier in (scale, y, x) order must be beaten strictly, a later one
 * non-strictly.  If D is given and limit2 > 0, Threshold #2 of eq (27) keeps
 * only candidates with sqrt(dx^2+dy^2) <= limit2.  Blobs are written in
 * (scale, y, x) order; returns the total count (may exceed cap; only the
 * first cap records are written). */
long ko_detect(const double *R, const double *D, int nscales, int H, int W,
               double T, int resp, int neigh, double limit2, int frame,
               ko_blob *out, long cap);

#ifdef __cplusplus
}
#endif
#endif
