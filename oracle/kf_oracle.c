/*
 * kf_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see the
 * header).  Kennedy, "Digital filters with vanishing moments for shape
 * analysis", arXiv:1912.07133.  Citations name the paper's section, equation
 * or table.
 */
#include "kf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ======================================================================= */
/* small helpers                                                            */
/* ======================================================================= */

static double binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
  return r;
}

/* Laurent polynomial product: c (2(Ka+Kb)+1) = a (2Ka+1) * b (2Kb+1). */
static void laurent_mul(const double *a, int Ka, const double *b, int Kb,
                        double *c) {
  int Kc = Ka + Kb;
  for (int i = 0; i < 2 * Kc + 1; ++i) c[i] = 0.0;
  for (int i = 0; i < 2 * Ka + 1; ++i)
    for (int j = 0; j < 2 * Kb + 1; ++j) c[i + j] += a[i] * b[j];
}

double ko_eulerian(int n, int k) {
  /* <n,k> = (k+1)<n-1,k> + (n-k)<n-1,k-1>, with <1,0> = 1. */
  if (n == 0) return k == 0 ? 1.0 : 0.0;
  if (k < 0 || k >= n || n > 60) return 0.0;
  double row[64], nxt[64];
  memset(row, 0, sizeof row);
  row[0] = 1.0; /* n = 1 */
  for (int r = 2; r <= n; ++r) {
    memset(nxt, 0, sizeof nxt);
    for (int j = 0; j < r; ++j) {
      double keep = (j < r - 1) ? row[j] : 0.0;
      double rise = (j >= 1) ? row[j - 1] : 0.0;
      nxt[j] = (double)(j + 1) * keep + (double)(r - j) * rise;
    }
    memcpy(row, nxt, sizeof row);
  }
  return row[k];
}

double ko_li_neg(int n, double z) {
  /* sum_{m>=1} m^n z^m = z A_n(z) / (1-z)^(n+1), A_0 = 1. */
  double A = 0.0, zk = 1.0;
  if (n == 0) A = 1.0;
  else
    for (int k = 0; k < n; ++k) {
      A += ko_eulerian(n, k) * zk;
      zk *= z;
    }
  return z * A / pow(1.0 - z, (double)(n + 1));
}

int ko_solve(int n, double *A, double *b) {
  double *rs = malloc(sizeof(double) * n), *cs = malloc(sizeof(double) * n);
  int rc = 0;
  /* equilibrate rows, then columns */
  for (int i = 0; i < n; ++i) {
    double m = 0.0;
    for (int j = 0; j < n; ++j) m = fmax(m, fabs(A[i * n + j]));
    rs[i] = m > 0 ? 1.0 / m : 1.0;
    for (int j = 0; j < n; ++j) A[i * n + j] *= rs[i];
    b[i] *= rs[i];
  }
  for (int j = 0; j < n; ++j) {
    double m = 0.0;
    for (int i = 0; i < n; ++i) m = fmax(m, fabs(A[i * n + j]));
    cs[j] = m > 0 ? 1.0 / m : 1.0;
    for (int i = 0; i < n; ++i) A[i * n + j] *= cs[j];
  }
  for (int k = 0; k < n; ++k) {
    int piv = k;
    double best = fabs(A[k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (fabs(A[i * n + k]) > best) best = fabs(A[i * n + k]), piv = i;
    if (best == 0.0) { rc = -1; goto done; }
    if (piv != k) {
      for (int j = 0; j < n; ++j) {
        double t = A[k * n + j]; A[k * n + j] = A[piv * n + j]; A[piv * n + j] = t;
      }
      double t = b[k]; b[k] = b[piv]; b[piv] = t;
    }
    for (int i = k + 1; i < n; ++i) {
      double f = A[i * n + k] / A[k * n + k];
      if (f == 0.0) continue;
      for (int j = k; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
      b[i] -= f * b[k];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int j = i + 1; j < n; ++j) s -= A[i * n + j] * b[j];
    b[i] = s / A[i * n + i];
  }
  for (int j = 0; j < n; ++j) b[j] *= cs[j];
done:
  free(rs); free(cs);
  return rc;
}

int ko_poly_roots(int d, const double *c, double *re, double *im) {
  /* Durand-Kerner on the monic polynomial, then Newton polish. */
  if (d < 1 || c[d] == 0.0) return -1;
  double mr[16], mi[16];
  if (d > 15) return -1;
  double cr[17];
  for (int i = 0; i <= d; ++i) cr[i] = c[i] / c[d];
  for (int k = 0; k < d; ++k) { /* (0.4 + 0.9i)^k */
    double r = 1.0, i0 = 0.0;
    for (int t = 0; t < k; ++t) {
      double nr = r * 0.4 - i0 * 0.9, ni = r * 0.9 + i0 * 0.4;
      r = nr; i0 = ni;
    }
    mr[k] = r; mi[k] = i0;
  }
  for (int it = 0; it < 2000; ++it) {
    double delta = 0.0;
    for (int k = 0; k < d; ++k) {
      /* p(x) by Horner */
      double pr = 1.0, pi = 0.0;
      for (int i = d - 1; i >= 0; --i) {
        double nr = pr * mr[k] - pi * mi[k] + cr[i];
        double ni = pr * mi[k] + pi * mr[k];
        pr = nr; pi = ni;
      }
      double qr = 1.0, qi = 0.0;
      for (int j = 0; j < d; ++j) {
        if (j == k) continue;
        double dr = mr[k] - mr[j], di = mi[k] - mi[j];
        double nr = qr * dr - qi * di, ni = qr * di + qi * dr;
        qr = nr; qi = ni;
      }
      double den = qr * qr + qi * qi;
      if (den == 0.0) den = 1e-300;
      double sr = (pr * qr + pi * qi) / den, si = (pi * qr - pr * qi) / den;
      mr[k] -= sr; mi[k] -= si;
      delta = fmax(delta, hypot(sr, si));
    }
    if (delta < 1e-15) break;
  }
  for (int k = 0; k < d; ++k) { /* Newton polish on the original polynomial */
    for (int it = 0; it < 5; ++it) {
      double pr = c[d], pi = 0.0, dr = 0.0, di = 0.0;
      for (int i = d - 1; i >= 0; --i) {
        double ndr = dr * mr[k] - di * mi[k] + pr, ndi = dr * mi[k] + di * mr[k] + pi;
        dr = ndr; di = ndi;
        double nr = pr * mr[k] - pi * mi[k] + c[i], ni = pr * mi[k] + pi * mr[k];
        pr = nr; pi = ni;
      }
      double den = dr * dr + di * di;
      if (den == 0.0) break;
      mr[k] -= (pr * dr + pi * di) / den;
      mi[k] -= (pi * dr - pr * di) / den;
    }
    re[k] = mr[k]; im[k] = mi[k];
  }
  return 0;
}

/* ======================================================================= */
/* Appendix (A13)-(A19): three-part decomposition                           */
/* ======================================================================= */

int ko_a17(int K, const double *b, const double *a, const double *aplus,
           double *btilde, double *a0circ, double *bplus, double *bminus,
           double *b0) {
  int M = 2 * K + 1;
  /* A^-(z) = A^+(1/z): a-_m = a+_m (symmetric responses, A19 text). */
  double ap_l[2 * KO_MAXK + 1], am_l[2 * KO_MAXK + 1], apm[4 * KO_MAXK + 1];
  if (K > KO_MAXK) return -1;
  for (int i = 0; i < M; ++i) ap_l[i] = am_l[i] = 0.0;
  for (int m = 0; m <= K; ++m) {
    ap_l[K - m] = aplus[m]; /* z^{-m} */
    am_l[K + m] = aplus[m]; /* z^{+m} */
  }
  laurent_mul(ap_l, K, am_l, K, apm); /* A^{+-} of eq (A18), powers -2K..2K */
  /* only powers -K..K are non-zero */
  double *apmK = apm + K; /* apmK[i] = coefficient of z^{i-K} */
  double a0pm = apmK[K];
  *a0circ = a[K] / a0pm;
  double *At = calloc((size_t)M * M, sizeof(double));
  /* columns 0..K-1: a0circ b+_{K-j} times A^-(z): rows (l - m) + K, value a-_l */
  for (int j = 0; j < K; ++j) {
    int m = K - j;
    for (int l = 0; l <= K; ++l) At[(l - m + K) * M + j] = aplus[l];
  }
  /* column K: b0circ times A^{+-}(z) */
  for (int i = 0; i < M; ++i) At[i * M + K] = apmK[i];
  /* columns K+m: a0circ b-_m times A^+(z): rows (m - l) + K, value a+_l */
  for (int m = 1; m <= K; ++m)
    for (int l = 0; l <= K; ++l) At[(m - l + K) * M + K + m] = aplus[l];
  for (int i = 0; i < M; ++i) btilde[i] = b[i];
  int rc = ko_solve(M, At, btilde);
  free(At);
  if (rc) return rc;
  bplus[0] = bminus[0] = 0.0;
  for (int m = 1; m <= K; ++m) {
    bplus[m] = btilde[K - m] / *a0circ;
    bminus[m] = btilde[K + m] / *a0circ;
  }
  *b0 = btilde[K] / *a0circ;
  return 0;
}

/* ======================================================================= */
/* Filter D: repeated-pole IIR blur, Sec. 4.3                               */
/* ======================================================================= */

int ko_design_repeated_pole(int L_D, int Lpi, double sigma, double *b0,
                            double *bplus, double *aplus, double *c) {
  if (!(sigma > 0.0) || L_D < 1 || Lpi < 0) return -1;
  const double p = exp(-1.0 / sigma);          /* p = e^{-1/sigma} */
  const int K = L_D + Lpi;                     /* K^lpf = L_D + Lpi */
  const int Ldc = L_D + 1;                     /* d = 0: L_D - Delta_d + 1 */
  const int NK = Ldc + Lpi;                    /* eq (13)-(14) sizes */
  if (K > KO_MAXK) return -1;
  /* F of eq (14)-(15): rows l = 2*lbar; basis k < NK-1 is |m|^k p^|m|
   * (eq 23), basis NK-1 is the unit impulse.  The l-th derivative of
   * F_k(w) = sum_m f_k(m) e^{-imw} at w = 0 is sum_m (-im)^l f_k(m), and at
   * w = pi it is sum_m (-im)^l (-1)^m f_k(m). */
  double *F = calloc((size_t)NK * NK, sizeof(double));
  double rho[32];
  for (int r = 0; r < NK; ++r) rho[r] = 0.0;
  rho[0] = 1.0; /* rho^dc_{0,0} = i^0 0! */
  for (int r = 0; r < NK; ++r) {
    int at_pi = r >= Ldc;
    int lbar = at_pi ? r - Ldc : r;
    int l = 2 * lbar;
    double sgn = (lbar % 2) ? -1.0 : 1.0; /* (-i)^l for even l */
    double z = at_pi ? -p : p;
    for (int k = 0; k < NK; ++k) {
      double v;
      if (k == NK - 1) v = (l == 0) ? 1.0 : 0.0; /* unit impulse */
      else {
        v = 2.0 * ko_li_neg(k + l, z);               /* m != 0, both sides */
        if (k == 0 && l == 0) v += 1.0;              /* f_0(0) = 1 */
      }
      F[r * NK + k] = sgn * v;
    }
  }
  double cc[32];
  for (int r = 0; r < NK; ++r) cc[r] = rho[r];
  int rc = ko_solve(NK, F, cc);
  free(F);
  if (rc) return -1;
  if (c)
    for (int k = 0; k < NK; ++k) c[k] = cc[k];
  /* The DE of eq (A10): A+(z) = (1 - p z^-1)^K (the K-fold pole of eq 23b);
   * the causal part B+(z)/A+(z) is the one-sided IR h(m), m >= 1, of eq (12a),
   * so B+ = A+ . H+ truncated to degree K; the centre term is h(0).  In exact
   * arithmetic this equals rearranging eq (12b) to B(z)/A(z) and solving eq
   * (A17); in FP64 that route cancels B(1) ~ (1-p)^{2K} and loses up to six
   * digits at coarse scale, so the IR route is used (ko_a17 stays available
   * and is cross-checked against it where it is well conditioned). */
  double hm[KO_MAXK + 1];
  for (int m = 0; m <= K; ++m) {
    double v = 0.0;
    for (int k = 0; k < NK - 1; ++k)
      v += cc[k] * (m == 0 ? (k == 0 ? 1.0 : 0.0) : pow((double)m, k)) * pow(p, m);
    if (m == 0) v += cc[NK - 1]; /* unit impulse */
    hm[m] = v;
  }
  for (int m = 0; m <= K; ++m) aplus[m] = binom(K, m) * pow(-p, m);
  *b0 = hm[0];
  bplus[0] = 0.0;
  for (int m = 1; m <= K; ++m) {
    double v = 0.0;
    for (int j = 0; j < m; ++j) v += aplus[j] * hm[m - j];
    bplus[m] = v;
  }
  return K;
}

/* ======================================================================= */
/* Filter E: discrete Butterworth IIR blur, Sec. 4.4                        */
/* ======================================================================= */

int ko_design_butterworth(int L_D, double sigma, double *b0, double *bplus,
                          double *aplus, double *omega_c_out) {
  if (!(sigma > 0.0) || L_D < 1) return -1;
  const int LB = 2 * (L_D + 1);
  const int n = LB / 2; /* exponent of (-s^2/wc^2) in eq (25) */
  const int K = n;      /* K^lpf = L_D + 1 */
  if (K > KO_MAXK) return -1;
  const double wc = sqrt(2.0 * log(2.0)) / sigma;
  if (omega_c_out) *omega_c_out = wc;
  /* s = 2(z-1)/(z+1): H = wc^{2n}(z+1)^{2n} / (wc^{2n}(z+1)^{2n} + (-4)^n (z-1)^{2n});
   * numerator and denominator times z^{-n} give Laurent polynomials. */
  double a[2 * KO_MAXK + 1];
  double wpow = pow(wc, 2.0 * n), m4 = pow(-4.0, n);
  for (int j = 0; j <= 2 * n; ++j) { /* coefficient of z^{j-n} */
    double cp = binom(2 * n, j);                          /* (z+1)^{2n} */
    double cm = binom(2 * n, j) * (((2 * n - j) % 2) ? -1.0 : 1.0); /* (z-1)^{2n} */
    a[j] = wpow * cp + m4 * cm; /* numerator: wpow * cp */
  }
  /* Poles (eq A19 roots inside the unit circle): 1 + (-s^2/wc^2)^n = 0 gives
   * s = +-i wc e^{i pi (2k+1)/(2n)}; the left-half-plane ones map to |z| < 1
   * under z = (2+s)/(2-s), the inverse of s = 2(z-1)/(z+1). */
  double pr[KO_MAXK + 1], pi_[KO_MAXK + 1];
  int cnt = 0;
  for (int k = 0; k < n; ++k)
    for (int sg = -1; sg <= 1; sg += 2) {
      double th = M_PI * (2.0 * k + 1.0) / (2.0 * n);
      double sr = -sg * wc * sin(th), si = sg * wc * cos(th); /* +-i wc e^{i th} */
      if (sr >= 0.0) continue;
      double nr = 2.0 + sr, ni = si, dr = 2.0 - sr, di = -si;
      double den = dr * dr + di * di;
      if (cnt >= K) return -1;
      pr[cnt] = (nr * dr + ni * di) / den;
      pi_[cnt] = (ni * dr - nr * di) / den;
      ++cnt;
    }
  if (cnt != K) return -1;
  /* A+(z) = prod (1 - p_i z^-1) */
  double cr[KO_MAXK + 1], ci[KO_MAXK + 1];
  for (int i = 0; i <= K; ++i) cr[i] = ci[i] = 0.0;
  cr[0] = 1.0;
  for (int r = 0; r < K; ++r) {
    for (int i = r + 1; i >= 1; --i) {
      double nr = cr[i] - (pr[r] * cr[i - 1] - pi_[r] * ci[i - 1]);
      double ni = ci[i] - (pr[r] * ci[i - 1] + pi_[r] * cr[i - 1]);
      cr[i] = nr; ci[i] = ni;
    }
  }
  for (int i = 0; i <= K; ++i) aplus[i] = cr[i]; /* imaginary parts cancel */
  /* Causal IR h(m) = sum_i rho_i p_i^m (m >= 1) with p_i rho_i the residue of
   * H(z) = z^n B(z) / (z^n A(z)) at p_i.  Then, as for Filter D,
   * B+ = A+ . H+ truncated and h(0) = H(1) - 2 sum_{m>=1} h(m), H(1) = 1. */
  double rr[KO_MAXK + 1], ri[KO_MAXK + 1];
  for (int i = 0; i < K; ++i) {
    /* numerator z^n B(z) = wc^{2n} (z+1)^{2n}; denominator derivative from its
     * 2n roots: all poles of z^n A(z) are the images of the 2n s-poles. */
    double zr = pr[i], zi = pi_[i];
    double numr = 1.0, numi = 0.0, ur = zr + 1.0, ui = zi;
    for (int t = 0; t < 2 * n; ++t) {
      double tr = numr * ur - numi * ui, ti = numr * ui + numi * ur;
      numr = tr; numi = ti;
    }
    numr *= wpow; numi *= wpow;
    /* derivative of lead * prod_j (z - z_j) at z_i: lead * prod_{j != i} (z_i - z_j);
     * the outer poles are 1/conj-pairs of the inner ones: z_j^out = 1 / z_j. */
    double lead = a[2 * n];
    double dr_ = lead, di_ = 0.0;
    for (int j = 0; j < K; ++j) {
      double qr, qi;
      if (j != i) {
        qr = zr - pr[j]; qi = zi - pi_[j];
        double tr = dr_ * qr - di_ * qi, ti = dr_ * qi + di_ * qr;
        dr_ = tr; di_ = ti;
      }
      double den = pr[j] * pr[j] + pi_[j] * pi_[j];
      double or_ = pr[j] / den, oi = -pi_[j] / den; /* 1 / p_j */
      qr = zr - or_; qi = zi - oi;
      double tr = dr_ * qr - di_ * qi, ti = dr_ * qi + di_ * qr;
      dr_ = tr; di_ = ti;
    }
    double den = dr_ * dr_ + di_ * di_;
    double resr = (numr * dr_ + numi * di_) / den, resi = (numi * dr_ - numr * di_) / den;
    double zden = zr * zr + zi * zi; /* rho_i = residue / p_i */
    rr[i] = (resr * zr + resi * zi) / zden;
    ri[i] = (resi * zr - resr * zi) / zden;
  }
  double hm[KO_MAXK + 1], tail = 0.0;
  for (int m = 1; m <= K; ++m) {
    double v = 0.0;
    for (int i = 0; i < K; ++i) {
      /* Re(rho_i p_i^m) */
      double wr = 1.0, wi = 0.0;
      for (int t = 0; t < m; ++t) {
        double tr = wr * pr[i] - wi * pi_[i], ti = wr * pi_[i] + wi * pr[i];
        wr = tr; wi = ti;
      }
      v += rr[i] * wr - ri[i] * wi;
    }
    hm[m] = v;
  }
  for (int i = 0; i < K; ++i) { /* sum_{m>=1} rho_i p_i^m = rho_i p_i / (1 - p_i) */
    double nr = rr[i] * pr[i] - ri[i] * pi_[i], ni = rr[i] * pi_[i] + ri[i] * pr[i];
    double dr2 = 1.0 - pr[i], di2 = -pi_[i], den = dr2 * dr2 + di2 * di2;
    tail += (nr * dr2 + ni * di2) / den;
  }
  *b0 = 1.0 - 2.0 * tail;
  bplus[0] = 0.0;
  for (int m = 1; m <= K; ++m) {
    double v = 0.0;
    for (int j = 0; j < m; ++j) v += aplus[j] * hm[m - j];
    bplus[m] = v;
  }
  return K;
}

/* ======================================================================= */
/* Filter C: colored Savitzky-Golay FIR blur, Sec. 4.2                      */
/* ======================================================================= */

int ko_design_colored_sg_raw(int L_D, int K, double wc, double *h) {
  if (K < L_D || L_D < 1 || wc < 0.0 || wc >= M_PI) return -1;
  const int M = 2 * K + 1;
  const int NK = K + 1;
  const int Ldc = L_D + 1;
  /* S-bar of eq (22b), indexed by m1 + K, m2 + K */
  double *Sb = malloc(sizeof(double) * M * M);
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < M; ++j) {
      int dlt = i - j;
      Sb[i * M + j] = dlt == 0
                          ? (M_PI - wc) / M_PI
                          : (sin(M_PI * dlt) / dlt - sin(wc * dlt) / dlt) / M_PI;
    }
  /* S = T Sbar T^T with T_{k, K+m} = delta_{k,|m|} (eq 22c) */
  const int N = NK + Ldc;
  double *A = calloc((size_t)N * N, sizeof(double));
  double *rhs = calloc((size_t)N, sizeof(double));
  for (int k1 = 0; k1 < NK; ++k1)
    for (int k2 = 0; k2 < NK; ++k2) {
      double s = 0.0;
      for (int s1 = -1; s1 <= 1; s1 += 2) {
        if (k1 == 0 && s1 == 1) continue;
        for (int s2 = -1; s2 <= 1; s2 += 2) {
          if (k2 == 0 && s2 == 1) continue;
          s += Sb[(K + s1 * k1) * M + (K + s2 * k2)];
        }
      }
      A[k1 * N + k2] = s;
    }
  /* F^dc of the pure-delay basis (eq 16c-d): 2 mu_k (-1)^lbar k^{2 lbar} */
  for (int lb = 0; lb < Ldc; ++lb)
    for (int k = 0; k < NK; ++k) {
      double mu = (k == 0) ? 0.5 : 1.0;
      double kp = (lb == 0) ? 1.0 : pow((double)k, 2.0 * lb);
      double v = 2.0 * mu * ((lb % 2) ? -1.0 : 1.0) * kp;
      A[(NK + lb) * N + k] = v;      /* F   */
      A[k * N + (NK + lb)] = v;      /* F^T */
    }
  rhs[NK] = 1.0; /* rho^dc = e_0 */
  int rc = ko_solve(N, A, rhs);      /* eq (20) */
  if (!rc)
    for (int k = 0; k < NK; ++k) h[k] = rhs[k]; /* h(0)=c_0, h(+-k)=c_k */
  free(Sb); free(A); free(rhs);
  return rc ? -1 : K;
}

int ko_design_colored_sg(int L_D, double sigma, int Kmax, double *h) {
  if (!(sigma > 0.0) || (L_D != 1 && L_D != 2)) return -1;
  double wc = 3.0 / sigma;
  if (wc >= M_PI) return -1;
  int K = (int)ceil((L_D == 1 ? 5.0 : 7.0) * sigma);
  if (Kmax > 0 && K > Kmax) K = Kmax;
  return ko_design_colored_sg_raw(L_D, K, wc, h);
}

/* ======================================================================= */
/* 1-D realisations, Appendix A4-A10 and A32                                */
/* ======================================================================= */

void ko_iir1d(const double *x, long n, long sx, double *y, long sy, int K,
              double b0, const double *bplus, const double *aplus, double sym,
              int boundary) {
  double *yp = malloc(sizeof(double) * (n > 0 ? n : 1));
  double *ym = malloc(sizeof(double) * (n > 0 ? n : 1));
  /* steady-state gain of each one-sided part: B(1)/A(1) */
  double sb = 0.0, sa = 0.0;
  for (int m = 1; m <= K; ++m) sb += bplus[m];
  for (int m = 0; m <= K; ++m) sa += aplus[m];
  double gp = sb / sa, gm = sym * sb / sa;
  double x0 = 0.0, xN = 0.0;
  if (n > 0 && boundary == KO_BOUNDARY_HOLD) {
    x0 = x[0];
    xN = x[(n - 1) * sx];
  }
  /* (A10a) forward/causal: y+(i) = sum b+_m x(i-m) - sum a+_m y+(i-m);
   * outside the frame x = x0 and y+ = its steady state (A32). */
  for (long i = 0; i < n; ++i) {
    double s = 0.0;
    for (int m = 1; m <= K; ++m) {
      long j = i - m;
      double xv = j >= 0 ? x[j * sx] : x0;
      double yv = j >= 0 ? yp[j] : x0 * gp;
      s += bplus[m] * xv - aplus[m] * yv;
    }
    yp[i] = s;
  }
  /* (A10b) backward/anticausal, b-_m = sym b+_m, a-_m = a+_m */
  for (long i = n - 1; i >= 0; --i) {
    double s = 0.0;
    for (int m = 1; m <= K; ++m) {
      long j = i + m;
      double xv = j < n ? x[j * sx] : xN;
      double yv = j < n ? ym[j] : xN * gm;
      s += sym * bplus[m] * xv - aplus[m] * yv;
    }
    ym[i] = s;
  }
  /* (A6), (A10c) */
  for (long i = 0; i < n; ++i) y[i * sy] = yp[i] + ym[i] + b0 * x[i * sx];
  free(yp); free(ym);
}

void ko_fir1d(const double *x, long n, long sx, double *y, long sy, int K,
              const double *h, int boundary) {
  /* (A5): y(i) = sum_{m=-K..K} b_m x(i-m), b_m = h(|m|) */
  for (long i = 0; i < n; ++i) {
    double s = 0.0;
    for (int m = -K; m <= K; ++m) {
      long j = i - m;
      double xv;
      if (j >= 0 && j < n) xv = x[j * sx];
      else if (boundary == KO_BOUNDARY_HOLD) xv = x[(j < 0 ? 0 : n - 1) * sx];
      else xv = 0.0;
      s += h[m < 0 ? -m : m] * xv;
    }
    y[i * sy] = s;
  }
}

/* Filter A: eq 9 (d = 0) sampled at T_s = 1, renormalised by eq 11. */
int ko_design_gaussian(double sigma, int fir_kmax, double *h) {
  if (!(sigma > 0.0)) return -1;
  int K = (int)ceil(5.0 * sigma);
  if (fir_kmax > 0 && K > fir_kmax) K = fir_kmax;
  const double norm = 1.0 / (sigma * sqrt(2.0 * M_PI));
  double dc = 0.0; /* H0 at dc of the sampled prototype: sum over m = -K..K */
  for (int m = 0; m <= K; ++m) {
    h[m] = norm * exp(-(double)m * (double)m / (2.0 * sigma * sigma));
    dc += m == 0 ? h[m] : 2.0 * h[m];
  }
  const double cg = 1.0 / dc; /* eq 11 */
  for (int m = 0; m <= K; ++m) h[m] *= cg;
  return K;
}

/* ======================================================================= */
/* Filter bank (Sec. 5)                                                      */
/* ======================================================================= */

typedef struct {
  int type, K;
  double b0, bplus[KO_MAXK + 1], aplus[KO_MAXK + 1];
  double *h; /* FIR taps */
} design_t;

static int make_design(int type, int order, double sigma, int fir_kmax,
                       const double *taps, int tapK, design_t *d) {
  d->type = type;
  d->h = NULL;
  if (type == KO_FIR_COLORED_SG && taps) { /* taps designed by the caller */
    d->K = tapK;
    d->h = malloc(sizeof(double) * (tapK + 1));
    memcpy(d->h, taps, sizeof(double) * (tapK + 1));
    return 0;
  }
  if (type == KO_IIR_REPEATED_POLE) {
    /* order = K^lpf = L_D + Lpi with L_D = 1 (D = 3) */
    d->K = ko_design_repeated_pole(1, order - 1, sigma, &d->b0, d->bplus,
                                   d->aplus, NULL);
  } else if (type == KO_IIR_BUTTERWORTH) {
    /* order = L_B / 2 = L_D + 1 */
    d->K = ko_design_butterworth(order - 1, sigma, &d->b0, d->bplus, d->aplus,
                                 NULL);
  } else if (type == KO_FIR_COLORED_SG) {
    int cap = (int)ceil((order == 2 ? 7.0 : 5.0) * sigma);
    if (fir_kmax > 0 && cap > fir_kmax) cap = fir_kmax;
    d->h = malloc(sizeof(double) * (cap + 1));
    d->K = ko_design_colored_sg(order, sigma, fir_kmax, d->h);
  } else if (type == KO_FIR_GAUSSIAN) {
    int cap = (int)ceil(5.0 * sigma);
    if (fir_kmax > 0 && cap > fir_kmax) cap = fir_kmax;
    d->h = malloc(sizeof(double) * (cap + 1));
    d->K = ko_design_gaussian(sigma, fir_kmax, d->h);
  } else
    d->K = -1;
  return d->K < 0 ? -1 : 0;
}

static void filt1d(const design_t *d, const double *x, long n, long sx,
                   double *y, long sy, int boundary) {
  if (d->type == KO_FIR_COLORED_SG || d->type == KO_FIR_GAUSSIAN) ko_fir1d(x, n, sx, y, sy, d->K, d->h, boundary);
  else ko_iir1d(x, n, sx, y, sy, d->K, d->b0, d->bplus, d->aplus, 1.0, boundary);
}

int ko_bank(const double *img, int H, int W, int nscales, const double *lambdas,
            int type, int order, int resp, int boundary, int fir_kmax,
            const double *taps, const int *tapK, int tap_stride, double *R,
            double *D) {
  const long Hp = H + 2, Wp = W + 2;
  /* frame extended by one pixel on each side by the boundary rule */
  double *P = malloc(sizeof(double) * Hp * Wp);
  for (long y = 0; y < Hp; ++y)
    for (long x = 0; x < Wp; ++x) {
      long yy = y - 1, xx = x - 1;
      int out = yy < 0 || yy >= H || xx < 0 || xx >= W;
      if (out && boundary == KO_BOUNDARY_ZERO) { P[y * Wp + x] = 0.0; continue; }
      yy = yy < 0 ? 0 : (yy >= H ? H - 1 : yy);
      xx = xx < 0 ? 0 : (xx >= W ? W - 1 : xx);
      P[y * Wp + x] = img[yy * (long)W + xx];
    }
  double *T = malloc(sizeof(double) * Hp * Wp);
  double *B = malloc(sizeof(double) * Hp * Wp);
  int status = 0;
  for (int s = 0; s < nscales && !status; ++s) {
    double sigma = lambdas[s] / 2.0; /* lambda = 2 sigma (Sec. 5) */
    design_t d;
    if (make_design(type, order, sigma, fir_kmax,
                    taps ? taps + (long)s * tap_stride : NULL, taps ? tapK[s] : 0, &d)) {
      status = -1;
      break;
    }
    /* rows (x) then columns (y) */
#pragma omp parallel for schedule(static)
    for (long y = 0; y < Hp; ++y) filt1d(&d, P + y * Wp, Wp, 1, T + y * Wp, 1, boundary);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < Wp; ++x) filt1d(&d, T + x, Hp, Wp, B + x, Wp, boundary);
    free(d.h);
    /* derivative bank (Table I, Sec. 5) and response */
    double s2 = sigma * sigma;
#pragma omp parallel for schedule(static)
    for (long y = 0; y < H; ++y)
      for (long x = 0; x < W; ++x) {
        const double *c = B + (y + 1) * Wp + (x + 1);
        double d10 = 0.5 * (c[1] - c[-1]);
        double d01 = 0.5 * (c[Wp] - c[-Wp]);
        double d20 = c[1] - 2.0 * c[0] + c[-1];
        double d02 = c[Wp] - 2.0 * c[0] + c[-Wp];
        double d11 = 0.25 * (c[Wp + 1] - c[Wp - 1] - c[-Wp + 1] + c[-Wp - 1]);
        double r = resp == KO_RESP_HESSIAN ? s2 * s2 * (d20 * d02 - d11 * d11)
                                           : -s2 * (d20 + d02);
        R[((long)s * H + y) * W + x] = r;
        if (D) {
          long base = ((long)s * 5) * H * W + y * (long)W + x;
          long pl = (long)H * W;
          D[base + 0 * pl] = d10;
          D[base + 1 * pl] = d01;
          D[base + 2 * pl] = d20;
          D[base + 3 * pl] = d02;
          D[base + 4 * pl] = d11;
        }
      }
  }
  free(P); free(T); free(B);
  return status;
}

/* ======================================================================= */
/* Detector (Sec. 5, eqs 26-27)                                             */
/* ======================================================================= */

void ko_eq27(double d10, double d01, double d20, double d02, double d11,
             double *dx, double *dy, double *det) {
  *det = d20 * d02 - d11 * d11;          /* |H| of eq (26) */
  *dx = (d01 * d11 - d02 * d10) / *det;  /* eq (27a) */
  *dy = (d10 * d11 - d20 * d01) / *det;  /* eq (27b) */
}

int ko_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

long ko_detect(const double *R, const double *D, int S, int H, int W, double T,
               int resp, int neigh, double limit2, int frame, ko_blob *out,
               long cap) {
  long count = 0;
  const long plane = (long)H * W;
  for (int s = 0; s < S; ++s)
    for (int y = 0; y < H; ++y)
      for (int x = 0; x < W; ++x) {
        double v = R[s * plane + (long)y * W + x];
        int pol = 0;
        if (v > T) pol = 1;
        else if (resp == KO_RESP_LAPLACIAN && v < -T) pol = -1;
        if (!pol) continue;
        int s_lo = neigh == KO_NEIGH_ADJACENT ? s - 1 : 0;
        int s_hi = neigh == KO_NEIGH_ADJACENT ? s + 1 : S - 1;
        int ok = 1;
        for (int t = s_lo; t <= s_hi && ok; ++t) {
          if (t < 0 || t >= S) continue;
          for (int yy = y - 1; yy <= y + 1 && ok; ++yy) {
            if (yy < 0 || yy >= H) continue;
            for (int xx = x - 1; xx <= x + 1 && ok; ++xx) {
              if (xx < 0 || xx >= W) continue;
              if (t == s && yy == y && xx == x) continue;
              double q = R[t * plane + (long)yy * W + xx];
              int earlier = t < s || (t == s && (yy < y || (yy == y && xx < x)));
              double a = pol * v, b = pol * q;
              ok = earlier ? (a > b) : (a >= b);
            }
          }
        }
        if (!ok) continue;
        double dx = 0.0, dy = 0.0, det = 0.0;
        if (D) {
          long base = ((long)s * 5) * plane + (long)y * W + x;
          double d10 = D[base], d01 = D[base + plane], d20 = D[base + 2 * plane];
          double d02 = D[base + 3 * plane], d11 = D[base + 4 * plane];
          ko_eq27(d10, d01, d20, d02, d11, &dx, &dy, &det);
          if (limit2 > 0.0 && !(sqrt(dx * dx + dy * dy) <= limit2)) continue;
        }
        if (count < cap) {
          ko_blob *b = out + count;
          b->frame = frame; b->x = x; b->y = y; b->scale = s;
          b->polarity = pol; b->response = v;
          b->dx = dx; b->dy = dy; b->det = det;
        }
        ++count;
      }
  return count;
}
