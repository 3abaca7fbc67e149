// kf_design.cu -- FP64 design of the blurs on the GPU (Kennedy,
// arXiv:1912.07133, Sec. 4) and their realisation for the FP32 filter
// kernels.  One CTA per scale.
#include <math.h>

#include "kf_common.cuh"
#include "kf_internal.h"

namespace kf {

namespace {

struct cd {
  double r, i;
};
__device__ inline cd cmul(cd a, cd b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
__device__ inline cd cdiv(cd a, cd b) {
  double d = b.r * b.r + b.i * b.i;
  return {(a.r * b.r + a.i * b.i) / d, (a.i * b.r - a.r * b.i) / d};
}
__device__ inline cd csub(cd a, cd b) { return {a.r - b.r, a.i - b.i}; }
__device__ inline cd cpow(cd z, long n) {
  cd r = {1.0, 0.0};
  while (n > 0) {
    if (n & 1) r = cmul(r, z);
    z = cmul(z, z);
    n >>= 1;
  }
  return r;
}

// Eulerian number <n,k> by the recurrence <n,k> = (k+1)<n-1,k> + (n-k)<n-1,k-1>.
__device__ double eulerian(int n, int k) {
  if (n == 0) return k == 0 ? 1.0 : 0.0;
  if (k < 0 || k >= n || n > 24) return 0.0;
  double row[25];
  for (int i = 0; i < 25; ++i) row[i] = 0.0;
  row[0] = 1.0;
  for (int r = 2; r <= n; ++r)
    for (int j = r - 1; j >= 0; --j) {
      double keep = (j < r - 1) ? row[j] : 0.0;
      double rise = (j >= 1) ? row[j - 1] : 0.0;
      row[j] = (double)(j + 1) * keep + (double)(r - j) * rise;
    }
  return row[k];
}

// sum_{m>=1} m^n z^m = z A_n(z) / (1 - z)^(n+1)  (|z| < 1)
__device__ double li_neg(int n, double z) {
  double A = (n == 0) ? 1.0 : 0.0, zk = 1.0;
  for (int k = 0; k < n; ++k) {
    A += eulerian(n, k) * zk;
    zk *= z;
  }
  return z * A / pow(1.0 - z, (double)(n + 1));
}

__device__ double binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
  return r;
}

// C(n, i) p^(n-i) without overflow for large n.
__device__ double binom_pow(long n, int i, double p) {
  if (i > n) return 0.0;
  double lc = lgamma((double)n + 1.0) - lgamma((double)i + 1.0) - lgamma((double)(n - i) + 1.0);
  return exp(lc + (double)(n - i) * log(p));
}

// Small dense solve, single thread: equilibrated Gaussian elimination with
// partial pivoting.  n <= 10.
__device__ int solve_small(int n, double *A, double *b) {
  double rs[10], cs[10];
  for (int i = 0; i < n; ++i) {
    double m = 0.0;
    for (int j = 0; j < n; ++j) m = fmax(m, fabs(A[i * n + j]));
    rs[i] = m > 0.0 ? 1.0 / m : 1.0;
    for (int j = 0; j < n; ++j) A[i * n + j] *= rs[i];
    b[i] *= rs[i];
  }
  for (int j = 0; j < n; ++j) {
    double m = 0.0;
    for (int i = 0; i < n; ++i) m = fmax(m, fabs(A[i * n + j]));
    cs[j] = m > 0.0 ? 1.0 / m : 1.0;
    for (int i = 0; i < n; ++i) A[i * n + j] *= cs[j];
  }
  for (int k = 0; k < n; ++k) {
    int piv = k;
    double best = fabs(A[k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (fabs(A[i * n + k]) > best) best = fabs(A[i * n + k]), piv = i;
    if (!(best > 0.0)) return -1;
    if (piv != k) {
      for (int j = 0; j < n; ++j) {
        double t = A[k * n + j];
        A[k * n + j] = A[piv * n + j];
        A[piv * n + j] = t;
      }
      double t = b[k];
      b[k] = b[piv];
      b[piv] = t;
    }
    for (int i = k + 1; i < n; ++i) {
      double f = A[i * n + k] / A[k * n + k];
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
  return 0;
}

// ---------------------------------------------------------------------------
// Filter D (Sec. 4.3): basis |m|^k p^|m| (k < N_K - 1) plus the unit impulse,
// constraints at dc (l = 0, 2, .., 2 L_D) and Nyquist (l = 0, 2, ..,
// 2(Lpi-1)) (eqs 13-15, 23-24), c = F^-1 rho, with order = K^lpf = L_D + Lpi.
// The pole used is the FP32-rounded p, so the realised recursion satisfies
// the constraints exactly.
// ---------------------------------------------------------------------------
__device__ void design_D(Coef &c, int order, double lambda, int ld) {
  const double sigma = lambda / 2.0;
  const int K = order, Ldc = ld + 1, NK = order + 1;
  if (!(sigma > 0.0) || ld < 1 || order < ld || order > MAXK) { c.status = 1; return; }
  const float pf = (float)exp(-1.0 / sigma);
  const double p = (double)pf, q = 1.0 - p;
  double F[10 * 10], cc[10];
  for (int r = 0; r < NK; ++r) {
    const bool at_pi = r >= Ldc;
    const int lbar = at_pi ? r - Ldc : r, l = 2 * lbar;
    const double sgn = (lbar & 1) ? -1.0 : 1.0, z = at_pi ? -p : p;
    for (int k = 0; k < NK; ++k) {
      double v;
      if (k == NK - 1) v = (l == 0) ? 1.0 : 0.0;
      else v = 2.0 * li_neg(k + l, z) + ((k == 0 && l == 0) ? 1.0 : 0.0);
      F[r * NK + k] = sgn * v;
    }
    cc[r] = (r == 0) ? 1.0 : 0.0;
  }
  if (solve_small(NK, F, cc)) { c.status = 2; return; }
  double hm[MAXK + 1];
  for (int m = 0; m <= K; ++m) {
    double v = 0.0;
    for (int k = 0; k < NK - 1; ++k) v += cc[k] * (m == 0 ? (k == 0 ? 1.0 : 0.0) : pow((double)m, k)) * pow(p, m);
    if (m == 0) v += cc[NK - 1];
    hm[m] = v;
  }
  // delayed chain: IR of t_j at lag n is C(n, j-1) p^(n-j+1); the output
  // sum_j w_j t_j(n-1) has IR sum_j w_j C(m-1, j-1) p^(m-j) at m >= 1.
  double w[MAXK + 1];
  for (int m = 1; m <= K; ++m) {
    double acc = hm[m];
    for (int j = 1; j < m; ++j) acc -= w[j] * binom(m - 1, j - 1) * pow(p, m - j);
    w[m] = acc;
  }
  double gplus = 0.0;  // one-sided dc gain: sum_j w_j / q^j
  for (int j = 1; j <= K; ++j) {
    c.w[j - 1] = (float)w[j];
    c.hold[j - 1] = (float)pow(q, -(double)j);
    gplus += w[j] * pow(q, -(double)j);
  }
  for (int i = 0; i < K; ++i) {
    for (int m = 1; m <= WARPM; ++m) c.phiM[m - 1][i] = (float)binom_pow((long)CH * m, i, p);
  }
  c.p = pf;
  c.b0 = (float)hm[0];
  c.db0 = hm[0];
  c.param = p;
  for (int m = 0; m <= K; ++m) c.daplus[m] = binom(K, m) * pow(-p, m);
  c.dbplus[0] = 0.0;
  for (int m = 1; m <= K; ++m) {
    double v = 0.0;
    for (int j = 0; j < m; ++j) v += c.daplus[j] * hm[m - j];
    c.dbplus[m] = v;
  }
  c.dc_gain = hm[0] + 2.0 * gplus;
  // second moment by direct summation of eq (12a)
  double m2 = 0.0;
  long M = (long)(80.0 * sigma) + 200;
  for (long m = 1; m <= M; ++m) {
    double v = 0.0, mk = 1.0;
    for (int k = 0; k < NK - 1; ++k) {
      v += cc[k] * mk;
      mk *= (double)m;
    }
    m2 += 2.0 * (double)m * (double)m * v * pow(p, (double)m);
  }
  c.moment2 = m2;
  c.K = K;
}

// ---------------------------------------------------------------------------
// Filter E (Sec. 4.4): H(s) = 1/(1 + (-s^2/wc^2)^n), n = L_B/2, bilinear
// s = 2(z-1)/(z+1), no pre-warp, wc = sqrt(2 ln 2)/sigma.  Poles inside the
// unit circle are the images of the left-half-plane s-poles; the one-sided
// IR is sum_i rho_i z_i^m with z_i rho_i the residue of H(z) at z_i.
// ---------------------------------------------------------------------------
__device__ void design_E(Coef &c, int order, double lambda) {
  const double sigma = lambda / 2.0;
  const int n = order;
  if (!(sigma > 0.0) || n < 1 || n > MAXK) { c.status = 1; return; }
  const double wc = sqrt(2.0 * log(2.0)) / sigma;
  cd z[MAXK];
  int cnt = 0;
  for (int k = 0; k < n; ++k)
    for (int sg = -1; sg <= 1; sg += 2) {
      const double th = M_PI * (2.0 * k + 1.0) / (2.0 * n);
      cd s = {-sg * wc * sin(th), sg * wc * cos(th)};  // sg * i * wc * e^{i th}
      if (s.r >= 0.0) continue;
      z[cnt++] = cdiv(cd{2.0 + s.r, s.i}, cd{2.0 - s.r, -s.i});
    }
  if (cnt != n) { c.status = 3; return; }
  const double w2n = pow(wc, 2.0 * n);
  const double lead = w2n + pow(-4.0, (double)n);
  cd rho[MAXK];
  for (int i = 0; i < n; ++i) {
    cd num = {1.0, 0.0};
    for (int t = 0; t < 2 * n; ++t) num = cmul(num, cd{z[i].r + 1.0, z[i].i});
    num.r *= w2n;
    num.i *= w2n;
    cd den = {lead, 0.0};
    for (int j = 0; j < n; ++j) {
      if (j != i) den = cmul(den, csub(z[i], z[j]));
      den = cmul(den, csub(z[i], cdiv(cd{1.0, 0.0}, z[j])));
    }
    rho[i] = cdiv(cdiv(num, den), z[i]);
  }
  double hm[MAXK + 1], gexact = 0.0;
  for (int m = 1; m <= n; ++m) {
    double v = 0.0;
    for (int i = 0; i < n; ++i) v += cmul(rho[i], cpow(z[i], m)).r;
    hm[m] = v;
  }
  for (int i = 0; i < n; ++i) gexact += cdiv(cmul(rho[i], z[i]), csub(cd{1.0, 0.0}, z[i])).r;
  hm[0] = 1.0 - 2.0 * gexact;  // H(1) = 1
  // modes: one per conjugate pair (factor 2) and one per real pole
  int nm = 0;
  double greal = 0.0;
  cd gm[MAXK], zm[MAXK];
  for (int i = 0; i < n; ++i) {
    if (z[i].i < -1e-12) continue;
    const bool real = fabs(z[i].i) <= 1e-12;
    cd zf = {(double)(float)z[i].r, real ? 0.0 : (double)(float)z[i].i};
    cd g = cmul(rho[i], z[i]);
    if (!real) g = cd{2.0 * g.r, 2.0 * g.i};
    else g.i = 0.0;
    zm[nm] = zf;
    gm[nm] = g;
    greal += cdiv(g, csub(cd{1.0, 0.0}, zf)).r;
    ++nm;
  }
  const double fix = gexact / greal;  // unity dc gain with the FP32 poles
  for (int i = 0; i < nm; ++i) {
    c.zr[i] = (float)zm[i].r;
    c.zi[i] = (float)zm[i].i;
    c.gr[i] = (float)(gm[i].r * fix);
    c.gi[i] = (float)(gm[i].i * fix);
    cd hh = cdiv(cd{1.0, 0.0}, csub(cd{1.0, 0.0}, zm[i]));
    c.hr[i] = (float)hh.r;
    c.hi[i] = (float)hh.i;
    for (int m = 1; m <= WARPM; ++m) {
      cd zs = cpow(zm[i], (long)CH * m);
      c.zMr[m - 1][i] = (float)zs.r;
      c.zMi[m - 1][i] = (float)zs.i;
    }
  }
  c.K = nm;
  c.b0 = (float)hm[0];
  c.db0 = hm[0];
  c.param = wc;
  // DE of eq (A10): A+(z) = prod (1 - z_i z^-1), B+ = A+ . H+ truncated
  cd ap[MAXK + 1];
  for (int i = 0; i <= n; ++i) ap[i] = cd{0.0, 0.0};
  ap[0] = cd{1.0, 0.0};
  for (int r = 0; r < n; ++r)
    for (int i = r + 1; i >= 1; --i) ap[i] = csub(ap[i], cmul(z[r], ap[i - 1]));
  for (int m = 0; m <= n; ++m) c.daplus[m] = ap[m].r;
  c.dbplus[0] = 0.0;
  for (int m = 1; m <= n; ++m) {
    double v = 0.0;
    for (int j = 0; j < m; ++j) v += c.daplus[j] * hm[m - j];
    c.dbplus[m] = v;
  }
  c.dc_gain = hm[0] + 2.0 * gexact;
  double rmax = 0.0;
  for (int i = 0; i < n; ++i) rmax = fmax(rmax, sqrt(z[i].r * z[i].r + z[i].i * z[i].i));
  long M = (long)(50.0 / (1.0 - rmax)) + 100;
  double m2 = 0.0;
  for (int i = 0; i < n; ++i) {
    cd zp = z[i];
    for (long m = 1; m <= M; ++m) {
      m2 += 2.0 * (double)m * (double)m * cmul(rho[i], zp).r;
      zp = cmul(zp, z[i]);
    }
  }
  c.moment2 = m2;
}

// ---------------------------------------------------------------------------
// double-double arithmetic (about 32 significant digits from FP64 pairs;
// error-free transformations of Knuth/Dekker, fma-based products)
// ---------------------------------------------------------------------------
struct dd {
  double hi, lo;
};
__device__ __forceinline__ dd two_sum(double a, double b) {
  const double s = __dadd_rn(a, b), bb = __dsub_rn(s, a);
  return {s, __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb))};
}
__device__ __forceinline__ dd quick_two_sum(double a, double b) {
  const double s = __dadd_rn(a, b);
  return {s, __dsub_rn(b, __dsub_rn(s, a))};
}
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi), t = two_sum(a.lo, b.lo);
  s.lo = __dadd_rn(s.lo, t.hi);
  s = quick_two_sum(s.hi, s.lo);
  s.lo = __dadd_rn(s.lo, t.lo);
  return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dd dd_neg(dd a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  const double p = __dmul_rn(a.hi, b.hi);
  double e = fma(a.hi, b.hi, -p);
  e = fma(a.hi, b.lo, e);
  e = fma(a.lo, b.hi, e);
  return quick_two_sum(p, e);
}
__device__ __forceinline__ dd dd_mul_d(dd a, double b) { return dd_mul(a, dd{b, 0.0}); }
__device__ dd dd_div(dd a, dd b) {
  const double q1 = a.hi / b.hi;
  dd r = dd_sub(a, dd_mul_d(b, q1));
  const double q2 = r.hi / b.hi;
  r = dd_sub(r, dd_mul_d(b, q2));
  const double q3 = r.hi / b.hi;
  dd q = quick_two_sum(q1, q2);
  return dd_add(q, dd{q3, 0.0});
}
__device__ __forceinline__ dd dd_from(double a) { return {a, 0.0}; }
__device__ __forceinline__ double dd_abs_hi(dd a) { return fabs(a.hi); }

// pi/2 and pi as double-double constants
__device__ __forceinline__ dd dd_pi2() { return {1.5707963267948966, 6.123233995736766e-17}; }
__device__ __forceinline__ dd dd_pi() { return {3.141592653589793, 1.2246467991473532e-16}; }

// sin of a double-double argument |x| < ~1e3: reduce by k pi/2 (Cody-Waite
// with the double-double pi/2), Taylor series on |r| <= pi/4.
__device__ dd dd_sin(dd x) {
  const double kf = rint(x.hi / 1.5707963267948966);
  const dd r = dd_sub(x, dd_mul_d(dd_pi2(), kf));
  const int q = ((long long)kf % 4 + 4) % 4;
  const dd r2 = dd_mul(r, r);
  dd s, c;
  {  // sin r = r - r^3/3! + ...
    dd term = r, sum = r;
    for (int n = 1; n < 20; ++n) {
      term = dd_div(dd_mul(term, r2), dd_from(-(double)(2 * n) * (double)(2 * n + 1)));
      sum = dd_add(sum, term);
      if (dd_abs_hi(term) < 1e-36) break;
    }
    s = sum;
  }
  {  // cos r = 1 - r^2/2! + ...
    dd term = dd_from(1.0), sum = dd_from(1.0);
    for (int n = 1; n < 20; ++n) {
      term = dd_div(dd_mul(term, r2), dd_from(-(double)(2 * n - 1) * (double)(2 * n)));
      sum = dd_add(sum, term);
      if (dd_abs_hi(term) < 1e-36) break;
    }
    c = sum;
  }
  switch (q) {
    case 0: return s;
    case 1: return c;
    case 2: return dd_neg(s);
    default: return dd_neg(c);
  }
}

// ---------------------------------------------------------------------------
// Filter C (Sec. 4.2): minimise (1/pi) int_wc^pi |H|^2 subject to the dc
// constraints (eq 20), pure-delay basis (eq 16), S = T Sbar T^T (eq 22).
// Near sigma = 1 (wc = 3 close to pi) the KKT matrix has a condition number
// of about 1e17, so the matrix is built and solved in double-double
// (equilibrated Gaussian elimination with partial pivoting, one CTA).
// A, b: N x N and N double-double entries of workspace (as 2 doubles each).
// ---------------------------------------------------------------------------
__device__ void design_C(Coef &c, int order, double lambda, int kmax, dd *A, dd *b, int Nmax) {
  const int tid = threadIdx.x, nt = blockDim.x;
  __shared__ int s_K, s_bad, s_piv;
  __shared__ double s_red[256];
  __shared__ int s_redi[256];
  const double sigma = lambda / 2.0;
  const int LD = order;
  if (tid == 0) {
    s_bad = 0;
    const double wc = 3.0 / sigma;
    if (!(sigma > 0.0) || (LD != 1 && LD != 2) || !(wc < M_PI)) s_bad = 1;
    int K = (int)ceil((LD == 1 ? 5.0 : 7.0) * sigma);
    if (kmax > 0 && K > kmax) K = kmax;
    if (K > MAX_FIR_K || K < LD) s_bad = 1;
    s_K = K;
  }
  __syncthreads();
  if (s_bad) {
    if (tid == 0) c.status = 1;
    return;
  }
  const int K = s_K, NK = K + 1, Ldc = LD + 1, N = NK + Ldc;
  if (N > Nmax) {
    if (tid == 0) c.status = 1;
    return;
  }
  // wc = 3 / sigma with sigma = lambda / 2 exact in binary: wc = 6 / lambda
  const dd wcd = dd_div(dd_from(6.0), dd_from(lambda));
  const dd pid = dd_pi();
  // Sbar(delta) of eq (22b): (sin(pi d) - sin(wc d)) / (pi d); sin(pi d) = 0
  // for integer d; the diagonal is (pi - wc) / pi.
  for (int idx = tid; idx < N * N; idx += nt) {
    const int i = idx / N, j = idx % N;
    dd v = dd_from(0.0);
    if (i < NK && j < NK) {
      for (int s1 = -1; s1 <= 1; s1 += 2) {
        if (i == 0 && s1 == 1) continue;
        for (int s2 = -1; s2 <= 1; s2 += 2) {
          if (j == 0 && s2 == 1) continue;
          const int d = s1 * i - s2 * j;
          dd t;
          if (d == 0) t = dd_div(dd_sub(pid, wcd), pid);
          else t = dd_neg(dd_div(dd_sin(dd_mul_d(wcd, (double)d)), dd_mul_d(pid, (double)d)));
          v = dd_add(v, t);
        }
      }
    } else if (i < NK || j < NK) {
      const int lb = (i < NK) ? j - NK : i - NK, k = (i < NK) ? i : j;
      const double mu = (k == 0) ? 0.5 : 1.0;
      const double kp = (lb == 0) ? 1.0 : pow((double)k, 2.0 * lb);  // exact integers
      v = dd_from(2.0 * mu * ((lb & 1) ? -1.0 : 1.0) * kp);
    }
    A[idx] = v;
  }
  for (int i = tid; i < N; i += nt) b[i] = dd_from((i == NK) ? 1.0 : 0.0);
  __syncthreads();
  // equilibrate rows and columns by powers of two (exact)
  for (int i = tid; i < N; i += nt) {
    double m = 0.0;
    for (int j = 0; j < N; ++j) m = fmax(m, fabs(A[i * N + j].hi));
    const double sc = m > 0.0 ? exp2(-(double)ilogb(m)) : 1.0;
    for (int j = 0; j < N; ++j) A[i * N + j] = dd_mul_d(A[i * N + j], sc);
    b[i] = dd_mul_d(b[i], sc);
  }
  __syncthreads();
  double *colscale = s_red;  // reused below only after this loop's last read
  __shared__ double s_cs[MAX_FIR_K + 8];
  for (int j = tid; j < N; j += nt) {
    double m = 0.0;
    for (int i = 0; i < N; ++i) m = fmax(m, fabs(A[i * N + j].hi));
    const double sc = m > 0.0 ? exp2(-(double)ilogb(m)) : 1.0;
    s_cs[j] = sc;
    for (int i = 0; i < N; ++i) A[i * N + j] = dd_mul_d(A[i * N + j], sc);
  }
  (void)colscale;
  __syncthreads();
  for (int k = 0; k < N; ++k) {
    double best = -1.0;
    int bi = k;
    for (int i = k + tid; i < N; i += nt) {
      const double a = fabs(A[i * N + k].hi);
      if (a > best) best = a, bi = i;
    }
    s_red[tid] = best;
    s_redi[tid] = bi;
    __syncthreads();
    for (int off = nt / 2; off > 0; off >>= 1) {
      if (tid < off && s_red[tid + off] > s_red[tid]) {
        s_red[tid] = s_red[tid + off];
        s_redi[tid] = s_redi[tid + off];
      }
      __syncthreads();
    }
    if (tid == 0) {
      s_piv = s_redi[0];
      if (!(s_red[0] > 0.0)) s_bad = 2;
    }
    __syncthreads();
    if (s_bad) break;
    const int piv = s_piv;
    if (piv != k) {
      for (int j = tid; j < N; j += nt) {
        const dd t = A[k * N + j];
        A[k * N + j] = A[piv * N + j];
        A[piv * N + j] = t;
      }
      if (tid == 0) {
        const dd t = b[k];
        b[k] = b[piv];
        b[piv] = t;
      }
    }
    __syncthreads();
    const dd akk = A[k * N + k];
    for (int i = k + 1 + tid; i < N; i += nt) {
      const dd f = dd_div(A[i * N + k], akk);
      if (f.hi != 0.0) {
        for (int j = k; j < N; ++j) A[i * N + j] = dd_sub(A[i * N + j], dd_mul(f, A[k * N + j]));
        b[i] = dd_sub(b[i], dd_mul(f, b[k]));
      }
    }
    __syncthreads();
  }
  if (s_bad) {
    if (tid == 0) c.status = 2;
    return;
  }
  for (int i = N - 1; i >= 0; --i) {
    if (tid == 0) b[i] = dd_div(b[i], A[i * N + i]);
    __syncthreads();
    const dd xi = b[i];
    for (int r = tid; r < i; r += nt) b[r] = dd_sub(b[r], dd_mul(A[r * N + i], xi));
    __syncthreads();
  }
  for (int k = tid; k < NK; k += nt) {
    const dd hk = dd_mul_d(b[k], s_cs[k]);
    c.dh[k] = hk.hi + hk.lo;
    c.h[k] = (float)(hk.hi + hk.lo);
  }
  __syncthreads();
  if (tid == 0) {
    double dc = c.dh[0], m2 = 0.0;
    for (int k = 1; k <= K; ++k) {
      dc += 2.0 * c.dh[k];
      m2 += 2.0 * (double)k * (double)k * c.dh[k];
    }
    c.dc_gain = dc;
    c.moment2 = m2;
    c.K = K;
    c.b0 = c.h[0];
    c.db0 = c.dh[0];
    c.param = wcd.hi;
  }
}

// Filter A (Sec. 3.1): eq 9 with d = 0, the Gaussian of standard deviation
// sigma sampled at the integers |m| <= K, K = ceil(5 sigma) capped at kmax, and
// renormalised to unit gain at dc by eq 11 (c_g = 1 / sum_m g0(m)).  One thread.
__device__ void design_A(Coef &c, double lambda, int kmax) {
  const double sigma = lambda / 2.0;
  int K = (int)ceil(5.0 * sigma);
  if (kmax > 0 && K > kmax) K = kmax;
  if (!(sigma > 0.0) || K < 1 || K > MAX_FIR_K) {
    c.status = 1;
    return;
  }
  const double norm = 1.0 / (sigma * sqrt(2.0 * M_PI));
  double dc = 0.0;
  for (int m = 0; m <= K; ++m) {
    c.dh[m] = norm * exp(-(double)m * (double)m / (2.0 * sigma * sigma));
    dc += m == 0 ? c.dh[m] : 2.0 * c.dh[m];
  }
  const double cg = 1.0 / dc;
  double dcg = 0.0, m2 = 0.0;
  for (int m = 0; m <= K; ++m) {
    c.dh[m] *= cg;
    c.h[m] = (float)c.dh[m];
    dcg += m == 0 ? c.dh[m] : 2.0 * c.dh[m];
    m2 += 2.0 * (double)m * (double)m * c.dh[m];
  }
  c.K = K;
  c.b0 = c.h[0];
  c.db0 = c.dh[0];
  c.dc_gain = dcg;
  c.moment2 = m2;
  c.param = sigma;
}

__global__ void __launch_bounds__(256) k_design(int type, int order, int ld, const double *lambdas,
                                                int fir_kmax, Coef *out, double *work,
                                                int Nmax) {
  const int s = blockIdx.x;
  Coef &c = out[s];
  const double lambda = lambdas[s];
  if (threadIdx.x == 0) {
    c.type = type;
    c.status = 0;
    c.lambda = lambda;
    c.sigma = lambda / 2.0;
    c.sigma2 = (float)(c.sigma * c.sigma);
    c.K = 0;
  }
  __syncthreads();
  if (type == T_C) {
    dd *A = reinterpret_cast<dd *>(work) + (size_t)s * ((size_t)Nmax * Nmax + Nmax);
    design_C(c, order, lambda, fir_kmax, A, A + (size_t)Nmax * Nmax, Nmax);
  } else if (threadIdx.x == 0) {
    if (type == T_D) design_D(c, order, lambda, ld);
    else if (type == T_E) design_E(c, order, lambda);
    else if (type == T_A) design_A(c, lambda, fir_kmax);
    else c.status = 1;
  }
}

}  // namespace

int launch_design(int type, int order, const double *d_lambdas, int S, int fir_kmax, Coef *d_out,
                  double *d_work, int Nmax, cudaStream_t st, int ld) {
  k_design<<<S, 256, 0, st>>>(type, order, ld, d_lambdas, fir_kmax, d_out, d_work, Nmax);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace kf
