// kf_deriv.cu -- response and detector of the derivative bank (Kennedy,
// arXiv:1912.07133, Sec. 5): the blurred derivatives D20, D02, D11 (and D10,
// D01 for the eq 27 offsets), each produced as its own channel by the row and
// column passes (Table I taps before the blur, planes sigma^2 D), are combined
// into R_H = sigma^4 (D20 D02 - D11^2) (eq 26) or R_L = -sigma^2 (D20 + D02),
// and the scale-space extremum detector runs on tiles of R.
#include <math_constants.h>

#include "kf_batch.cuh"
#include "kf_common.cuh"
#include "kf_detect.cuh"
#include "kf_internal.h"

namespace kf {

namespace {

constexpr int DT = 32;  // tile side with the 1-pixel halo (30 x 30 interior)

// Item: a 30 x 30 interior tile of a frame, all scales.  c20 ... are the
// channel planes (response layout: frame at F.roff, then scale s, row, column).
__global__ void __launch_bounds__(256) k_combine_detect(const FrameDev *__restrict__ fr, Items it, int S,
                                                        int hessian, const float *__restrict__ c20,
                                                        const float *__restrict__ c02,
                                                        const float *__restrict__ c11,
                                                        const float *__restrict__ c10,
                                                        const float *__restrict__ c01, float limit2,
                                                        DetectArgs da) {
  extern __shared__ float sm[];
  float *buf = sm;                     // [S][32][32] responses
  float *red = sm + (long)S * DT * DT;  // detector scratch
  __shared__ FrameDev s_fr;
  const int tid = threadIdx.x;
  int k = 0;
  const int nitems = items_total(it);
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    int local;
    k = item_frame(it, item, k, local);
    stage_frame(&s_fr, fr, it, k);  // the previous item ended with __syncthreads
    __syncthreads();
    const FrameDev &F = s_fr;
    const int H = F.H, W = F.W;
    const int ntx = (W + TW - 1) / TW;
    const int x0 = (local % ntx) * TW - 1, r0 = (local / ntx) * TW - 1;
    const long plane = (long)H * W;
    for (int p = tid; p < S * DT * DT; p += blockDim.x) {
      const int s = p / (DT * DT), i = (p / DT) % DT, lane = p % DT;
      const int y = r0 + i, x = x0 + lane;
      float v = 0.f;
      if (y >= 0 && y < H && x >= 0 && x < W) {
        const long q = F.roff + s * plane + (long)y * W + x;
        const float a = __ldg(c20 + q), b = __ldg(c02 + q);
        if (hessian) {
          const float c = __ldg(c11 + q);
          v = a * b - c * c;  // planes carry sigma^2: sigma^4 (D20 D02 - D11^2)
        } else {
          v = -(a + b);
        }
      }
      buf[p] = v;
    }
    __syncthreads();
    DetectArgs a = da;
    a.S = S;
    a.NR = DT;
    a.x0 = x0;
    a.r0 = r0;
    a.H = H;
    a.W = W;
    a.frame = F.index;
    a.resp = F.resp;
    a.dark = hessian ? 0 : 1;  // R_H: bright maxima only
    a.raw = 0;
    if (c10) {
      a.d10 = c10 + F.roff;
      a.d01 = c01 + F.roff;
      a.d20 = c20 + F.roff;
      a.d02 = c02 + F.roff;
      a.d11 = c11 + F.roff;
      a.limit2 = limit2;
    }
    detect_tile(buf, red, a);
    __syncthreads();
  }
}

}  // namespace

int deriv_items(int H, int W) { return ((W + TW - 1) / TW) * ((H + TW - 1) / TW); }

int launch_combine_detect(const Plan &p, const Launch &l, const BankArgs &a, int hessian, const float *c20,
                          const float *c02, const float *c11, const float *c10, const float *c01, float limit2,
                          cudaStream_t st) {
  const size_t smem = ((size_t)a.S * DT * DT + (size_t)DT * DT * 2) * sizeof(float) + (size_t)DT * DT * 2;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_combine_detect, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  DetectArgs da;
  da.thr = a.threshold;
  da.neigh = a.neigh;
  da.dark = 1;
  da.out = a.blobs;
  da.cap = a.cap;
  da.status = a.status;
  da.resp = nullptr;
  const int nb = persistent_blocks((const void *)k_combine_detect, 256, smem, l.it.total, 0);
  a.prof->begin("deriv_detect", st);
  k_combine_detect<<<nb, 256, smem, st>>>(p.fr, l.it, a.S, hessian, c20, c02, c11, c10, c01, limit2, da);
  a.prof->end(st);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}


// ---------------------------------------------------------------------------
// Shape descriptors (Sec. 5): at a detection the blurred image's Hessian
// H = [[D20, D11], [D11, D02]] read as minus the Fisher information of the
// blob taken as a pdf; P = (-pol H)^-1 its covariance, pol = +1 for a bright
// blob (D20 + D02 < 0: an intensity maximum), -1 for a dark one (the
// detection's own polarity under R_H is that of |H|).  Eigenvalues of P
// p1 >= p2 (pixels^2), orientation of the p1 axis (radians from +x towards
// +y, in (-pi/2, pi/2]), |H|; NaN where -pol H is not positive definite.
// In closed form (FP64): M = -pol H = [[a, c], [c, b]] has eigenvalues
// (a + b)/2 -+ sqrt(((a - b)/2)^2 + c^2); its larger eigenvalue's axis is at
// phi = atan2(2c, a - b) / 2, P's major axis (M's smaller eigenvalue) at
// phi + pi/2.
namespace {

// lay[3 f .. 3 f + 2]: offset of frame f's planes in a channel, H, W
__global__ void k_shapes(const Blob *__restrict__ b, long n, const float *__restrict__ c20,
                         const float *__restrict__ c02, const float *__restrict__ c11,
                         const long *__restrict__ lay, const Coef *__restrict__ coef, float4 *__restrict__ out) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Blob r = b[i];
  const long H = lay[3 * r.frame + 1], W = lay[3 * r.frame + 2];
  const long o = lay[3 * r.frame] + ((long)r.scale * H + r.y) * W + r.x;
  const double s2 = (double)coef[r.scale].sigma2;  // the planes carry sigma^2 D
  const double d20 = c20[o] / s2, d02 = c02[o] / s2, d11 = c11[o] / s2;
  const double det = d20 * d02 - d11 * d11;
  const double pol = d20 + d02 < 0.0 ? 1.0 : -1.0;
  const double a = -pol * d20, bb = -pol * d02, c = -pol * d11;
  const double half = 0.5 * (a - bb), disc = sqrt(half * half + c * c), mid = 0.5 * (a + bb);
  const double mu_min = mid - disc, mu_max = mid + disc;
  float4 v;
  if (mu_min > 0.0) {
    double th = 0.5 * atan2(2.0 * c, a - bb) + 0.5 * M_PI;
    if (th > 0.5 * M_PI) th -= M_PI;
    v = make_float4((float)(1.0 / mu_min), (float)(1.0 / mu_max), (float)th, (float)det);
  } else {
    v = make_float4(CUDART_NAN_F, CUDART_NAN_F, CUDART_NAN_F, (float)det);
  }
  out[i] = v;
}

}  // namespace

int launch_shapes(const Blob *b, long n, const float *c20, const float *c02, const float *c11, const long *lay,
                  const Coef *coef, void *out, cudaStream_t st) {
  if (n <= 0) return 0;
  k_shapes<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(b, n, c20, c02, c11, lay, coef, static_cast<float4 *>(out));
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace kf
