// kf_fir.cu -- non-recursive colored Savitzky-Golay blur bank (Filter C,
// Kennedy, arXiv:1912.07133, Sec. 4.2) with the derivative stage of Table I
// and the Sec. 5 detector.
//
// As for the recursive banks, the hpf pair is applied first (5-point
// Laplacian L = U + V of the edge-held frame), then the symmetric taps
// h(0..K) (eq A5) along x, then along y.  Outside the frame U is zero beyond
// the left/right edges and V is held; in y the roles swap (the y-blur input
// outside the frame is blur_x(U) of the first/last row, held).
//
//   k_rowfir    one CTA per (row, 1024-pixel segment): L with a K-pixel halo
//               in shared memory, 4 outputs per thread with a sliding register
//               window, all scales.
//   k_rowfir<EDGE> the same on U alone for rows 0 and H-1.
//   k_colfir    64 rows x 32 columns x all scales per CTA: per scale the
//               input block (64 + 2K rows) is staged in shared memory, each
//               warp slides an 8-row register window down its column; then
//               the detector.
#include "kf_common.cuh"
#include "kf_detect.cuh"
#include "kf_internal.h"

namespace kf {

namespace {

constexpr int RSEG = 1024;  // outputs per row CTA
constexpr int RNT = 256;    // threads per row CTA (4 outputs each)
constexpr int CROWS = 64;   // output rows per column CTA (incl. 2 halo rows)

template <bool EDGE>
__global__ void __launch_bounds__(RNT) k_rowfir(const float *__restrict__ X, long xpitch, int H, int W,
                                                const Coef *__restrict__ coef, int S, int kmax,
                                                float *__restrict__ P, long PW, float *__restrict__ edge) {
  extern __shared__ float sm[];
  const int tid = threadIdx.x;
  const int y = EDGE ? (blockIdx.y == 0 ? 0 : H - 1) : blockIdx.y;
  const int xs = blockIdx.x * RSEG;
  // L on [xs - kmax - 1, xs + RSEG + kmax + 7): the sliding window reads one
  // element past the taps on each side in its last step
  const int n = RSEG + 2 * kmax + 8;
  float *sL = sm;
  float *sh = sm + n;
  const float *rm = X + (long)max(y - 1, 0) * xpitch;
  const float *r0 = X + (long)y * xpitch;
  const float *rp = X + (long)min(y + 1, H - 1) * xpitch;
  const float vlo = __ldg(rp) - 2.f * __ldg(r0) + __ldg(rm);
  const float vhi = __ldg(rp + W - 1) - 2.f * __ldg(r0 + W - 1) + __ldg(rm + W - 1);
  for (int j = tid; j < n; j += RNT) {
    const int e = xs - kmax - 1 + j;
    float v;
    if (e < 0) v = EDGE ? 0.f : vlo;
    else if (e >= W) v = EDGE ? 0.f : vhi;
    else {
      const float c0 = __ldg(r0 + e);
      const float u = __ldg(r0 + min(e + 1, W - 1)) - 2.f * c0 + __ldg(r0 + max(e - 1, 0));
      v = EDGE ? u : u + (__ldg(rp + e) - 2.f * c0 + __ldg(rm + e));
    }
    sL[j] = v;
  }
  for (int s = 0; s < S; ++s) {
    const Coef &c = coef[s];
    const int K = c.K;
    __syncthreads();
    for (int k = tid; k <= K; k += RNT) sh[k] = c.h[k];
    __syncthreads();
    const int xl = 4 * tid;             // local output index
    const float *base = sL + kmax + 1 + xl;  // L at output xl
    float acc[4], lw[4], rw[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      acc[j] = sh[0] * base[j];
      lw[j] = base[j - 1];
      rw[j] = base[j + 1];
    }
    for (int k = 1; k <= K; ++k) {
      const float hk = sh[k];
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[j] = fmaf(hk, lw[j] + rw[j], acc[j]);
      // slide: left window one step further left, right window one step right
      lw[3] = lw[2];
      lw[2] = lw[1];
      lw[1] = lw[0];
      lw[0] = base[-k - 1];
      rw[0] = rw[1];
      rw[1] = rw[2];
      rw[2] = rw[3];
      rw[3] = base[3 + k + 1];
    }
    float *dst = EDGE ? edge + ((long)s * 2 + blockIdx.y) * PW : P + (long)s * H * PW + (long)y * PW;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int e = xs + xl + j;
      if (e < W) dst[e] = acc[j];
    }
  }
}

__global__ void __launch_bounds__(256) k_colfir(const float *__restrict__ P, long PW, int H, int W,
                                                const float *__restrict__ edge,
                                                const Coef *__restrict__ coef, int S, int kmax,
                                                DetectArgs da) {
  extern __shared__ float sm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int NIN = CROWS + 2 * kmax + 2;
  float *in = sm;                               // [NIN][32]
  float *buf = sm + (long)NIN * 32;             // [S][CROWS][32]
  float *red = buf + (long)S * CROWS * 32;
  const int x = blockIdx.x * TW - 1 + lane;
  const int xv = min(max(x, 0), W - 1);
  const int r0 = blockIdx.y * (CROWS - 2) - 1;  // frame row of output row 0
  for (int s = 0; s < S; ++s) {
    const Coef &c = coef[s];
    const int K = c.K;
    const float *Pc = P + (long)s * H * PW + xv;
    const float top = edge[((long)s * 2 + 0) * PW + xv], bot = edge[((long)s * 2 + 1) * PW + xv];
    __syncthreads();
    // in[j] = input row r0 - K - 1 + j, j < CROWS + 2K + 2 (the sliding window
    // reads one row past the taps on each side in its last step)
    for (int j = warp; j < CROWS + 2 * K + 2; j += 8) {
      const int r = r0 - K - 1 + j;
      in[j * 32 + lane] = r < 0 ? top : (r >= H ? bot : __ldg(Pc + (long)r * PW));
    }
    __syncthreads();
    const float *col = in + lane + (K + 1 + 8 * warp) * 32;  // output row 8*warp
    float acc[8], lw[8], rw[8];
    const float h0 = c.h[0];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      acc[j] = h0 * col[j * 32];
      lw[j] = col[(j - 1) * 32];
      rw[j] = col[(j + 1) * 32];
    }
    for (int k = 1; k <= K; ++k) {
      const float hk = __ldg(&c.h[k]);
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j] = fmaf(hk, lw[j] + rw[j], acc[j]);
#pragma unroll
      for (int j = 7; j > 0; --j) lw[j] = lw[j - 1];
      lw[0] = col[(-k - 1) * 32];
#pragma unroll
      for (int j = 0; j < 7; ++j) rw[j] = rw[j + 1];
      rw[7] = col[(7 + k + 1) * 32];
    }
    const float ms2 = -c.sigma2;
#pragma unroll
    for (int j = 0; j < 8; ++j) buf[((long)s * CROWS + 8 * warp + j) * 32 + lane] = ms2 * acc[j];
  }
  __syncthreads();
  DetectArgs a = da;
  a.S = S;
  a.NR = CROWS;
  a.x0 = blockIdx.x * TW - 1;
  a.r0 = r0;
  detect_tile(buf, red, a);
}

}  // namespace

int launch_fir_frame(const FrameGeom &g, const BankArgs &a, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_rowfir<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    cudaFuncSetAttribute(k_rowfir<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    cudaFuncSetAttribute(k_colfir, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    attr = true;
  }
  const int kmax = a.kmax;
  const size_t rsm = (size_t)(RSEG + 2 * kmax + 8 + kmax + 1) * sizeof(float);
  dim3 gr((g.W + RSEG - 1) / RSEG, g.H);
  a.prof->begin("fir_row", st);
  k_rowfir<false><<<gr, RNT, rsm, st>>>(g.X, g.xpitch, g.H, g.W, a.coef, a.S, kmax, a.P, g.PW, a.edge);
  a.prof->end(st);
  dim3 ge((g.W + RSEG - 1) / RSEG, 2);
  a.prof->begin("fir_row_edge", st);
  k_rowfir<true><<<ge, RNT, rsm, st>>>(g.X, g.xpitch, g.H, g.W, a.coef, a.S, kmax, a.P, g.PW, a.edge);
  a.prof->end(st);
  DetectArgs da;
  da.H = g.H;
  da.W = g.W;
  da.thr = a.threshold;
  da.neigh = a.neigh;
  da.dark = 1;
  da.frame = g.frame;
  da.out = a.blobs;
  da.cap = a.cap;
  da.status = a.status;
  da.resp = a.responses ? a.responses + g.resp_off : nullptr;
  const size_t csm = ((size_t)(CROWS + 2 * kmax + 2) * 32 + (size_t)a.S * CROWS * 32 +
                      (size_t)CROWS * 32 * 2) * sizeof(float) + (size_t)CROWS * 32 * 2;
  if (csm > 220 * 1024) return -1;
  dim3 gc((g.W + TW - 1) / TW, (g.H + CROWS - 3) / (CROWS - 2));
  a.prof->begin("fir_coldet", st);
  k_colfir<<<gc, 256, csm, st>>>(a.P, g.PW, g.H, g.W, a.edge, a.coef, a.S, kmax, da);
  a.prof->end(st);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace kf
