// kf_quartic.cu -- the kernels of the D = 5 derivative bank (L_D = 2).
//
// The bank estimates D_{dx,dy} (eq 3) for every dx + dy <= 4 at each scale
// by separable filtering (Sec. 2): the differentiator g_dx along x and g_dy
// along y (Sec. 4.1), then the L_D = 2 blur along x and along y (the bank's
// row and column passes over the 15 channel planes as the frames of one
// call, channel CH_ID).  The differentiators run first, in k_hpf5, over the
// frame held beyond its edges: their output is formed on a frame padded by
// two pixels on every side (x = -2 .. W + 1, y = -2 .. H + 1), and beyond that
// padding it is constant, so holding the padded plane at its edges is exactly
// the differentiated held frame.  The planes keep the frame's width: the two
// values beyond each row end enter the row passes as a pre-roll of their
// recursion (or window); the two rows beyond each column end are plane rows.
// The column passes write the blurred channels, without those rows, into the
// caller's array.  k_steer forms
// the steered derivatives of Sec. 2 (after eq 3).
#include <cuda_runtime.h>

#include <algorithm>

#include "kf_common.cuh"
#include "kf_internal.h"

namespace kf {

namespace {

// The differentiators of a D = 5 bank: eqs (13)-(17) with the pure-delay
// basis and dc constraints only (moments l < 5 of g_d equal to d! delta_{l,d},
// Sec. 4.1), in correlation form y(n) = sum_j g(j) x(n + j), j = -2..2:
// integer weights over a common denominator (the denominator divides once,
// at the end).
__host__ __device__ constexpr int g5(int d, int j) {
  constexpr int w[5][5] = {
      {0, 0, 1, 0, 0},        // d = 0: the unit impulse
      {1, -8, 0, 8, -1},      // d = 1, / 12
      {-1, 16, -30, 16, -1},  // d = 2, / 12
      {-1, 2, 0, -2, 1},      // d = 3, / 2
      {1, -4, 6, -4, 1},      // d = 4
  };
  return w[d][j];
}
__host__ __device__ constexpr double den5(int d) { return d == 1 || d == 2 ? 12.0 : (d == 3 ? 2.0 : 1.0); }

constexpr int HTX = 32, HTY = 8;  // outputs per block

// Compensated dot products (Ogita, Rump and Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 26 (2005), algorithm Dot2): each product is
// split exactly by an FMA (TwoProduct), each sum by Knuth's TwoSum, and the
// rounding errors are accumulated beside the sum, so the result is as
// accurate as if computed in twice the working precision and then rounded.
// The _rn intrinsics are never contracted into FMAs, which the error-free
// transformations rely on.
struct Acc2 {
  float p = 0.f, s = 0.f;  // running sum and accumulated errors
  __device__ __forceinline__ void add_prod(float w, float x) {
    const float h = __fmul_rn(w, x), e = fmaf(w, x, -h);  // w x = h + e exactly
    const float t = __fadd_rn(p, h), z = __fsub_rn(t, p);
    s += __fadd_rn(__fsub_rn(p, __fsub_rn(t, z)), __fsub_rn(h, z)) + e;  // p + h = t + that exactly
    p = t;
  }
  __device__ __forceinline__ void add_small(float w, float x) { s = fmaf(w, x, s); }
  // p + s as an unevaluated pair hi + lo (TwoSum)
  __device__ __forceinline__ float2 pair() const {
    const float hi = __fadd_rn(p, s), z = __fsub_rn(hi, p);
    return make_float2(hi, __fadd_rn(__fsub_rn(p, __fsub_rn(hi, z)), __fsub_rn(s, z)));
  }
};

// every channel U_{dx,dy} = g_dx (x) g_dy of the held frame at x = -2 .. W + 1,
// y = -2 .. H + 1 (Hp = H + 4 rows): plane c of out (W x Hp, stride W Hp)
// holds at py * W + x the value at (x, py - 2) for x = 0 .. W - 1, and
// xpre[c * Hp + py] the values at x = -2, -1, W, W + 1.  The four nontrivial
// x-differences of the block's rows are formed once, as unevaluated sums
// hi + lo, and shared by the channels.  The differences cancel most of the
// frame's magnitude; the compensated sums keep U accurate relative to itself
// (a few units of its last place) whatever the cancellation.
__global__ void __launch_bounds__(HTX *HTY) k_hpf5(const void *__restrict__ X, int dtype, float vs, long pitch,
                                                   int W, int H, float *__restrict__ out,
                                                   float *__restrict__ xpre) {
  __shared__ float xs[HTY + 4][HTX + 4];
  __shared__ float2 ts[4][HTY + 4][HTX];  // dx = 1..4 (dx = 0 reads xs)
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * HTX + tx;
  const int px0 = blockIdx.x * HTX, py0 = blockIdx.y * HTY;
  const int Wp = W + 4, Hp = H + 4;
  // frame pixels x = px0 - 4 + c, y = py0 - 4 + r, clamped into the frame
  with_input_type(X, dtype, [&](auto Xt) {
    for (int i = tid; i < (HTY + 4) * (HTX + 4); i += HTX * HTY) {
      const int r = i / (HTX + 4), c = i % (HTX + 4);
      const int x = min(max(px0 - 4 + c, 0), W - 1), y = min(max(py0 - 4 + r, 0), H - 1);
      xs[r][c] = vs * in_f32(__ldg(Xt + (long)y * pitch + x));
    }
  });
  __syncthreads();
  for (int i = tid; i < (HTY + 4) * HTX; i += HTX * HTY) {
    const int r = i / HTX, c = i % HTX;
    float v[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) v[j] = xs[r][c + j];
#pragma unroll
    for (int d = 1; d < 5; ++d) {
      Acc2 a;
#pragma unroll
      for (int j = 0; j < 5; ++j)
        if (g5(d, j) != 0) a.add_prod((float)g5(d, j), v[j]);
      ts[d - 1][r][c] = a.pair();
    }
  }
  __syncthreads();
  const int px = px0 + tx, py = py0 + ty;
  if (px >= Wp || py >= Hp) return;
  // x = px - 2: inside the frame into the plane, else into the row's pre-roll
  const bool in = px >= 2 && px < W + 2;
  const int k = px < 2 ? px : px - W;  // pre-roll slot 0, 1 (left) or 2, 3 (right)
  const long plane = (long)W * Hp, o = in ? (long)py * W + px - 2 : 0;
#pragma unroll
  for (int n = 0, c = 0; n <= 4; ++n) {
#pragma unroll
    for (int dy = 0; dy <= n; ++dy, ++c) {
      const int dx = n - dy;
      Acc2 a;
#pragma unroll
      for (int j = 0; j < 5; ++j) {
        if (g5(dy, j) == 0) continue;
        const float w = (float)g5(dy, j);
        if (dx == 0) {
          a.add_prod(w, xs[ty + j][tx + 2]);
        } else {
          const float2 t = ts[dx - 1][ty + j][tx];
          a.add_prod(w, t.x);
          a.add_small(w, t.y);
        }
      }
      const float u = __fadd_rn(a.p, a.s) / (float)(den5(dx) * den5(dy));
      if (in) out[c * plane + o] = u;
      else xpre[((long)c * Hp + py) * 4 + k] = u;
    }
  }
}

struct SteerMat {
  float m[55];  // per order n = 0..4, an (n + 1) x (n + 1) block, row-major
};

// per set and pixel, each order's n + 1 channels through its block (all 15
// read before any is written: in == out is allowed)
__global__ void k_steer(const float *in, long npix, int nsets, SteerMat M, float *out) {
  const long n = npix * nsets;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const long set = i / npix, p = i - set * npix;
    const float *src = in + set * QUARTIC_NCH * npix + p;
    float *dst = out + set * QUARTIC_NCH * npix + p;
    float v[QUARTIC_NCH];
#pragma unroll
    for (int c = 0; c < QUARTIC_NCH; ++c) v[c] = src[c * npix];
    int base = 0, mb = 0;
#pragma unroll
    for (int o = 0; o < 5; ++o) {
#pragma unroll
      for (int a = 0; a <= o; ++a) {
        float acc = 0.f;
#pragma unroll
        for (int b = 0; b <= o; ++b) acc = fmaf(M.m[mb + a * (o + 1) + b], v[base + b], acc);
        dst[(base + a) * npix] = acc;
      }
      base += o + 1;
      mb += (o + 1) * (o + 1);
    }
  }
}

int grid_for(long n, int threads) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long want = (n + threads - 1) / threads, cap = 8L * std::max(nsm, 1);
  return (int)std::max(1L, std::min(want, cap));
}

}  // namespace

int launch_hpf5(const void *X, int dtype, float vs, long pitch, int W, int H, float *out, float *xpre,
                cudaStream_t st) {
  if (W < 1 || H < 1 || H + 4 > 8 * 65535) return -1;
  const dim3 grid((W + 4 + HTX - 1) / HTX, (H + 4 + HTY - 1) / HTY), block(HTX, HTY);
  k_hpf5<<<grid, block, 0, st>>>(X, dtype, vs, pitch, W, H, out, xpre);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

int launch_steer(const float *in, long npix, int nsets, const float *m55, float *out, cudaStream_t st) {
  SteerMat M;
  for (int i = 0; i < 55; ++i) M.m[i] = m55[i];
  const long n = npix * nsets;
  k_steer<<<grid_for(n, 256), 256, 0, st>>>(in, npix, nsets, M, out);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace kf
