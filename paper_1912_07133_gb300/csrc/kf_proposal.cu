// kf_proposal.cu -- the proposal network that gates the filter bank (no
// counterpart in the paper): 8 x 8 mean pooling of the frame, three 3 x 3
// convolutions (1 -> 16 -> 16 -> 8 channels, ReLU after the first two) on the
// pooled frame, and a max over each tile's 8 x 8 pooled pixels giving one
// logit per (64 x 64-pixel tile, scale).  Weights are used in bf16 (rounded
// from FP32 masters), every sum in FP32.  Training: weighted BCE with logits,
// backward through the max and the convolutions, Adam on the masters.
//
// Layouts: images [N][C][h][w] row-major; weights per layer W[co][ci][3][3]
// then b[co], layers back to back (3640 values); logits [N][8][th][tw].
#include <cuda_bf16.h>
#include <math_constants.h>

#include "kf_batch.cuh"
#include "kf_common.cuh"
#include "kf_internal.h"

namespace kf {

namespace {

constexpr int CT = 16;  // output tile side of the convolution kernels

// ---------------------------------------------------------------------------
// pooling
// ---------------------------------------------------------------------------
// one thread per pooled pixel: mean of the frame's 8 x 8 block (clipped),
// times the value scale
template <class T>
__global__ void __launch_bounds__(256) k_pool8(const T *__restrict__ X, long xpitch, int H, int W, float vs,
                                               float *__restrict__ out, int h, int w) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= w) return;
  const int r0 = 8 * y, c0 = 8 * x, r1 = min(r0 + 8, H), c1 = min(c0 + 8, W);
  float s = 0.f;
  for (int r = r0; r < r1; ++r)
    for (int c = c0; c < c1; ++c) s += in_f32(__ldg(X + (long)r * xpitch + c));
  out[(long)y * w + x] = vs * s / (float)((r1 - r0) * (c1 - c0));
}

// the same for frame f of a call's frame table (the frame pointer is read on
// the device, so a captured launch serves later calls with other frames)
__global__ void __launch_bounds__(256) k_pool8_tab(const FrameDev *__restrict__ fr, int f,
                                                   float *__restrict__ out) {
  const FrameDev &F = fr[f];
  const int H = F.H, W = F.W, h = (H + 7) / 8, w = (W + 7) / 8;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= w || y >= h) return;
  const int r0 = 8 * y, c0 = 8 * x, r1 = min(r0 + 8, H), c1 = min(c0 + 8, W);
  const long xpitch = F.xpitch;
  float s = 0.f;
  with_input_type(F.X, F.dtype, [&](auto Xt) {
    for (int r = r0; r < r1; ++r)
      for (int c = c0; c < c1; ++c) s += in_f32(__ldg(Xt + (long)r * xpitch + c));
  });
  out[(long)y * w + x] = F.vscale * s / (float)((r1 - r0) * (c1 - c0));
}

// ---------------------------------------------------------------------------
// convolution, forward: out[n][co] = b[co] + sum_ci,dy,dx W[co][ci][dy][dx] in[n][ci][y+dy-1][x+dx-1]
// ---------------------------------------------------------------------------
template <int CI, int CO, bool RELU>
__global__ void __launch_bounds__(CT * CT) k_conv_fwd(const float *__restrict__ in,
                                                      const __nv_bfloat16 *__restrict__ Wb,
                                                      const __nv_bfloat16 *__restrict__ bb, float *__restrict__ out,
                                                      int h, int w) {
  __shared__ float s_in[CI][CT + 2][CT + 3];
  __shared__ float s_w[CO * CI * 9];
  const int n = blockIdx.z, x0 = blockIdx.x * CT, y0 = blockIdx.y * CT, tid = threadIdx.x;
  const long plane = (long)h * w;
  const float *inn = in + (long)n * CI * plane;
  for (int i = tid; i < CO * CI * 9; i += CT * CT) s_w[i] = __bfloat162float(Wb[i]);
  for (int i = tid; i < CI * (CT + 2) * (CT + 2); i += CT * CT) {
    const int ci = i / ((CT + 2) * (CT + 2)), r = (i / (CT + 2)) % (CT + 2), c = i % (CT + 2);
    const int y = y0 + r - 1, x = x0 + c - 1;
    s_in[ci][r][c] = (y >= 0 && y < h && x >= 0 && x < w) ? __ldg(inn + ci * plane + (long)y * w + x) : 0.f;
  }
  __syncthreads();
  const int tx = tid % CT, ty = tid / CT, x = x0 + tx, y = y0 + ty;
  float acc[CO];
#pragma unroll
  for (int co = 0; co < CO; ++co) acc[co] = __bfloat162float(bb[co]);
#pragma unroll 1
  for (int ci = 0; ci < CI; ++ci)
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const float v = s_in[ci][ty + k / 3][tx + k % 3];
#pragma unroll
      for (int co = 0; co < CO; ++co) acc[co] = fmaf(s_w[(co * CI + ci) * 9 + k], v, acc[co]);
    }
  if (x < w && y < h) {
    float *o = out + (long)n * CO * plane + (long)y * w + x;
#pragma unroll
    for (int co = 0; co < CO; ++co) o[co * plane] = RELU ? fmaxf(acc[co], 0.f) : acc[co];
  }
}

// The same convolution, two pixels per thread (rows y and y + 16 of a 16 x 32
// tile) with the weights in shared memory as [ci][k][co]: per input tap a
// thread reads its two inputs and the CO weights as float4 (broadcast across
// the warp) for 2 CO fused multiply-adds.  Dynamic shared memory: the input
// tile (CI x 34 x 19) and the weights.
constexpr int CT2 = 2 * CT;  // tile rows
template <int CI, int CO>
constexpr size_t conv2_smem() {
  return sizeof(float) * ((size_t)CI * (CT2 + 2) * (CT + 3) + (size_t)CI * 9 * CO);
}

template <int CI, int CO, bool RELU>
__global__ void __launch_bounds__(CT * CT) k_conv_fwd2(const float *__restrict__ in,
                                                       const __nv_bfloat16 *__restrict__ Wb,
                                                       const __nv_bfloat16 *__restrict__ bb, float *__restrict__ out,
                                                       int h, int w) {
  static_assert(CO % 4 == 0, "float4 weight loads");
  extern __shared__ __align__(16) float sm2[];
  float *s_w = sm2;                                   // [CI * 9][CO]
  float(*s_in)[CT2 + 2][CT + 3] = reinterpret_cast<float(*)[CT2 + 2][CT + 3]>(sm2 + CI * 9 * CO);
  const int n = blockIdx.z, x0 = blockIdx.x * CT, y0 = blockIdx.y * CT2, tid = threadIdx.x;
  const long plane = (long)h * w;
  const float *inn = in + (long)n * CI * plane;
  for (int i = tid; i < CO * CI * 9; i += CT * CT) {
    const int co = i / (CI * 9), r = i % (CI * 9);  // global layout W[co][ci][k]
    s_w[r * CO + co] = __bfloat162float(Wb[i]);
  }
  for (int i = tid; i < CI * (CT2 + 2) * (CT + 2); i += CT * CT) {
    const int ci = i / ((CT2 + 2) * (CT + 2)), r = (i / (CT + 2)) % (CT2 + 2), c = i % (CT + 2);
    const int y = y0 + r - 1, x = x0 + c - 1;
    s_in[ci][r][c] = (y >= 0 && y < h && x >= 0 && x < w) ? __ldg(inn + ci * plane + (long)y * w + x) : 0.f;
  }
  __syncthreads();
  const int tx = tid % CT, ty = tid / CT, x = x0 + tx;
  float a0[CO], a1[CO];
#pragma unroll
  for (int co = 0; co < CO; ++co) a0[co] = a1[co] = __bfloat162float(bb[co]);
#pragma unroll 1
  for (int ci = 0; ci < CI; ++ci)
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const float v0 = s_in[ci][ty + k / 3][tx + k % 3];
      const float v1 = s_in[ci][ty + CT + k / 3][tx + k % 3];
      const float4 *wv = reinterpret_cast<const float4 *>(s_w + (ci * 9 + k) * CO);
#pragma unroll
      for (int q = 0; q < CO / 4; ++q) {
        const float4 wq = wv[q];
        a0[4 * q + 0] = fmaf(wq.x, v0, a0[4 * q + 0]);
        a0[4 * q + 1] = fmaf(wq.y, v0, a0[4 * q + 1]);
        a0[4 * q + 2] = fmaf(wq.z, v0, a0[4 * q + 2]);
        a0[4 * q + 3] = fmaf(wq.w, v0, a0[4 * q + 3]);
        a1[4 * q + 0] = fmaf(wq.x, v1, a1[4 * q + 0]);
        a1[4 * q + 1] = fmaf(wq.y, v1, a1[4 * q + 1]);
        a1[4 * q + 2] = fmaf(wq.z, v1, a1[4 * q + 2]);
        a1[4 * q + 3] = fmaf(wq.w, v1, a1[4 * q + 3]);
      }
    }
  if (x >= w) return;
  float *o = out + (long)n * CO * plane + x;
  const int ya = y0 + ty, yb = y0 + ty + CT;
#pragma unroll
  for (int co = 0; co < CO; ++co) {
    if (ya < h) o[co * plane + (long)ya * w] = RELU ? fmaxf(a0[co], 0.f) : a0[co];
    if (yb < h) o[co * plane + (long)yb * w] = RELU ? fmaxf(a1[co], 0.f) : a1[co];
  }
}

// ---------------------------------------------------------------------------
// tile max: z[n][c][ty][tx] = max over the 8 x 8 block (first maximum in
// row-major order; its flat index y w + x is kept for the backward pass)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_tilemax(const float *__restrict__ o, int C, int h, int w, int th, int tw,
                                                 long total, float *__restrict__ z, int *__restrict__ arg) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int tx = (int)(i % tw), ty = (int)((i / tw) % th);
  const long nc = i / ((long)tw * th);
  const float *p = o + nc * h * w;
  float best = -CUDART_INF_F;
  int bi = 0;
  for (int by = 8 * ty; by < min(8 * ty + 8, h); ++by)
    for (int bx = 8 * tx; bx < min(8 * tx + 8, w); ++bx) {
      const float v = __ldg(p + (long)by * w + bx);
      if (v > best) best = v, bi = by * w + bx;
    }
  z[i] = best;
  if (arg) arg[i] = bi;
}

// ---------------------------------------------------------------------------
// backward
// ---------------------------------------------------------------------------
// weighted BCE with logits: dz = (pw t (s - 1) + (1 - t) s) / M, s = sigmoid(z);
// per-block partial sums of the loss terms (reduced in a fixed order)
__global__ void __launch_bounds__(256) k_bce(const float *__restrict__ z, const unsigned char *__restrict__ t,
                                             long M, float pw, float *__restrict__ dz, float *__restrict__ part) {
  __shared__ float red[256];
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (i < M) {
    const float zi = z[i], ti = t[i] ? 1.f : 0.f;
    const float sp_pos = log1pf(expf(-fabsf(zi))) + fmaxf(zi, 0.f);  // softplus(z)
    const float sp_neg = sp_pos - zi;                                 // softplus(-z)
    l = pw * ti * sp_neg + (1.f - ti) * sp_pos;
    const float s = 1.f / (1.f + expf(-zi));
    dz[i] = (pw * ti * (s - 1.f) + (1.f - ti) * s) / (float)M;
  }
  red[threadIdx.x] = l;
  __syncthreads();
  for (int d = 128; d > 0; d >>= 1) {
    if (threadIdx.x < d) red[threadIdx.x] += red[threadIdx.x + d];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// sum of n partials in a fixed order (one block), times `scale`
__global__ void __launch_bounds__(256) k_sum(const float *__restrict__ part, long n, float scale,
                                             float *__restrict__ out) {
  __shared__ float red[256];
  float s = 0.f;
  for (long i = threadIdx.x; i < n; i += 256) s += part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int d = 128; d > 0; d >>= 1) {
    if (threadIdx.x < d) red[threadIdx.x] += red[threadIdx.x + d];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0] * scale;
}

// gradient of the tile max: each logit's gradient goes to its argmax (do3 zeroed before)
__global__ void __launch_bounds__(256) k_tilemax_bwd(const float *__restrict__ dz, const int *__restrict__ arg,
                                                     long total, int th, int tw, long plane, float *__restrict__ d) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const long nc = i / ((long)tw * th);
  d[nc * plane + arg[i]] = dz[i];
}

// d_in[n][ci][y][x] = (act[n][ci][y][x] > 0) sum_co,dy,dx W[co][ci][dy][dx] d_out[n][co][y-dy+1][x-dx+1]
template <int CI, int CO>
__global__ void __launch_bounds__(CT * CT) k_conv_bwd_data(const float *__restrict__ dout,
                                                           const __nv_bfloat16 *__restrict__ Wb,
                                                           const float *__restrict__ act, float *__restrict__ din,
                                                           int h, int w) {
  __shared__ float s_d[CO][CT + 2][CT + 3];
  __shared__ float s_w[CO * CI * 9];
  const int n = blockIdx.z, x0 = blockIdx.x * CT, y0 = blockIdx.y * CT, tid = threadIdx.x;
  const long plane = (long)h * w;
  const float *dn = dout + (long)n * CO * plane;
  for (int i = tid; i < CO * CI * 9; i += CT * CT) s_w[i] = __bfloat162float(Wb[i]);
  for (int i = tid; i < CO * (CT + 2) * (CT + 2); i += CT * CT) {
    const int co = i / ((CT + 2) * (CT + 2)), r = (i / (CT + 2)) % (CT + 2), c = i % (CT + 2);
    const int y = y0 + r - 1, x = x0 + c - 1;
    s_d[co][r][c] = (y >= 0 && y < h && x >= 0 && x < w) ? __ldg(dn + co * plane + (long)y * w + x) : 0.f;
  }
  __syncthreads();
  const int tx = tid % CT, ty = tid / CT, x = x0 + tx, y = y0 + ty;
  if (x >= w || y >= h) return;
  float acc[CI];
#pragma unroll
  for (int ci = 0; ci < CI; ++ci) acc[ci] = 0.f;
#pragma unroll 1
  for (int co = 0; co < CO; ++co)
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      // d_out at (y - dy + 1, x - dx + 1) sits at tile (ty - dy + 2, tx - dx + 2)
      const float g = s_d[co][ty + 2 - k / 3][tx + 2 - k % 3];
#pragma unroll
      for (int ci = 0; ci < CI; ++ci) acc[ci] = fmaf(s_w[(co * CI + ci) * 9 + k], g, acc[ci]);
    }
  const long o = (long)n * CI * plane + (long)y * w + x;
#pragma unroll
  for (int ci = 0; ci < CI; ++ci) din[o + ci * plane] = __ldg(act + o + ci * plane) > 0.f ? acc[ci] : 0.f;
}

// Partial weight and bias gradients of one 16 x 16 tile of one image:
// part[tile][(co CI + ci) 9 + k] = sum_px d_out[co][px] in[ci][px + k], part[tile][CO CI 9 + co] = sum_px d_out[co][px]
template <int CI, int CO>
__global__ void __launch_bounds__(CT * CT) k_conv_bwd_w(const float *__restrict__ in, const float *__restrict__ dout,
                                                        int h, int w, float *__restrict__ part) {
  constexpr int NE = CO * CI * 9 + CO;
  __shared__ float s_in[CI][CT + 2][CT + 3];
  __shared__ float s_d[CO][CT][CT + 1];
  const int n = blockIdx.z, x0 = blockIdx.x * CT, y0 = blockIdx.y * CT, tid = threadIdx.x;
  const long plane = (long)h * w;
  const float *inn = in + (long)n * CI * plane, *dn = dout + (long)n * CO * plane;
  for (int i = tid; i < CI * (CT + 2) * (CT + 2); i += CT * CT) {
    const int ci = i / ((CT + 2) * (CT + 2)), r = (i / (CT + 2)) % (CT + 2), c = i % (CT + 2);
    const int y = y0 + r - 1, x = x0 + c - 1;
    s_in[ci][r][c] = (y >= 0 && y < h && x >= 0 && x < w) ? __ldg(inn + ci * plane + (long)y * w + x) : 0.f;
  }
  for (int i = tid; i < CO * CT * CT; i += CT * CT) {
    const int co = i / (CT * CT), r = (i / CT) % CT, c = i % CT;
    const int y = y0 + r, x = x0 + c;
    s_d[co][r][c] = (y < h && x < w) ? __ldg(dn + co * plane + (long)y * w + x) : 0.f;
  }
  __syncthreads();
  const long tile = ((long)n * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  for (int e = tid; e < NE; e += CT * CT) {
    float s = 0.f;
    if (e < CO * CI * 9) {
      const int co = e / (CI * 9), ci = (e / 9) % CI, k = e % 9, dy = k / 3, dx = k % 3;
      for (int r = 0; r < CT; ++r)
#pragma unroll 4
        for (int c = 0; c < CT; ++c) s = fmaf(s_d[co][r][c], s_in[ci][r + dy][c + dx], s);
    } else {
      const int co = e - CO * CI * 9;
      for (int r = 0; r < CT; ++r)
        for (int c = 0; c < CT; ++c) s += s_d[co][r][c];
    }
    part[tile * NE + e] = s;
  }
}

// g[e] = sum over tiles of part[tile][e], in tile order
__global__ void __launch_bounds__(256) k_reduce_tiles(const float *__restrict__ part, long ntiles, int NE,
                                                      float *__restrict__ g) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= NE) return;
  float s = 0.f;
  for (long t = 0; t < ntiles; ++t) s += __ldg(part + t * NE + e);
  g[e] = s;
}

// Adam on the FP32 masters; the bf16 working copy follows
__global__ void __launch_bounds__(256) k_adam(float *__restrict__ master, float *__restrict__ m,
                                              float *__restrict__ v, const float *__restrict__ g, int n, float lr,
                                              float c1, float c2, __nv_bfloat16 *__restrict__ wb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float th = master[i] - lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
  master[i] = th;
  wb[i] = __float2bfloat16_rn(th);
}

__global__ void k_to_bf16(const float *__restrict__ x, int n, __nv_bfloat16 *__restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = __float2bfloat16_rn(x[i]);
}

// labels[frame][s][y / 64][x / 64] = 1 for every candidate with |R| > thr
__global__ void k_labels(const Blob *__restrict__ b, long n, float thr, const long *__restrict__ loff,
                         const int *__restrict__ ltw, int S, unsigned char *__restrict__ lab,
                         const int *__restrict__ lth) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Blob r = b[i];
  if (!(fabsf(r.response) > thr)) return;
  const int tw = ltw[r.frame], th = lth[r.frame];
  lab[loff[r.frame] + ((long)r.scale * th + r.y / 64) * tw + r.x / 64] = 1;
}

// ---------------------------------------------------------------------------
// gating
// ---------------------------------------------------------------------------
// act[ty][tx] = 1 if a logit of scale s < S exceeds zthr in the tile (dil = 0)
// or in its 3 x 3 tile neighbourhood (dil = 1)
__global__ void k_gate_tiles(const float *__restrict__ z, int S, int th, int tw, float zthr, int dil,
                             unsigned char *__restrict__ act) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= th * tw) return;
  const int ty = i / tw, tx = i % tw;
  unsigned char a = 0;
  for (int s = 0; s < S && !a; ++s)
    for (int yy = max(ty - dil, 0); yy <= min(ty + dil, th - 1) && !a; ++yy)
      for (int xx = max(tx - dil, 0); xx <= min(tx + dil, tw - 1); ++xx)
        if (z[((long)s * th + yy) * tw + xx] > zthr) {
          a = 1;
          break;
        }
  act[i] = a;
}

// position in it.fl of the frame holding item `item` (binary search; one thread)
__device__ __forceinline__ int find_frame(const Items &it, int item) {
  int lo = 0, hi = it.n;  // pre[lo] <= item < pre[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(it.pre + mid) <= item) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Items of a column pass (tiles of tw x th interior pixels, tile (tx, ty) =
// item ty ntx + tx) whose interior overlaps an active tile
__global__ void k_sel_tiles(const FrameDev *__restrict__ fr, Items full, const unsigned char *__restrict__ act,
                            int tw, int th, int2 *__restrict__ sel, int *__restrict__ count) {
  const int item = blockIdx.x * blockDim.x + threadIdx.x;
  if (item >= full.total) return;
  const int k = find_frame(full, item);
  const FrameDev &F = fr[__ldg(full.fl + k)];
  const int local = item - __ldg(full.pre + k);
  const int ntx = (F.W + tw - 1) / tw;
  const int x0 = (local % ntx) * tw, y0 = (local / ntx) * th;
  if (any_active(F, act, x0, x0 + tw, y0, y0 + th)) sel[atomicAdd(count, 1)] = make_int2(k, local);
}

// Items of the FIR row pass (rrows virtual rows x rseg outputs, item =
// row block nxs + segment; a block holding the U-only edge rows H and H+1 is
// always kept): a block is needed if an active tile lies within `reach` rows
// of it in the segment's columns +- 64
__global__ void k_sel_rows(const FrameDev *__restrict__ fr, Items full, const unsigned char *__restrict__ act,
                           int rseg, int rrows, int reach, int2 *__restrict__ sel, int *__restrict__ count) {
  const int item = blockIdx.x * blockDim.x + threadIdx.x;
  if (item >= full.total) return;
  const int k = find_frame(full, item);
  const FrameDev &F = fr[__ldg(full.fl + k)];
  const int local = item - __ldg(full.pre + k);
  const int nxs = (F.W + rseg - 1) / rseg;
  const int xs = (local % nxs) * rseg, y0 = (local / nxs) * rrows;
  if (y0 + rrows > F.H || any_active(F, act, xs - 64, xs + rseg + 64, y0 - reach, y0 + rrows + reach))
    sel[atomicAdd(count, 1)] = make_int2(k, local);
}

}  // namespace

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
namespace {

constexpr int W1 = 0, B1 = 144, W2 = 160, B2 = 2464, W3 = 2480, B3 = 3632;  // offsets in the flat vector
static_assert(B3 + 8 == NET_NPARAM, "parameter layout");

dim3 conv_grid(int N, int h, int w) { return dim3((w + CT - 1) / CT, (h + CT - 1) / CT, N); }

struct Carve {
  float *x1, *a2, *o3, *d2, *d1, *z, *dz, *part, *lossp, *loss;
  int *arg;
};

// workspace of a batch: a1 | a2 | o3 (= its gradient) | d(a2) | d(a1) | z | dz | arg | tile partials | loss partials | loss
Carve carve(float *work, int N, int h, int w) {
  const long P = (long)N * h * w;
  const long T = (long)N * 8 * ((h + 7) / 8) * ((w + 7) / 8);
  const long tiles = (long)N * ((h + CT - 1) / CT) * ((w + CT - 1) / CT);
  Carve c;
  float *p = work;
  c.x1 = p, p += 16 * P;
  c.a2 = p, p += 16 * P;
  c.o3 = p, p += 8 * P;
  c.d2 = p, p += 16 * P;
  c.d1 = p, p += 16 * P;
  c.z = p, p += T;
  c.dz = p, p += T;
  c.arg = reinterpret_cast<int *>(p), p += T;
  c.part = p, p += tiles * (16 * 16 * 9 + 16);
  c.lossp = p, p += (T + 255) / 256;
  c.loss = p;
  return c;
}

}  // namespace

size_t net_work_floats(int N, int h, int w) {
  const long P = (long)N * h * w;
  const long T = (long)N * 8 * ((h + 7) / 8) * ((w + 7) / 8);
  const long tiles = (long)N * ((h + CT - 1) / CT) * ((w + CT - 1) / CT);
  return (size_t)(72 * P + 3 * T + tiles * (16 * 16 * 9 + 16) + (T + 255) / 256 + 1);
}

int net_pool(const void *X, int dtype, float vs, long xpitch, int H, int W, float *out, cudaStream_t st) {
  const int h = (H + 7) / 8, w = (W + 7) / 8;
  dim3 g((w + 255) / 256, h);
  switch (dtype) {
    case IN_F16: k_pool8<<<g, 256, 0, st>>>(static_cast<const __half *>(X), xpitch, H, W, vs, out, h, w); break;
    case IN_BF16: k_pool8<<<g, 256, 0, st>>>(static_cast<const __nv_bfloat16 *>(X), xpitch, H, W, vs, out, h, w); break;
    case IN_U16: k_pool8<<<g, 256, 0, st>>>(static_cast<const unsigned short *>(X), xpitch, H, W, vs, out, h, w); break;
    default: k_pool8<<<g, 256, 0, st>>>(static_cast<const float *>(X), xpitch, H, W, vs, out, h, w);
  }
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

// logits of N pooled images x [N][h][w] into z_out [N][8][th][tw] (z_out may
// be the workspace's own logits: pass nullptr)
int net_forward(const float *x, int N, int h, int w, const __nv_bfloat16 *wb, float *work, float *z_out,
                cudaStream_t st) {
  Carve c = carve(work, N, h, w);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_conv_fwd2<16, 16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)conv2_smem<16, 16>());
    cudaFuncSetAttribute(k_conv_fwd2<16, 8, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)conv2_smem<16, 8>());
    attr = true;
  }
  const dim3 g = conv_grid(N, h, w), g2((w + CT - 1) / CT, (h + CT2 - 1) / CT2, N);
  k_conv_fwd<1, 16, true><<<g, CT * CT, 0, st>>>(x, wb + W1, wb + B1, c.x1, h, w);
  k_conv_fwd2<16, 16, true><<<g2, CT * CT, conv2_smem<16, 16>(), st>>>(c.x1, wb + W2, wb + B2, c.a2, h, w);
  k_conv_fwd2<16, 8, false><<<g2, CT * CT, conv2_smem<16, 8>(), st>>>(c.a2, wb + W3, wb + B3, c.o3, h, w);
  const int th = (h + 7) / 8, tw = (w + 7) / 8;
  const long T = (long)N * 8 * th * tw;
  k_tilemax<<<(unsigned)((T + 255) / 256), 256, 0, st>>>(c.o3, 8, h, w, th, tw, T, z_out ? z_out : c.z, c.arg);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

// forward, weighted BCE against labels t [N][8][th][tw], backward: the mean
// loss into *loss_dev and the gradient (3640 floats) into g
int net_grad(const float *x, const unsigned char *t, int N, int h, int w, float pw, const __nv_bfloat16 *wb,
             float *work, float *g, float *loss_dev, cudaStream_t st) {
  if (net_forward(x, N, h, w, wb, work, nullptr, st)) return -1;
  Carve c = carve(work, N, h, w);
  const int th = (h + 7) / 8, tw = (w + 7) / 8;
  const long T = (long)N * 8 * th * tw;
  const long P = (long)h * w;
  const unsigned nb = (unsigned)((T + 255) / 256);
  k_bce<<<nb, 256, 0, st>>>(c.z, t, T, pw, c.dz, c.lossp);
  k_sum<<<1, 256, 0, st>>>(c.lossp, nb, 1.f / (float)T, loss_dev);
  cudaMemsetAsync(c.o3, 0, sizeof(float) * 8 * P * N, st);  // o3 becomes its own gradient
  k_tilemax_bwd<<<nb, 256, 0, st>>>(c.dz, c.arg, T, th, tw, P, c.o3);
  const dim3 gr = conv_grid(N, h, w);
  const long tiles = (long)gr.x * gr.y * gr.z;
  // layer 3 (16 -> 8)
  k_conv_bwd_w<16, 8><<<gr, CT * CT, 0, st>>>(c.a2, c.o3, h, w, c.part);
  k_reduce_tiles<<<(8 * 16 * 9 + 8 + 255) / 256, 256, 0, st>>>(c.part, tiles, 8 * 16 * 9 + 8, g + W3);
  k_conv_bwd_data<16, 8><<<gr, CT * CT, 0, st>>>(c.o3, wb + W3, c.a2, c.d2, h, w);
  // layer 2 (16 -> 16)
  k_conv_bwd_w<16, 16><<<gr, CT * CT, 0, st>>>(c.x1, c.d2, h, w, c.part);
  k_reduce_tiles<<<(16 * 16 * 9 + 16 + 255) / 256, 256, 0, st>>>(c.part, tiles, 16 * 16 * 9 + 16, g + W2);
  k_conv_bwd_data<16, 16><<<gr, CT * CT, 0, st>>>(c.d2, wb + W2, c.x1, c.d1, h, w);
  // layer 1 (1 -> 16)
  k_conv_bwd_w<1, 16><<<gr, CT * CT, 0, st>>>(x, c.d1, h, w, c.part);
  k_reduce_tiles<<<(16 * 9 + 16 + 255) / 256, 256, 0, st>>>(c.part, tiles, 16 * 9 + 16, g + W1);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

int net_adam(float *master, float *m, float *v, const float *g, int step, float lr, __nv_bfloat16 *wb,
             cudaStream_t st) {
  const float c1 = 1.f - powf(0.9f, (float)step), c2 = 1.f - powf(0.999f, (float)step);
  k_adam<<<(NET_NPARAM + 255) / 256, 256, 0, st>>>(master, m, v, g, NET_NPARAM, lr, c1, c2, wb);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

int net_to_bf16(const float *x, __nv_bfloat16 *y, cudaStream_t st) {
  k_to_bf16<<<(NET_NPARAM + 255) / 256, 256, 0, st>>>(x, NET_NPARAM, y);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

int net_pool_table(const FrameDev *fr, int f, int H, int W, float *out, cudaStream_t st) {
  const int h = (H + 7) / 8, w = (W + 7) / 8;
  k_pool8_tab<<<dim3((w + 255) / 256, h), 256, 0, st>>>(fr, f, out);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

int gate_tiles(const float *z, int S, int th, int tw, float zthr, int dilate, unsigned char *act,
               cudaStream_t st) {
  k_gate_tiles<<<(th * tw + 255) / 256, 256, 0, st>>>(z, S, th, tw, zthr, dilate, act);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

int gate_select_tiles(const FrameDev *fr, const Items &full, const unsigned char *act, int tw, int th, int2 *sel,
                      int *count, cudaStream_t st) {
  if (full.total > 0)
    k_sel_tiles<<<(full.total + 255) / 256, 256, 0, st>>>(fr, full, act, tw, th, sel, count);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

int gate_select_rows(const FrameDev *fr, const Items &full, const unsigned char *act, int rseg, int rrows,
                     int reach, int2 *sel, int *count, cudaStream_t st) {
  if (full.total > 0)
    k_sel_rows<<<(full.total + 255) / 256, 256, 0, st>>>(fr, full, act, rseg, rrows, reach, sel, count);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

int net_labels(const Blob *b, long n, float thr, const long *loff, const int *ltw, const int *lth, int S,
               unsigned char *lab, cudaStream_t st) {
  if (n <= 0) return 0;
  k_labels<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(b, n, thr, loff, ltw, S, lab, lth);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace kf
