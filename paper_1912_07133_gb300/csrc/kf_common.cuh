// kf_common.cuh -- device-side records and helpers shared by the product
// kernels of the shape-filter bank (Kennedy, arXiv:1912.07133).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace kf {

constexpr int MAXK = 8;          // largest recursive order / number of modes
constexpr int MAXS = 16;         // scales per bank call
constexpr int CH = 32;           // row-kernel pixels per thread (chunk)
constexpr int TW = 30;           // column-kernel tile interior width (32 with halo)
constexpr int WARPM = 32;        // powers Phi^(CH m), m = 1..32, for the row scan
constexpr int MAX_FIR_K = 160;   // largest colored-SG half-length

enum { T_D = 0, T_E = 1, T_C = 2, T_A = 3 };

// Derivative channels of the row passes (Table I taps applied to the
// edge-held frame before the blur): the Laplacian L = U + V of the fused path,
// or one derivative of the derivative bank (R_H of eq 26, the eq 27 offsets).
//   U = X[x+1] - 2X + X[x-1]   V = X[y+1] - 2X + X[y-1]
//   W = (X[x+1,y+1] - X[x-1,y+1] - X[x+1,y-1] + X[x-1,y-1]) / 4
//   DX = (X[x+1] - X[x-1]) / 2  DY = (X[y+1] - X[y-1]) / 2
// Beyond the left/right edges the x-differences (U, W, DX) vanish and V, DY
// keep their row-end value; beyond the top/bottom the y-differences (V, W, DY)
// vanish and U, DX keep the value of the first/last row.  CH_ZERO: the edge
// rows of the y-vanishing channels.  CH_ID: the frame itself, held beyond
// every edge (the blur alone: the D = 5 bank differentiates before the bank).
enum { CH_LAP = 0, CH_U = 1, CH_V = 2, CH_W = 3, CH_DX = 4, CH_DY = 5, CH_ZERO = 6, CH_ID = 7 };

// channels of the D = 5 bank: every D_{dx,dy} with dx + dy <= 4
constexpr int QUARTIC_NCH = 15;

// the channel the U-only edge rows carry (the y-held part of the channel)
__host__ __device__ __forceinline__ int edge_chan(int c) {
  return (c == CH_LAP || c == CH_U) ? CH_U : (c == CH_DX ? CH_DX : (c == CH_ID ? CH_ID : CH_ZERO));
}

// channel c at column e (0 <= e < W) from rows y-1 (m), y (o), y+1 (p);
// at(row, e) returns the element with e clamped into the row
template <class AM, class AO, class AP>
__device__ __forceinline__ float chan_at(int c, AM m, AO o, AP p, int e) {
  switch (c) {
    case CH_LAP: return (o(e + 1) - 2.f * o(e) + o(e - 1)) + (p(e) - 2.f * o(e) + m(e));
    case CH_U: return o(e + 1) - 2.f * o(e) + o(e - 1);
    case CH_V: return p(e) - 2.f * o(e) + m(e);
    case CH_W: return 0.25f * ((p(e + 1) - p(e - 1)) - (m(e + 1) - m(e - 1)));
    case CH_DX: return 0.5f * (o(e + 1) - o(e - 1));
    case CH_DY: return 0.5f * (p(e) - m(e));
    case CH_ID: return o(e);
    default: return 0.f;
  }
}

// channel c beyond the row end at column e (e = 0: left, e = W - 1: right)
template <class AM, class AO, class AP>
__device__ __forceinline__ float chan_beyond(int c, AM m, AO o, AP p, int e) {
  switch (c) {
    case CH_LAP:
    case CH_V: return p(e) - 2.f * o(e) + m(e);
    case CH_DY: return 0.5f * (p(e) - m(e));
    case CH_ID: return o(e);
    default: return 0.f;
  }
}

// element types of input frames (same values as KF_DTYPE_*) and of the
// one-sided planes between the row and column passes
enum { IN_F32 = 0, IN_F16 = 1, IN_BF16 = 2, IN_U16 = 3 };
enum { ST_F32 = 0, ST_F16 = 1, ST_BF16 = 2 };

template <int ST>
struct Store;
template <>
struct Store<ST_F32> {
  using T = float;
  static __device__ __forceinline__ float ld(T v) { return v; }
  static __device__ __forceinline__ T cv(float x) { return x; }
};
template <>
struct Store<ST_F16> {
  using T = __half;
  static __device__ __forceinline__ float ld(T v) { return __half2float(v); }
  static __device__ __forceinline__ T cv(float x) { return __float2half_rn(x); }
};
template <>
struct Store<ST_BF16> {
  using T = __nv_bfloat16;
  static __device__ __forceinline__ float ld(T v) { return __bfloat162float(v); }
  static __device__ __forceinline__ T cv(float x) { return __float2bfloat16_rn(x); }
};

// largest finite f16 value: stored planes beyond it are reported, not clipped
constexpr float F16_MAX = 65504.f;

__host__ __device__ __forceinline__ int store_bytes(int st) { return st == ST_F32 ? 4 : 2; }
__host__ __device__ __forceinline__ int in_bytes(int dt) { return dt == IN_F32 ? 4 : 2; }

// one input element as f32 (before the value scale)
__device__ __forceinline__ float in_f32(float v) { return v; }
__device__ __forceinline__ float in_f32(__half v) { return __half2float(v); }
__device__ __forceinline__ float in_f32(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float in_f32(unsigned short v) { return (float)v; }

// Call f(p) with the frame pointer cast to its element type; the dispatch
// sits outside the caller's loops.
template <class F>
__device__ __forceinline__ void with_input_type(const void *X, int dt, F &&f) {
  switch (dt) {
    case IN_F16: f(static_cast<const __half *>(X)); break;
    case IN_BF16: f(static_cast<const __nv_bfloat16 *>(X)); break;
    case IN_U16: f(static_cast<const unsigned short *>(X)); break;
    default: f(static_cast<const float *>(X));
  }
}

// element i of a one-sided plane buffer of storage type st
__device__ __forceinline__ float load_plane(const void *P, long i, int st) {
  switch (st) {
    case ST_F16: return __half2float(__ldg(static_cast<const __half *>(P) + i));
    case ST_BF16: return __bfloat162float(__ldg(static_cast<const __nv_bfloat16 *>(P) + i));
    default: return __ldg(static_cast<const float *>(P) + i);
  }
}
__device__ __forceinline__ void store_plane(void *P, long i, int st, float v) {
  switch (st) {
    case ST_F16: static_cast<__half *>(P)[i] = __float2half_rn(v); break;
    case ST_BF16: static_cast<__nv_bfloat16 *>(P)[i] = __float2bfloat16_rn(v); break;
    default: static_cast<float *>(P)[i] = v;
  }
}

// Per-scale realisation of one designed blur.  Written by the FP64 design
// kernel; read by the filter kernels.  All recursive realisations are sums of
// one-sided parts (Appendix, eq A6): y = y+ + y- + b0 x, where y+ runs over
// the input left-to-right (top-to-bottom) and y- right-to-left, both on the
// INPUT (eq A10a-b), so the two directions are independent.
struct Coef {
  int type;      // T_D / T_E / T_C / T_A
  int K;         // D: chain length = K^lpf; E: number of modes; C: FIR half-length
  int status;    // 0 ok, else design failure code
  int pad0;
  float sigma2;  // sigma^2: R_L = -sigma^2 (D20 + D02)
  float b0;      // centre coefficient of the DE
  // Filter D: the K-fold pole p = exp(-1/sigma) realised as a delayed chain of
  // first-order sections t_1(n) = p t_1(n-1) + x(n), t_j(n) = p t_j(n-1) +
  // t_{j-1}(n-1); the one-sided output is sum_j w_j t_j(n-1).
  float p;
  float w[MAXK];
  float hold[MAXK];              // steady state per unit constant input: 1/q^j
  float phiM[WARPM][MAXK];       // first column of Phi^(CH m), m = 1..32
  // Filter E: complex (or real) one-pole modes t(n) = z t(n-1) + x(n);
  // one-sided output Re(sum_i g_i t_i(n-1)).
  float zr[MAXK], zi[MAXK];
  float gr[MAXK], gi[MAXK];
  float hr[MAXK], hi[MAXK];      // steady state per unit input: 1/(1-z)
  float zMr[WARPM][MAXK], zMi[WARPM][MAXK];  // z^(CH m), m = 1..32
  // FIR taps h[0..K] (Filter C or A)
  float h[MAX_FIR_K + 1];
  // FP64 design, copied to the host by kf_design
  double lambda, sigma, param, db0;
  double dbplus[MAXK + 1], daplus[MAXK + 1];
  double dh[MAX_FIR_K + 1];
  double dc_gain, moment2;
};

// Candidate record written by the detector kernels (matches kf_blob).
struct Blob {
  int32_t frame, x, y, scale, polarity;
  float response;
  float dx, dy;  // eq (27) offset (derivative bank; 0 otherwise)
};

// Bounded device-side status word shared by the kernels of one call.
struct DevStatus {
  unsigned long long count;  // candidates found (may exceed capacity)
  int error;                 // first error code seen by a kernel
  int range;                 // 1: a value exceeded the range of 16-bit (f16) plane storage
};

}  // namespace kf
