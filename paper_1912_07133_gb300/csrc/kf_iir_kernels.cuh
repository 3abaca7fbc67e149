// kf_iir_kernels.cuh -- recursive (IIR) blur banks: Filter D (repeated pole,
// Sec. 4.3) and Filter E (discrete Butterworth, Sec. 4.4) of Kennedy,
// arXiv:1912.07133, with the derivative stage of Table I and the Sec. 5
// detector.  Included by kf_iir_d.cu (Filter D realisations) and kf_iir_e.cu
// (Filter E), which instantiate run_iir for their recursions.
//
// The derivative filters are applied first: the hpf pair [1,-2,1] along x and
// along y (Table I, d = 2) turns the frame into the 5-point Laplacian L = U + V
// (U = d2/dx2, V = d2/dy2, edge-held frame); the blur commutes with them, so
// D20 + D02 = blur_y(blur_x(L)).  Because the frame is held outside its
// edges, U vanishes beyond the left/right edges and V beyond the top/bottom
// ones: the x-recursion starts from the steady state of V at the row ends and
// the y-recursion from the steady state of blur_x(U) at the first/last row.
//
// Each one-sided recursion (eq A10a-b) runs on the input in FP32 as a chain of
// first-order sections (Filter D) or complex one-pole modes (Filter E) whose
// states keep unit-dc-gain accuracy; the three-term sum (eq A6) adds them.
//
// Passes (each persistent over the work items of the frames it covers, see
// kf_batch.cuh):
//   k_row      one CTA per row: chunk of CH pixels per thread, zero-state end
//              states, warp scan + fold of the carries across the CTA, then
//              both directions with exact starting states; all scales.  The
//              two extra items of a frame are its first and last rows on U
//              alone (column boundary).
//   k_colseg   zero-state end states of every LC-row column segment.
//   k_colfold  carries: sequential fold of the segment states per column.
//   k_coldet   LC+2 rows x 32 columns x all scales per CTA: both column
//              directions from the carries, response, extremum detector.
// The column segment length LC (32 or 64 rows, a template parameter) is the
// scan block length the autotuner chooses.
#pragma once
#include "kf_batch.cuh"
#include "kf_common.cuh"
#include "kf_detect.cuh"
#include "kf_internal.h"
#include "kf_tma.cuh"

#include <cooperative_groups.h>

namespace kf {

namespace {

// ---------------------------------------------------------------------------
// one-sided recursions
// ---------------------------------------------------------------------------
template <int KK>
struct Chain {
  static constexpr int NF = KK;
  // two independent chains (e.g. the two directions of a recursion) advanced
  // together by packed FP32 instructions (fma.rn.f32x2): per component the
  // same IEEE operations in the same order as push() and out()
  static constexpr bool kPacked = true;
  struct Pair {
    // the coefficients duplicated into both halves of a register pair
    struct Coefs {
      float2 p2, w2[KK];
      template <class V>
      __device__ __forceinline__ explicit Coefs(const V &v) {
        p2 = make_float2(v.p, v.p);
#pragma unroll
        for (int j = 0; j < KK; ++j) w2[j] = make_float2(v.w[j], v.w[j]);
      }
    };
    float2 t[KK];
    __device__ __forceinline__ void zero() {
#pragma unroll
      for (int j = 0; j < KK; ++j) t[j] = make_float2(0.f, 0.f);
    }
    __device__ __forceinline__ void push(const Coefs &c, float2 x2) {
#pragma unroll
      for (int j = KK - 1; j > 0; --j) t[j] = __ffma2_rn(c.p2, t[j], t[j - 1]);
      t[0] = __ffma2_rn(c.p2, t[0], x2);
    }
    __device__ __forceinline__ float2 out(const Coefs &c) const {
      float2 y = make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < KK; ++j) y = __ffma2_rn(c.w2[j], t[j], y);
      return y;
    }
    __device__ __forceinline__ void set(const Chain &a, const Chain &b) {
#pragma unroll
      for (int j = 0; j < KK; ++j) t[j] = make_float2(a.t[j], b.t[j]);
    }
    __device__ __forceinline__ void get(Chain &a, Chain &b) const {
#pragma unroll
      for (int j = 0; j < KK; ++j) a.t[j] = t[j].x, b.t[j] = t[j].y;
    }
  };
  static constexpr int kColdetRegs32 = 80;  // k_coldet with 32-row segments: registers per thread
  struct View {
    float p, b0, w[KK];
    __device__ void load(const Coef &c) {
      p = c.p;
      b0 = c.b0;
#pragma unroll
      for (int j = 0; j < KK; ++j) w[j] = c.w[j];
    }
  };
  float t[KK];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int j = 0; j < KK; ++j) t[j] = 0.f;
  }
  __device__ __forceinline__ void hold(const Coef &c, float x) {
#pragma unroll
    for (int j = 0; j < KK; ++j) t[j] = c.hold[j] * x;
  }
  __device__ __forceinline__ float out(const View &v) const {
    float y = 0.f;
#pragma unroll
    for (int j = 0; j < KK; ++j) y = fmaf(v.w[j], t[j], y);
    return y;
  }
  __device__ __forceinline__ void push(const View &v, float x) {
#pragma unroll
    for (int j = KK - 1; j > 0; --j) t[j] = fmaf(v.p, t[j], t[j - 1]);
    t[0] = fmaf(v.p, t[0], x);
  }
  // this <- Phi^n prev + this, Phi^n lower-triangular Toeplitz, first column phi
  __device__ __forceinline__ void combine(const float *phi, const Chain &prev) {
#pragma unroll
    for (int j = 0; j < KK; ++j) {
      float acc = t[j];
#pragma unroll
      for (int i = 0; i <= j; ++i) acc = fmaf(phi[i], prev.t[j - i], acc);
      t[j] = acc;
    }
  }
  // this <- Phi^(CH m) prev + this, 1 <= m <= 32
  __device__ __forceinline__ void combine_m(const Coef &c, int m, const Chain &prev) {
    float phi[KK];
#pragma unroll
    for (int i = 0; i < KK; ++i) phi[i] = c.phiM[m - 1][i];
    combine(phi, prev);
  }
  __device__ __forceinline__ void store(float *dst, long stride) const {
#pragma unroll
    for (int j = 0; j < KK; ++j) dst[j * stride] = t[j];
  }
  __device__ __forceinline__ void load(const float *src, long stride) {
#pragma unroll
    for (int j = 0; j < KK; ++j) t[j] = src[j * stride];
  }
  // powers of Phi as records (the first column of the lower-triangular
  // Toeplitz Phi^n): identity, Phi^(CH m) from the design's table, and
  // this += pw x v (pw a power, v a state or another power)
  __device__ __forceinline__ void identity() {
#pragma unroll
    for (int j = 0; j < KK; ++j) t[j] = j == 0 ? 1.f : 0.f;
  }
  __device__ __forceinline__ void load_pow(const Coef &c, int m) {
#pragma unroll
    for (int i = 0; i < KK; ++i) t[i] = c.phiM[m - 1][i];
  }
  __device__ __forceinline__ void mac(const Chain &pw, const Chain &v) { combine(pw.t, v); }
  // state published by another CTA of the grid (read past L1)
  __device__ __forceinline__ void load_cg(const float *src, long stride) {
#pragma unroll
    for (int j = 0; j < KK; ++j) t[j] = __ldcg(src + j * stride);
  }
  __device__ __forceinline__ Chain shfl_up(int d) const {
    Chain r;
#pragma unroll
    for (int j = 0; j < KK; ++j) r.t[j] = __shfl_up_sync(0xffffffffu, t[j], d);
    return r;
  }
  __device__ __forceinline__ Chain shfl_down(int d) const {
    Chain r;
#pragma unroll
    for (int j = 0; j < KK; ++j) r.t[j] = __shfl_down_sync(0xffffffffu, t[j], d);
    return r;
  }
};

template <int NM>
struct Modes {
  static constexpr int NF = 2 * NM;
  // two independent sets of modes advanced by packed FP32 instructions, with
  // per component the operations of push() and out()
  static constexpr bool kPacked = true;
  struct Pair {
    struct Coefs {
      float2 zr[NM], zi[NM], mzi[NM], gr[NM], mgi[NM];
      template <class V>
      __device__ __forceinline__ explicit Coefs(const V &v) {
#pragma unroll
        for (int i = 0; i < NM; ++i) {
          zr[i] = make_float2(v.zr[i], v.zr[i]);
          zi[i] = make_float2(v.zi[i], v.zi[i]);
          mzi[i] = make_float2(-v.zi[i], -v.zi[i]);
          gr[i] = make_float2(v.gr[i], v.gr[i]);
          mgi[i] = make_float2(-v.gi[i], -v.gi[i]);
        }
      }
    };
    float2 tr[NM], ti[NM];
    __device__ __forceinline__ void zero() {
#pragma unroll
      for (int i = 0; i < NM; ++i) tr[i] = ti[i] = make_float2(0.f, 0.f);
    }
    __device__ __forceinline__ void push(const Coefs &c, float2 x2) {
#pragma unroll
      for (int i = 0; i < NM; ++i) {
        const float2 nr = __ffma2_rn(c.zr[i], tr[i], __ffma2_rn(c.mzi[i], ti[i], x2));
        const float2 ni = __ffma2_rn(c.zr[i], ti[i], __fmul2_rn(c.zi[i], tr[i]));
        tr[i] = nr;
        ti[i] = ni;
      }
    }
    __device__ __forceinline__ float2 out(const Coefs &c) const {
      float2 y = make_float2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < NM; ++i) y = __ffma2_rn(c.gr[i], tr[i], __ffma2_rn(c.mgi[i], ti[i], y));
      return y;
    }
    __device__ __forceinline__ void set(const Modes &a, const Modes &b) {
#pragma unroll
      for (int i = 0; i < NM; ++i) tr[i] = make_float2(a.tr[i], b.tr[i]), ti[i] = make_float2(a.ti[i], b.ti[i]);
    }
    __device__ __forceinline__ void get(Modes &a, Modes &b) const {
#pragma unroll
      for (int i = 0; i < NM; ++i) a.tr[i] = tr[i].x, a.ti[i] = ti[i].x, b.tr[i] = tr[i].y, b.ti[i] = ti[i].y;
    }
  };
  static constexpr int kColdetRegs32 = NM < 3 ? 80 : 128;  // three modes need more
  struct View {
    float zr[NM], zi[NM], gr[NM], gi[NM], b0;
    __device__ void load(const Coef &c) {
      b0 = c.b0;
#pragma unroll
      for (int i = 0; i < NM; ++i) zr[i] = c.zr[i], zi[i] = c.zi[i], gr[i] = c.gr[i], gi[i] = c.gi[i];
    }
  };
  float tr[NM], ti[NM];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < NM; ++i) tr[i] = ti[i] = 0.f;
  }
  __device__ __forceinline__ void hold(const Coef &c, float x) {
#pragma unroll
    for (int i = 0; i < NM; ++i) tr[i] = c.hr[i] * x, ti[i] = c.hi[i] * x;
  }
  __device__ __forceinline__ float out(const View &v) const {
    float y = 0.f;
#pragma unroll
    for (int i = 0; i < NM; ++i) y = fmaf(v.gr[i], tr[i], fmaf(-v.gi[i], ti[i], y));
    return y;
  }
  __device__ __forceinline__ void push(const View &v, float x) {
#pragma unroll
    for (int i = 0; i < NM; ++i) {
      const float nr = fmaf(v.zr[i], tr[i], fmaf(-v.zi[i], ti[i], x));
      const float ni = fmaf(v.zr[i], ti[i], v.zi[i] * tr[i]);
      tr[i] = nr;
      ti[i] = ni;
    }
  }
  __device__ __forceinline__ void combine_z(const float *zr, const float *zi, const Modes &prev) {
#pragma unroll
    for (int i = 0; i < NM; ++i) {
      tr[i] = fmaf(zr[i], prev.tr[i], fmaf(-zi[i], prev.ti[i], tr[i]));
      ti[i] = fmaf(zr[i], prev.ti[i], fmaf(zi[i], prev.tr[i], ti[i]));
    }
  }
  __device__ __forceinline__ void combine_m(const Coef &c, int m, const Modes &prev) {
    float zr[NM], zi[NM];
#pragma unroll
    for (int i = 0; i < NM; ++i) zr[i] = c.zMr[m - 1][i], zi[i] = c.zMi[m - 1][i];
    combine_z(zr, zi, prev);
  }
  __device__ __forceinline__ void store(float *dst, long stride) const {
#pragma unroll
    for (int i = 0; i < NM; ++i) dst[(2 * i) * stride] = tr[i], dst[(2 * i + 1) * stride] = ti[i];
  }
  __device__ __forceinline__ void load(const float *src, long stride) {
#pragma unroll
    for (int i = 0; i < NM; ++i) tr[i] = src[(2 * i) * stride], ti[i] = src[(2 * i + 1) * stride];
  }
  // powers of Phi (diagonal: z^n per mode), as for Chain
  __device__ __forceinline__ void identity() {
#pragma unroll
    for (int i = 0; i < NM; ++i) tr[i] = 1.f, ti[i] = 0.f;
  }
  __device__ __forceinline__ void load_pow(const Coef &c, int m) {
#pragma unroll
    for (int i = 0; i < NM; ++i) tr[i] = c.zMr[m - 1][i], ti[i] = c.zMi[m - 1][i];
  }
  __device__ __forceinline__ void mac(const Modes &pw, const Modes &v) { combine_z(pw.tr, pw.ti, v); }
  __device__ __forceinline__ void load_cg(const float *src, long stride) {
#pragma unroll
    for (int i = 0; i < NM; ++i) tr[i] = __ldcg(src + (2 * i) * stride), ti[i] = __ldcg(src + (2 * i + 1) * stride);
  }
  __device__ __forceinline__ Modes shfl_up(int d) const {
    Modes r;
#pragma unroll
    for (int i = 0; i < NM; ++i)
      r.tr[i] = __shfl_up_sync(0xffffffffu, tr[i], d), r.ti[i] = __shfl_up_sync(0xffffffffu, ti[i], d);
    return r;
  }
  __device__ __forceinline__ Modes shfl_down(int d) const {
    Modes r;
#pragma unroll
    for (int i = 0; i < NM; ++i)
      r.tr[i] = __shfl_down_sync(0xffffffffu, tr[i], d), r.ti[i] = __shfl_down_sync(0xffffffffu, ti[i], d);
    return r;
  }
};

// Block-wide carry scan over the chunks of CH samples of one row.  `u` is
// this thread's zero-state end state; `k` its position in scan order (0 =
// first chunk of the direction); `init` the state before chunk 0.  Returns
// the state before this thread's chunk:
//   1. inclusive scan inside each warp (u_k <- A^d u_{k-d} + u_k, A = Phi^CH),
//   2. one thread folds the warp aggregates: C_0 = init,
//      C_{w+1} = A^32 C_w + G_w,
//   3. carry_k = C_w (lane 0) or A^lane C_w + (scan value of lane - 1).
// REV: scan order is the reverse thread order.  sm: 64 * NF floats.
template <class Rec, bool REV>
__device__ Rec carry_scan(Rec u, const Coef &c, int k, int NT, float *sm, const Rec &init) {
  const int lane = k & 31, wid = k >> 5, NW = NT >> 5;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const Rec o = REV ? u.shfl_down(d) : u.shfl_up(d);
    if (lane >= d) u.combine_m(c, d, o);
  }
  float *G = sm, *Cw = sm + 32 * Rec::NF;
  if (lane == 31) u.store(G + wid, 32);
  __syncthreads();
  if (k == 0) {
    Rec C = init;
    for (int w = 0; w < NW; ++w) {
      C.store(Cw + w, 32);
      Rec g;
      g.load(G + w, 32);
      g.combine_m(c, 32, C);  // A^32 C_w + G_w
      C = g;
    }
  }
  __syncthreads();
  Rec carry;
  carry.load(Cw + wid, 32);
  const Rec prev = REV ? u.shfl_down(1) : u.shfl_up(1);
  if (lane > 0) {
    Rec t = prev;
    t.combine_m(c, lane, carry);
    carry = t;
  }
  __syncthreads();
  return carry;
}

__host__ __device__ __forceinline__ int pad32(int e) { return e + (e >> 5); }

// ---------------------------------------------------------------------------
// row pass
// ---------------------------------------------------------------------------
// One row of one frame: row yw, or (EDGE) the U-only first (yw = 0) or last
// (yw = 1) row for the column boundary.  One body for both cases keeps the
// kernel's code small.  All threads of the block; ends with __syncthreads.
template <class Rec, bool ID>
__device__ __forceinline__ void row_body(const FrameDev &F, bool EDGE, int yw, int chan,
                                         const Coef *__restrict__ coef, int S, void *__restrict__ P, int st,
                                         long PWb, float *__restrict__ edge, bool &ovf, float *sm) {
  const int NT = blockDim.x, tid = threadIdx.x;
  const int H = F.H, W = F.W;
  const int RP = pad32(NT * CH) + 1;
  float *s_m = sm, *s_0 = sm + RP, *s_p = sm + 2 * RP, *s_scan = sm + 3 * RP;
  const int y = EDGE ? (yw == 0 ? 0 : H - 1) : yw;
  const float vs = F.vscale;
  const long xpitch = F.xpitch;
  // ID: the identity channel (CH_ID), which reads its own row only
  constexpr bool one = ID;
  with_input_type(F.X, F.dtype, [&](auto Xt) {
    const auto *r0 = Xt + (long)y * xpitch;
    const auto *rm = one ? r0 : Xt + (long)max(y - 1, 0) * xpitch;
    const auto *rp = one ? r0 : Xt + (long)min(y + 1, H - 1) * xpitch;
    // 8 elements (24 loads) per thread in flight before they are stored
    for (int e0 = tid; e0 < W; e0 += 8 * NT) {
      float a[8], b[8], c[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = min(e0 + u * NT, W - 1);
        b[u] = in_f32(__ldg(r0 + e));
        a[u] = one ? b[u] : in_f32(__ldg(rm + e));
        c[u] = one ? b[u] : in_f32(__ldg(rp + e));
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * NT;
        if (e < W) {
          const int q = pad32(e);
          s_m[q] = vs * a[u];
          s_0[q] = vs * b[u];
          s_p[q] = vs * c[u];
        }
      }
    }
  });
  __syncthreads();
  float L[CH];
  const int x0 = tid * CH;
  float in_lo, in_hi;
  // two-sample pre-rolls (CH_ID with xpre): the left carry is the steady state
  // of U(-2) advanced by U(-1); the right one that of U(W + 1), advanced by
  // U(W) when the chunks end at W (otherwise U(W) is a chunk element)
  const float4 xp = (one && F.xpre) ? F.xpre[y] : make_float4(0.f, 0.f, 0.f, 0.f);
  const bool pre = one && F.xpre, pre_hi = pre && NT * CH == W;
  if (one && pre) {
#pragma unroll
    for (int i = 0; i < CH; ++i) {
      const int e = x0 + i;
      L[i] = e < W ? s_0[pad32(e)] : (e == W ? xp.z : xp.w);
    }
    in_lo = xp.x;
    in_hi = xp.w;
  } else if (chan == CH_LAP) {
    const float v_lo = s_p[0] - 2.f * s_0[0] + s_m[0];
    const int eW = pad32(W - 1);
    const float v_hi = s_p[eW] - 2.f * s_0[eW] + s_m[eW];
#pragma unroll
    for (int i = 0; i < CH; ++i) {
      const int e = x0 + i;
      if (e < W) {
        const float c0 = s_0[pad32(e)];
        const float u = s_0[pad32(min(e + 1, W - 1))] - 2.f * c0 + s_0[pad32(max(e - 1, 0))];
        const float v = s_p[pad32(e)] - 2.f * c0 + s_m[pad32(e)];
        L[i] = EDGE ? u : u + v;
      } else {
        L[i] = EDGE ? 0.f : v_hi;  // beyond the right edge only the held V part
      }
    }
    in_lo = EDGE ? 0.f : v_lo;
    in_hi = EDGE ? 0.f : v_hi;
  } else {  // one derivative channel of the derivative bank
    const int cin = EDGE ? edge_chan(chan) : chan;
    auto am = [&](int e) { return s_m[pad32(min(max(e, 0), W - 1))]; };
    auto ao = [&](int e) { return s_0[pad32(min(max(e, 0), W - 1))]; };
    auto ap = [&](int e) { return s_p[pad32(min(max(e, 0), W - 1))]; };
#pragma unroll
    for (int i = 0; i < CH; ++i) {
      const int e = x0 + i;
      L[i] = e < W ? chan_at(cin, am, ao, ap, e) : chan_beyond(cin, am, ao, ap, W - 1);
    }
    in_lo = chan_beyond(cin, am, ao, ap, 0);
    in_hi = chan_beyond(cin, am, ao, ap, W - 1);
  }
  __syncthreads();
  float *s_out = sm;
  for (int s = 0; s < S; ++s) {
    const Coef &c = coef[s];
    typename Rec::View v;
    v.load(c);
    Rec ef, eb;
    if constexpr (Rec::kPacked) {  // both directions in one packed chain
      typename Rec::Pair e2;
      const typename Rec::Pair::Coefs pc(v);
      e2.zero();
#pragma unroll
      for (int i = 0; i < CH; ++i) e2.push(pc, make_float2(L[i], L[CH - 1 - i]));
      e2.get(ef, eb);
    } else {
      ef.zero();
      eb.zero();
#pragma unroll
      for (int i = 0; i < CH; ++i) ef.push(v, L[i]);
#pragma unroll
      for (int i = CH - 1; i >= 0; --i) eb.push(v, L[i]);
    }
    Rec hlo, hhi;
    hlo.hold(c, in_lo);
    hhi.hold(c, in_hi);
    if (one && pre) hlo.push(v, xp.y);
    if (one && pre_hi) hhi.push(v, xp.z);
    const Rec cf = carry_scan<Rec, false>(ef, c, tid, NT, s_scan, hlo);
    const Rec cb = carry_scan<Rec, true>(eb, c, NT - 1 - tid, NT, s_scan, hhi);
    float yv[CH];
    if constexpr (Rec::kPacked) {
      // step i advances the causal chain at pixel i and the anticausal one at
      // pixel CH-1-i; a pixel's two outputs meet when the second arrives:
      // yv = y+ + (b0 L + y-), the same operations as the scalar passes
      typename Rec::Pair r2;
      const typename Rec::Pair::Coefs pc(v);
      r2.set(cf, cb);
#pragma unroll
      for (int i = 0; i < CH; ++i) {
        const int k = CH - 1 - i;
        const float2 o = r2.out(pc);
        if (i < k) {
          yv[i] = o.x;  // y+ first
          yv[k] = o.y;  // y- first
        } else {
          yv[i] = o.x + fmaf(v.b0, L[i], yv[i]);
          yv[k] = yv[k] + fmaf(v.b0, L[k], o.y);
        }
        r2.push(pc, make_float2(L[i], L[k]));
      }
    } else {
      Rec r = cf;
#pragma unroll
      for (int i = 0; i < CH; ++i) {
        yv[i] = r.out(v);
        r.push(v, L[i]);
      }
      r = cb;
#pragma unroll
      for (int i = CH - 1; i >= 0; --i) {
        yv[i] += fmaf(v.b0, L[i], r.out(v));
        r.push(v, L[i]);
      }
    }
    // planes hold sigma^2 x the one-sided blur: the column pass then only
    // negates (R_L = -sigma^2 (D20 + D02)), and 16-bit planes keep the
    // magnitude of R at every scale (the blur alone for CH_ID)
    const float s2 = one ? 1.f : c.sigma2;
#pragma unroll
    for (int i = 0; i < CH; ++i) s_out[pad32(x0 + i)] = s2 * yv[i];
    __syncthreads();
    const long row = (F.prow + (long)s * H + y) * PWb;
    if (EDGE) {
      float *dst = edge + F.eoff + ((long)s * 2 + yw) * PWb;
      for (int e = tid; e < W; e += NT) dst[e] = s_out[pad32(e)];
    } else if (st == ST_F32) {
      float *dst = static_cast<float *>(P) + row;
      for (int e = tid; e < W; e += NT) dst[e] = s_out[pad32(e)];
    } else if (st == ST_F16) {
      __half *dst = static_cast<__half *>(P) + row;
      for (int e = tid; e < W; e += NT) {
        const float val = s_out[pad32(e)];
        ovf |= fabsf(val) > F16_MAX;
        dst[e] = __float2half_rn(val);
      }
    } else {
      __nv_bfloat16 *dst = static_cast<__nv_bfloat16 *>(P) + row;
      for (int e = tid; e < W; e += NT) dst[e] = __float2bfloat16_rn(s_out[pad32(e)]);
    }
    __syncthreads();
  }
}

// Row pass: one block per row, persistent over the rows of the launch's
// frames; items H and H + 1 of a frame are its two U-only edge rows.  All
// frames of a launch share the block width (chunks of CH pixels per thread).
// ID: the identity channel of the D = 5 bank (a separate instance keeps the
// other channels' code as it is).
template <class Rec, bool ID>
__global__ void __launch_bounds__(256) k_row(const FrameDev *__restrict__ fr, Items it,
                                             const Coef *__restrict__ coef, int S, void *__restrict__ P,
                                             int st, long PWb, float *__restrict__ edge,
                                             DevStatus *__restrict__ status, int chan) {
  extern __shared__ float sm[];
  __shared__ FrameDev s_fr;
  bool ovf = false;  // a value beyond the f16 range
  int k = 0;
  const int nitems = items_total(it);
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    int local;
    k = item_frame(it, item, k, local);
    stage_frame(&s_fr, fr, it, k);  // the previous item ended with __syncthreads
    __syncthreads();
    const FrameDev &F = s_fr;
    const bool e = local >= F.H;
    row_body<Rec, ID>(F, e, e ? local - F.H : local, chan, coef, S, P, st, PWb, edge, ovf, sm);
  }
  if (ovf) atomicExch(&status->range, 1);
}

// ---------------------------------------------------------------------------
// column passes
// ---------------------------------------------------------------------------
// input of the column recursion at row r (phantom rows use the held one-sided
// rows of U at the frame's first/last row)
template <int ST>
__device__ __forceinline__ float col_in(const typename Store<ST>::T *Pc, long PWb, int r, int H, float top,
                                        float bot) {
  return r < 0 ? top : (r >= H ? bot : Store<ST>::ld(Pc[(long)r * PWb]));
}

// Zero-state end states of every LC-row column segment, both directions.
// Item: (128-column block, segment, scale) of a frame.
template <class Rec, int ST, int LC>
__global__ void __launch_bounds__(128) k_colseg(const FrameDev *__restrict__ fr, Items it,
                                                const typename Store<ST>::T *__restrict__ P, long PWb,
                                                const float *__restrict__ edge,
                                                const Coef *__restrict__ coef, float *__restrict__ E) {
  int k = 0;
  const int nitems = items_total(it);
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    int local;
    k = item_frame(it, item, k, local);
    const FrameDev F = fr[__ldg(it.fl + k)];  // by value: fields stay in registers
    const int H = F.H, W = F.W, nseg = F.nseg;
    const int nxb = (W + 127) / 128;
    const int xb = local % nxb, rest = local / nxb;
    const int c = rest % nseg, s = rest / nseg;
    const int x = xb * 128 + threadIdx.x;
    if (x >= W) continue;
    typename Rec::View v;
    v.load(coef[s]);
    const typename Store<ST>::T *Pc = P + (F.prow + (long)s * H) * PWb + x;
    const float *ed = edge + F.eoff + (long)s * 2 * PWb + x;
    const float top = ed[0], bot = ed[PWb];
    Rec r;
    const long fs = (long)Rec::NF * PWb;
    float *Ef = E + F.coff + (((long)s * nseg + c) * 2 + 0) * fs + x;
    // causal segment: rows [c LC - 1, (c+1) LC - 1); anticausal: rows (c+1) LC
    // down to c LC + 1.  Inside the frame the two directions run side by
    // side (two independent recursions), their loads unconditional and issued
    // 8 rows of each at a time ahead of the steps.
    const int rf = c * LC - 1, rb = (c + 1) * LC;
    if (rf >= 0 && rb < H) {
      const typename Store<ST>::T *pf = Pc + (long)rf * PWb, *pb = Pc + (long)rb * PWb;
      Rec q;
      if constexpr (Rec::kPacked) {
        typename Rec::Pair r2;
        const typename Rec::Pair::Coefs pc(v);
        r2.zero();
#pragma unroll
        for (int i0 = 0; i0 < LC; i0 += 8) {
          float inf[8], inb[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            inf[u] = Store<ST>::ld(pf[(long)(i0 + u) * PWb]);
            inb[u] = Store<ST>::ld(pb[-(long)(i0 + u) * PWb]);
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) r2.push(pc, make_float2(inf[u], inb[u]));
        }
        r2.get(r, q);
      } else {
        r.zero();
        q.zero();
#pragma unroll
        for (int i0 = 0; i0 < LC; i0 += 8) {
          float inf[8], inb[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            inf[u] = Store<ST>::ld(pf[(long)(i0 + u) * PWb]);
            inb[u] = Store<ST>::ld(pb[-(long)(i0 + u) * PWb]);
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            r.push(v, inf[u]);
            q.push(v, inb[u]);
          }
        }
      }
      r.store(Ef, PWb);
      q.store(Ef + fs, PWb);
    } else {
      r.zero();
#pragma unroll 8
      for (int i = 0; i < LC; ++i) r.push(v, col_in<ST>(Pc, PWb, rf + i, H, top, bot));
      r.store(Ef, PWb);
      r.zero();
#pragma unroll 8
      for (int i = 0; i < LC; ++i) r.push(v, col_in<ST>(Pc, PWb, rb - i, H, top, bot));
      r.store(Ef + fs, PWb);
    }
  }
}

// Carries of the column segments, one thread per (column, scale, direction):
// C_0 = steady state of the held row, C_{k+1} = Phi^LC C_k + e_k in the
// direction's segment order; the segment states e_k are replaced by the C_k.
// Segment states are read 8 at a time ahead of the sequential fold.
// Item: (128-column block, scale, direction) of a frame.
template <class Rec, int LC>
__global__ void __launch_bounds__(128) k_colfold(const FrameDev *__restrict__ fr, Items it, long PWb,
                                                 const float *__restrict__ edge,
                                                 const Coef *__restrict__ coef, float *__restrict__ E, int S) {
  int k = 0;
  const int nitems = items_total(it);
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    int local;
    k = item_frame(it, item, k, local);
    const FrameDev F = fr[__ldg(it.fl + k)];  // by value: fields stay in registers
    const int W = F.W, nseg = F.nseg;
    const int nxb = (W + 127) / 128;
    const int xb = local % nxb, rest = local / nxb;
    const int s = rest % S, dir = rest / S;  // dir 0: top-down, 1: bottom-up
    const int x = xb * 128 + threadIdx.x;
    if (x >= W) continue;
    const Coef &c = coef[s];
    const long fs = (long)Rec::NF * PWb;
    float *base = E + F.coff + ((long)s * nseg * 2 + dir) * fs + x;  // segment k at base + 2 k fs
    Rec st;
    st.hold(c, edge[F.eoff + ((long)s * 2 + dir) * PWb + x]);
    // segment k's end state is read, then its slot receives the carry into
    // segment k; batches of 8 alternate, the next batch's loads in flight
    // while the current one is folded
    constexpr int BATCH = 8;
    auto slot = [&](int kk) { return base + 2L * (dir ? nseg - 1 - kk : kk) * fs; };
    auto fetch = [&](Rec (&e)[BATCH], int k0) {
#pragma unroll
      for (int u = 0; u < BATCH; ++u)
        if (k0 + u < nseg) e[u].load(slot(k0 + u), PWb);
    };
    auto fold = [&](const Rec (&e)[BATCH], int k0) {
#pragma unroll
      for (int u = 0; u < BATCH; ++u) {
        const int kk = k0 + u;
        if (kk >= nseg) break;
        st.store(slot(kk), PWb);
        Rec n = e[u];
        n.combine_m(c, LC / CH, st);  // Phi^LC st + e (LC a multiple of CH)
        st = n;
      }
    };
    Rec ea[BATCH], eb[BATCH];
    fetch(ea, 0);
    for (int k0 = 0; k0 < nseg; k0 += 2 * BATCH) {
      fetch(eb, k0 + BATCH);
      fold(ea, k0);
      fetch(ea, k0 + 2 * BATCH);
      fold(eb, k0 + BATCH);
    }
  }
}

// Column pass + detector.  Item: a (32-column, LC+2-row) tile of a frame; one
// warp per scale, one thread per (column, scale).  The tile of every scale's
// one-sided plane arrives by TMA into shared memory; rows outside the frame
// take the held values.  Both recursions run from shared memory, the causal
// outputs stay in registers, and R overwrites the input in place for the
// detector.
//
// f32 planes: box 36 x 66 (the TMA x coordinate must be a multiple of 4
// floats, so the tile starts up to 3 columns early), rows of 36 floats.
// 16-bit planes: box 40 x NR (x a multiple of 8 elements) lands at byte
// coldet_c16b(NR) of the scale's region; the causal pass widens it row by row
// into f32 rows of 32 floats from the region's start.  f32 row i ends at
// 128 (i + 1) and 16-bit row j starts at c16b + 80 j; the warp is
// synchronised every 8 rows, so the offset is the least multiple of 128 with
// which no write of a group reaches a 16-bit row of that group or later.
constexpr int CLD = 36;
constexpr int CBOX16 = 40;  // 16-bit box width (elements)
constexpr uint32_t CWAIT_LIMIT = 1u << 20;

// f32 rows reserved per scale: NR rounded up to 8 (8 rows of 144 B = 9 x 128 B)
__host__ __device__ constexpr int coldet_cnrp(int NR) { return (NR + 7) / 8 * 8; }
__host__ __device__ constexpr int coldet_c16b(int NR) {
  int m = 0;
  for (int g = 0; 8 * g < NR; ++g) {
    const int end = 128 * (8 * (g + 1) < NR ? 8 * (g + 1) : NR);  // end of the group's f32 writes
    const int need = end - 80 * 8 * g;                              // minus start of its first 16-bit row
    m = need > m ? need : m;
  }
  return (m + 127) / 128 * 128;
}
__host__ __device__ constexpr int coldet_c16reg(int NR) {
  const int a = coldet_c16b(NR) + NR * CBOX16 * 2, b = NR * 128;
  return ((a > b ? a : b) + 127) / 128 * 128;
}
static_assert(coldet_c16b(66) == 3712 && coldet_c16b(34) == 2176, "16-bit box offsets");

template <int ST, int LC>
__host__ __device__ constexpr int coldet_region_floats() {
  return ST == ST_F32 ? coldet_cnrp(LC + 2) * CLD : coldet_c16reg(LC + 2) / 4;
}

template <class Rec, int ST, int LC>
__global__ void __launch_bounds__(512) __maxnreg__(LC == 32 ? Rec::kColdetRegs32 : 128) k_coldet(const __grid_constant__ CUtensorMap map,
                                                const FrameDev *__restrict__ fr, Items it, long PWb,
                                                const float *__restrict__ edge,
                                                const Coef *__restrict__ coef, int S,
                                                const float *__restrict__ E, DetectArgs da) {
  using T = typename Store<ST>::T;
  constexpr bool F32 = ST == ST_F32;
  constexpr int NR = LC + 2;
  constexpr int REG = coldet_region_floats<ST, LC>();  // floats per scale
  constexpr int LD = F32 ? CLD : 32;                   // f32 row stride
  constexpr int C16B = coldet_c16b(NR);
  static_assert((coldet_cnrp(NR) * CLD * 4) % TMA_SMEM_ALIGN == 0 && C16B % TMA_SMEM_ALIGN == 0 &&
                    (REG * 4) % TMA_SMEM_ALIGN == 0,
                "scale regions and boxes 128-byte aligned");
  extern __shared__ __align__(128) float sm_raw[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ FrameDev s_fr;
  float *buf = align_smem(sm_raw);  // [S][REG]
  float *red = buf + (long)S * REG;  // detector scratch
  const int tid = threadIdx.x, lane = tid & 31, s = tid >> 5;
  constexpr int XA = F32 ? 4 : 8;  // TMA x alignment in elements
  constexpr int BW = F32 ? CLD : CBOX16;
  if (tid == 0) {
    mbar_init(&mbar, 1);
    fence_proxy_async();
  }
  __syncthreads();  // no thread polls the barrier before it is initialised
  const Coef &cf = coef[s];
  typename Rec::View v;
  v.load(cf);
  const long fs = (long)Rec::NF * PWb;
  const float sgn = da.raw ? 1.f : -1.f;
  uint32_t phase = 0;
  int k = 0;
  const int nitems = items_total(it);
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    int local;
    k = item_frame(it, item, k, local);
    stage_frame(&s_fr, fr, it, k);  // the previous item ended with __syncthreads
    __syncthreads();
    const FrameDev &F = s_fr;
    const int H = F.H, W = F.W, nseg = F.nseg;
    const int ntx = (W + TW - 1) / TW;
    const int c = local / ntx;
    const int x0 = (local % ntx) * TW - 1;
    const int off = ((x0 % XA) + XA) % XA;
    const int xv = min(max(x0 + lane, 0), W - 1);
    const int r0 = c * LC - 1;
    const long prow = F.prow;
    if (tid == 0 && !da.wait_test) {
      fence_proxy_async();  // earlier generic accesses of the buffer before the async writes
      mbar_arrive_expect_tx(&mbar, (uint32_t)(S * NR * BW * sizeof(T)));
      for (int t = 0; t < S; ++t) {
        void *dst = F32 ? (void *)(buf + (long)t * REG) : (void *)((char *)(buf + (long)t * REG) + C16B);
        if (!tma_load_2d(dst, &map, x0 - off, (int)(prow + (long)t * H + r0), &mbar, (int)sizeof(T)))
          atomicExch(&da.status->error, 2);
      }
    }
    const float *Ef = E + F.coff + (((long)s * nseg + c) * 2) * fs + xv;
    Rec r;
    r.load(Ef, PWb);
    const bool ok = mbar_wait_bounded(&mbar, phase, da.wait_test ? da.wait_test : CWAIT_LIMIT);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicExch(&da.status->error, 1);
      return;
    }
    float *b = buf + (long)s * REG + (F32 ? off : 0) + lane;
    const bool outside = r0 < 0 || r0 + NR > H;
    float top = 0.f, bot = 0.f;
    if (outside) {
      const float *ed = edge + F.eoff + (long)s * 2 * PWb + xv;
      top = ed[0];
      bot = ed[PWb];
    }
    // causal pass; rows outside the frame take the held one-sided rows of U
    // (written back for the anticausal pass), 16-bit input is widened in place
    const T *b16 = reinterpret_cast<const T *>(reinterpret_cast<const char *>(buf + (long)s * REG) + C16B) +
                   off + lane;
    float yp[NR];
    if constexpr (Rec::kPacked) {
      // rows outside the frame take the held rows, 16-bit input is widened
      // in place (top-down, the warp in step every 8 rows), then step i
      // advances the causal chain at row i and the anticausal one at row
      // NR-1-i; a row's R is formed when its second output arrives, with the
      // operations of the scalar passes: sgn (y+ + (b0 x + y-))
      if (!F32 || outside) {
#pragma unroll
        for (int i = 0; i < NR; ++i) {
          const int y = r0 + i;
          float in = F32 ? b[i * LD] : Store<ST>::ld(b16[i * CBOX16]);
          if (outside) in = y < 0 ? top : (y >= H ? bot : in);
          b[i * LD] = in;
          if ((i & 7) == 7) __syncwarp();
        }
        __syncwarp();
      }
      Rec q;
      q.load(Ef + fs, PWb);
      typename Rec::Pair r2;
      const typename Rec::Pair::Coefs pc(v);
      r2.set(r, q);
#pragma unroll
      for (int i = 0; i < NR; ++i) {
        const int k = NR - 1 - i;
        const float xi = b[i * LD], xk = b[k * LD];
        const float2 o = r2.out(pc);
        if (i < k) {
          yp[i] = o.x;  // y+ first
          yp[k] = o.y;  // y- first
        } else {
          // R_L = -sigma^2 (D20 + D02) (planes carry sigma^2); raw channel: +sigma^2 D
          b[i * LD] = sgn * (o.x + fmaf(v.b0, xi, yp[i]));
          b[k * LD] = sgn * (yp[k] + fmaf(v.b0, xk, o.y));
        }
        r2.push(pc, make_float2(xi, xk));
      }
    } else {
#pragma unroll
      for (int i = 0; i < NR; ++i) {
        const int y = r0 + i;
        float in = F32 ? b[i * LD] : Store<ST>::ld(b16[i * CBOX16]);
        if (outside) in = y < 0 ? top : (y >= H ? bot : in);
        if (!F32 || outside) b[i * LD] = in;
        yp[i] = r.out(v);
        r.push(v, in);
        if ((i & 7) == 7) __syncwarp();
      }
      __syncwarp();
      r.load(Ef + fs, PWb);
#pragma unroll
      for (int i = NR - 1; i >= 0; --i) {
        const float in = b[i * LD];
        // R_L = -sigma^2 (D20 + D02) (planes carry sigma^2); raw channel: +sigma^2 D
        b[i * LD] = sgn * (yp[i] + fmaf(v.b0, in, r.out(v)));
        r.push(v, in);
      }
    }
    __syncthreads();
    DetectArgs a = da;
    a.S = S;
    a.NR = NR;
    a.x0 = x0;
    a.r0 = r0;
    a.H = H;
    a.W = W;
    a.frame = F.index;
    a.resp = F.resp;
    a.rplane = F.rplane;
    a.rpitch = F.rpitch;
    a.rmx = F.rmx;
    a.rmy = F.rmy;
    a.ld = LD;
    a.coff = F32 ? off : 0;
    a.srows = REG / LD;
    detect_tile(buf, red, a);
    fence_proxy_async();  // this thread's writes of the tile before the next item's async copies
    __syncthreads();      // the tile is read before the next item's copies overwrite it
  }
}

// ---------------------------------------------------------------------------
// single-read column pass
// ---------------------------------------------------------------------------
// k_colscan reads every plane once: the carries of the column recursions are
// found while the tiles sit in shared memory, instead of by a separate pass
// over the planes (k_colseg + k_colfold).  A cluster of SCAN_G CTAs takes a
// super-tile: SCAN_G consecutive 32-row tiles (34 rows with the detector's
// halo) of one 32-column strip, all scales.  Per super-tile:
//   1. each CTA loads its tile (TMA) and runs both recursions from the zero
//      state over its segment (the same segments as k_colseg): e+, e-;
//   2. through distributed shared memory each CTA folds the end states of the
//      tiles above it (P = sum_i Phi^(32(r-1-i)) e+_i) and below it (Q); the
//      bottom and top CTAs form the super-tile's end states A+ and A- and
//      publish them in global memory (a flag per super-tile and direction);
//   3. the bottom CTA folds the carry entering the super-tile from above,
//      C+ = Phi^256 (... (Phi^256 hold(top) + A+_0) ...) + A+_(k-1), from
//      the published end states of the strip's super-tiles above it, in
//      that fixed order; the top CTA folds C- from the super-tiles below,
//      starting at the held bottom.  A fixed order makes the result the same
//      on every run and for every schedule of the super-tiles;
//   4. each CTA's carries are Phi^(32 r) C+ + P and Phi^(32 (n-1-r)) C- + Q,
//      and the final recursions, the response and the detector run on the
//      tile in shared memory as in k_coldet.
// Super-tiles are taken in ticket order, strip by strip from the top, so a
// super-tile waits only on super-tiles that already hold a cluster or that
// need none of its results; the host launches this pass only when twice the
// super-tiles of a strip fit on the GPU at once.  Every wait is bounded by
// wall time; a wait that gives up (or a call that has already failed) turns
// the rest of the launch into no-ops that still pass every cluster barrier.
constexpr int SCAN_G = 8;           // tiles (CTAs) per cluster
constexpr int SCAN_LC = 32;         // rows per tile (one CH chunk: Phi^32 = phiM[0])
constexpr unsigned long long SCAN_WAIT_NS = 2000000000ull;  // 2 s
constexpr int SCAN_BATCH = 4;       // end states of other super-tiles loaded at once

struct ScanArgs {
  int *ticket;     // launch ticket counter (zero before the launch)
  unsigned *flag;  // [2][U]: 1 once the super-tile's end state of the direction is published
  float *data;     // [U][2 dir][NF][S][32]: the super-tiles' zero-state end states
  int U;           // super-tiles of the launch
  // gated calls: the active-tile maps (64 x 64 tiles, FrameDev.aoff); the
  // final recursions and the detector run only on tiles whose interior meets
  // an active tile (the loads and end states run everywhere: the carries need
  // every tile).  Null: every tile.
  const unsigned char *act;
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait until the n flags flag[0..n) are all >= 1 (the warp polls 32 at a
// time).  Returns false if a wait gave up (error 4 recorded) or the call has
// already failed.
__device__ __forceinline__ bool scan_wait_all(const unsigned *flag, int n, DevStatus *st) {
  const int lane = threadIdx.x & 31;
  for (int j0 = 0; j0 < n; j0 += 32) {
    const int j = j0 + lane;
    unsigned long long t0 = 0;
    for (unsigned i = 0;; ++i) {
      const bool ok = j >= n || ld_acquire_u32(flag + j) >= 1u;
      if (__all_sync(0xffffffffu, ok)) break;
      if (*reinterpret_cast<volatile int *>(&st->error)) return false;
      const unsigned long long now = global_ns();
      if (i == 0) {
        t0 = now;
      } else if (now - t0 > SCAN_WAIT_NS) {
        if (lane == 0) atomicCAS(&st->error, 0, 4);
        return false;
      }
      __nanosleep(100);
    }
  }
  return true;
}

// Step 3 of k_colscan for direction dir (0: causal, by the super-tile's
// bottom CTA; 1: anticausal, by its top CTA), all threads of the CTA: the
// super-tile's end state A = Phi^32 P + e of this tile (P: the folded end
// states of the cluster's other tiles on the far side), published in global
// memory; then the carry entering the super-tile, folded in a fixed order
// from the held edge row and the published end states of the strip's
// super-tiles on the near side, and stored into every CTA of the cluster.
// Kept out of line: the kernel's main path needs its registers.
template <class Rec>
__device__ __noinline__ void colscan_publish(int dir, const Coef &cf, const float *agg, const float *pq,
                                             float *cin, ScanArgs sa, long DS, int u, int sup, int nsup,
                                             int ntile, int nreal, float edge_row, DevStatus *status) {
  namespace cg = cooperative_groups;
  const int lane = threadIdx.x & 31, s = threadIdx.x >> 5;
  const long SS = DS / Rec::NF, o = (long)dir * DS + s * 32 + lane;
  Rec A, P;
  A.load(agg + o, SS);
  P.load(pq + o, SS);
  A.combine_m(cf, 1, P);
  A.store(sa.data + (long)u * 2 * DS + o, SS);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) st_release_u32(sa.flag + (long)dir * sa.U + u, 1u);
  Rec C;
  C.hold(cf, edge_row);
  // causal: the super-tiles above, from the strip's first; anticausal: those
  // below, from the strip's last (nlast tiles) up
  const int n = dir == 0 ? sup : nsup - 1 - sup;
  const int ufar = dir == 0 ? u - sup : u - sup + nsup - 1, step = dir == 0 ? 1 : -1;
  const int nlast = ntile - (nsup - 1) * SCAN_G;
  if (scan_wait_all(sa.flag + (dir == 0 ? (long)ufar : (long)sa.U + u + 1), n, status))
    for (int j0 = 0; j0 < n; j0 += SCAN_BATCH) {
      Rec e[SCAN_BATCH];
#pragma unroll
      for (int q = 0; q < SCAN_BATCH; ++q)
        if (j0 + q < n) e[q].load_cg(sa.data + (long)(ufar + step * (j0 + q)) * 2 * DS + o, SS);
#pragma unroll
      for (int q = 0; q < SCAN_BATCH; ++q)
        if (j0 + q < n) {
          // C enters the super-tile being added: whole (SCAN_G tiles) unless
          // it is the strip's last
          e[q].combine_m(cf, (dir == 1 && j0 + q == 0) ? nlast : SCAN_G, C);
          C = e[q];
        }
    }
  cg::cluster_group cl = cg::this_cluster();
  for (int i = 0; i < nreal; ++i) C.store(cl.map_shared_rank(cin, i) + o, SS);
}

template <class Rec, int ST>
__host__ __device__ constexpr int colscan_scratch_floats(int S) {
  // detector scratch, or (aliasing it before the detector runs) the tile's
  // end states, the super-tile carries and the end states of the tiles above
  // and below: 3 x [2][NF][S][32]
  return (SCAN_LC + 2) * 32 * 2 + ((SCAN_LC + 2) * 32 * 2 + 3) / 4 > 6 * Rec::NF * S * 32
             ? (SCAN_LC + 2) * 32 * 2 + ((SCAN_LC + 2) * 32 * 2 + 3) / 4
             : 6 * Rec::NF * S * 32;
}

template <class Rec, int ST>
__global__ void __launch_bounds__(512) __maxnreg__(Rec::kColdetRegs32) k_colscan(const __grid_constant__ CUtensorMap map,
                                                const FrameDev *__restrict__ fr, Items it, long PWb,
                                                const float *__restrict__ edge,
                                                const Coef *__restrict__ coef, int S, ScanArgs sa,
                                                DetectArgs da) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  using T = typename Store<ST>::T;
  constexpr bool F32 = ST == ST_F32;
  constexpr int LC = SCAN_LC, NR = LC + 2, G = SCAN_G, NF = Rec::NF;
  constexpr int REG = coldet_region_floats<ST, LC>();
  constexpr int LD = F32 ? CLD : 32;
  constexpr int C16B = coldet_c16b(NR);
  extern __shared__ __align__(128) float sm_raw[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ FrameDev s_fr;
  __shared__ int s_ticket, s_bad;
  float *buf = align_smem(sm_raw);   // [S][REG]
  float *red = buf + (long)S * REG;  // detector scratch
  const long SS = (long)S * 32;      // stride of a state component in agg / cin
  float *agg = red;                  // [2][NF][S][32] this tile's zero-state end states
  float *cin = red + 2 * NF * SS;    // [2][NF][S][32] carries entering the super-tile
  float *pq = red + 4 * NF * SS;     // [2][NF][S][32] end states of the tiles above (P) and below (Q)
  const int rank = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, s = tid >> 5;
  constexpr int XA = F32 ? 4 : 8;
  constexpr int BW = F32 ? CLD : CBOX16;
  if (tid == 0) {
    mbar_init(&mbar, 1);
    fence_proxy_async();
  }
  __syncthreads();
  const Coef &cf = coef[s];
  const long DS = (long)NF * SS;  // floats of one (dir, kind) record of a super-tile
  uint32_t phase = 0;
  int k = 0;
  for (;;) {
    if (rank == 0 && tid == 0) {
      const int u = atomicAdd(sa.ticket, 1);
      for (int i = 0; i < G; ++i) *cl.map_shared_rank(&s_ticket, i) = u;
    }
    cl.sync();  // B0: the ticket is known; the previous super-tile is done everywhere
    const int u = s_ticket;
    if (u >= sa.U) break;
    int local;
    k = item_frame(it, u, k, local);
    stage_frame(&s_fr, fr, it, k);
    if (tid == 0) s_bad = *reinterpret_cast<volatile int *>(&da.status->error);
    __syncthreads();
    const FrameDev &F = s_fr;
    const bool bad = s_bad != 0;
    const int H = F.H, W = F.W;
    const int ntile = (H + LC - 1) / LC, nsup = (ntile + G - 1) / G;
    const int strip = local / nsup, sup = local % nsup;
    const int nreal = min(G, ntile - sup * G);
    const bool real = rank < nreal;
    const int t = sup * G + rank;
    const int x0 = strip * TW - 1;
    const int off = ((x0 % XA) + XA) % XA;
    const int xv = min(max(x0 + lane, 0), W - 1);
    const int r0 = t * LC - 1;
    const float *ed = edge + F.eoff + (long)s * 2 * PWb + xv;
    float *b = buf + (long)s * REG + (F32 ? off : 0) + lane;
    // 1. load and zero-state end states
    if (real && !bad) {
      typename Rec::View v;  // loaded where used: fewer registers live across the loop
      v.load(cf);
      if (tid == 0 && !da.wait_test) {
        fence_proxy_async();
        mbar_arrive_expect_tx(&mbar, (uint32_t)(S * NR * BW * sizeof(T)));
        for (int q = 0; q < S; ++q) {
          void *dst = F32 ? (void *)(buf + (long)q * REG) : (void *)((char *)(buf + (long)q * REG) + C16B);
          if (!tma_load_2d(dst, &map, x0 - off, (int)(F.prow + (long)q * H + r0), &mbar, (int)sizeof(T)))
            atomicExch(&da.status->error, 2);
        }
      }
      const bool ok = mbar_wait_bounded(&mbar, phase, da.wait_test ? da.wait_test : CWAIT_LIMIT);
      phase ^= 1u;
      if (!ok && tid == 0) atomicCAS(&da.status->error, 0, 1);
      const bool outside = r0 < 0 || r0 + NR > H;
      float top = 0.f, bot = 0.f;
      if (outside) {
        top = ed[0];
        bot = ed[PWb];
      }
      // causal segment: tile rows 0 .. LC-1; every row is widened to f32 (and
      // rows outside the frame take the held edge rows) in place
      const T *b16 = reinterpret_cast<const T *>(reinterpret_cast<const char *>(buf + (long)s * REG) + C16B) +
                     off + lane;
      Rec e;
      e.zero();
#pragma unroll
      for (int i = 0; i < NR; ++i) {
        const int y = r0 + i;
        float in = F32 ? b[i * LD] : Store<ST>::ld(b16[i * CBOX16]);
        if (outside) in = y < 0 ? top : (y >= H ? bot : in);
        if (!F32 || outside) b[i * LD] = in;
        if (i < LC) e.push(v, in);
        if ((i & 7) == 7) __syncwarp();
      }
      __syncwarp();
      e.store(agg + s * 32 + lane, SS);
      // anticausal segment: tile rows NR-1 down to 2
      e.zero();
#pragma unroll
      for (int i = NR - 1; i >= 2; --i) e.push(v, b[i * LD]);
      e.store(agg + DS + s * 32 + lane, SS);
    }
    cl.sync();  // B1: every tile's end states are visible to the cluster
    // 2. end states of the tiles above (P) and below (Q) this one, kept in
    // shared memory until the carries arrive
    if (real) {
      Rec P;
      P.zero();
      for (int i = 0; i < rank; ++i) {
        Rec n;
        n.load(cl.map_shared_rank(agg, i) + s * 32 + lane, SS);
        n.combine_m(cf, 1, P);  // Phi^32 P + e_i
        P = n;
      }
      P.store(pq + s * 32 + lane, SS);
      P.zero();
      for (int i = nreal - 1; i > rank; --i) {
        Rec n;
        n.load(cl.map_shared_rank(agg, i) + DS + s * 32 + lane, SS);
        n.combine_m(cf, 1, P);
        P = n;
      }
      P.store(pq + DS + s * 32 + lane, SS);
    }
    // 3. the super-tile's end states and the carries entering it
    if (rank == nreal - 1)
      colscan_publish<Rec>(0, cf, agg, pq, cin, sa, DS, u, sup, nsup, ntile, nreal, ed[0], da.status);
    if (rank == 0)
      colscan_publish<Rec>(1, cf, agg, pq, cin, sa, DS, u, sup, nsup, ntile, nreal, ed[PWb], da.status);
    cl.sync();  // B2: the super-tile's carries are in every CTA
    // 4. this tile's carries, final recursions, response, detector
    if (real && !bad && (!sa.act || any_active(F, sa.act, strip * TW, strip * TW + TW, t * LC, t * LC + LC))) {
      Rec cp, cq;
      cp.load(cin + s * 32 + lane, SS);
      cq.load(cin + DS + s * 32 + lane, SS);
      if (rank > 0) {
        Rec n;
        n.load(pq + s * 32 + lane, SS);
        n.combine_m(cf, rank, cp);
        cp = n;
      }
      if (rank < nreal - 1) {
        Rec n;
        n.load(pq + DS + s * 32 + lane, SS);
        n.combine_m(cf, nreal - 1 - rank, cq);
        cq = n;
      }
      typename Rec::View v;
      v.load(cf);
      const float sgn = da.raw ? 1.f : -1.f;
      float yp[NR];
      Rec r = cp;
#pragma unroll
      for (int i = 0; i < NR; ++i) {
        yp[i] = r.out(v);
        r.push(v, b[i * LD]);
      }
      r = cq;
#pragma unroll
      for (int i = NR - 1; i >= 0; --i) {
        const float in = b[i * LD];
        b[i * LD] = sgn * (yp[i] + fmaf(v.b0, in, r.out(v)));
        r.push(v, in);
      }
      __syncthreads();
      DetectArgs a = da;
      a.S = S;
      a.NR = NR;
      a.x0 = x0;
      a.r0 = r0;
      a.H = H;
      a.W = W;
      a.frame = F.index;
      a.resp = F.resp;
      a.rplane = F.rplane;
      a.rpitch = F.rpitch;
      a.rmx = F.rmx;
      a.rmy = F.rmy;
      a.ld = LD;
      a.coff = F32 ? off : 0;
      a.srows = REG / LD;
      detect_tile(buf, red, a);
      fence_proxy_async();  // generic accesses of the buffer before the next tile's async copies
    }
    __syncthreads();
  }
}

template <class Rec, int ST>
size_t colscan_smem(int S) {
  return ((size_t)S * coldet_region_floats<ST, SCAN_LC>() + colscan_scratch_floats<Rec, ST>(S)) * sizeof(float) +
         TMA_SMEM_ALIGN;
}

template <class Rec, int ST>
cudaLaunchConfig_t colscan_config(int S, int nclusters, cudaStream_t st, cudaLaunchAttribute *attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nclusters * SCAN_G));
  cfg.blockDim = dim3((unsigned)(32 * S));
  cfg.dynamicSmemBytes = colscan_smem<Rec, ST>(S);
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = SCAN_G;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// clusters of k_colscan<Rec, ST> resident on the current device at once (0:
// the kernel cannot run), cached per (device, S)
template <class Rec, int ST>
int colscan_clusters(int S) {
  constexpr int kMaxDev = 64;
  static int cache[kMaxDev][MAXS + 1];
  static bool attr_set[kMaxDev];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= kMaxDev || S < 1 || S > MAXS) return 0;
  if (cache[dev][S]) return cache[dev][S] > 0 ? cache[dev][S] : 0;
  if (!attr_set[dev]) {
    cudaFuncSetAttribute(k_colscan<Rec, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set[dev] = true;
  }
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t cfg = colscan_config<Rec, ST>(S, 1, nullptr, at);
  int n = 0;
  if (cfg.dynamicSmemBytes > 200 * 1024 ||
      cudaOccupancyMaxActiveClusters(&n, (void *)k_colscan<Rec, ST>, &cfg) != cudaSuccess)
    n = 0;
  cudaGetLastError();  // a failed query leaves no sticky error
  cache[dev][S] = n > 0 ? n : -1;
  return n;
}

// whether every super-tile of a strip of a frame of height maxH (and a
// second such bank running at the same time) fits on the device at once
template <class Rec, int ST>
bool colscan_fits(int S, int maxH) {
  const int nt = (maxH + SCAN_LC - 1) / SCAN_LC, nsup = (nt + SCAN_G - 1) / SCAN_G;
  return colscan_clusters<Rec, ST>(S) >= 2 * nsup;
}

template <class Rec>
bool colscan_fits_st(int storage, int S, int maxH) {
  switch (storage) {
    case ST_F32: return colscan_fits<Rec, ST_F32>(S, maxH);
    case ST_F16: return colscan_fits<Rec, ST_F16>(S, maxH);
    case ST_BF16: return colscan_fits<Rec, ST_BF16>(S, maxH);
    default: return false;
  }
}

template <class Rec, int ST, int LC>
int run_iir_st(const Plan &p, const BankArgs &a, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_row<Rec, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_row<Rec, ST == ST_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_coldet<Rec, ST, LC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_colscan<Rec, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  constexpr int NR = LC + 2;
  const size_t det_smem = ((size_t)a.S * coldet_region_floats<ST, LC>() + (size_t)NR * 32 * 2) * sizeof(float) +
                          (size_t)NR * 32 * 2 + TMA_SMEM_ALIGN;
  CUtensorMap map;
  if (encode_plane_map(&map, a.P, ST, p.PWb, p.prows, ST == ST_F32 ? CLD : CBOX16, NR)) return -1;
  DetectArgs da;
  da.thr = a.threshold;
  da.neigh = a.neigh;
  da.dark = 1;
  da.out = a.blobs;
  da.cap = a.cap;
  da.status = a.status;
  da.resp = nullptr;
  da.raw = a.raw;
  da.wait_test = a.wait_test;
  using TS = typename Store<ST>::T;
  // the identity channel (the D = 5 bank, f32 planes only) has its own instance
  if (a.chan == CH_ID && ST != ST_F32) return -1;
  auto row = [&](const Launch &l) {
    const size_t smem = (size_t)(3 * (pad32(l.nt * CH) + 1) + 64 * Rec::NF) * sizeof(float);
    if (smem > 200 * 1024) return false;
    const auto kfn = a.chan == CH_ID ? k_row<Rec, ST == ST_F32> : k_row<Rec, false>;
    const int nb = persistent_blocks((const void *)kfn, l.nt, smem, l.it.total, p.mult[PASS_ROW]);
    a.prof->begin("iir_row", st);
    kfn<<<nb, l.nt, smem, st>>>(p.fr, l.it, a.coef, a.S, a.P, a.storage, p.PWb, a.edge, a.status, a.chan);
    a.prof->end(st);
    return true;
  };
  auto seg = [&](const Launch &l) {
    const int nb = persistent_blocks((const void *)k_colseg<Rec, ST, LC>, 128, 0, l.it.total, p.mult[PASS_SEG]);
    a.prof->begin("iir_colseg", st);
    k_colseg<Rec, ST, LC><<<nb, 128, 0, st>>>(p.fr, l.it, static_cast<const TS *>(a.P), p.PWb, a.edge, a.coef,
                                          a.carry);
    a.prof->end(st);
  };
  auto fold = [&](const Launch &l) {
    const int nb = persistent_blocks((const void *)k_colfold<Rec, LC>, 128, 0, l.it.total, p.mult[PASS_FOLD]);
    a.prof->begin("iir_colfold", st);
    k_colfold<Rec, LC><<<nb, 128, 0, st>>>(p.fr, l.it, p.PWb, a.edge, a.coef, a.carry, a.S);
    a.prof->end(st);
  };
  auto det = [&](const Launch &l) {
    const int nb =
        persistent_blocks((const void *)k_coldet<Rec, ST, LC>, 32 * a.S, det_smem, l.it.total, p.mult[PASS_DET]);
    a.prof->begin("iir_coldet", st);
    k_coldet<Rec, ST, LC><<<nb, 32 * a.S, det_smem, st>>>(map, p.fr, l.it, p.PWb, a.edge, a.coef, a.S, a.carry, da);
    a.prof->end(st);
  };
  // single-read column pass: ticket and flags cleared, then one persistent
  // launch of clusters over every super-tile of the call
  auto scan = [&](const Launch &l) -> bool {
    const int U = l.it.total;
    const int ncl = colscan_clusters<Rec, ST>(a.S);
    if (ncl < 1) return false;
    CUtensorMap smap;
    if (encode_plane_map(&smap, a.P, ST, p.PWb, p.prows, ST == ST_F32 ? CLD : CBOX16, SCAN_LC + 2)) return false;
    ScanArgs sa;
    sa.ticket = static_cast<int *>(a.scan);
    sa.flag = reinterpret_cast<unsigned *>(static_cast<int *>(a.scan) + 32);
    sa.data = reinterpret_cast<float *>(static_cast<char *>(a.scan) + ((size_t)(32 + 2 * (size_t)U) * 4 + 255) / 256 * 256);
    sa.U = U;
    sa.act = a.gate_act;
    if (cudaMemsetAsync(a.scan, 0, (32 + 2 * (size_t)U) * sizeof(int), st) != cudaSuccess) return false;
    cudaLaunchAttribute at[1];
    const cudaLaunchConfig_t cfg = colscan_config<Rec, ST>(a.S, std::min(ncl, std::max(U, 1)), st, at);
    a.prof->begin("iir_colscan", st);
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_colscan<Rec, ST>, smap, p.fr, l.it, p.PWb,
                                             (const float *)a.edge, a.coef, a.S, sa, da);
    a.prof->end(st);
    return e == cudaSuccess;
  };
  if (a.scan) {
    if (p.per_frame) {
      for (int f = 0; f < p.nframes; ++f)
        if (!row(p.pass[PASS_ROW][f]) || !scan(p.scan[f])) return -1;
    } else {
      for (const Launch &l : p.pass[PASS_ROW])
        if (!row(l)) return -1;
      if (!scan(p.scan[0])) return -1;
    }
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
  }
  if (p.per_frame) {
    for (int f = 0; f < p.nframes; ++f) {
      if (!row(p.pass[PASS_ROW][f])) return -1;
      seg(p.pass[PASS_SEG][f]);
      fold(p.pass[PASS_FOLD][f]);
      det(p.pass[PASS_DET][f]);
    }
  } else {
    for (const Launch &l : p.pass[PASS_ROW])
      if (!row(l)) return -1;
    seg(p.pass[PASS_SEG][0]);
    fold(p.pass[PASS_FOLD][0]);
    det(p.pass[PASS_DET][0]);
  }
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

template <class Rec, int ST>
int run_iir_lc(const Plan &p, const BankArgs &a, cudaStream_t st) {
  switch (p.lc) {
    case 32: return run_iir_st<Rec, ST, 32>(p, a, st);
    case 64: return run_iir_st<Rec, ST, 64>(p, a, st);
    default: return -2;
  }
}

// all passes of a recursive bank for one recursion realisation
template <class Rec>
int run_iir(const Plan &p, const BankArgs &a, cudaStream_t st) {
  switch (a.storage) {
    case ST_F32: return run_iir_lc<Rec, ST_F32>(p, a, st);
    case ST_F16: return run_iir_lc<Rec, ST_F16>(p, a, st);
    case ST_BF16: return run_iir_lc<Rec, ST_BF16>(p, a, st);
    default: return -2;
  }
}

}  // namespace

}  // namespace kf
