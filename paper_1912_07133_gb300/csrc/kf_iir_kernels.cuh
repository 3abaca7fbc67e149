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

namespace kf {

namespace {

// ---------------------------------------------------------------------------
// one-sided recursions
// ---------------------------------------------------------------------------
template <int KK>
struct Chain {
  static constexpr int NF = KK;
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
    ef.zero();
    eb.zero();
#pragma unroll
    for (int i = 0; i < CH; ++i) ef.push(v, L[i]);
#pragma unroll
    for (int i = CH - 1; i >= 0; --i) eb.push(v, L[i]);
    Rec hlo, hhi;
    hlo.hold(c, in_lo);
    hhi.hold(c, in_hi);
    if (one && pre) hlo.push(v, xp.y);
    if (one && pre_hi) hhi.push(v, xp.z);
    const Rec cf = carry_scan<Rec, false>(ef, c, tid, NT, s_scan, hlo);
    const Rec cb = carry_scan<Rec, true>(eb, c, NT - 1 - tid, NT, s_scan, hhi);
    float yv[CH];
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

template <class Rec, int ST, int LC>
int run_iir_st(const Plan &p, const BankArgs &a, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_row<Rec, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_row<Rec, ST == ST_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_coldet<Rec, ST, LC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
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
