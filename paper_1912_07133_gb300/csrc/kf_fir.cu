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
// Passes (each persistent over the work items of the frames it covers, see
// kf_batch.cuh):
//   k_rowfir      (row, 2048-pixel segment) items: L with a K-pixel halo in
//                 shared memory, 16 outputs per thread in 8-tap register
//                 blocks, all scales in groups of three that share the
//                 symmetric pair sums; two extra rows per frame on U alone.
//   k_colfir_tma  128 rows x 32 columns x all scales per item, TMA-staged,
//                 all-scales detector.
//   k_colfir      64 rows x 32 columns, adjacent-scales detector.
#include <cudaTypedefs.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "kf_batch.cuh"
#include "kf_common.cuh"
#include "kf_detect.cuh"
#include "kf_internal.h"
#include "kf_tma.cuh"

namespace kf {

namespace {

constexpr int NOUT = 16;             // outputs per thread (register block)
constexpr int TB = 8;                // taps per block of the inner loop
constexpr int RNT = 128;             // threads per row CTA
constexpr int RLD = 8;               // row staging: elements per thread in flight (5 loads each)
constexpr int RSEG = RNT * NOUT;     // outputs per row CTA (2048)
constexpr int CNT = 128;             // threads per column CTA (4 warps x 32 columns)
constexpr int CROWS = 4 * NOUT;      // output rows per column CTA (64, incl. 2 halo rows)
constexpr int BOXW = 36;             // TMA box width (floats): 32 columns + alignment offset <= 3
constexpr int BOXH = 48;             // TMA box height (rows)
constexpr uint32_t WAIT_LIMIT = 1u << 20;

// taps h[0..K] padded with zeros to a multiple of TB beyond K
__device__ __forceinline__ void stage_taps(float *sh, const Coef &c, int K, int tid, int nt) {
  const int KP = ((K + TB - 1) / TB) * TB;
  for (int k = tid; k <= KP; k += nt) sh[k] = (k <= K) ? c.h[k] : 0.f;
}

// Taps for the tensor-core column pass as a zero-padded band,
// band[u] = h(|u - BAND0 - K|) for |u - BAND0 - K| <= K and 0 elsewhere, so
// that the Toeplitz entry A[r][q] = h(|q - r - K|) is band[BAND0 + q - r]
// without an absolute value or a range test.  Each tap is split into TF32
// parts, hi = tf32(h) and lo = tf32(h - hi), after multiplying by sgn (+-1,
// exact).
constexpr int BAND0 = 16;  // band[0..BAND0) pads the smallest index a fragment reads (q - r >= -15)

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return u;
}

__device__ __forceinline__ void stage_taps_band(float *th, float *tl, const Coef &c, int K, int len, float sgn,
                                                int tid, int nt) {
  for (int u = tid; u < len; u += nt) {
    const int m = abs(u - BAND0 - K);
    const float v = m <= K ? sgn * c.h[m] : 0.f;
    const uint32_t hi = to_tf32(v);
    th[u] = __uint_as_float(hi);
    tl[u] = __uint_as_float(to_tf32(v - __uint_as_float(hi)));
  }
}

// D += A B, one m16n8k8 TF32 tensor-core product (A 16 x 8 row-major, B 8 x 8)
__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Symmetric FIR on a register block of NOUT consecutive outputs.
// at(t) returns the input at offset t from the first output (t may be
// negative); the window loads for taps [k0, k0+TB) are statically indexed.
template <class At>
__device__ __forceinline__ void fir_block(const float *sh, int K, At at, float (&acc)[NOUT]) {
  const float h0 = sh[0];
#pragma unroll
  for (int j = 0; j < NOUT; ++j) acc[j] = h0 * at(j);
  for (int k0 = 1; k0 <= K; k0 += TB) {
    float A[NOUT + TB - 1], B[NOUT + TB - 1], hk[TB];
#pragma unroll
    for (int u = 0; u < TB; ++u) hk[u] = sh[k0 + u];
    // A[m] = x(m - k0 - TB + 1): left operands x(j - k) = A[j - u + TB - 1]
    // B[m] = x(k0 + m):          right operands x(j + k) = B[j + u]
#pragma unroll
    for (int m = 0; m < NOUT + TB - 1; ++m) {
      A[m] = at(m - k0 - TB + 1);
      B[m] = at(k0 + m);
    }
#pragma unroll
    for (int u = 0; u < TB; ++u)
#pragma unroll
      for (int j = 0; j < NOUT; ++j) acc[j] = fmaf(hk[u], A[j - u + TB - 1] + B[j + u], acc[j]);
  }
}

// Row layout in shared memory: 16 elements then 4 unused floats (20 per 16),
// so 128-bit loads of quads that start at multiples of 4 never straddle a gap
// and a quarter-warp whose threads start 16 elements apart hits 8 distinct
// 4-bank groups.
__host__ __device__ __forceinline__ constexpr int pad20(int e) { return e + ((e >> 4) << 2); }

// Scales of one group of the row pass: the pair sums x(j - k) + x(j + k) are
// the same for every scale, so a group forms each sum once and applies the
// taps of all its scales whose half-length reaches k.  The scales are ordered
// by K, largest first; groups of three keep the accumulators at 48 registers.
constexpr int RGS = ROW_GS;
constexpr int RWIN = NOUT + TB;  // window length of a block of 8 taps

// The two windows of one block of 8 taps: pa / pb point at the padded
// positions of the 16-element groups holding the left / right windows; OA / OB
// (0 or 8) are the windows' offsets inside them, so every load address is a
// compile-time offset from the two pointers.
template <int OA, int OB>
__device__ __forceinline__ void fir_row_windows(const float *pa, const float *pb, float (&A)[RWIN],
                                                float (&B)[RWIN]) {
#pragma unroll
  for (int q = 0; q < RWIN / 4; ++q) {
    const float4 a = *reinterpret_cast<const float4 *>(pa + pad20(OA + 4 * q));  // A[m] = x(base + m - k0 - 7)
    const float4 b = *reinterpret_cast<const float4 *>(pb + pad20(OB + 4 * q));  // B[m] = x(base + m + k0 - 1)
    A[4 * q + 0] = a.x, A[4 * q + 1] = a.y, A[4 * q + 2] = a.z, A[4 * q + 3] = a.w;
    B[4 * q + 0] = b.x, B[4 * q + 1] = b.y, B[4 * q + 2] = b.z, B[4 * q + 3] = b.w;
  }
}

// One block of 8 taps for NOUT consecutive outputs of the first NA scales of
// a group.  T[u]: the taps k0 + u of the group's scales (.x, .y, .z; zero
// beyond a scale's K).  Per scale the products are accumulated in increasing
// k, as a one-scale pass would.
template <int NA>
__device__ __forceinline__ void fir_row_mac8(const float (&A)[RWIN], const float (&B)[RWIN], const float4 *T,
                                             float (&acc)[RGS][NOUT]) {
  // output j, tap k0 + u: x(j - k0 - u) = A[j - u + 7], x(j + k0 + u) = B[j + u + 1]
#pragma unroll
  for (int u = 0; u < TB; ++u) {
    const float4 h = T[u];
#pragma unroll
    for (int j = 0; j < NOUT; ++j) {
      const float v = A[j - u + TB - 1] + B[j + u + 1];
      acc[0][j] = fmaf(h.x, v, acc[0][j]);
      if (NA > 1) acc[1][j] = fmaf(h.y, v, acc[1][j]);
      if (NA > 2) acc[2][j] = fmaf(h.z, v, acc[2][j]);
    }
  }
}

// Symmetric FIR of NOUT consecutive outputs for the scales of one group from
// a padded row: `row` points at element 0, `base` (a multiple of 16) is the
// first output, T[k] = the group's taps h_k (half-lengths K0 >= K1 >= K2; -1
// for a missing scale).  Taps are used 8 at a time: block i reads the left
// window x(base-8(i+1) .. +23) and the right window x(base+8i .. +23), six
// 128-bit loads each; the windows move by one 16-element group every second
// block.  The block's scales are those whose half-length reaches its first
// tap (the first na of the group).
__device__ __forceinline__ void fir_row_group(const float4 *T, int K0, int K1, int K2, const float *row, int base,
                                              float (&acc)[RGS][NOUT]) {
  const float4 h0 = T[0];
  const float *p0 = row + pad20(base);
#pragma unroll
  for (int q = 0; q < NOUT / 4; ++q) {
    const float4 v = *reinterpret_cast<const float4 *>(p0 + pad20(4 * q));
    const float x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      acc[0][4 * q + e] = h0.x * x[e];
      acc[1][4 * q + e] = h0.y * x[e];
      acc[2][4 * q + e] = h0.z * x[e];
    }
  }
  // block 2n reads its left window at 16(m - n - 1) + 8 and its right one at
  // 16(m + n); block 2n + 1 at 16(m - n - 1) and 16(m + n) + 8 (m = base / 16)
  const float *pa = row + 20 * ((base >> 4) - 1), *pb = row + 20 * (base >> 4);
  for (int k0 = 1, odd = 0; k0 <= K0; k0 += TB, odd ^= 1) {
    float A[RWIN], B[RWIN];
    if (odd) fir_row_windows<0, 8>(pa, pb, A, B);
    else fir_row_windows<8, 0>(pa, pb, A, B);
    const int na = 1 + (K1 >= k0) + (K2 >= k0);
    if (na == 3) fir_row_mac8<3>(A, B, T + k0, acc);
    else if (na == 2) fir_row_mac8<2>(A, B, T + k0, acc);
    else fir_row_mac8<1>(A, B, T + k0, acc);
    if (odd) pa -= 20, pb += 20;
  }
}

// halo of the row kernel: >= kmax + TB, a multiple of 16
__host__ __device__ __forceinline__ int row_halo(int kmax) { return (kmax + TB + 15) / 16 * 16; }
// tap table of the row kernel: entries per group (taps 0 .. K rounded up to
// whole 8-tap blocks) and its offset (floats, 16-byte aligned) after the
// padded row of n elements
__host__ __device__ __forceinline__ int row_taps_len(int kmax) { return (kmax + TB - 1) / TB * TB + 1; }
__host__ __device__ __forceinline__ int row_taps_offset(int n) { return (pad20(n) + 3) / 4 * 4; }

// Row pass.  Item: a segment of RSEG outputs of one row of a frame; items
// beyond the frame's H rows are its U-only first and last rows.
__global__ void __launch_bounds__(RNT, 512 / RNT) k_rowfir(const FrameDev *__restrict__ fr, Items it,
                                                const Coef *__restrict__ coef, const float4 *__restrict__ taps,
                                                RowGroups rg, int kmax,
                                                void *__restrict__ P, int st, long PWb, float *__restrict__ edge,
                                                DevStatus *__restrict__ status, int chan, int zero) {
  extern __shared__ __align__(16) float sm[];
  const int tid = threadIdx.x;
  // L on [xs - G, xs + RSEG + G): the 8-tap blocks read up to TB elements past
  // the last tap on each side
  const int G = row_halo(kmax);
  const int n = RSEG + 2 * G;
  float *sL = sm;                       // padded: element j at pad20(j)
  // taps of the scale groups: T[g * TK + k] = h_k of the group's scales
  float4 *T = reinterpret_cast<float4 *>(sm + row_taps_offset(n));
  const int S = rg.S, NG = rg.NG, TK = rg.TK;
  __shared__ int s_ord[ROW_MAXS];       // scales by half-length, largest first
  __shared__ int s_K[ROW_MAXS + 2];     // half-length of group slot i (-1: empty)
  __shared__ FrameDev s_fr;
  if (tid == 0) {
#pragma unroll
    for (int i = 0; i < ROW_MAXS; ++i) s_ord[i] = rg.ord[i];
#pragma unroll
    for (int i = 0; i < ROW_MAXS + 2; ++i) s_K[i] = rg.K[i];
  }
  for (int e = tid; e < NG * TK; e += RNT) T[e] = taps[e];
  bool ovf = false;                     // a value beyond the f16 range
  int k = 0, staged = -1;
  const int nitems = items_total(it);
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    int local;
    k = item_frame(it, item, k, local);
    __syncthreads();  // the previous item is done with s_fr and sL
    if (k != staged) {  // the frame record, staged again only for another frame
      stage_frame(&s_fr, fr, it, k);
      staged = k;
      __syncthreads();
    }
    const FrameDev &F = s_fr;
    const int H = F.H, W = F.W;
    const int nxs = (W + RSEG - 1) / RSEG;
    const int xs = (local % nxs) * RSEG, ri = local / nxs;
    const bool EDGE = ri >= H;            // U alone: first (ri = H) or last (ri = H + 1) row
    const int which = ri - H;
    const int y = EDGE ? (which == 0 ? 0 : H - 1) : ri;
    const float vs = F.vscale;
    const long xpitch = F.xpitch;
    with_input_type(F.X, F.dtype, [&](auto Xt) {
      const auto *rm = Xt + (long)max(y - 1, 0) * xpitch;
      const auto *r0 = Xt + (long)y * xpitch;
      const auto *rp = Xt + (long)min(y + 1, H - 1) * xpitch;
      auto ld = [&](const decltype(Xt) row, int e) { return vs * in_f32(__ldg(row + e)); };
      const float vlo = ld(rp, 0) - 2.f * ld(r0, 0) + ld(rm, 0);
      const float vhi = ld(rp, W - 1) - 2.f * ld(r0, W - 1) + ld(rm, W - 1);
      if (chan == CH_ID && F.xpre) {  // D = 5 channel row with its two-sample pre-rolls
        const float4 xp = F.xpre[y];
        for (int j = tid; j < n; j += RNT) {
          const int e = xs - G + j;
          sL[pad20(j)] = e < -1 ? xp.x : (e == -1 ? xp.y : (e < W ? ld(r0, e) : (e == W ? xp.z : xp.w)));
        }
        return;
      }
      if (zero) {
        // zero boundary (fused Laplacian): the frame extended by zeros, so U
        // and V take zero neighbours beyond the edges and L is X(0) and
        // X(W - 1) one pixel beyond the row ends and zero further out; the
        // edge items carry the first / last input row itself (the Laplacian
        // one row beyond the frame), zero beyond its ends
        auto ldz = [&](const decltype(Xt) row, int e, bool rowin) {
          return (rowin && e >= 0 && e < W) ? ld(row, e) : 0.f;
        };
        const bool hm = y - 1 >= 0, hp = y + 1 < H;
        for (int j = tid; j < n; j += RNT) {
          const int e = xs - G + j;
          float v;
          if (EDGE) {
            v = ldz(r0, e, true);
          } else if (e < -1 || e > W) {
            v = 0.f;
          } else if (e == -1 || e == W) {
            v = ld(r0, e < 0 ? 0 : W - 1);
          } else {
            const float c0 = ld(r0, e);
            v = (ldz(r0, e + 1, true) - 2.f * c0 + ldz(r0, e - 1, true)) +
                (ldz(rp, e, hp) - 2.f * c0 + ldz(rm, e, hm));
          }
          sL[pad20(j)] = v;
        }
        return;
      }
      if (chan != CH_LAP) {  // one derivative channel of the derivative bank
        const int cin = EDGE ? edge_chan(chan) : chan;
        auto am = [&](int e) { return ld(rm, min(max(e, 0), W - 1)); };
        auto ao = [&](int e) { return ld(r0, min(max(e, 0), W - 1)); };
        auto ap = [&](int e) { return ld(rp, min(max(e, 0), W - 1)); };
        for (int j = tid; j < n; j += RNT) {
          const int e = xs - G + j;
          sL[pad20(j)] = e < 0 ? chan_beyond(cin, am, ao, ap, 0)
                               : (e >= W ? chan_beyond(cin, am, ao, ap, W - 1) : chan_at(cin, am, ao, ap, e));
        }
        return;
      }
      // RLD elements (5 RLD loads, clamped into the row) per thread in flight
      for (int j0 = tid; j0 < n; j0 += RLD * RNT) {
        float cm[RLD], c0[RLD], cp[RLD], um[RLD], up[RLD];
#pragma unroll
        for (int u = 0; u < RLD; ++u) {
          const int e = min(max(xs - G + j0 + u * RNT, 0), W - 1);
          c0[u] = ld(r0, e);
          um[u] = ld(r0, max(e - 1, 0));
          up[u] = ld(r0, min(e + 1, W - 1));
          cm[u] = ld(rm, e);
          cp[u] = ld(rp, e);
        }
#pragma unroll
        for (int u = 0; u < RLD; ++u) {
          const int j = j0 + u * RNT, e = xs - G + j;
          if (j >= n) continue;
          float v;
          if (e < 0) v = EDGE ? 0.f : vlo;
          else if (e >= W) v = EDGE ? 0.f : vhi;
          else {
            const float uu = up[u] - 2.f * c0[u] + um[u];
            v = EDGE ? uu : uu + (cp[u] - 2.f * c0[u] + cm[u]);
          }
          sL[pad20(j)] = v;
        }
      }
    });
    __syncthreads();  // L staged
    const int base = G + NOUT * tid;  // local index of this thread's first output
    const int x0 = xs + NOUT * tid;
    // one plane row of scale s from NOUT outputs (f32 or 16-bit planes)
    auto store = [&](int s, const float (&v)[NOUT]) {
      const long row = (F.prow + (long)s * H + y) * PWb;
      if (EDGE || st == ST_F32) {
        float *dst = EDGE ? edge + F.eoff + ((long)s * 2 + which) * PWb : static_cast<float *>(P) + row;
        if (x0 + NOUT <= W) {
#pragma unroll
          for (int j = 0; j < NOUT; j += 4)
            *reinterpret_cast<float4 *>(dst + x0 + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        } else {
#pragma unroll
          for (int j = 0; j < NOUT; ++j)
            if (x0 + j < W) dst[x0 + j] = v[j];
        }
      } else {
        // 16-bit planes: four values per 8-byte store
        unsigned short *dst = static_cast<unsigned short *>(P) + row;
        unsigned short h[NOUT];
#pragma unroll
        for (int j = 0; j < NOUT; ++j) {
          if (st == ST_F16) {
            ovf |= x0 + j < W && fabsf(v[j]) > F16_MAX;
            h[j] = __half_as_ushort(__float2half_rn(v[j]));
          } else {
            h[j] = __bfloat16_as_ushort(__float2bfloat16_rn(v[j]));
          }
        }
        if (x0 + NOUT <= W) {
#pragma unroll
          for (int j = 0; j < NOUT; j += 4)
            *reinterpret_cast<uint2 *>(dst + x0 + j) =
                make_uint2(h[j] | ((unsigned)h[j + 1] << 16), h[j + 2] | ((unsigned)h[j + 3] << 16));
        } else {
#pragma unroll
          for (int j = 0; j < NOUT; ++j)
            if (x0 + j < W) dst[x0 + j] = h[j];
        }
      }
    };
    for (int g = 0; g < NG; ++g) {
      float acc[RGS][NOUT];
      fir_row_group(T + g * TK, s_K[g * RGS], s_K[g * RGS + 1], s_K[g * RGS + 2], sL, base, acc);
#pragma unroll
      for (int i = 0; i < RGS; ++i) {
        if (g * RGS + i >= S) break;
        const int sc = s_ord[g * RGS + i];
        // planes hold sigma^2 x the one-sided blur (the column pass only
        // negates; the blur alone for CH_ID)
        const float s2 = chan == CH_ID ? 1.f : coef[sc].sigma2;
#pragma unroll
        for (int j = 0; j < NOUT; ++j) acc[i][j] *= s2;
        store(sc, acc[i]);
      }
    }
  }
  if (ovf) atomicExch(&status->range, 1);
}

// Column FIR + detector, adjacent-scales neighbourhood.  Item: 64 rows x 32
// columns of a frame, all scales: per scale the input block (64 + 2(K+8)
// rows) is staged in shared memory, each warp slides an 8-row register window
// down its column; then the detector on the R tile of every scale.
__global__ void __launch_bounds__(CNT) k_colfir(const FrameDev *__restrict__ fr, Items it,
                                                const void *__restrict__ P, int st, long PWb,
                                                const float *__restrict__ edge,
                                                const Coef *__restrict__ coef, int S, int kmax,
                                                DetectArgs da) {
  extern __shared__ float sm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int G = kmax + TB;
  const int zero = da.zero;
  const int NIN = CROWS + 2 * G;
  float *in = sm;                               // [NIN][32]
  float *buf = sm + (long)NIN * 32;             // [S][CROWS][32]
  float *red = buf + (long)S * CROWS * 32;
  float *sh = red + CROWS * 32 * 2 + CROWS * 32 * 2 / 4;
  const float sgn = da.raw ? 1.f : -1.f;  // R_L = -(column blur); raw channel: +
  __shared__ FrameDev s_fr;
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
    const int x = (local % ntx) * TW - 1 + lane;
    const int xv = min(max(x, 0), W - 1);
    const int r0 = (local / ntx) * (CROWS - 2) - 1;  // frame row of output row 0
    for (int s = 0; s < S; ++s) {
      const Coef &c = coef[s];
      const int K = c.K;
      const long pc = (F.prow + (long)s * H) * PWb + xv;
      const float *ed = edge + F.eoff + (long)s * 2 * PWb + xv;
      const float top = ed[0], bot = ed[PWb];
      __syncthreads();
      stage_taps(sh, c, K, threadIdx.x, CNT);
      // in[j] = input row r0 - G + j
      for (int j = warp; j < NIN; j += CNT / 32) {
        const int r = r0 - G + j;
        in[j * 32 + lane] =
            (r < 0 || r >= H) ? col_outside(r, H, top, bot, zero) : load_plane(P, pc + (long)r * PWb, st);
      }
      __syncthreads();
      const float *col = in + lane + (G + NOUT * warp) * 32;  // output row NOUT*warp
      float acc[NOUT];
      fir_block(sh, K, [&](int t) { return col[t * 32]; }, acc);
#pragma unroll
      for (int j = 0; j < NOUT; ++j) buf[((long)s * CROWS + NOUT * warp + j) * 32 + lane] = sgn * acc[j];
    }
    __syncthreads();
    DetectArgs a = da;
    a.S = S;
    a.NR = CROWS;
    a.x0 = (local % ntx) * TW - 1;
    a.r0 = r0;
    a.H = H;
    a.W = W;
    a.frame = F.index;
    a.resp = F.resp;
    a.rplane = F.rplane;
    a.rpitch = F.rpitch;
    a.rmx = F.rmx;
    a.rmy = F.rmy;
    detect_tile(buf, red, a);
    __syncthreads();
  }
}

// Column FIR + detector, all-scales neighbourhood.  Item: 32 columns x 128
// rows of a frame (row 0 and row 127 are halo), a CTA of 8 warps; per scale
// the input block (128 + 2(K+8) rows of the one-sided plane) arrives by TMA
// while an earlier scale is filtered; rows outside the frame take the held
// values.  Each thread keeps the running maximum / minimum over scales of its
// 16 pixels in registers (their first scale in shared memory); the spatial
// 3 x 3 test runs once at the end on those extremes.
//
// f32 planes: two stages of 36-float rows (x a multiple of 4 floats), the
// filter reads the stage itself after the held rows are written into it.
// 16-bit planes: two landing stages of 40-element rows (x a multiple of 8
// elements); each is widened once into one f32 work tile of 32-float rows,
// after which its next scale (two ahead) is issued.
constexpr int CNT2 = 256;
constexpr int CROWS2 = 8 * NOUT;  // 128
constexpr int BOXW16 = 40;        // 16-bit box width (elements): 32 columns + alignment offset <= 7

// floats of the stages (f32: 2 stages; 16-bit: 2 landing stages + work tile)
template <int ST>
__host__ __device__ constexpr int colfir_stage_floats(int stage_rows) {
  return ST == ST_F32 ? 2 * stage_rows * BOXW : stage_rows * BOXW16 + stage_rows * 32;
}

// pixel of output j (0..15) of a thread in the tensor-core accumulator layout:
// tile nb = j / 4 holds rows g, g + 8 and columns n = 2 tig, 2 tig + 1 of the
// warp's 16 x 8 block nb (g = lane / 4, tig = lane % 4).  Column n of block nb
// is tile column bcol<PERM>(n, nb): with PERM (the 36-float rows of the f32
// stages) (n & 3) + 4 nb + 16 (n >> 2), so that the eight columns of a block
// and the four rows tig of a fragment load fall in 32 different banks;
// without it (the 32-float work tile, whose rows are XOR-swizzled instead)
// n + 8 nb.
template <bool PERM>
__device__ __forceinline__ int bcol(int n, int nb) { return PERM ? (n & 3) + 4 * nb + 16 * (n >> 2) : n + 8 * nb; }
__device__ __forceinline__ int mma_row(int warp, int lane, int j) { return 16 * warp + (lane >> 2) + 8 * ((j & 3) >> 1); }
template <bool PERM>
__device__ __forceinline__ int mma_col(int lane, int j) { return bcol<PERM>(2 * (lane & 3) + (j & 1), j >> 2); }

template <int ST>
__global__ void __launch_bounds__(CNT2, 2) k_colfir_tma(const __grid_constant__ CUtensorMap map,
                                                        const FrameDev *__restrict__ fr, Items it,
                                                        const float *__restrict__ edge, long PWb,
                                                        const Coef *__restrict__ coef, int S, int stage_rows,
                                                        int taps_len, DetectArgs da) {
  using T = typename Store<ST>::T;
  constexpr bool F32 = ST == ST_F32;
  constexpr int BW = F32 ? BOXW : BOXW16;  // box width (elements)
  constexpr int XA = F32 ? 4 : 8;          // TMA x alignment (elements)
  constexpr int LDW = F32 ? BOXW : 32;     // row stride of the f32 tile the filter reads
  extern __shared__ __align__(128) float sm_raw[];
  __shared__ __align__(8) uint64_t mbar[2];
  float *sm = align_smem(sm_raw);  // boxes: 48 rows x 144 B (f32) or x 80 B (16-bit), multiples of 128 B
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  auto land = [&](int b) { return reinterpret_cast<T *>(sm) + (long)b * stage_rows * BW; };
  float *work = sm + stage_rows * BOXW16;  // 16-bit planes only
  const int SF = colfir_stage_floats<ST>(stage_rows);
  // two bands of taps (hi parts, then lo parts), alternating with the stages:
  // a scale writes its band while the previous scale may still read the other
  float *taps0 = sm + SF;
  unsigned char *amx = reinterpret_cast<unsigned char *>(sm + SF + 4 * taps_len);
  unsigned char *amn = amx + CROWS2 * 32;
  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    fence_proxy_async();
  }
  __syncthreads();
  __shared__ FrameDev s_fr;
  const float sgn = da.raw ? 1.f : -1.f;
  uint32_t ph0 = 0u, ph1 = 0u;  // phase to wait for, per barrier
  int k = 0;
  const int nitems = items_total(it);
  // The stages alternate over the block's whole sequence of (item, scale)
  // loads: `base` counts the scales of the earlier items.  f32 planes: the
  // next item's first scale is loaded during this item's last scale
  // (`pre`), and this item's extremes go to the stage of its last scale.
  int base = 0;
  bool pre = false;
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    int local;
    k = item_frame(it, item, k, local);
    stage_frame(&s_fr, fr, it, k);  // the previous item ended with __syncthreads
    __syncthreads();
    const FrameDev &F = s_fr;
    const int H = F.H, W = F.W;
    const long prow = F.prow;
    const int ntx = (W + TW - 1) / TW;
    const int x0 = (local % ntx) * TW - 1;     // frame column of lane 0
    const int off = ((x0 % XA) + XA) % XA;
    const int xa = x0 - off;
    const int r0 = (local / ntx) * (CROWS2 - 2) - 1;  // frame row of output row 0
    const int x = x0 + lane, xv = min(max(x, 0), W - 1);
    const bool inside = x0 >= 0 && x0 + 32 <= W && r0 >= 0 && r0 + CROWS2 <= H;  // the whole 128 x 32 tile
    float *resp = F.resp;
    float mxr[NOUT], mnr[NOUT];
#pragma unroll
    for (int j = 0; j < NOUT; ++j) {
      const int p = mma_row(warp, lane, j) * 32 + mma_col<F32>(lane, j);
      mxr[j] = -CUDART_INF_F;
      mnr[j] = CUDART_INF_F;
      amx[p] = (unsigned char)S;
      amn[p] = (unsigned char)S;
    }
    // scale s of a tile (plane rows of frame row r0_, box column xa_) into stage b
    auto issue_at = [&](int s, int b, long prow_, int H_, int r0_, int xa_) {  // thread 0 only
      const int G = coef[s].K + TB;
      const int nb = (CROWS2 + 2 * G + BOXH - 1) / BOXH;
      fence_proxy_async();
      mbar_arrive_expect_tx(&mbar[b], (uint32_t)(nb * BOXH * BW * sizeof(T)));
      const int y0 = (int)(prow_ + (long)s * H_ + r0_ - G);
      for (int i = 0; i < nb; ++i)
        if (!tma_load_2d(land(b) + i * BOXH * BW, &map, xa_, y0 + i * BOXH, &mbar[b], (int)sizeof(T)))
          atomicExch(&da.status->error, 2);
    };
    auto issue = [&](int s, int b) { issue_at(s, b, prow, H, r0, xa); };
    const int next = item + gridDim.x;
    // scales from the longest filter down (the order of the caller's scales is
    // kept for ties: the first scale attaining an extreme is the one reported)
    if (tid == 0) {
      if (!pre) issue(S - 1, base & 1);
      if (!F32 && S > 1) issue(S - 2, (base + 1) & 1);
    }
    const long plane = (long)H * W;
    // f32: one barrier per scale (after the scale's load and taps); the next
    // load into a stage is issued after the following scale's barrier, when
    // every warp is done with that stage.  16-bit: the scales share one work
    // tile, and each scale also ends with a barrier.
    for (int is = 0; is < S; ++is) {
      const int s = S - 1 - is;
      const int b = (base + is) & 1;
      float *taps = taps0 + 2 * b * taps_len;
      const Coef &c = coef[s];
      const int K = c.K, G = K + TB, nin = CROWS2 + 2 * G;
      // R_L = -sigma^2 (D20 + D02) with the planes carrying sigma^2: the taps
      // carry the sign (a raw derivative channel keeps +)
      stage_taps_band(taps, taps + taps_len, c, K, taps_len, sgn, tid, CNT2);
      const bool ok = mbar_wait_bounded(&mbar[b], b ? ph1 : ph0, WAIT_LIMIT);
      if (b) ph1 ^= 1u;
      else ph0 ^= 1u;
      if (__syncthreads_or(!ok)) {
        // a load never completed: report, let the other stage's load finish, stop
        if (tid == 0) {
          atomicExch(&da.status->error, 1);
          if (!F32 && is + 1 < S) mbar_wait_bounded(&mbar[b ^ 1], b ? ph0 : ph1, WAIT_LIMIT);
        }
        __syncthreads();
        return;
      }
      if (F32 && tid == 0) {
        if (is + 1 < S) {
          issue(s - 1, b ^ 1);
        } else if (next < nitems) {  // the next item's first scale
          int ln;
          const int kq = item_frame(it, next, k, ln);
          const FrameDev &Fn = fr[__ldg(it.fl + kq)];
          const int Hn = Fn.H, ntxn = (Fn.W + TW - 1) / TW;
          const int x0n = (ln % ntxn) * TW - 1, r0n = (ln / ntxn) * (CROWS2 - 2) - 1;
          issue_at(S - 1, b ^ 1, Fn.prow, Hn, r0n, x0n - ((x0n % XA) + XA) % XA);
        }
      }
      const bool outside = r0 - G < 0 || r0 + CROWS2 + G > H;
      float top = 0.f, bot = 0.f;
      if (outside) {
        const float *ed = edge + F.eoff + (long)s * 2 * PWb + xv;
        top = ed[0];
        bot = ed[PWb];
      }
      const float *tile;
      if constexpr (F32) {
        float *stg = land(b);
        if (outside) {  // rows outside the frame: held values (uniform over the block)
          for (int j = warp; j < nin; j += CNT2 / 32) {
            const int r = r0 - G + j;
            if (r < 0 || r >= H) stg[j * BOXW + off + lane] = col_outside(r, H, top, bot, da.zero);
          }
          fence_proxy_async();  // before the stage's next async copy
          __syncthreads();
        }
        tile = stg + off;
      } else {
        const T *src = land(b) + off + lane;
        for (int j = warp; j < nin; j += CNT2 / 32) {
          const int r = r0 - G + j;
          const float v = Store<ST>::ld(src[j * BW]);
          work[j * 32 + (lane ^ (8 * (j & 3)))] =
              (r < 0 || r >= H) ? col_outside(r, H, top, bot, da.zero) : v;  // XOR-swizzled rows
        }
        tile = work;
        __syncthreads();  // landing stage b is free again
        if (tid == 0 && is + 2 < S) issue(s - 2, b);
      }
      // Banded Toeplitz product on the tensor cores: warp w computes output rows
      // o = 16w + r (r < 16) x 32 columns as four m16n8k8 tiles,
      // out[o] = sum_q A[r][q] stage[16w + 8 + q] over q in [0, 16 + 2K) with
      // A[r][q] = h(|q - r - K|) (zero beyond K): the same A for every row
      // block.  Three TF32 products per tap: lo x hi, hi x lo, hi x hi.
      const int g = lane >> 2, tig = lane & 3;
      const int J = (16 + 2 * K + 7) / 8;  // k-steps of 8 input rows
      // A(g, tig) at k-step j is band[BAND0 + 8j + tig - g]; the fragment's other
      // entries, A(g + 8, tig), A(g, tig + 4) and A(g + 8, tig + 4), sit 8 below,
      // 4 above and 4 below it: the two below are the previous k-step's first
      // and third
      const float *ph = taps + BAND0 + tig - g, *pl = ph + taps_len;
      uint32_t h1 = __float_as_uint(ph[-8]), h3 = __float_as_uint(ph[-4]);
      uint32_t l1 = __float_as_uint(pl[-8]), l3 = __float_as_uint(pl[-4]);
      // B(k, g) of block nb is window row 8j + k (k = tig, tig + 4), tile column
      // bcol(g, nb); the work tile's row R holds column c at c ^ 8 (R & 3), and
      // R & 3 = tig here
      const float *tb = tile + (16 * warp + 8 + tig) * LDW;
      int cb[4];
#pragma unroll
      for (int nb = 0; nb < 4; ++nb) cb[nb] = F32 ? bcol<true>(g, nb) : g + 8 * (nb ^ tig);
      float d[4][4];
#pragma unroll
      for (int nb = 0; nb < 4; ++nb)
#pragma unroll
        for (int e = 0; e < 4; ++e) d[nb][e] = 0.f;
#pragma unroll 2
      for (int j = 0; j < J; ++j) {
        const uint32_t h0 = __float_as_uint(ph[8 * j]), h2 = __float_as_uint(ph[8 * j + 4]);
        const uint32_t l0 = __float_as_uint(pl[8 * j]), l2 = __float_as_uint(pl[8 * j + 4]);
        const float *rp = tb + 8 * j * LDW;
#pragma unroll
        for (int nb = 0; nb < 4; ++nb) {
          const float x0v = rp[cb[nb]], x1v = rp[4 * LDW + cb[nb]];
          // hi: x with the 13 bits below the TF32 mantissa cleared; lo = x - hi
          // (exact), of which the tensor core reads the top 19 bits
          const uint32_t bh0 = __float_as_uint(x0v) & 0xffffe000u, bh1 = __float_as_uint(x1v) & 0xffffe000u;
          const uint32_t bl0 = __float_as_uint(x0v - __uint_as_float(bh0));
          const uint32_t bl1 = __float_as_uint(x1v - __uint_as_float(bh1));
          mma_tf32(d[nb], l0, l1, l2, l3, bh0, bh1);
          mma_tf32(d[nb], h0, h1, h2, h3, bl0, bl1);
          mma_tf32(d[nb], h0, h1, h2, h3, bh0, bh1);
        }
        h1 = h0;
        h3 = h2;
        l1 = l0;
        l3 = l2;
      }
      // scales arrive in decreasing order: >= keeps the smallest scale of a tie;
      // items wholly inside the frame skip the per-pixel frame test
      auto extremes = [&](auto check) {
#pragma unroll
        for (int j = 0; j < NOUT; ++j) {
          const int i = mma_row(warp, lane, j), cc = mma_col<F32>(lane, j);
          if (decltype(check)::value) {
            const int y = r0 + i, xj = x0 + cc;
            if (xj < 0 || xj >= W || y < 0 || y >= H) continue;
          }
          const float v = d[j >> 2][j & 3];
          if (v >= mxr[j]) mxr[j] = v, amx[i * 32 + cc] = (unsigned char)s;
          if (v <= mnr[j]) mnr[j] = v, amn[i * 32 + cc] = (unsigned char)s;
        }
      };
      if (inside) extremes(std::false_type());
      else extremes(std::true_type());
      if (resp) {
#pragma unroll
        for (int j = 0; j < NOUT; ++j) {
          const int i = mma_row(warp, lane, j), cc = mma_col<F32>(lane, j), y = r0 + i, xj = x0 + cc;
          if (xj >= 0 && xj < W && y >= 0 && y < H && i >= 1 && i <= CROWS2 - 2 && cc >= 1 && cc <= TW)
            resp[s * plane + (long)y * W + xj] = d[j >> 2][j & 3];
        }
      }
      if (!F32) {
        fence_proxy_async();
        __syncthreads();  // the work tile and the landing stage are free again
      }
    }
    if (F32) __syncthreads();  // every warp is done with the last scale's stage
    const int blast = (base + S - 1) & 1;  // stage of the last scale
    pre = F32 && next < nitems;
    base += S;
    if (da.raw) {  // a derivative channel: written above, no detection (uniform over the block)
      fence_proxy_async();
      __syncthreads();
      continue;
    }
    // the extremes go to shared memory for the 3 x 3 test: f32, the last
    // scale's stage (the other one holds the next item's first load); 16-bit,
    // the landing stages
    float *mx = F32 ? reinterpret_cast<float *>(land(blast)) : sm, *mn = mx + CROWS2 * 32;
#pragma unroll
    for (int j = 0; j < NOUT; ++j) {
      const int p = mma_row(warp, lane, j) * 32 + mma_col<F32>(lane, j);
      mx[p] = mxr[j];
      mn[p] = mnr[j];
    }
    __syncthreads();
    DetectArgs a = da;
    a.S = S;
    a.NR = CROWS2;
    a.x0 = x0;
    a.r0 = r0;
    a.H = H;
    a.W = W;
    a.frame = F.index;
    a.resp = resp;
    spatial_detect(mx, mn, ArgBytes{amx, amn}, a);
    fence_proxy_async();  // extremes written over the stages before the next item's copies
    __syncthreads();
  }
}

template <int ST>
int launch_colfir_tma(const Plan &p, const Launch &l, const BankArgs &a, const DetectArgs &da, int G, int KP,
                      cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_colfir_tma<ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  CUtensorMap map;
  if (encode_plane_map(&map, a.P, ST, p.PWb, p.prows, ST == ST_F32 ? BOXW : BOXW16, BOXH)) return -1;
  // whole boxes; f32: a stage holds the 2 x 128 x 32 extremes of an item
  const int stage_rows = std::max((CROWS2 + 2 * G + BOXH - 1) / BOXH * BOXH, ST == ST_F32 ? 240 : 0);
  // band length >= BAND0 + 2K + 23: one past the largest index a fragment reads
  const int taps_len = (BAND0 + 2 * KP + 23 + 3) / 4 * 4;
  const int SF = colfir_stage_floats<ST>(stage_rows);
  // stages (>= 2 x 128 x 32 floats for the final extremes) + taps + first-scale bytes
  const size_t tsm = ((size_t)SF + 4 * taps_len) * sizeof(float) + (size_t)CROWS2 * 32 * 2 + TMA_SMEM_ALIGN;
  if (tsm > 200 * 1024 || SF < 2 * CROWS2 * 32) return -1;
  const int nb = persistent_blocks((const void *)k_colfir_tma<ST>, CNT2, tsm, l.it.total, p.mult[PASS_DET]);
  a.prof->begin("fir_coldet", st);
  k_colfir_tma<ST><<<nb, CNT2, tsm, st>>>(map, p.fr, l.it, a.edge, p.PWb, a.coef, a.S, stage_rows, taps_len, da);
  a.prof->end(st);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace

// 2-D tensor map over the plane row space (x, plane row), box boxw x boxh
int encode_plane_map(CUtensorMap *m, void *P, int storage, long PWb, long prows, int boxw, int boxh) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void *fn = nullptr;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return -1;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t eb = (cuuint64_t)store_bytes(storage);
  const cuuint64_t dims[2] = {(cuuint64_t)PWb, (cuuint64_t)prows};
  const cuuint64_t strides[1] = {(cuuint64_t)PWb * eb};
  const cuuint32_t box[2] = {(cuuint32_t)boxw, (cuuint32_t)boxh};
  const cuuint32_t es[2] = {1, 1};
  const CUtensorMapDataType ty = storage == ST_F16    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                 : storage == ST_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                      : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const CUresult r = encode(m, ty, 2, P, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -1;
}

int persistent_blocks(const void *kernel, int threads, size_t smem, int items, int mult) {
  if (mult <= 0) return std::max(1, items);
  constexpr int kMaxDev = 64;
  static int nsm[kMaxDev];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= kMaxDev) dev = 0;
  if (!nsm[dev]) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    nsm[dev] = n > 0 ? n : 1;
  }
  // resident blocks per SM, cached per (device, kernel, block size, shared memory)
  struct Key {
    int dev;
    const void *kernel;
    int threads;
    size_t smem;
    bool operator<(const Key &o) const {
      return std::tie(dev, kernel, threads, smem) < std::tie(o.dev, o.kernel, o.threads, o.smem);
    }
  };
  static std::map<Key, int> cache;
  static std::mutex mu;
  int occ = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    const Key key{dev, kernel, threads, smem};
    auto f = cache.find(key);
    if (f != cache.end()) {
      occ = f->second;
    } else {
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem) != cudaSuccess || occ < 1)
        occ = 1;
      cache[key] = occ;
    }
  }
  // mult < 0: a share of -mult blocks on every SM (at most the resident limit)
  const long cap = mult < 0 ? (long)nsm[dev] * std::min(occ, -mult) : (long)nsm[dev] * occ * mult;
  return (int)std::max(1L, std::min((long)items, cap));
}

int fir_row_segment() { return RSEG; }
int fir_row_rows() { return 1; }
int fir_tile_rows(int neigh) { return neigh == 0 ? CROWS2 - 2 : CROWS - 2; }
int fir_halo(int kmax) { return kmax + TB + 1; }

int fir_items(int pass, int H, int W, int S, int neigh, bool tc) {
  const int tw = tc ? fir_tc_tile_cols() : TW;
  const int th = tc ? fir_tc_tile_rows(S) : (neigh == 0 ? CROWS2 - 2 : CROWS - 2);
  const int ntx = (W + tw - 1) / tw;
  switch (pass) {
    case PASS_ROW: return ((W + RSEG - 1) / RSEG) * (H + 2);
    case PASS_DET: return ntx * ((H + th - 1) / th);
    default: return 0;
  }
}

long row_groups(const Coef *h_coef, int S, RowGroups *g, std::vector<float> *table) {
  if (S < 1 || S > ROW_MAXS) return -1;
  RowGroups r;
  r.S = S;
  r.NG = (S + RGS - 1) / RGS;
  int kmax = 0;
  for (int i = 0; i < S; ++i) r.ord[i] = i, kmax = std::max(kmax, h_coef[i].K);
  std::stable_sort(r.ord, r.ord + S, [&](int a, int b) { return h_coef[a].K > h_coef[b].K; });
  for (int i = 0; i < ROW_MAXS + 2; ++i) r.K[i] = i < S ? h_coef[r.ord[i]].K : -1;
  r.TK = row_taps_len(kmax);
  table->assign((size_t)4 * r.NG * r.TK, 0.f);
  for (int gi = 0; gi < r.NG; ++gi)
    for (int i = 0; i < RGS; ++i) {
      const int slot = gi * RGS + i;
      if (slot >= S) continue;
      const Coef &c = h_coef[r.ord[slot]];
      for (int k = 0; k <= c.K; ++k) (*table)[((size_t)gi * r.TK + k) * 4 + i] = c.h[k];
    }
  *g = r;
  return (long)table->size();
}

int launch_fir(const Plan &p, const BankArgs &a, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_rowfir, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    cudaFuncSetAttribute(k_colfir, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  const int kmax = a.kmax;
  const int G = kmax + TB;
  const int KP = ((kmax + TB - 1) / TB) * TB;
  const int RG = row_halo(kmax);
  if (!a.row_taps || a.rg.S != a.S || a.rg.TK > row_taps_len(kmax)) return -1;
  const size_t rsm = (size_t)row_taps_offset(RSEG + 2 * RG) * sizeof(float) +
                     (size_t)a.rg.NG * a.rg.TK * sizeof(float4);
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
  da.zero = a.zero;
  // in + buf + detector scratch (2 float planes + 2 byte planes) + taps (adjacent neighbourhood)
  const size_t csm = ((size_t)(CROWS + 2 * G) * 32 + (size_t)a.S * CROWS * 32 + (size_t)CROWS * 32 * 2 +
                      (size_t)CROWS * 32 * 2 / 4 + KP + 1) * sizeof(float);
  if (a.neigh != 0 && csm > 200 * 1024) return -1;
  auto row = [&](const Launch &l) {
    const int nb = persistent_blocks((const void *)k_rowfir, RNT, rsm, l.it.total, p.mult[PASS_ROW]);
    a.prof->begin("fir_row", st);
    k_rowfir<<<nb, RNT, rsm, st>>>(p.fr, l.it, a.coef, reinterpret_cast<const float4 *>(a.row_taps), a.rg, kmax,
                                   a.P, a.storage, p.PWb, a.edge, a.status, a.chan, a.zero);
    a.prof->end(st);
  };
  auto det = [&](const Launch &l) -> int {
    if (a.tc_bands) return launch_colfir_tc(p, l, a, da, st);  // the tensor-core (tcgen05) pass
    if (a.neigh == 0) {
      switch (a.storage) {
        case ST_F32: return launch_colfir_tma<ST_F32>(p, l, a, da, G, KP, st);
        case ST_F16: return launch_colfir_tma<ST_F16>(p, l, a, da, G, KP, st);
        case ST_BF16: return launch_colfir_tma<ST_BF16>(p, l, a, da, G, KP, st);
        default: return -2;
      }
    }
    const int nb = persistent_blocks((const void *)k_colfir, CNT, csm, l.it.total, p.mult[PASS_DET]);
    a.prof->begin("fir_coldet", st);
    k_colfir<<<nb, CNT, csm, st>>>(p.fr, l.it, a.P, a.storage, p.PWb, a.edge, a.coef, a.S, kmax, da);
    a.prof->end(st);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
  };
  if (p.per_frame) {
    for (int f = 0; f < p.nframes; ++f) {
      row(p.pass[PASS_ROW][f]);
      if (int rc = det(p.pass[PASS_DET][f])) return rc;
    }
  } else {
    row(p.pass[PASS_ROW][0]);
    if (int rc = det(p.pass[PASS_DET][0])) return rc;
  }
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace kf
