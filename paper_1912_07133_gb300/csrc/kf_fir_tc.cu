// kf_fir_tc.cu -- column pass of the FIR banks (colored Savitzky-Golay,
// Filter C, Sec. 4.2; Gaussian, Filter A, Sec. 3.1) on the fifth-generation
// tensor cores (tcgen05, tensor memory), with the all-scales detector of
// Sec. 5.
//
// For one scale the column blur of a tile is a banded Toeplitz product
// (eq A5 along y).  A tile is 128 image columns (the MMA's M, tensor-memory
// lanes) by NR output rows (the MMA's N: 64, or 32 above six scales so that
// every scale's accumulator fits the tensor memory), rows r0 .. r0 + NR - 1;
// its input rows are r0 - Kp + q, q < Kd = NR + 2 Kp (Kp = K rounded up to 4;
// taps beyond K are zero).  Per scale one MMA chain
//   D[c][n] = sum_q A[c][q] B[n][q],   output row r0 + NR - 1 - n,
//   A[c][q] = plane (r0 - Kp + q, x0 + c)      (tensor memory),
//   B[n][q] = band[q + n],  band[u] = sgn h(|u - Kp - NR + 1|)   (shared memory).
// B is K-major without swizzle; because B[n][q] depends on q + n only, its
// 8-row x 16-byte core matrices are cut from one array of chunks -- chunk
// (g, i) at byte 16 (8 g + i) holds band[4 g + i .. 4 g + i + 3] -- with a
// K-direction core-matrix stride of 128 bytes and an N-direction one of 256
// bytes: the Toeplitz structure is the overlap of the core matrices, and a
// scale's whole B takes (Kd + NR + 7) / 4 x 128 bytes.  The A operand lives in
// tensor memory: each splitting thread owns one column (a lane), reads its
// column of a landed 32-row chunk from shared memory and stores it into
// tensor memory (tcgen05.st), so the MMAs read only the small B from shared
// memory.
//
// FP32 accuracy from TF32 products (three per tap product): the tensor core
// reads the top 19 bits of each 32-bit operand (truncation), so with
// x = hi + lo (hi = x with its low 13 bits cleared, lo = x - hi exactly) and
// the taps split once per design (hi = tf32(h), lo = tf32(h - hi)),
// out = A_lo B_hi + A_hi B_lo + A_hi B_hi leaves about 2^-21 of each product.
// A_hi is the raw data (the tensor core truncates it to hi).  16-bit planes
// (f16, bf16) hold values exact in TF32: two products, A_hi (B_lo + B_hi),
// except in chunks that reach the frame's held f32 edge rows.
//
// One CTA per SM, persistent over the call's tiles (interior 126 x (NR - 2)),
// warp-specialised:
//   warp 0      TMA producer: per scale the band pair (bulk copy, two slots)
//               and the 32-row chunks of the one-sided plane (2-D tensor
//               copies of 132 x 32 floats into a ring of landing slots);
//   warp 1      tensor-memory allocation and the MMA issue (one thread): per
//               chunk 4 k-steps x 3 products of M = 128, N = NR, K = 8;
//   warps 2-5   splitting: each thread takes one column of a landed chunk
//               (held rows substituted at the frame's top and bottom), splits
//               it and stores it into the chunk's tensor-memory slot;
//   warps 6-13  epilogue, two warps per tensor-memory lane quarter (each
//               reads one 32-row block of the accumulators): every scale of
//               the tile out of tensor memory (per-pixel extremes over the
//               scales, the optional responses), each scale's columns
//               released to the next tile's MMAs once its readers are done;
//               then the 3 x 3 spatial test (each warp half of the rows) and
//               the tile's candidate list.
// Tensor memory (512 columns): the accumulators of scale s at columns
// [NR s, NR (s + 1)) (at most 384), two operand slots of 64 columns (hi,
// lo) at 384 and 448.  Every wait is bounded; a wait that gives up sets the
// call's error status and the CTA stops taking tiles (copies and MMAs in
// flight are awaited, with a bound, before the tensor memory is released).
#include <cudaTypedefs.h>

#include <algorithm>

#include "kf_batch.cuh"
#include "kf_common.cuh"
#include "kf_detect.cuh"
#include "kf_internal.h"
#include "kf_tma.cuh"

namespace kf {

namespace {

constexpr int TC_M = 128;               // image columns per tile (MMA M, tensor-memory lanes)
constexpr int TC_CH = 32;               // input rows per chunk
constexpr int TC_BOXW = 132;            // landed chunk width (f32): 128 columns + TMA alignment offset <= 3
constexpr int TC_BOXW16 = 136;          // landed chunk width (16-bit): 128 columns + offset <= 7
constexpr int TC_THREADS = 448;         // warps 0 (loads), 1 (MMA), 2-5 (split), 6-13 (epilogue)
constexpr int TC_EPI = 256;             // epilogue threads: two warps per tensor-memory lane quarter
constexpr int TC_MAXL = 6;              // landing slots at most
constexpr int TC_ACOL = 384;            // tensor-memory column of the first operand slot
constexpr int XS = TC_M + 1;            // row stride (floats) of the per-pixel extremes
constexpr int XB = TC_M + 4;            // row stride (bytes) of their first-scale maps
constexpr uint32_t TC_WAIT = 1u << 20;  // polls of a bounded wait (each parks the warp up to ~1 us)
// landed chunk bytes: 16896 (f32 planes) or 8704 (16-bit planes)
__host__ __device__ constexpr size_t land_bytes(int st) {
  return st == ST_F32 ? (size_t)TC_BOXW * TC_CH * 4 : (size_t)TC_BOXW16 * TC_CH * 2;
}

__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  // shared-memory matrix descriptor: start >> 4, leading and stride byte
  // offsets >> 4, version 1, no swizzle
  return (uint64_t)((addr >> 4) & 0x3fffu) | ((uint64_t)((lbo >> 4) & 0x3fffu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3fffu) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor: kind::tf32, D f32, A and B tf32 (K-major), N, M = 128
__device__ __forceinline__ uint32_t tc_idesc(int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

// D (tensor memory) += A (tensor memory) x B (shared-memory descriptor)
__device__ __forceinline__ void tc_mma(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, int acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d),
      "r"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// 1-D bulk copy global -> shared (16-byte aligned, size a multiple of 16)
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// 32 consecutive tensor-memory columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// 32 values into 32 consecutive tensor-memory columns of this warp's lanes
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"
      "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]),
      "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]),
      "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}

// barrier of the 256 epilogue threads (warps 6-13), optionally with an OR of a predicate
__device__ __forceinline__ bool epi_sync_or(bool p) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred pi, po;\n\tsetp.ne.u32 pi, %1, 0;\n\tbar.red.or.pred po, 1, 256, pi;\n\t"
      "selp.u32 %0, 1, 0, po;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)p)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
// barrier of the 128 splitting threads (warps 2-5), with an OR of a predicate
__device__ __forceinline__ bool split_sync_or(bool p) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred pi, po;\n\tsetp.ne.u32 pi, %1, 0;\n\tbar.red.or.pred po, 2, 128, pi;\n\t"
      "selp.u32 %0, 1, 0, po;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)p)
      : "memory");
  return r != 0;
}

// Candidates of one tile, staged in shared memory and reserved in the call's
// list once per tile (a 128 x 64 tile of a textured frame holds a few hundred).
constexpr int TC_CANDS = 512;
struct TcList {
  int n;
  int pad[7];
  Blob rec[TC_CANDS];
};

__device__ __forceinline__ void tc_emit(const DetectArgs &a, TcList &tl, int s, int y, int x, int pol, float v) {
  Blob b;
  b.frame = a.frame;
  b.x = x;
  b.y = y;
  b.scale = s;
  b.polarity = pol;
  b.response = v;
  b.dx = b.dy = 0.f;
  const int slot = atomicAdd(&tl.n, 1);
  if (slot < TC_CANDS) {
    tl.rec[slot] = b;
  } else {
    const unsigned long long idx = atomicAdd(&a.status->count, 1ull);
    if (idx < (unsigned long long)a.cap) a.out[idx] = b;
  }
}

// tie rule of one candidate against its 8 neighbours' extremes (pol = -1
// mirrors the values): strictly above a neighbour earlier in (y, x) order or
// with an earlier first scale, at least equal to a later one
__device__ __forceinline__ bool tc_beats(const float *m, const unsigned char *am, int i, int c, int pol, float v,
                                         int s) {
  bool ok = true;
  for (int di = -1; di <= 1 && ok; ++di)
    for (int dl = -1; dl <= 1 && ok; ++dl) {
      if (di == 0 && dl == 0) continue;
      const float vn = m[(i + di) * XS + c + dl];
      const int sn = am[(i + di) * XB + c + dl];
      const bool after = di > 0 || (di == 0 && dl > 0);
      const float a1 = pol * v, b1 = pol * vn;
      ok = (a1 > b1) || (a1 == b1 && (sn > s || (sn == s && after)));
    }
  return ok;
}

// The spatial 3 x 3 test over the per-pixel extremes of an NR x 128 tile
// (rows 0 and NR - 1, columns 0 and 127 halo) by the 256 epilogue threads:
// warp ew takes columns [32 ew, 32 ew + 32), one per lane, and walks the
// interior rows [ib, ie) with the horizontal 3-maxima (3-minima) of three rows in
// registers (left and right neighbours read from shared memory: shuffles
// with the warp's edge lanes reading shared memory measured twice as slow);
// candidates are staged in the tile list.
__device__ void tc_detect(const float *mx, const float *mn, const unsigned char *amx, const unsigned char *amn,
                          TcList &tl, const DetectArgs &a, int ew, int lane, int ib, int ie) {
  const int c = 32 * ew + lane;
  const int x = a.x0 + c;
  const bool col = c >= 1 && c <= TC_M - 2 && x >= 0 && x < a.W;
  // consecutive columns: conflict-free; the tile's edge columns are halo and
  // never tested, so they read themselves
  const int cl = c > 0 ? c - 1 : c, cr = c < TC_M - 1 ? c + 1 : c;
  auto sidemax = [&](const float *m, int i) { return fmaxf(m[i * XS + cl], m[i * XS + cr]); };
  auto sidemin = [&](const float *m, int i) { return fminf(m[i * XS + cl], m[i * XS + cr]); };
  float vp = mx[(ib - 1) * XS + c], wp = mn[(ib - 1) * XS + c];
  float xa = fmaxf(vp, sidemax(mx, ib - 1)), na = fminf(wp, sidemin(mn, ib - 1));
  float vc = mx[ib * XS + c], wc = mn[ib * XS + c];
  float lx = sidemax(mx, ib), ln = sidemin(mn, ib);
  for (int i = ib; i < ie; ++i) {
    const float vn = mx[(i + 1) * XS + c], wn = mn[(i + 1) * XS + c];
    const float lxn = sidemax(mx, i + 1), lnn = sidemin(mn, i + 1);
    const int y = a.r0 + i;
    if (col && y >= 0 && y < a.H) {
      const float m8 = fmaxf(xa, fmaxf(lx, fmaxf(vn, lxn)));  // maximum of the 8 neighbours
      if (vc > a.thr && vc >= m8) {
        const int s = amx[i * XB + c];
        if (vc > m8 || tc_beats(mx, amx, i, c, 1, vc, s)) tc_emit(a, tl, s, y, x, 1, vc);
      }
      const float n8 = fminf(na, fminf(ln, fminf(wn, lnn)));
      if (a.dark && -wc > a.thr && wc <= n8) {
        const int s = amn[i * XB + c];
        if (wc < n8 || tc_beats(mn, amn, i, c, -1, wc, s)) tc_emit(a, tl, s, y, x, -1, wc);
      }
    }
    xa = fmaxf(vc, lx), na = fminf(wc, ln);
    vc = vn, wc = wn, lx = lxn, ln = lnn;
  }
}

// the tile list's candidates to the call's list (one global reservation)
__device__ void tc_flush(const DetectArgs &a, TcList &tl, unsigned long long &s_base, int t) {
  epi_sync();
  const int nloc = min(tl.n, TC_CANDS);
  if (t == 0 && nloc > 0) s_base = atomicAdd(&a.status->count, (unsigned long long)nloc);
  epi_sync();
  for (int i = t; i < nloc; i += TC_EPI) {
    const unsigned long long idx = s_base + i;
    if (idx < (unsigned long long)a.cap) a.out[idx] = tl.rec[i];
  }
}

struct TcSmem {
  uint64_t land_full[TC_MAXL], land_empty[TC_MAXL], a_full[2], a_empty[2], tap_full[2], tap_empty[2], d_full,
      d_empty[TC_MAXS], fin;
  uint32_t tmem;
  int abort;
  unsigned long long base;  // the tile's reservation in the call's candidate list
};

// geometry of an item (tile) of a frame
struct TcTile {
  int x0, r0;  // frame column of lane 0, frame row of output row 0
};
__device__ __forceinline__ TcTile tc_tile(int local, int W, int NR) {
  const int ntx = (W + TC_M - 3) / (TC_M - 2);
  return {(local % ntx) * (TC_M - 2) - 1, (local / ntx) * (NR - 2) - 1};
}

// 448 threads of one CTA per SM (at most 144 registers per thread)
template <int ST>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_colfir_tc(const __grid_constant__ CUtensorMap map, const FrameDev *__restrict__ fr, Items it,
                const float *__restrict__ edge, long PWb, const float *__restrict__ bands, TcGeom g, int NL,
                DetectArgs da) {
  using T = typename Store<ST>::T;
  constexpr bool F32 = ST == ST_F32;
  constexpr int BW = F32 ? TC_BOXW : TC_BOXW16;  // landed row (elements)
  constexpr int XA = F32 ? 4 : 8;                 // TMA x alignment (elements)
  constexpr size_t LAND = land_bytes(ST);
  extern __shared__ __align__(1024) unsigned char sm_raw[];
  __shared__ TcSmem sh;
  unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(sm_raw) + 1023) &
                                                          ~(uintptr_t)1023);
  const int NR = g.NR;
  const size_t tapb = ((size_t)2 * g.gmax * 128 + 1023) / 1024 * 1024;  // one band pair (hi, lo)
  unsigned char *taps = base;                                               // [2][tapb]
  T *land = reinterpret_cast<T *>(taps + 2 * tapb);                         // [NL][32][BW]
  float *mx = reinterpret_cast<float *>(taps + 2 * tapb + (size_t)NL * LAND);  // [NR][XS]
  float *mn = mx + (size_t)NR * XS;
  unsigned char *amx = reinterpret_cast<unsigned char *>(mn + (size_t)NR * XS);  // [NR][XB]
  unsigned char *amn = amx + (size_t)NR * XB;
  TcList &tl = *reinterpret_cast<TcList *>(amn + (size_t)NR * XB);  // 16-byte aligned (NR a multiple of 32)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int S = g.S;
  if (tid == 0) {
    for (int b = 0; b < NL; ++b) {
      mbar_init(&sh.land_full[b], 1);
      mbar_init(&sh.land_empty[b], 4);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sh.a_full[b], 4);
      mbar_init(&sh.a_empty[b], 1);
      mbar_init(&sh.tap_full[b], 1);
      mbar_init(&sh.tap_empty[b], 1);
    }
    mbar_init(&sh.d_full, 1);
    for (int t = 0; t < TC_MAXS; ++t) mbar_init(&sh.d_empty[t], 4 * (g.NR / 32));  // the warps that read it
    mbar_init(&sh.fin, 1);
    sh.abort = 0;
    fence_proxy_async();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&sh.tmem))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sh.tmem;
  volatile int *abort = &sh.abort;
  auto give_up = [&](int code) {
    *abort = 1;
    atomicExch(&da.status->error, code);
  };
  const uint32_t wlim = da.wait_test ? da.wait_test : TC_WAIT;
  const int nitems = items_total(it);

  if (warp == 0) {
    // ---------------- producer: band pairs and plane chunks ----------------
    if (lane == 0) {
      uint32_t nl = 0, nt = 0;
      int k = 0;
      for (int item = blockIdx.x; item < nitems && !*abort; item += gridDim.x) {
        int local;
        k = item_frame(it, item, k, local);
        const FrameDev &F = fr[__ldg(it.fl + k)];
        const TcTile t = tc_tile(local, F.W, NR);
        const int xa = t.x0 - (((t.x0 % XA) + XA) % XA);
        for (int s = 0; s < S && !*abort; ++s) {
          const int ts = nt & 1;
          if (!mbar_wait_bounded(&sh.tap_empty[ts], ((nt >> 1) & 1) ^ 1, wlim)) {
            give_up(3);
            break;
          }
          const uint32_t tbytes = (uint32_t)g.G[s] * 256u;
          if (!da.wait_test) {
            mbar_arrive_expect_tx(&sh.tap_full[ts], tbytes);
            bulk_load(taps + ts * tapb, bands + g.boff[s], tbytes, &sh.tap_full[ts]);
          }
          ++nt;
          const int nch = (g.Kd[s] + TC_CH - 1) / TC_CH;
          const long y0 = F.prow + (long)s * F.H + t.r0 - g.Kp[s];
          for (int c = 0; c < nch; ++c) {
            const int ls = nl % NL;
            if (!mbar_wait_bounded(&sh.land_empty[ls], ((nl / NL) & 1) ^ 1, wlim)) {
              give_up(3);
              break;
            }
            if (!da.wait_test) {
              fence_proxy_async();
              mbar_arrive_expect_tx(&sh.land_full[ls], (uint32_t)LAND);
              if (!tma_load_2d(land + (size_t)ls * BW * TC_CH, &map, xa, (int)(y0 + (long)c * TC_CH),
                               &sh.land_full[ls], (int)sizeof(T)))
                give_up(2);
            }
            ++nl;
          }
        }
      }
      // copies still in flight complete before the CTA ends (bounded)
      if (!da.wait_test) {
        for (uint32_t u = nl > (uint32_t)NL ? nl - NL : 0; u < nl; ++u)
          mbar_wait_bounded(&sh.land_full[u % NL], (u / NL) & 1, wlim);
        for (uint32_t u = nt > 2 ? nt - 2 : 0; u < nt; ++u) mbar_wait_bounded(&sh.tap_full[u & 1], (u >> 1) & 1, wlim);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issue (one thread) ----------------
    if (lane == 0) {
      uint32_t na = 0, nt = 0, ntile = 0;
      bool issued = false;
      const uint32_t idesc = tc_idesc(NR);
      int k = 0;
      for (int item = blockIdx.x; item < nitems && !*abort; item += gridDim.x) {
        int local;
        k = item_frame(it, item, k, local);
        const int H = fr[__ldg(it.fl + k)].H;
        const int r0 = tc_tile(local, fr[__ldg(it.fl + k)].W, NR).r0;
        for (int s = 0; s < S && !*abort; ++s) {
          const int ts = nt & 1;
          // the epilogue has read the previous tile's accumulators of scale s
          if (!mbar_wait_bounded(&sh.d_empty[s], (ntile & 1) ^ 1, wlim) ||
              !mbar_wait_bounded(&sh.tap_full[ts], (nt >> 1) & 1, wlim)) {
            give_up(1);
            break;
          }
          tc_fence_after();
          const uint32_t b_hi = smem_u32(taps + ts * tapb), b_lo = b_hi + (uint32_t)g.G[s] * 128u;
          const int nch = (g.Kd[s] + TC_CH - 1) / TC_CH;
          const uint32_t d = tmem + (uint32_t)(NR * s);
          for (int c = 0; c < nch; ++c) {
            const int as = na & 1;
            if (!mbar_wait_bounded(&sh.a_full[as], (na >> 1) & 1, wlim)) {
              give_up(4);
              break;
            }
            tc_fence_after();
            const uint32_t a_hi = tmem + (uint32_t)(TC_ACOL + 64 * as), a_lo = a_hi + 32u;
            const int nk = min(TC_CH / 8, (g.Kd[s] - c * TC_CH) / 8);
            // a chunk that reaches the held (f32) edge rows needs its low parts
            const int yq = r0 - g.Kp[s] + c * TC_CH;
            const bool three = F32 || yq < 0 || yq + TC_CH > H;
            for (int kk = 0; kk < nk; ++kk) {
              const uint32_t ks = (uint32_t)(4 * c + kk);
              const uint64_t bh = sdesc(b_hi + 256u * ks, 128, 256), bl = sdesc(b_lo + 256u * ks, 128, 256);
              if (three) {
                tc_mma(d, a_lo + 8u * kk, bh, idesc, ks > 0);
                tc_mma(d, a_hi + 8u * kk, bl, idesc, 1);
              } else {  // 16-bit planes are exact in TF32: no low part
                tc_mma(d, a_hi + 8u * kk, bl, idesc, ks > 0);
              }
              tc_mma(d, a_hi + 8u * kk, bh, idesc, 1);
            }
            issued = true;
            tc_commit(&sh.a_empty[as]);
            ++na;
          }
          tc_commit(&sh.tap_empty[ts]);
          ++nt;
        }
        tc_commit(&sh.d_full);
        ++ntile;
      }
      // every MMA issued completes before the tensor memory is released
      if (issued) {
        tc_commit(&sh.fin);
        mbar_wait_bounded(&sh.fin, 0, wlim);
      }
    }
  } else if (warp < 6) {
    // ---------------- split (warps 2-5): one column per thread ----------------
    const int quarter = warp & 3;        // tensor-memory lanes 32 quarter .. 32 quarter + 31
    const int c = 32 * quarter + lane;   // tile column of this thread
    const uint32_t lanes = (uint32_t)(32 * quarter) << 16;
    uint32_t nl = 0, na = 0;
    int k = 0;
    bool bad = false;
    for (int item = blockIdx.x; item < nitems && !bad; item += gridDim.x) {
      int local;
      k = item_frame(it, item, k, local);
      const FrameDev &F = fr[__ldg(it.fl + k)];
      const int H = F.H, W = F.W;
      const TcTile t = tc_tile(local, W, NR);
      const int off = ((t.x0 % XA) + XA) % XA;
      const int xc = min(max(t.x0 + c, 0), W - 1);
      for (int s = 0; s < S && !bad; ++s) {
        const int nch = (g.Kd[s] + TC_CH - 1) / TC_CH;
        // the held (or zero-boundary) edge values of this column, read once
        // per scale where the scale's rows reach beyond the frame
        float top = 0.f, bot = 0.f;
        if (t.r0 - g.Kp[s] < 0 || t.r0 - g.Kp[s] + g.Kd[s] > H) {
          const float *ed = edge + F.eoff + (long)s * 2 * PWb + xc;
          top = ed[0];
          bot = ed[PWb];
        }
        for (int ch = 0; ch < nch; ++ch) {
          const int ls = nl % NL, as = na & 1;
          bool ok = mbar_wait_bounded(&sh.land_full[ls], (nl / NL) & 1, wlim);
          ok = ok && mbar_wait_bounded(&sh.a_empty[as], ((na >> 1) & 1) ^ 1, wlim);
          if (split_sync_or(!ok)) {
            if (warp == 2 && lane == 0) give_up(1);
            bad = true;
            break;
          }
          tc_fence_after();
          const T *L = land + (size_t)ls * BW * TC_CH + off + c;
          const int yq = t.r0 - g.Kp[s] + ch * TC_CH;  // frame row of chunk row 0
          uint32_t hi[32], lo[32];
          if (yq >= 0 && yq + TC_CH <= H) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const float x = Store<ST>::ld(L[j * BW]);
              hi[j] = __float_as_uint(x);
              lo[j] = __float_as_uint(x - __uint_as_float(hi[j] & 0xffffe000u));
            }
          } else {  // rows outside the frame: the boundary rule (held or zero)
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const int y = yq + j;
              const float x = (y < 0 || y >= H) ? col_outside(y, H, top, bot, da.zero) : Store<ST>::ld(L[j * BW]);
              hi[j] = __float_as_uint(x);
              lo[j] = __float_as_uint(x - __uint_as_float(hi[j] & 0xffffe000u));
            }
          }
          const uint32_t ta = tmem + lanes + (uint32_t)(TC_ACOL + 64 * as);
          tmem_st32(ta, hi);
          // f32: the low parts; a 16-bit plane value is exact in TF32, but
          // the held edge rows (f32) need their low parts too
          if (F32 || yq < 0 || yq + TC_CH > H) tmem_st32(ta + 32u, lo);
          asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
          tc_fence_before();
          __syncwarp();
          if (lane == 0) {
            mbar_arrive(&sh.land_empty[ls]);
            mbar_arrive(&sh.a_full[as]);
          }
          ++nl;
          ++na;
        }
      }
    }
  } else {
    // ---------------- epilogue (warps 6-13) ----------------
    // warp ew reads accumulator columns [32 half, + 32) of its quarter's
    // lanes, then takes columns 32 (ew % 4) .. of the spatial test on half
    // of the tile's interior rows
    const int ew = warp - 6;            // 0..7
    const int half = ew >> 2;           // accumulator block and row half
    const int quarter = warp & 3;       // tensor-memory lanes 32 quarter ..
    const int c = 32 * quarter + lane;  // tile column of this lane's accumulators
    const uint32_t lanes = (uint32_t)(32 * quarter) << 16;
    uint32_t ntile = 0;
    int k = 0;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
      int local;
      k = item_frame(it, item, k, local);
      const FrameDev &F = fr[__ldg(it.fl + k)];
      const int H = F.H, W = F.W;
      const TcTile t = tc_tile(local, W, NR);
      const bool ok = mbar_wait_bounded(&sh.d_full, ntile & 1, wlim);
      if (epi_sync_or(!ok || *abort)) {
        if (!ok && ew == 0 && lane == 0) give_up(4);
        break;
      }
      __syncwarp();
      tc_fence_after();
      const int x = t.x0 + c;
      const bool xin = x >= 0 && x < W;
      float *resp = F.resp;
      const long plane = (long)H * W;
      // per-pixel extremes over the scales (first scale attaining them) and
      // the responses: accumulator column n is output row NR - 1 - n; this
      // warp reads the block of 32 at n0; once every reading warp has read a
      // scale its columns go to the next tile's MMAs
#pragma unroll 1
      for (int n0 = 32 * half; n0 < NR && n0 < 32 * (half + 1); n0 += 32) {
        const bool last = true;
        float vmax[32], vmin[32];
        uint32_t pmax[4] = {0, 0, 0, 0}, pmin[4] = {0, 0, 0, 0};  // 4 bits per row
#pragma unroll
        for (int j = 0; j < 32; ++j) vmax[j] = -CUDART_INF_F, vmin[j] = CUDART_INF_F;
        for (int s = 0; s < S; ++s) {
          float v[32];
          tmem_ld32(tmem + lanes + (uint32_t)(NR * s + n0), v);
          if (last) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh.d_empty[s]);  // scale s's columns free for the next tile
          }
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const uint32_t sh4 = 4u * (j & 7);
            if (v[j] > vmax[j]) vmax[j] = v[j], pmax[j >> 3] = (pmax[j >> 3] & ~(15u << sh4)) | ((uint32_t)s << sh4);
            if (v[j] < vmin[j]) vmin[j] = v[j], pmin[j >> 3] = (pmin[j >> 3] & ~(15u << sh4)) | ((uint32_t)s << sh4);
          }
          if (resp && xin && c >= 1 && c <= TC_M - 2) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const int o = NR - 1 - (n0 + j), y = t.r0 + o;
              if (o >= 1 && o <= NR - 2 && y >= 0 && y < H) resp[s * plane + (long)y * W + x] = v[j];
            }
          }
        }
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int o = NR - 1 - (n0 + j), y = t.r0 + o;
          const bool in = xin && y >= 0 && y < H;
          const uint32_t sh4 = 4u * (j & 7);
          mx[o * XS + c] = in ? vmax[j] : -CUDART_INF_F;
          mn[o * XS + c] = in ? vmin[j] : CUDART_INF_F;
          amx[o * XB + c] = in ? (unsigned char)((pmax[j >> 3] >> sh4) & 15u) : (unsigned char)S;
          amn[o * XB + c] = in ? (unsigned char)((pmin[j >> 3] >> sh4) & 15u) : (unsigned char)S;
        }
      }
      ++ntile;
      if (ew == 0 && lane == 0) tl.n = 0;
      epi_sync();
      const int ihalf = 1 + (NR - 2) / 2;  // interior rows [1, ihalf) and [ihalf, NR - 1)
      DetectArgs a = da;
      a.S = S;
      a.x0 = t.x0;
      a.r0 = t.r0;
      a.H = H;
      a.W = W;
      a.frame = F.index;
      tc_detect(mx, mn, amx, amn, tl, a, ew & 3, lane, half ? ihalf : 1, half ? NR - 1 : ihalf);
      tc_flush(a, tl, sh.base, 32 * ew + lane);
    }
  }
  // ---------------- release the tensor memory ----------------
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

__global__ void __launch_bounds__(256) k_tc_bands(const Coef *__restrict__ coef, TcGeom g, float sgn,
                                                  float *__restrict__ bands) {
  const int s = blockIdx.x;
  const Coef &c = coef[s];
  const int K = c.K, Kp = g.Kp[s], G = g.G[s];
  float *hi = bands + g.boff[s], *lo = hi + (long)G * 32;
  for (int e = threadIdx.x; e < G * 32; e += blockDim.x) {
    const int gg = e >> 5, i = (e >> 2) & 7, j = e & 3;
    const int m = abs(4 * gg + i + j - (Kp + g.NR - 1));
    const float v = m <= K ? sgn * c.h[m] : 0.f;
    uint32_t h;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(v));
    uint32_t l;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(v - __uint_as_float(h)));
    hi[e] = __uint_as_float(h);
    lo[e] = __uint_as_float(l);
  }
}

// dynamic shared memory of the pass with nl landing slots
size_t tc_smem_bytes(const TcGeom &g, int nl, int st) {
  const size_t tapb = ((size_t)2 * g.gmax * 128 + 1023) / 1024 * 1024;
  return 1024 + 2 * tapb + (size_t)nl * land_bytes(st) + (size_t)2 * g.NR * XS * 4 + (size_t)2 * g.NR * XB +
         sizeof(TcList);
}

// landing slots that fit 216 KB of dynamic shared memory (the rest of the
// 227 KB a block may have is its static part)
int tc_landing_slots(const TcGeom &g, int st) {
  int nl = TC_MAXL;
  while (nl > 2 && tc_smem_bytes(g, nl, st) > (size_t)216 * 1024) --nl;
  return nl;
}

}  // namespace

bool fir_tc_applies(int S, int storage, int neigh, int raw, long PWb, long prows) {
  // the tensor map's box (132 or 136 elements x 32 rows) fits the plane row space
  return S >= 1 && S <= TC_MAXS && storage >= ST_F32 && storage <= ST_BF16 && neigh == 0 && !raw &&
         PWb >= TC_BOXW16 && prows >= TC_CH;
}

int fir_tc_tile_cols() { return TC_M - 2; }
int fir_tc_tile_rows(int S) { return (S <= 6 ? 64 : 32) - 2; }

long tc_geometry(const int *K, int S, TcGeom *g) {
  if (S < 1 || S > TC_MAXS) return -1;
  g->S = S;
  g->NR = S <= 6 ? 64 : 32;  // S x NR accumulator columns <= 384
  g->gmax = 0;
  long off = 0;
  for (int s = 0; s < S; ++s) {
    g->K[s] = K[s];
    g->Kp[s] = (K[s] + 3) / 4 * 4;
    g->Kd[s] = g->NR + 2 * g->Kp[s];
    g->G[s] = (g->Kd[s] + g->NR + 3) / 4 + 1;
    g->boff[s] = off;
    off += 2L * g->G[s] * 32;
    g->gmax = std::max(g->gmax, g->G[s]);
  }
  g->floats = off;
  return off;
}

int launch_tc_bands(const Coef *d_coef, const TcGeom &g, float sgn, float *d_bands, cudaStream_t st) {
  k_tc_bands<<<g.S, 256, 0, st>>>(d_coef, g, sgn, d_bands);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

template <int ST>
int launch_colfir_tc_st(const Plan &p, const Launch &l, const BankArgs &a, const DetectArgs &da, cudaStream_t st) {
  // dynamic shared memory (<= 216 KB) plus the static part (barriers,
  // candidate list) within the 227 KB a block may have
  static size_t attr = 0;
  const int nl = tc_landing_slots(a.tc, ST);
  const size_t smem = tc_smem_bytes(a.tc, nl, ST);
  if (smem > 216 * 1024 || nl < 2) return -1;
  if (smem > attr) {
    if (cudaFuncSetAttribute(k_colfir_tc<ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return -1;
    attr = smem;
  }
  CUtensorMap map;
  if (encode_plane_map(&map, a.P, ST, p.PWb, p.prows, ST == ST_F32 ? TC_BOXW : TC_BOXW16, TC_CH)) return -1;
  // one CTA per SM (the tensor memory is allocated whole), persistent over the tiles
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm < 1) nsm = 1;
  }
  const int nb = std::max(1, std::min(l.it.total, nsm));
  a.prof->begin("fir_coldet", st);
  k_colfir_tc<ST><<<nb, TC_THREADS, smem, st>>>(map, p.fr, l.it, a.edge, p.PWb, a.tc_bands, a.tc, nl, da);
  a.prof->end(st);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

int launch_colfir_tc(const Plan &p, const Launch &l, const BankArgs &a, const DetectArgs &da, cudaStream_t st) {
  switch (a.storage) {
    case ST_F32: return launch_colfir_tc_st<ST_F32>(p, l, a, da, st);
    case ST_F16: return launch_colfir_tc_st<ST_F16>(p, l, a, da, st);
    case ST_BF16: return launch_colfir_tc_st<ST_BF16>(p, l, a, da, st);
    default: return -2;
  }
}

}  // namespace kf
