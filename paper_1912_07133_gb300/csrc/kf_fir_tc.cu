// kf_fir_tc.cu -- column pass of the FIR banks (colored Savitzky-Golay,
// Filter C, Sec. 4.2; Gaussian, Filter A, Sec. 3.1) on the fifth-generation
// tensor cores (tcgen05, tensor memory), with the all-scales detector of
// Sec. 5.
//
// For one scale the column blur of a tile is a banded Toeplitz product
// (eq A5 along y): out[o][c] = sum_q h(|q - Kp - o|) in[q][c], o the tile's
// output rows, q its input rows r0 - Kp + q, Kp = K rounded up to 4 (taps
// beyond K are zero).  As one MMA chain per scale:
//   D[m][c] (tensor memory, lane m = output row 127 - m, column c)
//     = sum_q A[m][q] B[c][q],  A[m][q] = band[q + m],  band[u] = sgn h(|u - Kp - 127|).
// A (M = 128 rows x K) is K-major without swizzle; because A[m][q] depends
// on q + m only, its 8-row x 16-byte core matrices are cut from one shared
// array of chunks -- chunk (g, i) at byte 16 (8 g + i) holds band[4 g + i ..
// 4 g + i + 3] -- with a K-direction core-matrix stride (LBO) of 128 bytes and
// an M-direction one (SBO) of 256 bytes: the Toeplitz structure is the
// overlap of the core matrices, so a whole scale's A takes (Kd + 131) / 4 x
// 128 bytes instead of 128 x Kd x 4.  B (N = 64 columns x K) is K-major
// without swizzle, written by the splitting warps from the TMA-landed rows.
//
// FP32 accuracy from TF32 products (three per tap product): the tensor core
// reads the top 19 bits of each 32-bit operand (truncation), so with
// x = hi + lo (hi = x with its low 13 bits cleared, lo = x - hi exactly) and
// the taps split the same way once per design (hi = tf32(h), lo = tf32(h - hi)),
// out = A_lo B_hi + A_hi B_lo + A_hi B_hi leaves about 2^-21 of each product.
// B_hi is the raw data (the tensor core truncates it to hi).
//
// One CTA per SM, persistent over the call's tiles (64 columns x 128 rows,
// interior 62 x 126), warp-specialised:
//   warp 0      TMA producer: per scale the band pair (bulk copy, two slots)
//               and the 32-row chunks of the one-sided plane (2-D tensor
//               copies of 68 x 32 floats into a ring of 8-12 landing slots,
//               as many as the shared memory holds: the chunks in flight
//               cover the copy latency);
//   warp 1      tensor-memory allocation and the MMA issue (one thread): per
//               chunk 4 k-steps x 3 products of M = 128, N = 64, K = 8;
//   warps 2-5   split each landed chunk into the B operands (raw and low
//               parts, transposed into core matrices, held rows substituted
//               at the frame's top and bottom), then the epilogue in two
//               passes (bright, then dark blobs): the per-pixel extreme over
//               all scales out of tensor memory (and the optional responses),
//               the 3 x 3 spatial test, and the tile's candidate list.
// Every wait is bounded; a wait that gives up sets the call's error status
// and the CTA stops taking tiles (copies in flight are awaited, with a
// bound, before the tensor memory is released).
#include <cudaTypedefs.h>

#include <algorithm>

#include "kf_batch.cuh"
#include "kf_common.cuh"
#include "kf_detect.cuh"
#include "kf_internal.h"
#include "kf_tma.cuh"

namespace kf {

namespace {

constexpr int TC_M = 128;         // output rows per tile (MMA M)
constexpr int TC_N = 64;          // columns per tile (MMA N)
constexpr int TC_CH = 32;         // input rows per chunk
constexpr int TC_BOXW = 68;       // landed chunk width (floats): 64 columns + TMA alignment offset <= 3
constexpr int TC_THREADS = 192;   // warps 0 (loads), 1 (MMA), 2-5 (split, epilogue)
constexpr int XS = 65;            // row stride (floats) of the per-pixel extremes
constexpr int XB = 68;            // row stride (bytes) of their first-scale maps
constexpr uint32_t TC_WAIT = 1u << 20;  // polls of a bounded wait (each parks the warp up to ~1 us)

constexpr size_t LAND_BYTES = (size_t)TC_BOXW * TC_CH * 4;  // 8704
constexpr size_t BOP_BYTES = (size_t)TC_N * TC_CH * 4;      // one B operand (hi or lo) of a chunk: 8 KB

__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  // shared-memory matrix descriptor: start >> 4, leading and stride byte
  // offsets >> 4, version 1, no swizzle
  return (uint64_t)((addr >> 4) & 0x3fffu) | ((uint64_t)((lbo >> 4) & 0x3fffu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3fffu) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor: kind::tf32, D f32, A and B tf32, both K-major, N, M
constexpr uint32_t TC_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                              ((uint32_t)(TC_M >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, int acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(TC_IDESC), "r"(acc)
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

// barrier of the 128 epilogue threads (warps 2-5) with an OR of a predicate
__device__ __forceinline__ bool epi_sync_or(bool p) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred pi, po;\n\tsetp.ne.u32 pi, %1, 0;\n\tbar.red.or.pred po, 1, 128, pi;\n\t"
      "selp.u32 %0, 1, 0, po;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)p)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// tie rule of one candidate against its 8 neighbours' extremes (strides XS, XB)
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

// The spatial 3 x 3 test of one polarity over a 128 x 64 tile (rows 0 and
// 127, columns 0 and 63 halo) by the 128 epilogue threads.  ext holds pol x
// the per-pixel extreme over the scales (-inf outside the frame), aext the
// first scale attaining it, so a candidate is a value above the threshold
// that beats its 8 neighbours with the tie rule (strictly an earlier
// neighbour in (scale, y, x) order, non-strictly a later one).  Each warp
// walks a band of rows, each lane two columns (lane, lane + 32), with the
// horizontal 3-maxima of three rows in registers; candidates are staged in
// the tile list.
__device__ void tc_detect(const float *ext, const unsigned char *aext, int pol, const DetectArgs &a, int ew,
                          int lane) {
  TileList &tl = g_tl;
  constexpr unsigned FULL = 0xffffffffu;
  const int ib = 1 + 32 * ew, ie = min(TC_M - 1, ib + 32);
  // maximum of the left and right neighbours of the two columns
  auto sides = [&](float v0, float v1, float &s0, float &s1) {
    const float u0 = __shfl_up_sync(FULL, v0, 1), d0 = __shfl_down_sync(FULL, v0, 1);
    const float u1 = __shfl_up_sync(FULL, v1, 1), d1 = __shfl_down_sync(FULL, v1, 1);
    const float b1 = __shfl_sync(FULL, v1, 0), e0 = __shfl_sync(FULL, v0, 31);
    const float l0 = lane == 0 ? -CUDART_INF_F : u0, r0 = lane == 31 ? b1 : d0;
    const float l1 = lane == 0 ? e0 : u1, r1 = lane == 31 ? -CUDART_INF_F : d1;
    s0 = fmaxf(l0, r0);
    s1 = fmaxf(l1, r1);
  };
  float xa0, xa1, vc0, vc1, lx0, lx1;
  {
    const float p0 = ext[(ib - 1) * XS + lane], p1 = ext[(ib - 1) * XS + lane + 32];
    float s0, s1;
    sides(p0, p1, s0, s1);
    xa0 = fmaxf(p0, s0), xa1 = fmaxf(p1, s1);  // row i - 1: 3-maxima
    vc0 = ext[ib * XS + lane], vc1 = ext[ib * XS + lane + 32];
    sides(vc0, vc1, lx0, lx1);                 // row i: the two side neighbours
  }
  for (int i = ib; i < ie; ++i) {
    const float vn0 = ext[(i + 1) * XS + lane], vn1 = ext[(i + 1) * XS + lane + 32];
    float lxn0, lxn1;
    sides(vn0, vn1, lxn0, lxn1);
    const int y = a.r0 + i;
    if (y >= 0 && y < a.H) {
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int c = lane + 32 * hh;
        const int x = a.x0 + c;
        if (c < 1 || c > TC_N - 2 || x < 0 || x >= a.W) continue;
        const float vc = hh ? vc1 : vc0;
        // maximum of the 8 neighbours: row i - 1 (3 columns), row i (2), row i + 1 (3)
        const float m8 = fmaxf(hh ? xa1 : xa0, fmaxf(hh ? lx1 : lx0, fmaxf(hh ? vn1 : vn0, hh ? lxn1 : lxn0)));
        if (vc > a.thr && vc >= m8) {
          const int s = aext[i * XB + c];
          if (vc > m8 || tc_beats(ext, aext, i, c, 1, vc, s)) emit_blob(a, tl, s, y, x, pol, pol * vc);
        }
      }
    }
    xa0 = fmaxf(vc0, lx0), xa1 = fmaxf(vc1, lx1);
    vc0 = vn0, vc1 = vn1, lx0 = lxn0, lx1 = lxn1;
  }
}

// the tile list's candidates to the call's list (one global reservation)
__device__ void tc_flush(const DetectArgs &a, int t) {
  TileList &tl = g_tl;
  unsigned long long &s_base = g_tl_base;
  epi_sync();
  const int nloc = min(tl.n, TILE_CANDS);
  if (t == 0 && nloc > 0) s_base = atomicAdd(&a.status->count, (unsigned long long)nloc);
  epi_sync();
  for (int i = t; i < nloc; i += 128) {
    const unsigned long long idx = s_base + i;
    if (idx < (unsigned long long)a.cap) a.out[idx] = tl.rec[i];
  }
}

constexpr int TC_MAXL = 12;  // landing slots at most

struct TcSmem {
  uint64_t land_full[TC_MAXL], land_empty[TC_MAXL], b_full[2], b_empty[2], tap_full[2], tap_empty[2], d_full,
      d_empty, fin;
  uint32_t tmem;
  int abort;
};

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_colfir_tc(const __grid_constant__ CUtensorMap map, const FrameDev *__restrict__ fr, Items it,
                const float *__restrict__ edge, long PWb, const float *__restrict__ bands, TcGeom g, int NL,
                DetectArgs da) {
  extern __shared__ __align__(1024) unsigned char sm_raw[];
  __shared__ TcSmem sh;
  unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(sm_raw) + 1023) &
                                                          ~(uintptr_t)1023);
  const size_t tapb = ((size_t)2 * g.gmax * 128 + 1023) / 1024 * 1024;  // one band pair (hi, lo)
  unsigned char *taps = base;                                               // [2][tapb]
  unsigned char *bop = taps + 2 * tapb;                                     // [2][hi 8 KB | lo 8 KB]
  float *land = reinterpret_cast<float *>(bop + 4 * BOP_BYTES);             // [NL][32][68]
  float *ext = land + (size_t)NL * TC_BOXW * TC_CH;                         // [128][XS]
  unsigned char *aext = reinterpret_cast<unsigned char *>(ext + TC_M * XS);  // [128][XB]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int S = g.S;
  if (tid == 0) {
    for (int b = 0; b < NL; ++b) {
      mbar_init(&sh.land_full[b], 1);
      mbar_init(&sh.land_empty[b], 4);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sh.b_full[b], 4);
      mbar_init(&sh.b_empty[b], 1);
      mbar_init(&sh.tap_full[b], 1);
      mbar_init(&sh.tap_empty[b], 1);
    }
    mbar_init(&sh.d_full, 1);
    mbar_init(&sh.d_empty, 4);
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
        const int H = F.H, W = F.W;
        const int ntx = (W + TC_N - 3) / (TC_N - 2);
        const int x0 = (local % ntx) * (TC_N - 2) - 1, r0 = (local / ntx) * (TC_M - 2) - 1;
        const int xa = x0 - (((x0 % 4) + 4) % 4);
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
          const long y0 = F.prow + (long)s * H + r0 - g.Kp[s];
          for (int c = 0; c < nch; ++c) {
            const int ls = nl % NL;
            if (!mbar_wait_bounded(&sh.land_empty[ls], ((nl / NL) & 1) ^ 1, wlim)) {
              give_up(3);
              break;
            }
            if (!da.wait_test) {
              fence_proxy_async();
              mbar_arrive_expect_tx(&sh.land_full[ls], (uint32_t)LAND_BYTES);
              if (!tma_load_2d(land + ls * TC_BOXW * TC_CH, &map, xa, (int)(y0 + (long)c * TC_CH), &sh.land_full[ls]))
                give_up(2);
            }
            ++nl;
          }
        }
      }
      // copies still in flight complete before the CTA ends (bounded)
      for (uint32_t u = nl > (uint32_t)NL ? nl - NL : 0; u < nl; ++u)
        if (!da.wait_test) mbar_wait_bounded(&sh.land_full[u % NL], (u / NL) & 1, wlim);
      for (uint32_t u = nt > 2 ? nt - 2 : 0; u < nt; ++u)
        if (!da.wait_test) mbar_wait_bounded(&sh.tap_full[u & 1], (u >> 1) & 1, wlim);
    }
  } else if (warp == 1) {
    // ---------------- MMA issue (one thread) ----------------
    if (lane == 0) {
      uint32_t nb = 0, nt = 0, ntile = 0;
      bool issued = false;
      for (int item = blockIdx.x; item < nitems && !*abort; item += gridDim.x) {
        if (!mbar_wait_bounded(&sh.d_empty, (ntile & 1) ^ 1, wlim)) {
          give_up(4);
          break;
        }
        tc_fence_after();
        for (int s = 0; s < S && !*abort; ++s) {
          const int ts = nt & 1;
          if (!mbar_wait_bounded(&sh.tap_full[ts], (nt >> 1) & 1, wlim)) {
            give_up(1);
            break;
          }
          const uint32_t a_hi = smem_u32(taps + ts * tapb), a_lo = a_hi + (uint32_t)g.G[s] * 128u;
          const int nch = (g.Kd[s] + TC_CH - 1) / TC_CH;
          const uint32_t d = tmem + (uint32_t)(TC_N * s);
          for (int c = 0; c < nch; ++c) {
            const int bs = nb & 1;
            if (!mbar_wait_bounded(&sh.b_full[bs], (nb >> 1) & 1, wlim)) {
              give_up(4);
              break;
            }
            tc_fence_after();
            const uint32_t b_hi = smem_u32(bop + (size_t)bs * 2 * BOP_BYTES), b_lo = b_hi + (uint32_t)BOP_BYTES;
            const int nk = min(TC_CH / 8, (g.Kd[s] - c * TC_CH) / 8);
            for (int kk = 0; kk < nk; ++kk) {
              const uint32_t ks = (uint32_t)(4 * c + kk);
              const uint64_t ah = sdesc(a_hi + 256u * ks, 128, 256), al = sdesc(a_lo + 256u * ks, 128, 256);
              const uint64_t bh = sdesc(b_hi + 256u * kk, 128, 1024), bl = sdesc(b_lo + 256u * kk, 128, 1024);
              tc_mma(d, al, bh, ks > 0);
              tc_mma(d, ah, bl, 1);
              tc_mma(d, ah, bh, 1);
            }
            issued = true;
            tc_commit(&sh.b_empty[bs]);
            ++nb;
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
  } else {
    // ---------------- split (warps 2-5), then the epilogue ----------------
    const int ew = warp - 2;              // 0..3: the warp's share of the chunk
    const int quarter = warp & 3;         // tensor-memory lanes 32 quarter ..
    uint32_t nl = 0, nb = 0, ntile = 0;
    int k = 0;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
      if (epi_sync_or(*abort != 0)) break;
      int local;
      k = item_frame(it, item, k, local);
      const FrameDev &F = fr[__ldg(it.fl + k)];
      const int H = F.H, W = F.W;
      const int ntx = (W + TC_N - 3) / (TC_N - 2);
      const int x0 = (local % ntx) * (TC_N - 2) - 1, r0 = (local / ntx) * (TC_M - 2) - 1;
      const int off = ((x0 % 4) + 4) % 4;
      bool bad = false;
      for (int s = 0; s < S && !bad; ++s) {
        const int nch = (g.Kd[s] + TC_CH - 1) / TC_CH;
        const float *ed = edge + F.eoff + (long)s * 2 * PWb;
        for (int c = 0; c < nch; ++c) {
          const int ls = nl % NL, bs = nb & 1;
          bool ok = mbar_wait_bounded(&sh.land_full[ls], (nl / NL) & 1, wlim);
          ok = ok && mbar_wait_bounded(&sh.b_empty[bs], ((nb >> 1) & 1) ^ 1, wlim);
          if (epi_sync_or(!ok)) {
            if (ew == 0 && lane == 0) give_up(1);
            bad = true;
            break;
          }
          const float *L = land + ls * TC_BOXW * TC_CH;
          float *bh = reinterpret_cast<float *>(bop + (size_t)bs * 2 * BOP_BYTES), *bl = bh + BOP_BYTES / 4;
          const int yq = r0 - g.Kp[s] + c * TC_CH;  // frame row of chunk row 0
          const bool outside = yq < 0 || yq + TC_CH > H;
          // core matrix (8 columns x 4 rows) per warp step: lane = 4 (column % 8) + row % 4
          const int cl = lane >> 2, ql = lane & 3;
#pragma unroll 4
          for (int cm = 16 * ew; cm < 16 * ew + 16; ++cm) {
            const int ccm = cm & 7, qcm = cm >> 3;
            const int cc = 8 * ccm + cl, qq = 4 * qcm + ql;
            float x = L[qq * TC_BOXW + off + cc];
            if (outside) {
              const int y = yq + qq;
              if (y < 0 || y >= H) {
                const float *e = ed + min(max(x0 + cc, 0), W - 1);
                x = col_outside(y, H, e[0], e[PWb], da.zero);
              }
            }
            const float hi = __uint_as_float(__float_as_uint(x) & 0xffffe000u);
            const int o = ccm * 256 + qcm * 32 + lane;  // float offset: 1024 B per column group, 128 B per row quad
            bh[o] = x;
            bl[o] = x - hi;
          }
          fence_proxy_async();
          __syncwarp();
          if (lane == 0) {
            mbar_arrive(&sh.land_empty[ls]);
            mbar_arrive(&sh.b_full[bs]);
          }
          ++nl;
          ++nb;
        }
      }
      if (bad) break;
      // ---- epilogue: extremes over the scales from tensor memory ----
      const bool ok = mbar_wait_bounded(&sh.d_full, ntile & 1, wlim);
      if (epi_sync_or(!ok)) {
        if (ew == 0 && lane == 0) give_up(4);
        break;
      }
      __syncwarp();
      tc_fence_after();
      const int m = 32 * quarter + lane, o = TC_M - 1 - m;  // output row of this lane
      const int y = r0 + o;
      const bool yin = y >= 0 && y < H;
      float *resp = F.resp;
      const long plane = (long)H * W;
      DetectArgs a = da;
      a.S = S;
      a.x0 = x0;
      a.r0 = r0;
      a.H = H;
      a.W = W;
      a.frame = F.index;
      if (ew == 0 && lane == 0) g_tl.n = 0;
      // pass 0: bright blobs (maxima of R over the scales); pass 1: dark ones
      // (minima, stored negated so that both passes test maxima).  The
      // second pass's reads of the tensor memory are its last.
#pragma unroll 1
      for (int pass = 0; pass < 2; ++pass) {
        const float pol = pass ? -1.f : 1.f;
        if (pass) epi_sync();  // the first pass's detector is done with ext
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
          float vx[32];
          uint32_t px[4] = {0, 0, 0, 0};  // first scale attaining the extreme, 4 bits per column
#pragma unroll
          for (int j = 0; j < 32; ++j) vx[j] = -CUDART_INF_F;
          for (int s = 0; s < S; ++s) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(TC_N * s + 32 * h), v);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const float w = pol * v[j];
              if (w > vx[j]) vx[j] = w, px[j >> 3] = (px[j >> 3] & ~(15u << (4 * (j & 7)))) | ((uint32_t)s << (4 * (j & 7)));
            }
            if (!pass && resp && yin && o >= 1 && o <= TC_M - 2) {
#pragma unroll
              for (int j = 0; j < 32; ++j) {
                const int c = 32 * h + j, x = x0 + c;
                if (c >= 1 && c <= TC_N - 2 && x >= 0 && x < W) resp[s * plane + (long)y * W + x] = v[j];
              }
            }
          }
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int c = 32 * h + j, x = x0 + c;
            const bool in = yin && x >= 0 && x < W;
            ext[o * XS + c] = in ? vx[j] : -CUDART_INF_F;
            aext[o * XB + c] = in ? (unsigned char)((px[j >> 3] >> (4 * (j & 7))) & 15u) : (unsigned char)S;
          }
        }
        if (pass) {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&sh.d_empty);  // tensor memory free for the next tile
        }
        epi_sync();
        if (pass == 0 || a.dark) tc_detect(ext, aext, pass ? -1 : 1, a, ew, lane);
      }
      ++ntile;
      tc_flush(a, 32 * ew + lane);
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
    const int m = abs(4 * gg + i + j - (Kp + TC_M - 1));
    const float v = m <= K ? sgn * c.h[m] : 0.f;
    uint32_t h;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(v));
    uint32_t l;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(v - __uint_as_float(h)));
    hi[e] = __uint_as_float(h);
    lo[e] = __uint_as_float(l);
  }
}

}  // namespace

bool fir_tc_applies(int S, int storage, int neigh, int raw, long PWb, long prows) {
  // the tensor map's box (68 x 32) fits the plane row space
  return S >= 1 && S <= TC_MAXS && storage == ST_F32 && neigh == 0 && !raw && PWb >= TC_BOXW && prows >= TC_CH;
}

int fir_tc_tile_cols() { return TC_N - 2; }

long tc_geometry(const int *K, int S, TcGeom *g) {
  if (S < 1 || S > TC_MAXS) return -1;
  g->S = S;
  g->gmax = 0;
  long off = 0;
  for (int s = 0; s < S; ++s) {
    g->K[s] = K[s];
    g->Kp[s] = (K[s] + 3) / 4 * 4;
    g->Kd[s] = TC_M + 2 * g->Kp[s];
    g->G[s] = (g->Kd[s] + TC_M + 3) / 4 + 1;
    g->boff[s] = off;
    off += 2L * g->G[s] * 32;
    g->gmax = std::max(g->gmax, g->G[s]);
  }
  g->floats = off;
  return off;
}

// dynamic shared memory of the pass with nl landing slots
size_t tc_smem_bytes(const TcGeom &g, int nl) {
  const size_t tapb = ((size_t)2 * g.gmax * 128 + 1023) / 1024 * 1024;
  return 1024 + 2 * tapb + 4 * BOP_BYTES + (size_t)nl * LAND_BYTES + (size_t)TC_M * XS * 4 + (size_t)TC_M * XB;
}

// landing slots that fit 216 KB of dynamic shared memory (the rest of the
// 227 KB a block may have is its static part): 10 for K <= 96, 8 for K <= 160
int tc_landing_slots(const TcGeom &g) {
  int nl = TC_MAXL;
  while (nl > 2 && tc_smem_bytes(g, nl) > (size_t)216 * 1024) --nl;
  return nl;
}

int launch_tc_bands(const Coef *d_coef, const TcGeom &g, float sgn, float *d_bands, cudaStream_t st) {
  k_tc_bands<<<g.S, 256, 0, st>>>(d_coef, g, sgn, d_bands);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

int launch_colfir_tc(const Plan &p, const Launch &l, const BankArgs &a, const DetectArgs &da, cudaStream_t st) {
  // dynamic shared memory (<= 206 KB for K <= 160) plus the static part
  // (barriers, candidate list) within the 227 KB a block may have
  static size_t attr = 0;
  const int nl = tc_landing_slots(a.tc);
  const size_t smem = tc_smem_bytes(a.tc, nl);
  if (smem > 216 * 1024) return -1;
  if (smem > attr) {
    if (cudaFuncSetAttribute(k_colfir_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return -1;
    attr = smem;
  }
  CUtensorMap map;
  if (encode_plane_map(&map, a.P, ST_F32, p.PWb, p.prows, TC_BOXW, TC_CH)) return -1;
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
  k_colfir_tc<<<nb, TC_THREADS, smem, st>>>(map, p.fr, l.it, a.edge, p.PWb, a.tc_bands, a.tc, nl, da);
  a.prof->end(st);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace kf
