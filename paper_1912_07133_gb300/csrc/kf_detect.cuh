// kf_detect.cuh -- scale-space extremum detector on a tile of responses held
// in shared memory (Kennedy, arXiv:1912.07133, Sec. 5, Threshold #1).
//
// The tile buffer holds R for all S scales on NR rows x 32 columns; row 0 and
// row NR-1, lane 0 and lane 31 are halo.  A candidate at (s, y, x) must beat
// every in-frame neighbour of its 3 x 3 x (scales) neighbourhood: strictly a
// neighbour earlier in (scale, y, x) order, non-strictly a later one, so that
// exactly one pixel of a plateau survives.  Bright: R > T; dark (Laplacian
// response only): R < -T, mirrored.
#pragma once
#include <math_constants.h>

#include "kf_common.cuh"

namespace kf {

struct DetectArgs {
  int S, NR;           // scales, buffer rows
  int x0;              // frame column of lane 0
  int r0;              // frame row of buffer row 0
  int H, W;
  float thr;
  int neigh;           // 0 all scales, 1 adjacent scales
  int dark;            // 1: also report minima (Laplacian response)
  int frame;
  Blob *out;
  long cap;
  DevStatus *status;
  float *resp;         // optional: R planes of this frame (S x H x W)
  long rplane = 0;     // with rplane > 0: the frame's cropped response layout (FrameDev)
  int rpitch = 0, rmx = 0, rmy = 0;
  int ld = 32;         // row stride of the response buffer (floats)
  int coff = 0;        // column of lane 0 inside a buffer row
  int srows = 0;       // rows per scale in the buffer (0: NR)
  int raw = 0;         // 1: the buffer holds a derivative channel: write it, no detection
  // derivative bank: sigma^2 D planes of the frame (S x H x W) for the eq (27)
  // offsets of the candidates (d10/d01 null: no offsets), Threshold #2 limit
  const float *d10 = nullptr, *d01 = nullptr, *d20 = nullptr, *d02 = nullptr, *d11 = nullptr;
  float limit2 = 0.f;
  // failure-detection test hook: > 0, the column pass issues no copy to its
  // load barrier (nothing is in flight) and its bounded wait gives up after
  // this many polls, so the call reports a timed-out wait
  unsigned wait_test = 0;
  int zero = 0;  // FIR column passes: the zero boundary (rows -1 and H from the edge rows, zero beyond)
};

// Input of a column pass at frame row y outside [0, H): the held one-sided
// edge rows (top, bot) for the hold boundary; for the zero boundary those
// rows one row beyond the frame and zero further out.
__device__ __forceinline__ float col_outside(int y, int H, float top, float bot, int zero) {
  if (y < 0) return (zero && y < -1) ? 0.f : top;
  return (zero && y > H) ? 0.f : bot;
}

constexpr int TILE_CANDS = 128;  // candidates staged per tile before one global reservation

struct TileList {
  int n;
  Blob rec[TILE_CANDS];
};

// one staged list per CTA (file-scope shared: every kernel gets its own)
static __shared__ TileList g_tl;
static __shared__ unsigned long long g_tl_base;

// Stage a candidate in the tile's list; when it is full, reserve globally.
static __device__ __forceinline__ void emit_blob(const DetectArgs &a, TileList &tl, int s, int y, int x,
                                                 int pol, float v) {
  Blob b;
  b.frame = a.frame;
  b.x = x;
  b.y = y;
  b.scale = s;
  b.polarity = pol;
  b.response = v;
  b.dx = b.dy = 0.f;
  if (a.d10) {  // eq (27): offset of the extremum of the local quadratic (sigma^2 factors cancel)
    const long i = ((long)s * a.H + y) * a.W + x;
    const float d10 = a.d10[i], d01 = a.d01[i], d20 = a.d20[i], d02 = a.d02[i], d11 = a.d11[i];
    const float det = d20 * d02 - d11 * d11;
    b.dx = (d01 * d11 - d02 * d10) / det;
    b.dy = (d10 * d11 - d20 * d01) / det;
    if (a.limit2 > 0.f && !(sqrtf(b.dx * b.dx + b.dy * b.dy) <= a.limit2)) return;  // Threshold #2
  }
  const int slot = atomicAdd(&tl.n, 1);
  if (slot < TILE_CANDS) {
    tl.rec[slot] = b;
  } else {
    const unsigned long long idx = atomicAdd(&a.status->count, 1ull);
    if (idx < (unsigned long long)a.cap) a.out[idx] = b;
  }
}

// First scale attaining a pixel's extreme, from per-pixel byte arrays.
struct ArgBytes {
  const unsigned char *amx, *amn;
  __device__ __forceinline__ int operator()(int p, int pol) const { return pol > 0 ? amx[p] : amn[p]; }
};

// The same found on demand by scanning the tile's scales (buffer row i =
// p / 32, column p % 32) for the first value equal to the extreme: the
// per-pixel pass then keeps only the extremes (two min/max per scale), and
// the scan runs for candidates and ties only.
struct ArgScan {
  const float *buf, *mx, *mn;
  int S, SR, ld, coff;
  __device__ __forceinline__ int operator()(int p, int pol) const {
    const float t = pol > 0 ? mx[p] : mn[p];
    const float *b = buf + (p >> 5) * ld + coff + (p & 31);
    for (int s = 0; s < S; ++s)
      if (b[(long)s * SR * ld] == t) return s;
    return S;  // outside the frame (+-inf)
  }
};

// The tie rule of one candidate against its 8 neighbours' extremes m (first
// scales from arg): strictly above a neighbour earlier in (y, x) order or with
// an earlier first scale, at least equal to a later one (pol = -1 mirrors the
// values).
template <class ArgF>
static __device__ __forceinline__ bool beats_neighbours(const float *m, const ArgF &arg, int p, int pol, float v,
                                                        int s) {
  bool ok = true;
  for (int di = -1; di <= 1 && ok; ++di)
    for (int dl = -1; dl <= 1 && ok; ++dl) {
      if (di == 0 && dl == 0) continue;
      const int pn = p + di * 32 + dl;
      const float vn = m[pn];
      if (pol * v != pol * vn) {  // no tie: the first scale does not matter
        ok = pol * v > pol * vn;
        continue;
      }
      const int sn = arg(pn, pol);
      const bool after = di > 0 || (di == 0 && dl > 0);
      const float a1 = pol * v, b1 = pol * vn;
      ok = (a1 > b1) || (a1 == b1 && (sn > s || (sn == s && after)));
    }
  return ok;
}

// Spatial part of the all-scales test.  mx/mn: per-pixel maximum/minimum of R
// over the scales of an NR x 32 tile (+-inf outside the frame), arg(p, pol):
// the first scale attaining them.  A pixel's candidate is its first argmax
// (argmin); it must beat the 8 neighbours' extremes with the tie rule.
// Each warp walks a band of interior rows, one column per lane, holding the
// horizontal 3-maxima (3-minima, by shuffles) of three consecutive rows in
// registers: a pixel below its 3 x 3 maximum cannot pass, one strictly above
// its 8 neighbours passes, and the rest (ties) take the exact tie test.  Candidates are staged in shared memory and reserved
// globally once per tile.  Must be called by all threads of the block
// (blockDim a multiple of 32; contains __syncthreads).
template <class ArgF>
static __device__ void spatial_detect(const float *mx, const float *mn, const ArgF &arg, const DetectArgs &a) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  TileList &tl = g_tl;
  unsigned long long &s_base = g_tl_base;
  if (tid == 0) tl.n = 0;
  __syncthreads();
  const int chunk = (a.NR - 2 + (nt >> 5) - 1) / (nt >> 5);
  const int ib = 1 + warp * chunk, ie = min(a.NR - 1, ib + chunk);  // rows [ib, ie), warp-uniform
  const int x = a.x0 + lane;
  const bool col = lane >= 1 && lane <= 30 && x >= 0 && x < a.W;
  constexpr unsigned FULL = 0xffffffffu;
  // maximum (minimum) of the left and right neighbours
  auto lrmax = [&](float v) { return fmaxf(__shfl_up_sync(FULL, v, 1), __shfl_down_sync(FULL, v, 1)); };
  auto lrmin = [&](float v) { return fminf(__shfl_up_sync(FULL, v, 1), __shfl_down_sync(FULL, v, 1)); };
  if (ib < ie) {
    float vp = mx[(ib - 1) * 32 + lane], wp = mn[(ib - 1) * 32 + lane];
    float xa = fmaxf(vp, lrmax(vp)), na = fminf(wp, lrmin(wp));  // row i - 1: 3-maximum (minimum)
    float vc = mx[ib * 32 + lane], wc = mn[ib * 32 + lane];
    float lx = lrmax(vc), ln = lrmin(wc);  // row i: the two side neighbours
    for (int i = ib; i < ie; ++i) {
      const float vn = mx[(i + 1) * 32 + lane], wn = mn[(i + 1) * 32 + lane];
      const float lxn = lrmax(vn), lnn = lrmin(wn);
      const float xc = fmaxf(vn, lxn), nc = fminf(wn, lnn);  // row i + 1
      const int y = a.r0 + i;
      if (col && y >= 0 && y < a.H) {
        const int p = i * 32 + lane;
        const float m8 = fmaxf(xa, fmaxf(lx, xc));  // maximum of the 8 neighbours
        if (vc > a.thr && vc >= m8) {
          const int s = arg(p, 1);
          if (vc > m8 || beats_neighbours(mx, arg, p, 1, vc, s)) emit_blob(a, tl, s, y, x, 1, vc);
        }
        const float n8 = fminf(na, fminf(ln, nc));
        if (a.dark && -wc > a.thr && wc <= n8) {
          const int s = arg(p, -1);
          if (wc < n8 || beats_neighbours(mn, arg, p, -1, wc, s)) emit_blob(a, tl, s, y, x, -1, wc);
        }
      }
      xa = fmaxf(vc, lx), na = fminf(wc, ln);
      vc = vn, wc = wn, lx = lxn, ln = lnn;
    }
  }
  __syncthreads();
  const int nloc = min(tl.n, TILE_CANDS);
  if (tid == 0 && nloc > 0) s_base = atomicAdd(&a.status->count, (unsigned long long)nloc);
  __syncthreads();
  for (int i = tid; i < nloc; i += nt) {
    const unsigned long long idx = s_base + i;
    if (idx < (unsigned long long)a.cap) a.out[idx] = tl.rec[i];
  }
}

// buf: [S][NR][32] responses; red: scratch of NR*32*(2 floats + 2 bytes).
// Must be called by all threads of the block (contains __syncthreads).
static __device__ void detect_tile(const float *buf, float *red, const DetectArgs &a) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int NP = a.NR * 32;
  const int NI = (a.NR - 2) * 30;  // interior pixels
  const int SR = a.srows ? a.srows : a.NR;
  if (a.resp) {
    const long plane = a.rplane > 0 ? a.rplane : (long)a.H * a.W;
    const int pitch = a.rplane > 0 ? a.rpitch : a.W, mx = a.rplane > 0 ? a.rmx : 0, my = a.rplane > 0 ? a.rmy : 0;
    for (int q = tid; q < NI; q += nt) {
      const int i = 1 + q / 30, lane = 1 + q % 30;
      const int y = a.r0 + i, x = a.x0 + lane;
      if (y < my || y >= a.H - my || x < mx || x >= a.W - mx) continue;
      for (int s = 0; s < a.S; ++s)
        a.resp[s * plane + (long)(y - my) * pitch + (x - mx)] = buf[(s * SR + i) * a.ld + a.coff + lane];
    }
  }
  if (a.raw) return;  // a derivative channel: written, not detected (uniform over the block)
  float *mx = red, *mn = red + NP;
  if (a.neigh == 0) {
    // per-pixel extremes over scales, out-of-frame -> +-inf (the first scale
    // attaining them is found on demand)
    for (int p = tid; p < NP; p += nt) {
      const int i = p >> 5, lane = p & 31;
      const int y = a.r0 + i, x = a.x0 + lane;
      float vmax = -CUDART_INF_F, vmin = CUDART_INF_F;
      if (y >= 0 && y < a.H && x >= 0 && x < a.W) {
        const float *b = buf + i * a.ld + a.coff + lane;
        for (int s = 0; s < a.S; ++s) {
          const float v = b[(long)s * SR * a.ld];
          vmax = fmaxf(vmax, v);
          vmin = fminf(vmin, v);
        }
      }
      mx[p] = vmax;
      mn[p] = vmin;
    }
    __syncthreads();
    ArgScan arg{buf, mx, mn, a.S, SR, a.ld, a.coff};
    spatial_detect(mx, mn, arg, a);
    return;
  }
  // adjacent scales: every (scale, pixel) against its 3 x 3 x 3 neighbourhood
  TileList &tl = g_tl;
  unsigned long long &s_base = g_tl_base;
  if (tid == 0) tl.n = 0;
  __syncthreads();
  for (int q = tid; q < NI; q += nt) {
    const int i = 1 + q / 30, lane = 1 + q % 30;
    const int y = a.r0 + i, x = a.x0 + lane;
    if (y < 0 || y >= a.H || x < 0 || x >= a.W) continue;
    for (int s = 0; s < a.S; ++s) {
      const float v = buf[(s * SR + i) * a.ld + a.coff + lane];
      const int pol = (v > a.thr) ? 1 : ((a.dark && v < -a.thr) ? -1 : 0);
      if (!pol) continue;
      bool ok = true;
      for (int t = max(0, s - 1); t <= min(a.S - 1, s + 1) && ok; ++t)
        for (int di = -1; di <= 1 && ok; ++di)
          for (int dl = -1; dl <= 1 && ok; ++dl) {
            if (t == s && di == 0 && dl == 0) continue;
            const int yn = y + di, xn = x + dl;
            if (yn < 0 || yn >= a.H || xn < 0 || xn >= a.W) continue;
            const float vn = buf[(t * SR + i + di) * a.ld + a.coff + lane + dl];
            const bool earlier = t < s || (t == s && (di < 0 || (di == 0 && dl < 0)));
            ok = earlier ? (pol * v > pol * vn) : (pol * v >= pol * vn);
          }
      if (ok) emit_blob(a, tl, s, y, x, pol, v);
    }
  }
  __syncthreads();
  const int nloc = min(tl.n, TILE_CANDS);
  if (tid == 0 && nloc > 0) s_base = atomicAdd(&a.status->count, (unsigned long long)nloc);
  __syncthreads();
  for (int i = tid; i < nloc; i += nt) {
    const unsigned long long idx = s_base + i;
    if (idx < (unsigned long long)a.cap) a.out[idx] = tl.rec[i];
  }
}

}  // namespace kf
