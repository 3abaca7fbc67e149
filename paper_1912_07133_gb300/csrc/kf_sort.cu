// kf_sort.cu -- ordering of the detector's candidate list on the GPU: the
// candidates arrive in arbitrary (atomic) order; the blob list is returned in
// (frame, scale, y, x) order.  Least-significant-digit radix sort of 64-bit
// keys with digits of up to 9 bits (stable per pass), then a gather of the records.
// Candidates at or below the re-threshold get the all-ones key and sort last.
// Every launch reads the candidate count from the device status and loops
// over the list's 1024-item tiles (grids of at most a few blocks per SM), so
// the ordering can be enqueued (and captured in a graph) before the count is
// known on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <utility>

#include "kf_common.cuh"
#include "kf_internal.h"

namespace kf {

namespace {

constexpr int SORT_NT = 256;               // threads per block
constexpr int SORT_ITEMS = 4;              // items per thread (1024-item tiles: enough blocks for 152 SMs)
constexpr int TILE = SORT_NT * SORT_ITEMS; // items per block
constexpr int NWARP = SORT_NT / 32;
constexpr int ITEMS_PER_WARP = TILE / NWARP;
constexpr int MAXBITS = 9;                 // digit width per pass (<= 9 bits: 512 digits)
constexpr int MAXD = 1 << MAXBITS;

// candidates to order: the device count, clamped to the list's capacity
__device__ __forceinline__ long list_n(const unsigned long long *count, long cap) {
  return (long)min(*count, (unsigned long long)cap);
}

__global__ void k_keys(const Blob *__restrict__ b, long cap, const unsigned long long *__restrict__ count, float thr,
                       int nscales, long hmax, long wmax, unsigned long long *__restrict__ key,
                       unsigned *__restrict__ idx, unsigned *__restrict__ npass) {
  const long n = list_n(count, cap);
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const Blob r = b[i];
    const bool pass = fabsf(r.response) > thr;
    unsigned long long k = ~0ull;
    if (pass) {
      k = (((unsigned long long)r.frame * nscales + r.scale) * hmax + r.y) * wmax + r.x;
      atomicAdd(npass, 1u);
    }
    key[i] = k;
    idx[i] = (unsigned)i;
  }
}

__device__ __forceinline__ int digit(unsigned long long k, int shift, int bits) {
  return (int)((k >> shift) & ((1ull << bits) - 1ull));
}

// per-tile digit histogram: hist[d * stride + tile]
__global__ void __launch_bounds__(SORT_NT) k_hist(const unsigned long long *__restrict__ key, long cap,
                                                  const unsigned long long *__restrict__ count, int shift, int bits,
                                                  unsigned *__restrict__ hist, int stride) {
  __shared__ unsigned h[MAXD];
  const long n = list_n(count, cap);
  const int tid = threadIdx.x, nd = 1 << bits;
  for (long t = blockIdx.x; t * TILE < n; t += gridDim.x) {  // uniform over the block
    for (int d = tid; d < nd; d += SORT_NT) h[d] = 0;
    __syncthreads();
    for (int j = 0; j < SORT_ITEMS; ++j) {
      const long i = t * TILE + (long)j * SORT_NT + tid;
      if (i < n) atomicAdd(&h[digit(key[i], shift, bits)], 1u);
    }
    __syncthreads();
    for (int d = tid; d < nd; d += SORT_NT) hist[(long)d * stride + t] = h[d];
  }
}

// One warp per digit d: exclusive scan of hist[d * stride + (0..nb)] over
// the nb blocks that hold items, in place, and the digit's total in tot[d].
__global__ void __launch_bounds__(SORT_NT) k_scan_digits(unsigned *__restrict__ hist, int stride, int nd, long cap,
                                                         const unsigned long long *__restrict__ count,
                                                         unsigned *__restrict__ tot) {
  const int lane = threadIdx.x & 31, d = blockIdx.x * NWARP + (threadIdx.x >> 5);
  if (d >= nd) return;
  const int nb = (int)((list_n(count, cap) + TILE - 1) / TILE);
  unsigned *h = hist + (long)d * stride;
  unsigned carry = 0;
  for (int b0 = 0; b0 < nb; b0 += 32) {
    const int b = b0 + lane;
    const unsigned v = b < nb ? h[b] : 0u;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (b < nb) h[b] = carry + x - v;
    carry += __shfl_sync(0xffffffffu, x, 31);
  }
  if (lane == 0) tot[d] = carry;
}

// stable scatter: items keep their order inside a digit; a digit's first
// position is the sum of the totals of the smaller digits (a block scan of
// tot) plus the earlier blocks' counts of it (hist, scanned)
__global__ void __launch_bounds__(SORT_NT) k_scatter(const unsigned long long *__restrict__ kin,
                                                     const unsigned *__restrict__ iin, long cap,
                                                     const unsigned long long *__restrict__ count, int shift,
                                                     int bits, const unsigned *__restrict__ off, int stride,
                                                     const unsigned *__restrict__ tot,
                                                     unsigned long long *__restrict__ kout,
                                                     unsigned *__restrict__ iout) {
  __shared__ unsigned cnt[NWARP][MAXD];
  __shared__ unsigned dbase[MAXD];
  __shared__ unsigned wsum[NWARP];
  const long n = list_n(count, cap);
  if ((long)blockIdx.x * TILE >= n) return;  // uniform over the block
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nd = 1 << bits;
  {  // digit bases: exclusive scan of tot[0..nd), two digits per thread
    const unsigned t0 = 2 * tid < nd ? tot[2 * tid] : 0u, t1 = 2 * tid + 1 < nd ? tot[2 * tid + 1] : 0u;
    unsigned x = t0 + t1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    unsigned before = x - t0 - t1;
    for (int ww = 0; ww < w; ++ww) before += wsum[ww];
    if (2 * tid < nd) dbase[2 * tid] = before;
    if (2 * tid + 1 < nd) dbase[2 * tid + 1] = before + t0;
  }
  const unsigned lt = (1u << lane) - 1u;
  for (long t = blockIdx.x; t * TILE < n; t += gridDim.x) {  // uniform over the block
    for (int d = lane; d < nd; d += 32) cnt[w][d] = 0;
    __syncthreads();
    const long wbase = t * TILE + (long)w * ITEMS_PER_WARP;
    // pass 1: per-warp digit counts
    for (int r = 0; r < ITEMS_PER_WARP / 32; ++r) {
      const long i = wbase + r * 32 + lane;
      const bool valid = i < n;
      const int d = valid ? digit(kin[i], shift, bits) : MAXD + lane;  // invalid lanes never match
      const unsigned m = __match_any_sync(0xffffffffu, d);
      if (valid && (m & lt) == 0) cnt[w][d] += __popc(m);
      __syncwarp();
    }
    __syncthreads();
    // exclusive prefix over warps, plus the tile's global offset for the digit
    for (int d = tid; d < nd; d += SORT_NT) {
      unsigned run = dbase[d] + off[(long)d * stride + t];
      for (int ww = 0; ww < NWARP; ++ww) {
        const unsigned c = cnt[ww][d];
        cnt[ww][d] = run;
        run += c;
      }
    }
    __syncthreads();
    // pass 2: positions
    for (int r = 0; r < ITEMS_PER_WARP / 32; ++r) {
      const long i = wbase + r * 32 + lane;
      const bool valid = i < n;
      unsigned long long k = valid ? kin[i] : 0ull;
      const int d = valid ? digit(k, shift, bits) : MAXD + lane;
      const unsigned m = __match_any_sync(0xffffffffu, d);
      if (valid) {
        const unsigned pos = cnt[w][d] + __popc(m & lt);
        kout[pos] = k;
        iout[pos] = iin[i];
      }
      __syncwarp();
      if (valid && (m & lt) == 0) cnt[w][d] += __popc(m);
      __syncwarp();
    }
    __syncthreads();  // cnt is reset for the next tile
  }
}

__global__ void k_gather(const Blob *__restrict__ b, const unsigned *__restrict__ idx, long cap,
                         const unsigned long long *__restrict__ count, Blob *__restrict__ out) {
  const long n = list_n(count, cap);
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    out[i] = b[idx[i]];
}

// ---------------------------------------------------------------------------
// row-bucket ordering: a counting sort of the passing candidates by (frame,
// scale, y) -- one bucket per frame row of a scale -- then within a bucket by
// x (keys are unique: one candidate per pixel and scale).  Six light launches
// instead of the radix's eleven; used while the buckets fit the workspace.
// ---------------------------------------------------------------------------
constexpr long ROW_BUCKETS_MAX = 1L << 22;
constexpr int SCAN_CHUNK = 4096;  // buckets per block of the scans

__device__ __forceinline__ unsigned row_bucket(const Blob &r, int nscales, long hmax) {
  return (unsigned)(((long)r.frame * nscales + r.scale) * hmax + r.y);
}

// bucket and slot of every passing candidate; the passing count
__global__ void __launch_bounds__(256) k_rows_count(const Blob *__restrict__ b, long cap,
                                                    const unsigned long long *__restrict__ count, float thr,
                                                    int nscales, long hmax, long wmax, long nrows,
                                                    unsigned *__restrict__ cnt,
                                                    unsigned *__restrict__ bid, unsigned *__restrict__ slot,
                                                    unsigned *__restrict__ npass) {
  const long n = list_n(count, cap);
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i - threadIdx.x < n;
       i += (long)gridDim.x * blockDim.x) {
    bool pass = false;
    if (i < n) {
      const Blob r = b[i];
      // a record outside the call's geometry (never written by the detectors)
      // takes no bucket: the bucket index addresses the count array
      pass = fabsf(r.response) > thr && r.frame >= 0 && r.scale >= 0 && r.scale < nscales && r.y >= 0 &&
             r.y < hmax && r.x >= 0 && r.x < wmax && ((long)r.frame * nscales + r.scale) * hmax + r.y < nrows;
      unsigned k = ~0u;
      if (pass) {
        k = row_bucket(r, nscales, hmax);
        slot[i] = atomicAdd(cnt + k, 1u);
      }
      bid[i] = k;
    }
    const unsigned m = __ballot_sync(0xffffffffu, pass);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(npass, (unsigned)__popc(m));
  }
}

// block sums of SCAN_CHUNK buckets
__global__ void __launch_bounds__(1024) k_rows_part(const unsigned *__restrict__ cnt, long nb,
                                                    unsigned *__restrict__ part) {
  __shared__ unsigned ws[32];
  const long c0 = (long)blockIdx.x * SCAN_CHUNK;
  unsigned v = 0;
  for (int j = threadIdx.x; j < SCAN_CHUNK; j += 1024)
    if (c0 + j < nb) v += cnt[c0 + j];
  v = __reduce_add_sync(0xffffffffu, v);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    const unsigned t = __reduce_add_sync(0xffffffffu, ws[threadIdx.x]);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
  }
}

// exclusive scan of the block sums (at most 1024 of them), in place
__global__ void __launch_bounds__(1024) k_rows_top(unsigned *__restrict__ part, int np) {
  __shared__ unsigned ws[32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const unsigned v = t < np ? part[t] : 0u;
  unsigned x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    unsigned z = ws[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, z, o);
      if (lane >= o) z += y;
    }
    ws[lane] = z - ws[lane];  // exclusive over warps
  }
  __syncthreads();
  if (t < np) part[t] = ws[w] + x - v;
}

// exclusive scan of the buckets: off[k] = first position of bucket k
__global__ void __launch_bounds__(1024) k_rows_off(const unsigned *__restrict__ cnt, long nb,
                                                   const unsigned *__restrict__ part, unsigned *__restrict__ off) {
  __shared__ unsigned ws[32];
  __shared__ unsigned carry;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const long c0 = (long)blockIdx.x * SCAN_CHUNK;
  if (t == 0) carry = part[blockIdx.x];
  for (int j0 = 0; j0 < SCAN_CHUNK; j0 += 1024) {
    const long k = c0 + j0 + t;
    const unsigned v = k < nb ? cnt[k] : 0u;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
      unsigned z = ws[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, z, o);
        if (lane >= o) z += y;
      }
      ws[lane] = z - ws[lane];
    }
    __syncthreads();
    if (k < nb) off[k] = carry + ws[w] + x - v;
    __syncthreads();
    if (t == 1023) carry += ws[w] + x;
    __syncthreads();
  }
}

// candidate i (passing) to its bucket, with its x
__global__ void __launch_bounds__(256) k_rows_scatter(const Blob *__restrict__ b, long cap,
                                                      const unsigned long long *__restrict__ count,
                                                      const unsigned *__restrict__ bid,
                                                      const unsigned *__restrict__ slot,
                                                      const unsigned *__restrict__ off, unsigned *__restrict__ tmp,
                                                      int *__restrict__ xs) {
  const long n = list_n(count, cap);
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const unsigned k = bid[i];
    if (k == ~0u) continue;
    const unsigned pos = off[k] + slot[i];
    tmp[pos] = (unsigned)i;
    xs[pos] = b[i].x;
  }
}

// each placed candidate's rank by x among its bucket's; the record to the
// ordered list
__global__ void __launch_bounds__(256) k_rows_rank(const Blob *__restrict__ b, const unsigned *__restrict__ tmp,
                                                   const int *__restrict__ xs, const unsigned *__restrict__ bid,
                                                   const unsigned *__restrict__ cnt,
                                                   const unsigned *__restrict__ off,
                                                   const unsigned *__restrict__ npass, Blob *__restrict__ out) {
  const long n = *npass;
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long)gridDim.x * blockDim.x) {
    const unsigned i = tmp[p];
    const unsigned k = bid[i];
    const unsigned lo = off[k], m = cnt[k];
    const int x = xs[p];
    unsigned r = 0;
    for (unsigned q = 0; q < m; ++q) r += xs[lo + q] < x;
    out[lo + r] = b[i];
  }
}

}  // namespace

size_t sort_workspace_bytes(long n, long nrows) {
  const long nb = (n + TILE - 1) / TILE;
  const size_t radix = (size_t)n * 2 * (sizeof(unsigned long long) + sizeof(unsigned)) +
                       ((size_t)MAXD * nb + MAXD) * sizeof(unsigned) + 256;
  if (nrows > ROW_BUCKETS_MAX) return radix;
  const size_t rows = ((size_t)2 * nrows + 1024 + (size_t)4 * n) * sizeof(unsigned) + 256;
  return std::max(radix, rows);
}

// Sort the first min(*count, cap) candidates of `blobs` (count: device) into
// `out` (device) and write the number of records with |response| > thr to
// *d_npass (device); only those records are ordered (the ones at or below
// thr are not used).  nrows = frames x scales x hmax row buckets: up to
// ROW_BUCKETS_MAX the row-bucket ordering runs, beyond it the radix sort:
// `keybits` bounds the real keys, frame, scale, y, x packed as ((frame S +
// scale) hmax + y) wmax + x, split into equal digits of at most MAXBITS bits.
// Work: sort_workspace_bytes(cap, nrows).
int launch_sort(const Blob *blobs, long cap, const unsigned long long *count, float thr, int nscales, long hmax,
                long wmax, int keybits, long nrows, void *work, Blob *out, unsigned *d_npass, Prof *prof,
                cudaStream_t st) {
  if (cap <= 0) return 0;
  if (nrows >= 1 && nrows <= ROW_BUCKETS_MAX) {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return -1;
    char *p = static_cast<char *>(work);
    auto *cnt = reinterpret_cast<unsigned *>(p);
    auto *off = cnt + nrows;
    auto *part = off + nrows;
    auto *bid = part + 1024;
    auto *slot = bid + cap;
    auto *tmp = slot + cap;
    auto *xs = reinterpret_cast<int *>(tmp + cap);
    const int np = (int)((nrows + SCAN_CHUNK - 1) / SCAN_CHUNK);
    const unsigned ng = (unsigned)std::min<long>((cap + 255) / 256, 8L * nsm);
    if (cudaMemsetAsync(d_npass, 0, sizeof(unsigned), st) != cudaSuccess ||
        cudaMemsetAsync(cnt, 0, (size_t)nrows * sizeof(unsigned), st) != cudaSuccess)
      return -1;
    prof->begin("sort_count", st);
    k_rows_count<<<ng, 256, 0, st>>>(blobs, cap, count, thr, nscales, hmax, wmax, nrows, cnt, bid, slot, d_npass);
    prof->end(st);
    prof->begin("sort_scan", st);
    k_rows_part<<<np, 1024, 0, st>>>(cnt, nrows, part);
    k_rows_top<<<1, 1024, 0, st>>>(part, np);
    k_rows_off<<<np, 1024, 0, st>>>(cnt, nrows, part, off);
    prof->end(st);
    prof->begin("sort_scatter", st);
    k_rows_scatter<<<ng, 256, 0, st>>>(blobs, cap, count, bid, slot, off, tmp, xs);
    prof->end(st);
    prof->begin("sort_gather", st);
    k_rows_rank<<<ng, 256, 0, st>>>(blobs, tmp, xs, bid, cnt, off, d_npass, out);
    prof->end(st);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
  }
  const long nb = (cap + TILE - 1) / TILE;
  char *p = static_cast<char *>(work);
  auto *k0 = reinterpret_cast<unsigned long long *>(p);
  auto *k1 = k0 + cap;
  auto *i0 = reinterpret_cast<unsigned *>(k1 + cap);
  auto *i1 = i0 + cap;
  auto *hist = i1 + cap;
  auto *tot = hist + (size_t)MAXD * nb;
  const int npass = std::max(1, (keybits + MAXBITS - 1) / MAXBITS);
  const int bits = (keybits + npass - 1) / npass;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return -1;
  const unsigned ng = (unsigned)std::min<long>((cap + 255) / 256, 4L * nsm);  // element loops
  const unsigned nt = (unsigned)std::min<long>(nb, 2L * nsm);                 // tile loops
  if (cudaMemsetAsync(d_npass, 0, sizeof(unsigned), st) != cudaSuccess) return -1;
  prof->begin("sort_keys", st);
  k_keys<<<ng, 256, 0, st>>>(blobs, cap, count, thr, nscales, hmax, wmax, k0, i0, d_npass);
  prof->end(st);
  for (int ps = 0; ps < npass; ++ps) {
    const int shift = ps * bits, nd = 1 << bits;
    prof->begin("sort_hist", st);
    k_hist<<<nt, SORT_NT, 0, st>>>(k0, cap, count, shift, bits, hist, (int)nb);
    prof->end(st);
    prof->begin("sort_scan", st);
    k_scan_digits<<<(unsigned)((nd + NWARP - 1) / NWARP), SORT_NT, 0, st>>>(hist, (int)nb, nd, cap, count, tot);
    prof->end(st);
    prof->begin("sort_scatter", st);
    k_scatter<<<nt, SORT_NT, 0, st>>>(k0, i0, cap, count, shift, bits, hist, (int)nb, tot, k1, i1);
    prof->end(st);
    std::swap(k0, k1);
    std::swap(i0, i1);
  }
  prof->begin("sort_gather", st);
  k_gather<<<ng, 256, 0, st>>>(blobs, i0, cap, count, out);
  prof->end(st);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace kf
