// kf_sort.cu -- ordering of the detector's candidate list on the GPU: the
// candidates arrive in arbitrary (atomic) order; the blob list is returned in
// (frame, scale, y, x) order.  Least-significant-digit radix sort of 64-bit
// keys with 8-bit digits (stable per pass), then a gather of the records.
// Candidates at or below the re-threshold get the all-ones key and sort last.
#include <cuda_runtime.h>

#include "kf_common.cuh"
#include "kf_internal.h"

namespace kf {

namespace {

constexpr int SORT_NT = 256;               // threads per block
constexpr int SORT_ITEMS = 4;              // items per thread (1024-item tiles: enough blocks for 152 SMs)
constexpr int TILE = SORT_NT * SORT_ITEMS; // items per block
constexpr int NWARP = SORT_NT / 32;
constexpr int ITEMS_PER_WARP = TILE / NWARP;

__global__ void k_keys(const Blob *__restrict__ b, long n, float thr, int nscales, long hmax, long wmax,
                       unsigned long long *__restrict__ key, unsigned *__restrict__ idx,
                       unsigned *__restrict__ npass) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
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

__device__ __forceinline__ int digit(unsigned long long k, int shift) { return (int)((k >> shift) & 0xff); }

// per-block digit histogram: hist[d * nblocks + block]
__global__ void __launch_bounds__(SORT_NT) k_hist(const unsigned long long *__restrict__ key, long n, int shift,
                                                  unsigned *__restrict__ hist) {
  __shared__ unsigned h[256];
  const int tid = threadIdx.x;
  h[tid] = 0;
  __syncthreads();
  const long base = (long)blockIdx.x * TILE;
  for (int j = 0; j < SORT_ITEMS; ++j) {
    const long i = base + (long)j * SORT_NT + tid;
    if (i < n) atomicAdd(&h[digit(key[i], shift)], 1u);
  }
  __syncthreads();
  hist[(long)tid * gridDim.x + blockIdx.x] = h[tid];
}

// Exclusive scan of m entries, one block of 1024 threads, in chunks of
// SCAN_CHUNK entries: a coalesced load into shared memory (padded by one word
// per 32 so that a thread's 32 consecutive entries sit in 32 banks), a serial
// scan of each thread's 32 entries, a block scan of the thread totals with a
// carried prefix, a coalesced write back.
constexpr int SCAN_NT = 1024;
constexpr int SCAN_CHUNK = 32 * SCAN_NT;
constexpr size_t SCAN_SMEM = (size_t)(SCAN_CHUNK + SCAN_CHUNK / 32) * sizeof(unsigned);

__device__ __forceinline__ int scan_pad(int i) { return i + (i >> 5); }

__global__ void __launch_bounds__(SCAN_NT) k_scan(unsigned *__restrict__ a, long m) {
  extern __shared__ unsigned sa[];
  __shared__ unsigned wsum[32];
  __shared__ unsigned carry;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) carry = 0;
  for (long r = 0; r < m; r += SCAN_CHUNK) {
    const int n = (int)min((long)SCAN_CHUNK, m - r);
    for (int i = tid; i < SCAN_CHUNK; i += SCAN_NT) sa[scan_pad(i)] = i < n ? a[r + i] : 0u;
    __syncthreads();
    unsigned tot = 0;  // this thread's 32 entries, scanned in place
#pragma unroll 8
    for (int j = 0; j < 32; ++j) {
      const int q = scan_pad(32 * tid + j);
      const unsigned v = sa[q];
      sa[q] = tot;
      tot += v;
    }
    unsigned x = tot;  // inclusive scan of the thread totals
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= d) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
      unsigned t = wsum[lane];
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, t, d);
        if (lane >= d) t += y;
      }
      wsum[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    const unsigned before = carry + (w > 0 ? wsum[w - 1] : 0u) + x - tot;
#pragma unroll 8
    for (int j = 0; j < 32; ++j) sa[scan_pad(32 * tid + j)] += before;
    __syncthreads();
    for (int i = tid; i < n; i += SCAN_NT) a[r + i] = sa[scan_pad(i)];
    if (tid == 0) carry += wsum[31];
    __syncthreads();
  }
}

// stable scatter: items keep their order inside a digit
__global__ void __launch_bounds__(SORT_NT) k_scatter(const unsigned long long *__restrict__ kin,
                                                     const unsigned *__restrict__ iin, long n, int shift,
                                                     const unsigned *__restrict__ off,
                                                     unsigned long long *__restrict__ kout,
                                                     unsigned *__restrict__ iout) {
  __shared__ unsigned cnt[NWARP][256];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  for (int d = lane; d < 256; d += 32) cnt[w][d] = 0;
  __syncwarp();
  const long wbase = (long)blockIdx.x * TILE + (long)w * ITEMS_PER_WARP;
  const unsigned lt = (1u << lane) - 1u;
  // pass 1: per-warp digit counts
  for (int r = 0; r < ITEMS_PER_WARP / 32; ++r) {
    const long i = wbase + r * 32 + lane;
    const bool valid = i < n;
    const int d = valid ? digit(kin[i], shift) : 256 + lane;  // invalid lanes never match
    const unsigned m = __match_any_sync(0xffffffffu, d);
    if (valid && (m & lt) == 0) cnt[w][d] += __popc(m);
    __syncwarp();
  }
  __syncthreads();
  // exclusive prefix over warps, plus the block's global offset for the digit
  for (int d = tid; d < 256; d += SORT_NT) {
    unsigned run = off[(long)d * gridDim.x + blockIdx.x];
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
    const int d = valid ? digit(k, shift) : 256 + lane;
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
}

__global__ void k_gather(const Blob *__restrict__ b, const unsigned *__restrict__ idx, long n,
                         Blob *__restrict__ out) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = b[idx[i]];
}

}  // namespace

size_t sort_workspace_bytes(long n) {
  const long nb = (n + TILE - 1) / TILE;
  return (size_t)n * 2 * (sizeof(unsigned long long) + sizeof(unsigned)) + (size_t)256 * nb * sizeof(unsigned) +
         256;
}

// Sort the n candidates of `blobs` into `out` (device) and write the number of
// records with |response| > thr to *d_npass (device).  `keybits` bounds the
// real keys: frame, scale, y, x packed as ((frame S + scale) hmax + y) wmax + x.
int launch_sort(const Blob *blobs, long n, float thr, int nscales, long hmax, long wmax, int keybits,
                void *work, Blob *out, unsigned *d_npass, Prof *prof, cudaStream_t st) {
  if (n <= 0) return 0;
  const long nb = (n + TILE - 1) / TILE;
  char *p = static_cast<char *>(work);
  auto *k0 = reinterpret_cast<unsigned long long *>(p);
  auto *k1 = k0 + n;
  auto *i0 = reinterpret_cast<unsigned *>(k1 + n);
  auto *i1 = i0 + n;
  auto *hist = i1 + n;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_scan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SCAN_SMEM);
    attr = true;
  }
  cudaMemsetAsync(d_npass, 0, sizeof(unsigned), st);
  prof->begin("sort_keys", st);
  k_keys<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(blobs, n, thr, nscales, hmax, wmax, k0, i0, d_npass);
  prof->end(st);
  for (int shift = 0; shift < keybits; shift += 8) {
    prof->begin("sort_pass", st);
    k_hist<<<(unsigned)nb, SORT_NT, 0, st>>>(k0, n, shift, hist);
    k_scan<<<1, SCAN_NT, SCAN_SMEM, st>>>(hist, 256 * nb);
    k_scatter<<<(unsigned)nb, SORT_NT, 0, st>>>(k0, i0, n, shift, hist, k1, i1);
    prof->end(st);
    std::swap(k0, k1);
    std::swap(i0, i1);
  }
  prof->begin("sort_gather", st);
  k_gather<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(blobs, i0, n, out);
  prof->end(st);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace kf
