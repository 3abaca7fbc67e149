// kf_batch.cuh -- frame table and work-item lists of a bank call.
//
// Every frame of a call keeps its one-sided planes resident in one "plane row
// space" of pitch PWb (the widest frame's pitch): scale s, row y of frame f is
// plane row F.prow + s F.H + y.  One 2-D tensor map covers the whole space, so
// the TMA kernels serve all frames with one map; a box that reaches past a
// frame's first or last row reads a neighbouring plane (or the fill value),
// and those rows are replaced by the held boundary values anyway.
//
// A launch covers a list of frames; its work items (rows, column tiles, ...)
// are numbered frame after frame.  Kernels run persistently: block b takes
// items b, b + gridDim.x, ... and finds the frame of an item by advancing a
// monotone index over the exclusive prefix sums of the items per frame.
#pragma once
#include "kf_common.cuh"

namespace kf {

struct FrameDev {
  const void *X;   // input frame (IN_* elements)
  float *resp;     // responses of this frame (S x H x W), or nullptr
  long xpitch;     // input elements between rows
  long prow;       // plane row of (scale 0, frame row 0)
  long eoff;       // floats: edge rows [S][2][PWb]
  long coff;       // floats: IIR column carries [S][nseg][2][NF][PWb]
  int dtype;       // IN_F32 / IN_F16 / IN_BF16 / IN_U16
  float vscale;    // input multiplier
  long aoff;       // gated calls: byte offset of the frame's active-tile map (64 x 64 tiles)
  long roff;       // float offset of the frame's planes in response-layout buffers (S x H x W)
  // response layout when rplane > 0: value (s, y, x) at resp[s * rplane +
  // (y - rmy) * rpitch + x - rmx], only for y at least rmy and x at least rmx
  // inside the frame (the D = 5 bank writes its padded channel frames cropped
  // into the caller's array); rplane = 0: S x H x W planes.  Honoured by
  // detect_tile (the IIR column pass and the FP32 FIR column pass, the
  // passes of the D = 5 bank), not by the tensor-core FIR column pass.
  long rplane;
  int rpitch, rmx, rmy;
  // CH_ID rows with two-sample pre-rolls (the D = 5 bank): per frame row,
  // the values at x = -2 (held beyond), -1, W and W + 1 (held beyond); null:
  // the row is held at its ends
  const float4 *xpre;
  int H, W;
  int nseg;        // IIR column segments
  int index;       // frame index in the call (blob records)
};

struct Items {
  const int *fl;   // frames of this launch: indices into the frame table
  const int *pre;  // exclusive prefix sums of the items per frame (n + 1 entries)
  int n;           // frames in the launch
  int total;       // items in the launch (pre[n]); with sel: the capacity of the list
  const int2 *sel = nullptr;    // gated launches: selected (position in fl, item of that frame) pairs
  const int *dcount = nullptr;  // gated launches: number of selected pairs (device)
};

// position in it.fl of the frame that holds `item`, starting the search at k
// (the items a block takes only increase, so k only advances)
__device__ __forceinline__ int advance_frame(const Items &it, int item, int k) {
  while (item >= __ldg(it.pre + k + 1)) ++k;
  return k;
}

// items of the launch (a gated launch reads its count from the device)
__device__ __forceinline__ int items_total(const Items &it) { return it.dcount ? __ldg(it.dcount) : it.total; }

// position in it.fl and item of that frame for launch item `item` (k: the
// previous position, for the monotone search of ungated launches)
__device__ __forceinline__ int item_frame(const Items &it, int item, int k, int &local) {
  if (it.sel) {
    const int2 e = __ldg(it.sel + item);
    local = e.y;
    return e.x;
  }
  k = advance_frame(it, item, k);
  local = item - __ldg(it.pre + k);
  return k;
}

// Gated calls: any active 64 x 64 tile in the pixel rectangle [x0, x1) x
// [y0, y1) of frame F (act: the call's active-tile maps)
__device__ __forceinline__ bool any_active(const FrameDev &F, const unsigned char *act, int x0, int x1, int y0,
                                           int y1) {
  const int tw = (F.W + 63) / 64, th = (F.H + 63) / 64;
  x0 = max(x0, 0), y0 = max(y0, 0), x1 = min(x1, F.W), y1 = min(y1, F.H);
  if (x0 >= x1 || y0 >= y1) return false;
  const unsigned char *a = act + F.aoff;
  for (int ty = y0 / 64; ty <= (y1 - 1) / 64 && ty < th; ++ty)
    for (int tx = x0 / 64; tx <= (x1 - 1) / 64 && tx < tw; ++tx)
      if (a[ty * tw + tx]) return true;
  return false;
}

// Heavy kernels (near their register limit) keep the current item's frame
// record in shared memory: the compiler may otherwise re-load its fields from
// global memory at every use.  Thread 0 copies it; the caller synchronises
// before and after (the previous item's readers must be done).
__device__ __forceinline__ void stage_frame(FrameDev *dst, const FrameDev *__restrict__ fr, const Items &it,
                                            int k) {
  if (threadIdx.x == 0) *dst = fr[__ldg(it.fl + k)];
}

}  // namespace kf
