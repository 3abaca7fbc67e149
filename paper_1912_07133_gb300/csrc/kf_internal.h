// kf_internal.h -- host-side declarations shared by the library's translation
// units (launchers of the CUDA kernels).  Not part of the C ABI.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include "kf_common.cuh"

namespace kf {

// FP64 design of S scales into d_out (device array of S Coef).  d_work holds
// S * 2 (Nmax^2 + Nmax) doubles (double-double KKT matrix and right-hand side
// of the colored-SG design).
int launch_design(int type, int order, const double *d_lambdas, int S, int fir_kmax, Coef *d_out,
                  double *d_work, int Nmax, cudaStream_t st);

// Geometry of one frame in the bank.
struct FrameGeom {
  const void *X;    // input frame (IN_* element type)
  int dtype;        // IN_F32 / IN_F16 / IN_BF16 / IN_U16
  float vscale;     // input multiplier
  long xpitch;      // elements between input rows
  int H, W;
  long PW;          // pitch of the intermediate planes (elements)
  int frame;        // frame index (for blob records)
  long resp_off;    // offset of this frame in the responses output
};

// Optional per-launch event recording (profiling) and launch counting.
struct Prof {
  cudaEvent_t *ev;        // 2 events per launch, or nullptr
  int cap;                // launches that fit in ev
  int n;                  // launches so far in this call
  const char *names[256]; // kernel name of each launch
  void begin(const char *name, cudaStream_t st) {
    if (n < 256) names[n] = name;
    if (ev && n < cap) cudaEventRecord(ev[2 * n], st);
  }
  void end(cudaStream_t st) {
    if (ev && n < cap) cudaEventRecord(ev[2 * n + 1], st);
    ++n;
  }
};

struct BankArgs {
  const Coef *coef;      // device, S entries
  int S;
  int type, nstate;      // filter type; D: chain length, E: number of modes
  int kmax;              // FIR: largest half-length over the scales
  float threshold;
  int neigh;
  void *P;               // S planes of H x PW, element type `storage`
  int storage;           // ST_F32 / ST_F16 / ST_BF16
  float *edge;           // S x 2 x PW: one-sided rows for the column boundary
  float *carry;          // S x nseg x 2 x NF x PW (IIR column carries)
  Blob *blobs;
  long cap;
  DevStatus *status;
  float *responses;      // optional
  Prof *prof;            // launch bookkeeping (never null)
};

int launch_iir_frame(const FrameGeom &g, const BankArgs &a, cudaStream_t st);
int launch_fir_frame(const FrameGeom &g, const BankArgs &a, cudaStream_t st);

// 3-D tensor map over S one-sided planes (x, y, scale) of pitch PW and
// element type `storage`, box boxw x boxh x 1 (kf_fir.cu)
int encode_plane_map(CUtensorMap *m, void *P, int storage, long PW, int H, int S, int boxw, int boxh);

// workspace needs (bytes) of one frame
size_t iir_carry_floats(int H, long PW, int S, int nf);

// candidate ordering (kf_sort.cu)
size_t sort_workspace_bytes(long n);
int launch_sort(const Blob *blobs, long n, float thr, int nscales, long hmax, long wmax, int keybits,
                void *work, Blob *out, unsigned *d_npass, Prof *prof, cudaStream_t st);

}  // namespace kf
