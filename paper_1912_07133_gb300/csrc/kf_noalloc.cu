// kf_noalloc.cu -- response planes of the recursive banks without any device
// allocation (kf_responses_noalloc in include/kf.h).
//
// Who needs this: programs whose device memory belongs to a host framework's
// pool allocator, or real-time loops that forbid cudaMalloc after start-up
// because it can synchronise the device and can fail under memory pressure.
// They pass the frame and the output buffer; every intermediate (designs,
// one-sided planes, edge rows, column carries, status word) lives in the one
// file-scope device array below, which each GPU that loads the library keeps
// until the process exits.  The paper has no counterpart to this entry point.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>

#include "kf.h"
#include "kf_common.cuh"
#include "kf_internal.h"

namespace {

constexpr size_t kScratchBytes = (size_t)KF_NOALLOC_SCRATCH_MB << 20;

// The shared scratch.  Host code must not use this name as a pointer: it is a
// host-side stand-in for the device symbol; cudaGetSymbolAddress gives the
// device address.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

thread_local char g_msg[256];
// failure-detection test hook (kf_set_wait_limit(NULL, polls)); 0: normal waits
unsigned g_wait_test = 0;

}  // namespace

namespace kf {
void set_global_error(const char *msg);
void set_noalloc_wait_test(unsigned polls) { g_wait_test = polls; }
}

namespace {

int nofail(int code, const char *msg) {
  std::snprintf(g_msg, sizeof g_msg, "kf_responses_noalloc: %s", msg);
  kf::set_global_error(g_msg);
  return code;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" int kf_responses_noalloc(const kf_frame *frame, const double *scales, int nscales, int type,
                                    int order, float *responses, void *cuda_stream) {
  g_msg[0] = 0;
  if (!frame || !scales || !responses) return nofail(KF_EINVAL, "NULL argument");
  if (type != KF_IIR_REPEATED_POLE && type != KF_IIR_BUTTERWORTH)
    return nofail(KF_EINVAL, "only the recursive banks (repeated pole, Butterworth) are supported");
  if (type == KF_IIR_REPEATED_POLE && (order < 2 || order > 6))
    return nofail(KF_EINVAL, "repeated-pole order must be 2..6");
  if (type == KF_IIR_BUTTERWORTH && (order < 1 || order > 6))
    return nofail(KF_EINVAL, "Butterworth order must be 1..6");
  if (nscales < 1 || nscales > KF_MAX_SCALES) return nofail(KF_EINVAL, "nscales must be 1..16");
  for (int s = 0; s < nscales; ++s)
    if (!(scales[s] > 0.0) || !std::isfinite(scales[s])) return nofail(KF_EINVAL, "scales must be > 0");
  if (!frame->data || frame->width < 1 || frame->height < 1 || frame->width > 8192 ||
      frame->pitch < frame->width || !std::isfinite(frame->value_scale))
    return nofail(KF_EINVAL, "frame needs data, 1 <= width <= 8192, pitch >= width, a finite value_scale");
  if (frame->dtype != KF_DTYPE_F32 && frame->dtype != KF_DTYPE_F16 && frame->dtype != KF_DTYPE_BF16 &&
      frame->dtype != KF_DTYPE_U16)
    return nofail(KF_EINVAL, "unknown frame dtype");
  if ((reinterpret_cast<uintptr_t>(frame->data) & (uintptr_t)(kf::in_bytes(frame->dtype) - 1)) != 0)
    return nofail(KF_EINVAL, "frame data is not aligned to its element size");
  const int W = frame->width, H = frame->height, S = nscales;
  const long PW = ((long)W + 31) / 32 * 32;
  // layout of the scratch: coefficients | scales | status | frame table | planes | edges | carries
  const int nstate_max = 6;  // chain length (repeated pole) or 2 x modes (Butterworth)
  const int nseg = kf::iir_segments(H, 64);
  // frame table: one frame, each of the four passes one launch over it
  struct Table {
    kf::FrameDev fd;
    int pool[4][3];  // per pass: frame list {0}, item prefix {0, items}
  } tab;
  const size_t b_coef = align256(sizeof(kf::Coef) * KF_MAX_SCALES);
  const size_t b_lam = align256(sizeof(double) * KF_MAX_SCALES);
  const size_t b_stat = align256(sizeof(kf::DevStatus));
  const size_t b_tab = align256(sizeof(Table));
  const size_t b_P = align256(sizeof(float) * (size_t)S * H * PW);
  const size_t b_edge = align256(sizeof(float) * (size_t)S * 2 * PW);
  const size_t b_carry = align256(sizeof(float) * (size_t)S * nseg * 2 * nstate_max * PW);
  const size_t need = b_coef + b_lam + b_stat + b_tab + b_P + b_edge + b_carry;
  if (need > kScratchBytes) {
    char m[200];
    std::snprintf(m, sizeof m, "%d scales of %dx%d need %zu bytes of scratch; the limit is %zu", S, W, H,
                  need, kScratchBytes);
    return nofail(KF_EINVAL, m);
  }
  if (kf::iir_row_threads(W) == 0) return nofail(KF_EINVAL, "frame too wide for the row pass");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return nofail(KF_ENODEV, "no usable CUDA device");
  // the device address of the scratch on the current device, looked up on
  // every call (after a device reset the module, and with it the array, is
  // loaded anew at another address; the lookup allocates nothing)
  void *addr = nullptr;
  {
    const cudaError_t e = cudaGetSymbolAddress(&addr, g_scratch);
    if (e != cudaSuccess || !addr) return nofail(KF_ECUDA, cudaGetErrorString(e));
  }
  unsigned char *base = static_cast<unsigned char *>(addr);
  auto *coef = reinterpret_cast<kf::Coef *>(base);
  auto *lam = reinterpret_cast<double *>(base + b_coef);
  auto *status = reinterpret_cast<kf::DevStatus *>(base + b_coef + b_lam);
  auto *d_tab = reinterpret_cast<Table *>(base + b_coef + b_lam + b_stat);
  auto *P = reinterpret_cast<float *>(base + b_coef + b_lam + b_stat + b_tab);
  auto *edge = reinterpret_cast<float *>(base + b_coef + b_lam + b_stat + b_tab + b_P);
  auto *carry = reinterpret_cast<float *>(base + b_coef + b_lam + b_stat + b_tab + b_P + b_edge);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e;
  // FP64 designs into the scratch; the host checks them (stack copy, no allocation)
  if ((e = cudaMemcpyAsync(lam, scales, sizeof(double) * S, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return nofail(KF_ECUDA, cudaGetErrorString(e));
  if (kf::launch_design(type, order, lam, S, 96, coef, nullptr, 1, st))
    return nofail(KF_ECUDA, "design kernel launch failed");
  // the frame table (copied before the synchronisation below, so the stack
  // copy may go away afterwards)
  std::memset(&tab, 0, sizeof tab);
  tab.fd.X = frame->data;
  tab.fd.resp = responses;
  tab.fd.xpitch = frame->pitch;
  tab.fd.prow = 0;
  tab.fd.eoff = 0;
  tab.fd.coff = 0;
  tab.fd.dtype = frame->dtype;
  tab.fd.vscale = frame->value_scale == 0.0f ? 1.0f : frame->value_scale;
  tab.fd.H = H;
  tab.fd.W = W;
  tab.fd.nseg = nseg;
  tab.fd.index = 0;
  for (int p = 0; p < 4; ++p) {
    tab.pool[p][0] = 0;
    tab.pool[p][1] = 0;
    tab.pool[p][2] = kf::iir_items(p, H, W, S, 64);
  }
  if ((e = cudaMemcpyAsync(d_tab, &tab, sizeof tab, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return nofail(KF_ECUDA, cudaGetErrorString(e));
  struct Check {
    int status, K;
    double dc;
  } chk[KF_MAX_SCALES];
  for (int s = 0; s < S; ++s) {
    if ((e = cudaMemcpyAsync(&chk[s].status, &coef[s].status, sizeof(int), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(&chk[s].K, &coef[s].K, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&chk[s].dc, &coef[s].dc_gain, sizeof(double), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess)
      return nofail(KF_ECUDA, cudaGetErrorString(e));
  }
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return nofail(KF_ECUDA, cudaGetErrorString(e));
  int nstate = 0;
  for (int s = 0; s < S; ++s) {
    if (chk[s].status == 1) return nofail(KF_EINVAL, "invalid design parameters");
    if (chk[s].status != 0 || !(std::fabs(chk[s].dc - 1.0) < 1e-6)) return nofail(KF_ECOND, "design failed");
    nstate = chk[s].K > nstate ? chk[s].K : nstate;
  }
  // the status word must start at zero; everything else is written before it is read
  if ((e = cudaMemsetAsync(status, 0, sizeof(kf::DevStatus), st)) != cudaSuccess)
    return nofail(KF_ECUDA, cudaGetErrorString(e));
  kf::Prof prof{};
  kf::BankArgs a;
  a.coef = coef;
  a.S = S;
  a.type = type;
  a.nstate = nstate;
  a.kmax = 0;
  a.threshold = INFINITY;  // responses only: no candidates
  a.neigh = KF_NEIGH_ALL_SCALES;
  a.P = P;
  a.storage = kf::ST_F32;
  a.edge = edge;
  a.carry = carry;
  a.blobs = nullptr;
  a.cap = 0;
  a.status = status;
  a.prof = &prof;
  a.wait_test = g_wait_test;
  kf::Plan plan;
  plan.fr = &d_tab->fd;
  plan.nframes = 1;
  plan.PWb = PW;
  plan.prows = (long)S * H;
  plan.per_frame = false;
  plan.lc = 64;
  for (int p = 0; p < 4; ++p) {
    kf::Launch l;
    l.it.fl = &d_tab->pool[p][0];
    l.it.pre = &d_tab->pool[p][1];
    l.it.n = 1;
    l.it.total = tab.pool[p][2];
    l.nt = p == kf::PASS_ROW ? kf::iir_row_threads(W) : 0;
    plan.pass[p].push_back(l);
  }
  const int rc = kf::launch_iir(plan, a, st);
  if (rc == -2) return nofail(KF_EINVAL, "no kernel instance for this order");
  if (rc) return nofail(KF_ECUDA, cudaGetErrorString(cudaGetLastError()));
  // the device status: a bounded wait of the column pass that gave up leaves
  // its tile's responses unwritten, which the caller must learn of
  kf::DevStatus hs{};
  if ((e = cudaMemcpyAsync(&hs, status, sizeof hs, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return nofail(KF_ECUDA, cudaGetErrorString(e));
  if (hs.error) {
    char m[96];
    std::snprintf(m, sizeof m, "a device wait gave up (code %d); the responses are incomplete", hs.error);
    return nofail(KF_ETIMEOUT, m);
  }
  return KF_OK;
}
