// kf_api.cu -- host implementation of the C ABI declared in include/kf.h:
// argument checks, workspace, design cache, kernel launches, candidate
// read-back.  Every arithmetic step of the filter bank runs in the kernels of
// kf_design.cu, kf_iir.cu and kf_fir.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "kf.h"
#include "kf_common.cuh"
#include "kf_internal.h"

struct kf_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  // workspace (grown on demand)
  float *P = nullptr;
  size_t P_floats = 0;
  float *edge = nullptr;
  size_t edge_floats = 0;
  float *carry = nullptr;
  size_t carry_floats = 0;
  double *lambdas = nullptr;
  double *dwork = nullptr;
  int dwork_nmax = 0;
  kf::DevStatus *status = nullptr;
  kf::Blob *blobs = nullptr;
  long blob_cap = 0;
  // design cache: (type, order, kmax, scales) -> coefficients, LRU
  struct Design {
    int type = -1, order = -1, kmax = -1, S = 0;
    double lam[KF_MAX_SCALES];
    kf::Coef *d_coef = nullptr;
    std::vector<kf::Coef> h_coef;
    unsigned long long used = 0;
  };
  std::vector<Design> designs;
  unsigned long long tick = 0;
  Design *cur = nullptr;
  // candidate ordering
  kf::Blob *sorted = nullptr;
  void *sort_work = nullptr;
  size_t sort_work_bytes = 0;
  unsigned *d_npass = nullptr;
  bool sorted_valid = false;
  double sorted_thr = 0.0;
  long sorted_n = 0;
  int last_nframes = 0;
  long last_hmax = 0, last_wmax = 0;
  // launch bookkeeping of the last bank call
  kf::Prof prof{};
  std::vector<cudaEvent_t> events;
  bool have_prof = false;
  // last bank call
  bool have_result = false;
  double last_threshold = 0.0;
  int last_S = 0;
};

namespace {

thread_local std::string g_err;

int fail(kf_ctx *ctx, int code, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
int fail(kf_ctx *ctx, int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf;
  else g_err = buf;
  return code;
}

int cuda_fail(kf_ctx *ctx, cudaError_t e, const char *what) {
  return fail(ctx, e == cudaErrorMemoryAllocation ? KF_ENOMEM : KF_ECUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

template <class T>
int grow(kf_ctx *ctx, T **p, size_t *have, size_t need, const char *what) {
  if (*have >= need && *p) return KF_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  cudaError_t e = cudaMalloc((void **)p, need * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_fail(ctx, e, what);
  }
  *have = need;
  return KF_OK;
}

int nmax_for(int type, int order, int kmax) {
  if (type != KF_FIR_COLORED_SG) return 1;
  return kmax + 1 + order + 1;
}

// Run the FP64 design kernel for (type, order, scales) unless the context
// already holds exactly this design (small LRU cache); ctx->cur points at it.
constexpr size_t kDesignSlots = 8;

int ensure_design(kf_ctx *ctx, int type, int order, const double *scales, int S, int kmax) {
  for (auto &d : ctx->designs)
    if (d.type == type && d.order == order && d.kmax == kmax && d.S == S &&
        std::equal(scales, scales + S, d.lam)) {
      d.used = ++ctx->tick;
      ctx->cur = &d;
      return KF_OK;
    }
  ctx->cur = nullptr;
  cudaError_t e;
  if (!ctx->lambdas) {
    if ((e = cudaMalloc(&ctx->lambdas, sizeof(double) * KF_MAX_SCALES)) != cudaSuccess)
      return cuda_fail(ctx, e, "cudaMalloc(lambdas)");
  }
  kf_ctx::Design *slot = nullptr;
  if (ctx->designs.size() < kDesignSlots) {
    ctx->designs.reserve(kDesignSlots);
    ctx->designs.emplace_back();
    slot = &ctx->designs.back();
  } else {
    slot = &*std::min_element(ctx->designs.begin(), ctx->designs.end(),
                              [](const kf_ctx::Design &a, const kf_ctx::Design &b) { return a.used < b.used; });
  }
  slot->type = -1;  // invalid until the design succeeds
  if (!slot->d_coef) {
    if ((e = cudaMalloc(&slot->d_coef, sizeof(kf::Coef) * KF_MAX_SCALES)) != cudaSuccess)
      return cuda_fail(ctx, e, "cudaMalloc(coef)");
  }
  const int nmax = nmax_for(type, order, kmax);
  if (nmax > ctx->dwork_nmax) {
    if (ctx->dwork) cudaFree(ctx->dwork);
    ctx->dwork = nullptr;
    // double-double KKT matrix and right-hand side per scale
    size_t n = (size_t)KF_MAX_SCALES * 2 * ((size_t)nmax * nmax + nmax);
    if ((e = cudaMalloc(&ctx->dwork, n * sizeof(double))) != cudaSuccess)
      return cuda_fail(ctx, e, "cudaMalloc(design work)");
    ctx->dwork_nmax = nmax;
  }
  if ((e = cudaMemcpyAsync(ctx->lambdas, scales, sizeof(double) * S, cudaMemcpyHostToDevice,
                           ctx->stream)) != cudaSuccess)
    return cuda_fail(ctx, e, "copy scales");
  if (kf::launch_design(type, order, ctx->lambdas, S, kmax, slot->d_coef, ctx->dwork, ctx->dwork_nmax,
                        ctx->stream))
    return cuda_fail(ctx, cudaGetLastError(), "design kernel launch");
  slot->h_coef.resize(S);
  if ((e = cudaMemcpyAsync(slot->h_coef.data(), slot->d_coef, sizeof(kf::Coef) * S,
                           cudaMemcpyDeviceToHost, ctx->stream)) != cudaSuccess)
    return cuda_fail(ctx, e, "copy design");
  if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return cuda_fail(ctx, e, "design");
  for (int s = 0; s < S; ++s) {
    const kf::Coef &c = slot->h_coef[s];
    if (c.status == 1)
      return fail(ctx, KF_EINVAL, "design: invalid parameters for scale %g (type %d, order %d)",
                  scales[s], type, order);
    if (c.status != 0)
      return fail(ctx, KF_ECOND, "design failed for scale %g (code %d)", scales[s], c.status);
    if (!(std::fabs(c.dc_gain - 1.0) < 1e-6))
      return fail(ctx, KF_ECOND, "design for scale %g has dc gain %.9g", scales[s], c.dc_gain);
  }
  slot->type = type;
  slot->order = order;
  slot->kmax = kmax;
  slot->S = S;
  std::copy(scales, scales + S, slot->lam);
  slot->used = ++ctx->tick;
  ctx->cur = slot;
  return KF_OK;
}

int check_type_order(kf_ctx *ctx, int type, int order) {
  if (type == KF_IIR_REPEATED_POLE && (order < 2 || order > 6))
    return fail(ctx, KF_EINVAL, "repeated-pole order must be 2..6 (got %d)", order);
  if (type == KF_IIR_BUTTERWORTH && (order < 1 || order > 6))
    return fail(ctx, KF_EINVAL, "Butterworth order (L_B/2) must be 1..6 (got %d)", order);
  if (type == KF_FIR_COLORED_SG && order != 1 && order != 2)
    return fail(ctx, KF_EINVAL, "colored SG order (L_D) must be 1 or 2 (got %d)", order);
  if (type < 0 || type > 2) return fail(ctx, KF_EINVAL, "unknown filter type %d", type);
  return KF_OK;
}

}  // namespace

namespace kf {
// message of a context-less failure, as read by kf_last_error(NULL)
void set_global_error(const char *msg) { g_err = msg; }
}  // namespace kf

extern "C" {

int kf_bank_opts_default(kf_bank_opts *o) {
  if (!o) return KF_EINVAL;
  std::memset(o, 0, sizeof *o);
  o->response = KF_RESP_LAPLACIAN;
  o->boundary = KF_BOUNDARY_HOLD;
  o->neighbourhood = KF_NEIGH_ALL_SCALES;
  o->storage = KF_DTYPE_F32;
  o->threshold = 0.05;
  o->fir_kmax = 96;
  o->responses = nullptr;
  return KF_OK;
}

int kf_create(kf_ctx **out, int device, void *stream) {
  if (!out) return fail(nullptr, KF_EINVAL, "kf_create: ctx is NULL");
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) return fail(nullptr, KF_ENODEV, "no CUDA device");
  if (device < 0 || device >= n) return fail(nullptr, KF_EINVAL, "device %d out of range", device);
  if ((e = cudaSetDevice(device)) != cudaSuccess) return cuda_fail(nullptr, e, "cudaSetDevice");
  kf_ctx *ctx = new kf_ctx();
  ctx->device = device;
  ctx->stream = (cudaStream_t)stream;
  if ((e = cudaMalloc(&ctx->status, sizeof(kf::DevStatus))) != cudaSuccess) {
    delete ctx;
    return cuda_fail(nullptr, e, "cudaMalloc(status)");
  }
  ctx->blob_cap = 1 << 20;
  if ((e = cudaMalloc(&ctx->blobs, sizeof(kf::Blob) * ctx->blob_cap)) != cudaSuccess) {
    cudaFree(ctx->status);
    delete ctx;
    return cuda_fail(nullptr, e, "cudaMalloc(blobs)");
  }
  *out = ctx;
  return KF_OK;
}

void kf_destroy(kf_ctx *ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  cudaFree(ctx->P);
  cudaFree(ctx->edge);
  cudaFree(ctx->carry);
  for (auto &d : ctx->designs) cudaFree(d.d_coef);
  cudaFree(ctx->sorted);
  cudaFree(ctx->sort_work);
  cudaFree(ctx->d_npass);
  cudaFree(ctx->lambdas);
  cudaFree(ctx->dwork);
  cudaFree(ctx->status);
  cudaFree(ctx->blobs);
  for (cudaEvent_t e : ctx->events) cudaEventDestroy(e);
  delete ctx;
}

const char *kf_last_error(const kf_ctx *ctx) { return ctx ? ctx->err.c_str() : g_err.c_str(); }

int kf_design(int type, int order, double scale, kf_coeffs *out) {
  if (!out) return fail(nullptr, KF_EINVAL, "kf_design: out is NULL");
  if (!(scale > 0.0) || !std::isfinite(scale))
    return fail(nullptr, KF_EINVAL, "kf_design: scale must be > 0");
  kf_ctx tmp;
  int rc = check_type_order(&tmp, type, order);
  if (rc) return fail(nullptr, rc, "%s", tmp.err.c_str());
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) return fail(nullptr, KF_ENODEV, "no CUDA device");
  cudaGetDevice(&tmp.device);
  rc = ensure_design(&tmp, type, order, &scale, 1, 96);
  kf::Coef c{};
  if (!rc) c = tmp.cur->h_coef[0];
  for (auto &d : tmp.designs) cudaFree(d.d_coef);
  cudaFree(tmp.lambdas);
  cudaFree(tmp.dwork);
  if (rc) return fail(nullptr, rc, "%s", tmp.err.c_str());
  std::memset(out, 0, sizeof *out);
  out->type = type;
  out->order = order;
  out->scale = scale;
  out->sigma = c.sigma;
  out->param = c.param;
  out->b0 = c.db0;
  out->dc_gain = c.dc_gain;
  out->moment2 = c.moment2;
  if (type == KF_FIR_COLORED_SG) {
    out->K = c.K;
    for (int k = 0; k <= c.K; ++k) out->h[k] = c.dh[k];
  } else {
    const int K = (type == KF_IIR_REPEATED_POLE) ? order : order;
    out->K = K;
    for (int m = 0; m <= K; ++m) {
      out->bplus[m] = c.dbplus[m];
      out->aplus[m] = c.daplus[m];
    }
  }
  return KF_OK;
}

int kf_filter_bank(kf_ctx *ctx, const kf_frame *frames, int nframes, const double *scales, int nscales,
                   int type, int order, const kf_bank_opts *opts_in) {
  if (!ctx) return fail(nullptr, KF_EINVAL, "kf_filter_bank: ctx is NULL");
  ctx->have_result = false;
  kf_bank_opts opts;
  if (opts_in) opts = *opts_in;
  else kf_bank_opts_default(&opts);
  if (!frames || nframes < 1) return fail(ctx, KF_EINVAL, "need at least one frame");
  if (!scales || nscales < 1 || nscales > KF_MAX_SCALES)
    return fail(ctx, KF_EINVAL, "nscales must be 1..%d", KF_MAX_SCALES);
  for (int s = 0; s < nscales; ++s)
    if (!(scales[s] > 0.0) || !std::isfinite(scales[s]))
      return fail(ctx, KF_EINVAL, "scale %d must be > 0", s);
  int rc = check_type_order(ctx, type, order);
  if (rc) return rc;
  if (opts.response != KF_RESP_LAPLACIAN)
    return fail(ctx, KF_EINVAL, "only the Laplacian response is implemented");
  if (opts.boundary != KF_BOUNDARY_HOLD) return fail(ctx, KF_EINVAL, "only the hold boundary is implemented");
  if (opts.neighbourhood != KF_NEIGH_ALL_SCALES && opts.neighbourhood != KF_NEIGH_ADJACENT)
    return fail(ctx, KF_EINVAL, "unknown neighbourhood %d", opts.neighbourhood);
  if (opts.storage != KF_DTYPE_F32 && opts.storage != KF_DTYPE_F16 && opts.storage != KF_DTYPE_BF16)
    return fail(ctx, KF_EINVAL, "storage must be f32, f16 or bf16");
  if (!(opts.threshold >= 0.0)) return fail(ctx, KF_EINVAL, "threshold must be >= 0");
  const int kmax_opt = opts.fir_kmax > 0 ? opts.fir_kmax : 96;
  if (kmax_opt > KF_MAX_FIR_K) return fail(ctx, KF_EINVAL, "fir_kmax must be <= %d", KF_MAX_FIR_K);
  long maxH = 0, maxPW = 0;
  size_t maxplane = 0;
  for (int f = 0; f < nframes; ++f) {
    const kf_frame &fr = frames[f];
    if (!fr.data) return fail(ctx, KF_EINVAL, "frame %d: data is NULL", f);
    if (fr.width < 1 || fr.height < 1 || fr.pitch < fr.width)
      return fail(ctx, KF_EINVAL, "frame %d: bad geometry %dx%d pitch %lld", f, fr.width, fr.height,
                  (long long)fr.pitch);
    if (fr.width > 8192) return fail(ctx, KF_EINVAL, "frame %d: width > 8192", f);
    if (fr.dtype != KF_DTYPE_F32 && fr.dtype != KF_DTYPE_F16 && fr.dtype != KF_DTYPE_BF16 &&
        fr.dtype != KF_DTYPE_U16)
      return fail(ctx, KF_EINVAL, "frame %d: unknown dtype %d", f, fr.dtype);
    if (!std::isfinite(fr.value_scale)) return fail(ctx, KF_EINVAL, "frame %d: value_scale is not finite", f);
    if ((reinterpret_cast<uintptr_t>(fr.data) & (uintptr_t)(kf::in_bytes(fr.dtype) - 1)) != 0)
      return fail(ctx, KF_EINVAL, "frame %d: data is not aligned to its element size", f);
    const long PW = ((long)fr.width + 31) / 32 * 32;
    maxH = std::max(maxH, (long)fr.height);
    maxPW = std::max(maxPW, PW);
    maxplane = std::max(maxplane, (size_t)fr.height * PW);
  }
  cudaError_t e;
  if ((e = cudaSetDevice(ctx->device)) != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  rc = ensure_design(ctx, type, order, scales, nscales, kmax_opt);
  if (rc) return rc;
  int nstate = 0, kmax = 0;
  for (int s = 0; s < nscales; ++s) {
    nstate = std::max(nstate, ctx->cur->h_coef[s].K);
    kmax = std::max(kmax, ctx->cur->h_coef[s].K);
  }
  const int nf = (type == KF_IIR_BUTTERWORTH) ? 2 * nstate : nstate;
  const size_t plane_floats = ((size_t)nscales * maxplane * kf::store_bytes(opts.storage) + 3) / 4;
  if ((rc = grow(ctx, &ctx->P, &ctx->P_floats, plane_floats, "planes"))) return rc;
  if ((rc = grow(ctx, &ctx->edge, &ctx->edge_floats, (size_t)nscales * 2 * maxPW, "edge rows"))) return rc;
  if (type != KF_FIR_COLORED_SG) {
    size_t need = 0;
    for (int f = 0; f < nframes; ++f) {
      const long PW = ((long)frames[f].width + 31) / 32 * 32;
      need = std::max(need, kf::iir_carry_floats(frames[f].height, PW, nscales, nf));
    }
    if ((rc = grow(ctx, &ctx->carry, &ctx->carry_floats, need, "carries"))) return rc;
  }
  if ((e = cudaMemsetAsync(ctx->status, 0, sizeof(kf::DevStatus), ctx->stream)) != cudaSuccess)
    return cuda_fail(ctx, e, "reset status");
  kf::BankArgs a;
  a.coef = ctx->cur->d_coef;
  a.S = nscales;
  a.type = type;
  a.nstate = nstate;
  a.kmax = kmax;
  a.threshold = (float)opts.threshold;
  a.neigh = opts.neighbourhood;
  a.P = ctx->P;
  a.storage = opts.storage;  // KF_DTYPE_F32 / F16 / BF16 equal ST_F32 / ST_F16 / ST_BF16
  a.edge = ctx->edge;
  a.carry = ctx->carry;
  a.blobs = ctx->blobs;
  a.cap = ctx->blob_cap;
  a.status = ctx->status;
  a.responses = opts.responses;
  ctx->prof = kf::Prof{};
  ctx->prof.ev = nullptr;
  if (opts.profile) {
    const int need = 2 * 256;
    while ((int)ctx->events.size() < need) {
      cudaEvent_t ev;
      if ((e = cudaEventCreate(&ev)) != cudaSuccess) return cuda_fail(ctx, e, "cudaEventCreate");
      ctx->events.push_back(ev);
    }
    ctx->prof.ev = ctx->events.data();
    ctx->prof.cap = 256;
  }
  a.prof = &ctx->prof;
  ctx->have_prof = true;
  long resp_off = 0;
  for (int f = 0; f < nframes; ++f) {
    const kf_frame &fr = frames[f];
    kf::FrameGeom g;
    g.X = fr.data;
    g.dtype = fr.dtype;
    g.vscale = fr.value_scale == 0.0f ? 1.0f : fr.value_scale;
    g.xpitch = fr.pitch;
    g.H = fr.height;
    g.W = fr.width;
    g.PW = ((long)fr.width + 31) / 32 * 32;
    g.frame = f;
    g.resp_off = resp_off;
    resp_off += (long)nscales * fr.height * fr.width;
    int lr = (type == KF_FIR_COLORED_SG) ? kf::launch_fir_frame(g, a, ctx->stream)
                                         : kf::launch_iir_frame(g, a, ctx->stream);
    if (lr == -2) return fail(ctx, KF_EINVAL, "no kernel instance for order %d", order);
    if (lr) return cuda_fail(ctx, cudaGetLastError(), "filter-bank kernel launch");
  }
  ctx->have_result = true;
  ctx->sorted_valid = false;
  ctx->last_threshold = opts.threshold;
  ctx->last_S = nscales;
  ctx->last_nframes = nframes;
  ctx->last_hmax = maxH;
  ctx->last_wmax = 0;
  for (int f = 0; f < nframes; ++f) ctx->last_wmax = std::max(ctx->last_wmax, (long)frames[f].width);
  return KF_OK;
}

int kf_kernel_times(kf_ctx *ctx, kf_kernel_time *out, int cap, int *n) {
  if (!ctx) return fail(nullptr, KF_EINVAL, "kf_kernel_times: ctx is NULL");
  if (!n || cap < 0 || (cap > 0 && !out)) return fail(ctx, KF_EINVAL, "kf_kernel_times: bad outputs");
  if (!ctx->have_prof) return fail(ctx, KF_EINVAL, "kf_kernel_times: no bank call yet");
  cudaError_t e;
  if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return cuda_fail(ctx, e, "sync");
  const kf::Prof &p = ctx->prof;
  std::vector<std::string> names;
  std::vector<int> launches;
  std::vector<float> ms;
  for (int i = 0; i < p.n && i < 256; ++i) {
    const std::string nm = p.names[i];
    size_t k = std::find(names.begin(), names.end(), nm) - names.begin();
    if (k == names.size()) {
      names.push_back(nm);
      launches.push_back(0);
      ms.push_back(0.f);
    }
    launches[k] += 1;
    if (p.ev && i < p.cap) {
      float t = 0.f;
      if ((e = cudaEventElapsedTime(&t, p.ev[2 * i], p.ev[2 * i + 1])) != cudaSuccess)
        return cuda_fail(ctx, e, "cudaEventElapsedTime");
      ms[k] += t;
    }
  }
  *n = (int)names.size();
  for (int i = 0; i < cap && i < (int)names.size(); ++i) {
    std::memset(out[i].name, 0, sizeof out[i].name);
    std::strncpy(out[i].name, names[i].c_str(), sizeof out[i].name - 1);
    out[i].launches = launches[i];
    out[i].ms = ms[i];
  }
  return KF_OK;
}

int kf_detect_blobs(kf_ctx *ctx, double threshold, kf_blob *out, int64_t capacity, int64_t *count) {
  if (!ctx) return fail(nullptr, KF_EINVAL, "kf_detect_blobs: ctx is NULL");
  if (!count || capacity < 0 || (capacity > 0 && !out))
    return fail(ctx, KF_EINVAL, "kf_detect_blobs: bad output arguments");
  if (!ctx->have_result) return fail(ctx, KF_EINVAL, "kf_detect_blobs: no filter-bank result");
  if (!(threshold >= ctx->last_threshold))
    return fail(ctx, KF_EINVAL, "threshold %g is below the bank threshold %g", threshold,
                ctx->last_threshold);
  cudaError_t e;
  if ((e = cudaSetDevice(ctx->device)) != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  kf::DevStatus st;
  if ((e = cudaMemcpyAsync(&st, ctx->status, sizeof st, cudaMemcpyDeviceToHost, ctx->stream)) != cudaSuccess)
    return cuda_fail(ctx, e, "read status");
  if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return cuda_fail(ctx, e, "filter bank");
  if (st.error) return fail(ctx, KF_ETIMEOUT, "device wait gave up (code %d)", st.error);
  if (st.range)
    return fail(ctx, KF_ERANGE,
                "a stored plane value exceeded the f16 range: scale the input (value_scale) or use bf16/f32 storage");
  if (st.count > (unsigned long long)ctx->blob_cap) {
    *count = (int64_t)st.count;
    // grow for the next call; this call's list is incomplete
    cudaFree(ctx->blobs);
    ctx->blobs = nullptr;
    long ncap = (long)st.count + (long)st.count / 4 + 1024;
    if ((e = cudaMalloc(&ctx->blobs, sizeof(kf::Blob) * ncap)) != cudaSuccess) {
      ctx->blob_cap = 0;
      return cuda_fail(ctx, e, "cudaMalloc(blobs)");
    }
    ctx->blob_cap = ncap;
    ctx->have_result = false;
    return fail(ctx, KF_ERERUN,
                "candidate list overflowed (%llu found); capacity raised, run the bank again",
                (unsigned long long)st.count);
  }
  const long n = (long)st.count;
  if (!ctx->sorted_valid || ctx->sorted_thr != threshold) {
    ctx->sorted_n = 0;
    if (n > 0) {
      const size_t wb = kf::sort_workspace_bytes(ctx->blob_cap);
      if (!ctx->sort_work || ctx->sort_work_bytes < wb) {
        cudaFree(ctx->sort_work);
        cudaFree(ctx->sorted);
        ctx->sort_work = nullptr;
        ctx->sorted = nullptr;
        ctx->sort_work_bytes = 0;
        if ((e = cudaMalloc(&ctx->sort_work, wb)) != cudaSuccess) return cuda_fail(ctx, e, "sort workspace");
        if ((e = cudaMalloc(&ctx->sorted, sizeof(kf::Blob) * ctx->blob_cap)) != cudaSuccess)
          return cuda_fail(ctx, e, "sorted blobs");
        ctx->sort_work_bytes = wb;
      }
      if (!ctx->d_npass && (e = cudaMalloc(&ctx->d_npass, sizeof(unsigned))) != cudaSuccess)
        return cuda_fail(ctx, e, "cudaMalloc(npass)");
      const unsigned long long span = (unsigned long long)ctx->last_nframes * ctx->last_S *
                                      (unsigned long long)ctx->last_hmax * ctx->last_wmax;
      int keybits = 0;
      while (keybits < 64 && (span >> keybits) != 0) ++keybits;
      kf::Prof none{};
      if (kf::launch_sort(ctx->blobs, n, (float)threshold, ctx->last_S, ctx->last_hmax, ctx->last_wmax,
                          keybits, ctx->sort_work, ctx->sorted, ctx->d_npass, &none, ctx->stream))
        return cuda_fail(ctx, cudaGetLastError(), "sort launch");
      unsigned np = 0;
      if ((e = cudaMemcpyAsync(&np, ctx->d_npass, sizeof np, cudaMemcpyDeviceToHost, ctx->stream)) !=
          cudaSuccess)
        return cuda_fail(ctx, e, "read count");
      if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return cuda_fail(ctx, e, "sort");
      ctx->sorted_n = np;
    }
    ctx->sorted_valid = true;
    ctx->sorted_thr = threshold;
  }
  *count = (int64_t)ctx->sorted_n;
  const int64_t ncopy = std::min<int64_t>(capacity, ctx->sorted_n);
  if (ncopy > 0) {
    static_assert(sizeof(kf_blob) == sizeof(kf::Blob), "record layout");
    if ((e = cudaMemcpyAsync(out, ctx->sorted, sizeof(kf::Blob) * ncopy, cudaMemcpyDeviceToHost,
                             ctx->stream)) != cudaSuccess)
      return cuda_fail(ctx, e, "copy blobs");
    if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return cuda_fail(ctx, e, "copy blobs");
  }
  if (ctx->sorted_n > capacity)
    return fail(ctx, KF_EOVERFLOW, "capacity %lld < %lld blobs", (long long)capacity,
                (long long)ctx->sorted_n);
  return KF_OK;
}

}  // extern "C"
