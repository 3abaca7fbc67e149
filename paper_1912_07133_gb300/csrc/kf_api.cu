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
  float *scan = nullptr;  // single-read column pass: ticket, flags, super-tile states
  size_t scan_floats = 0;
  double *lambdas = nullptr;
  double *dwork = nullptr;
  int dwork_nmax = 0;
  kf::DevStatus *status = nullptr;
  kf::Blob *blobs = nullptr;
  long blob_cap = 0;
  // design cache: (type, order, L_D, kmax, scales) -> coefficients, LRU
  struct Design {
    int type = -1, order = -1, ld = 1, kmax = -1, S = 0;
    double lam[KF_MAX_SCALES];
    kf::Coef *d_coef = nullptr;
    std::vector<kf::Coef> h_coef;
    unsigned long long used = 0;
    // FIR designs: the taps as band operands of the tensor-core column pass
    float *d_bands = nullptr;
    size_t bands_floats = 0;
    kf::TcGeom tc;
    bool tc_ok = false;
    // FIR designs: the grouped tap table of the row pass
    float *d_rowtaps = nullptr;
    size_t rowtaps_floats = 0;
    std::vector<float> h_rowtaps;
    kf::RowGroups rg;
  };
  std::vector<Design> designs;
  unsigned long long tick = 0;
  Design *cur = nullptr;
  // candidate ordering
  kf::Blob *sorted = nullptr;
  long sorted_cap = 0;
  void *sort_work = nullptr;
  size_t sort_work_bytes = 0;
  unsigned *d_npass = nullptr;
  // pinned landing place of the status and the count: read with the records
  // under one synchronisation
  struct HostRead {
    kf::DevStatus st;
    unsigned npass;
  };
  HostRead *h_read = nullptr;
  bool sorted_valid = false;  // an ordering at sorted_thr is enqueued (or done)
  bool npass_read = false;    // sorted_n holds its count
  long count_hint = 1 << 16;  // records copied with the first read (the previous count + margin)
  // the device status of the last bank call, read once
  kf::DevStatus last_status{};
  bool status_read = false;
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
  // frame table of a call (frames + work-item lists): device copy, uploaded
  // from a ring of pinned slots (a slot is reused once its copy has run)
  static constexpr int kRing = 4;
  unsigned char *d_table = nullptr;
  size_t table_cap = 0;
  unsigned char *h_table[kRing] = {};
  cudaEvent_t table_ev[kRing] = {};
  int table_next = 0;
  // graph-mode replays, per call geometry (LRU)
  struct Graph {
    std::vector<long long> key;
    cudaGraphExec_t exec = nullptr;
    kf::Prof prof{};
    unsigned long long used = 0;
  };
  std::vector<Graph> graphs;
  cudaStream_t cap_stream = nullptr;  // private stream for capture (the caller's may be the legacy stream)
  // launch shape per filter type and pass (kf_set_launch_shape / kf_autotune).
  // Default: one block per work item, which measured fastest or within noise
  // of the persistent shapes for every pass on GB300 (4096^2 and uneven
  // batches); the persistent shapes remain candidates of the autotuner.
  int grid_mult[KF_NTYPES][KF_NPASS] = {};
  int seg_len[KF_NTYPES] = {64, 64, 64, 64};  // recursive banks: column segment length (kf_set_segment_length)
  bool seg_chosen[KF_NTYPES] = {false, false, false, false};  // set by kf_set_segment_length or kf_autotune
  // recursive banks: column pass (kf_set_column_pass)
  int column_pass[KF_NTYPES] = {KF_COLUMN_SEGMENTS, KF_COLUMN_SEGMENTS, KF_COLUMN_SEGMENTS, KF_COLUMN_SEGMENTS};
  std::vector<int> last_H, last_W;  // frame sizes of the last bank call
  // proposal network: FP32 masters, Adam moments, bf16 working copy, gradient, loss
  float *net_master = nullptr, *net_m = nullptr, *net_v = nullptr, *net_g = nullptr, *net_loss = nullptr;
  __nv_bfloat16 *net_wb = nullptr;
  int net_step = 0;
  unsigned long long net_version = 0;  // bumped whenever the weights change
  // the gate of the last gated call that evaluated the network: frame sizes,
  // scale count, mode, threshold and weight version (for opts.gate_reuse)
  std::vector<long long> gate_sig;
  bool net_ready = false;
  float *net_work = nullptr;
  size_t net_work_floats = 0;
  long *d_loff = nullptr;  // labels: per-frame offsets and tile grid
  int *d_ltw = nullptr, *d_lth = nullptr;
  int lab_frames = 0;
  // gating buffers: pooled frames, logits, active-tile maps, selected items, counts
  float *g_pooled = nullptr, *g_logits = nullptr;
  size_t g_pooled_n = 0, g_logits_n = 0;
  unsigned char *g_act = nullptr;
  size_t g_act_n = 0;
  int2 *g_sel[2] = {nullptr, nullptr};
  size_t g_sel_n[2] = {0, 0};
  int *g_count = nullptr;
  size_t g_count_n = 0;
  float *ch_buf = nullptr;  // derivative bank: channel planes sigma^2 D (3 or 5 x responses layout)
  size_t ch_floats = 0;
  // the last call's derivative planes (kf_blob_shapes): channel stride, per
  // frame (plane offset, H, W) on the host and its device copy, the shapes
  bool have_dplanes = false;
  size_t dplane_per = 0;
  std::vector<long> dlay;
  long *d_dlay = nullptr;
  size_t d_dlay_n = 0;
  float *shape_buf = nullptr;
  size_t shape_floats = 0;
  // D = 5 bank (kf_quartic_bank): while it runs its channels through the
  // bank call, the call blurs channel q_chan of its frame as raw planes with
  // the L_D = q_ld designs; q_chan < 0 otherwise
  int q_chan = -1, q_ld = 1;
  float *q_out = nullptr;  // the caller's D array: channel frame f, scale s at (s * 15 + f) * H * W
  int q_H = 0, q_W = 0;
  float *q_pad = nullptr;  // the differentiated channels, W x (H + 4) each
  size_t q_pad_floats = 0;
  float *q_xpre = nullptr;  // their rows' pre-rolls (x = -2, -1, W, W + 1)
  size_t q_xpre_floats = 0;
  // per-kernel times of the last profiled kf_quartic_bank call (returned by
  // kf_kernel_times until the next kf_filter_bank call)
  bool q_times_valid = false;
  std::vector<std::string> q_names;
  std::vector<int> q_launches;
  std::vector<float> q_ms;
  cudaEvent_t q_ev[2] = {nullptr, nullptr};
  // failure-detection test hook (kf_set_wait_limit): 0, normal waits
  unsigned wait_test = 0;
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

void drop_graphs(kf_ctx *ctx) {
  for (auto &g : ctx->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  ctx->graphs.clear();
}

// Grow a device buffer; a reallocation invalidates the captured graphs (their
// kernels hold the old pointer).
template <class T>
int grow(kf_ctx *ctx, T **p, size_t *have, size_t need, const char *what) {
  if (*have >= need && *p) return KF_OK;
  drop_graphs(ctx);
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

// Ordering buffers for the context's candidate capacity (keys, indices, digit
// histograms, the ordered list, the count, the pinned read-back); a
// reallocation drops the captured graphs.
int ensure_sort(kf_ctx *ctx, long nrows) {
  cudaError_t e;
  const size_t wb = kf::sort_workspace_bytes(ctx->blob_cap, nrows);
  if (!ctx->sort_work || ctx->sort_work_bytes < wb || !ctx->sorted || ctx->sorted_cap < ctx->blob_cap) {
    drop_graphs(ctx);
    cudaFree(ctx->sort_work);
    cudaFree(ctx->sorted);
    ctx->sort_work = nullptr;
    ctx->sorted = nullptr;
    ctx->sort_work_bytes = 0;
    ctx->sorted_cap = 0;
    if ((e = cudaMalloc(&ctx->sort_work, wb)) != cudaSuccess) return cuda_fail(ctx, e, "sort workspace");
    ctx->sort_work_bytes = wb;
    if ((e = cudaMalloc(&ctx->sorted, sizeof(kf::Blob) * ctx->blob_cap)) != cudaSuccess)
      return cuda_fail(ctx, e, "sorted blobs");
    ctx->sorted_cap = ctx->blob_cap;
  }
  if (!ctx->d_npass && (e = cudaMalloc(&ctx->d_npass, sizeof(unsigned))) != cudaSuccess)
    return cuda_fail(ctx, e, "cudaMalloc(npass)");
  if (!ctx->h_read && (e = cudaMallocHost(&ctx->h_read, sizeof(kf_ctx::HostRead))) != cudaSuccess)
    return cuda_fail(ctx, e, "cudaMallocHost(status)");
  return KF_OK;
}

// Bits of the largest ordering key ((frame S + scale) H + y) W + x.
int sort_keybits(long nframes, long S, long hmax, long wmax) {
  const unsigned long long span = (unsigned long long)nframes * S * (unsigned long long)hmax * wmax;
  int keybits = 0;
  while (keybits < 64 && (span >> keybits) != 0) ++keybits;
  return keybits;
}

int nmax_for(int type, int order, int kmax) {
  if (type != KF_FIR_COLORED_SG) return 1;  // the Gaussian needs no solve
  return kmax + 1 + order + 1;
}

// Run the FP64 design kernel for (type, order, scales) unless the context
// already holds exactly this design (small LRU cache); ctx->cur points at it.
constexpr size_t kDesignSlots = 8;

int ensure_design(kf_ctx *ctx, int type, int order, const double *scales, int S, int kmax, int ld = 1) {
  for (auto &d : ctx->designs)
    if (d.type == type && d.order == order && d.ld == ld && d.kmax == kmax && d.S == S &&
        std::equal(scales, scales + S, d.lam)) {
      d.used = ++ctx->tick;
      ctx->cur = &d;
      return KF_OK;
    }
  ctx->cur = nullptr;
  drop_graphs(ctx);  // a slot may be overwritten: graphs hold coefficient pointers
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
                        ctx->stream, ld))
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
  // FIR designs: the row pass's grouped tap table
  if (type == KF_FIR_COLORED_SG || type == KF_FIR_GAUSSIAN) {
    const long nf = kf::row_groups(slot->h_coef.data(), S, &slot->rg, &slot->h_rowtaps);
    if (nf <= 0) return fail(ctx, KF_EINVAL, "row tap table: %d scales", S);
    if ((size_t)nf > slot->rowtaps_floats) {
      if (slot->d_rowtaps) cudaFree(slot->d_rowtaps);
      slot->d_rowtaps = nullptr;
      slot->rowtaps_floats = 0;
      if ((e = cudaMalloc(&slot->d_rowtaps, (size_t)nf * sizeof(float))) != cudaSuccess)
        return cuda_fail(ctx, e, "cudaMalloc(row tap table)");
      slot->rowtaps_floats = (size_t)nf;
    }
    if ((e = cudaMemcpyAsync(slot->d_rowtaps, slot->h_rowtaps.data(), (size_t)nf * sizeof(float),
                             cudaMemcpyHostToDevice, ctx->stream)) != cudaSuccess)
      return cuda_fail(ctx, e, "copy row tap table");
  }
  // FIR designs of at most 8 scales: the band operands of the tensor-core
  // column pass (R_L = -sigma^2 (...): the taps carry the sign)
  slot->tc_ok = false;
  if ((type == KF_FIR_COLORED_SG || type == KF_FIR_GAUSSIAN) && S <= kf::TC_MAXS) {
    int Ks[kf::TC_MAXS];
    for (int s = 0; s < S; ++s) Ks[s] = slot->h_coef[s].K;
    const long nf = kf::tc_geometry(Ks, S, &slot->tc);
    if (nf > 0) {
      if ((size_t)nf > slot->bands_floats) {
        if (slot->d_bands) cudaFree(slot->d_bands);
        slot->d_bands = nullptr;
        slot->bands_floats = 0;
        if ((e = cudaMalloc(&slot->d_bands, (size_t)nf * sizeof(float))) != cudaSuccess)
          return cuda_fail(ctx, e, "cudaMalloc(tap bands)");
        slot->bands_floats = (size_t)nf;
      }
      if (kf::launch_tc_bands(slot->d_coef, slot->tc, -1.f, slot->d_bands, ctx->stream))
        return cuda_fail(ctx, cudaGetLastError(), "tap band launch");
      slot->tc_ok = true;
    }
  }
  slot->type = type;
  slot->order = order;
  slot->ld = ld;
  slot->kmax = kmax;
  slot->S = S;
  std::copy(scales, scales + S, slot->lam);
  slot->used = ++ctx->tick;
  ctx->cur = slot;
  return KF_OK;
}

bool is_fir(int type) { return type == KF_FIR_COLORED_SG || type == KF_FIR_GAUSSIAN; }

int check_type_order(kf_ctx *ctx, int type, int order) {
  if (type == KF_IIR_REPEATED_POLE && (order < 2 || order > 6))
    return fail(ctx, KF_EINVAL, "repeated-pole order must be 2..6 (got %d)", order);
  if (type == KF_IIR_BUTTERWORTH && (order < 1 || order > 6))
    return fail(ctx, KF_EINVAL, "Butterworth order (L_B/2) must be 1..6 (got %d)", order);
  if (type == KF_FIR_COLORED_SG && order != 1 && order != 2)
    return fail(ctx, KF_EINVAL, "colored SG order (L_D) must be 1 or 2 (got %d)", order);
  if (type == KF_FIR_GAUSSIAN && order != 1)
    return fail(ctx, KF_EINVAL, "Gaussian FIR order must be 1 (got %d)", order);
  if (type < 0 || type >= KF_NTYPES) return fail(ctx, KF_EINVAL, "unknown filter type %d", type);
  return KF_OK;
}

// Upload the call's frame table through the next pinned slot of the ring
// (waiting, in the rare case, until that slot's previous copy has run).
int upload_table(kf_ctx *ctx, const void *bytes, size_t n) {
  cudaError_t e;
  if (n > ctx->table_cap) {
    drop_graphs(ctx);  // graphs hold pointers into the old table
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->d_table);
    ctx->d_table = nullptr;
    ctx->table_cap = 0;
    for (int i = 0; i < kf_ctx::kRing; ++i) {
      if (ctx->h_table[i]) cudaFreeHost(ctx->h_table[i]);
      ctx->h_table[i] = nullptr;
    }
    const size_t cap = std::max(n + n / 2, (size_t)64 << 10);
    if ((e = cudaMalloc(&ctx->d_table, cap)) != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(frame table)");
    for (int i = 0; i < kf_ctx::kRing; ++i) {
      if ((e = cudaHostAlloc(&ctx->h_table[i], cap, cudaHostAllocDefault)) != cudaSuccess)
        return cuda_fail(ctx, e, "cudaHostAlloc(frame table)");
      if (!ctx->table_ev[i] && (e = cudaEventCreateWithFlags(&ctx->table_ev[i], cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(ctx, e, "cudaEventCreate(frame table)");
    }
    ctx->table_cap = cap;
  }
  const int slot = ctx->table_next++ % kf_ctx::kRing;
  if ((e = cudaEventSynchronize(ctx->table_ev[slot])) != cudaSuccess) return cuda_fail(ctx, e, "frame table slot");
  std::memcpy(ctx->h_table[slot], bytes, n);
  if ((e = cudaMemcpyAsync(ctx->d_table, ctx->h_table[slot], n, cudaMemcpyHostToDevice, ctx->stream)) != cudaSuccess)
    return cuda_fail(ctx, e, "upload frame table");
  if ((e = cudaEventRecord(ctx->table_ev[slot], ctx->stream)) != cudaSuccess)
    return cuda_fail(ctx, e, "cudaEventRecord(frame table)");
  return KF_OK;
}

// everything a captured launch sequence depends on besides the frame table
std::vector<long long> call_key(const kf_ctx *ctx, const kf_frame *frames, int nframes, const double *scales, int S,
                                int type, int order, int kmax, const kf_bank_opts &o) {
  std::vector<long long> k = {type, order, kmax, S, o.storage, o.neighbourhood, o.schedule, nframes,
                              (long long)(intptr_t)ctx->cur, o.gate, o.boundary, o.gate_reuse};
  if (o.gate) {
    long long gt;
    double g = o.gate_threshold;
    std::memcpy(&gt, &g, sizeof gt);
    k.push_back(gt);
  }
  for (int p = 0; p < KF_NPASS; ++p) k.push_back(ctx->grid_mult[type][p]);
  k.push_back(ctx->seg_len[type]);
  k.push_back(ctx->column_pass[type]);
  long long t;
  std::memcpy(&t, &o.threshold, sizeof t);
  k.push_back(t);
  for (int s = 0; s < S; ++s) {
    std::memcpy(&t, &scales[s], sizeof t);
    k.push_back(t);
  }
  for (int f = 0; f < nframes; ++f) {
    k.push_back(frames[f].width);
    k.push_back(frames[f].height);
  }
  return k;
}

constexpr size_t kGraphSlots = 4;
constexpr int TW_COL = kf::TW;  // interior columns of a column-pass tile

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
  o->gate_threshold = 0.25f;
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
  cudaFree(ctx->scan);
  for (auto &d : ctx->designs) cudaFree(d.d_coef), cudaFree(d.d_bands), cudaFree(d.d_rowtaps);
  cudaFree(ctx->sorted);
  cudaFree(ctx->sort_work);
  cudaFree(ctx->d_npass);
  if (ctx->h_read) cudaFreeHost(ctx->h_read);
  cudaFree(ctx->lambdas);
  cudaFree(ctx->dwork);
  cudaFree(ctx->status);
  cudaFree(ctx->blobs);
  for (cudaEvent_t e : ctx->events) cudaEventDestroy(e);
  drop_graphs(ctx);
  cudaFree(ctx->d_table);
  cudaFree(ctx->ch_buf);
  cudaFree(ctx->d_dlay);
  cudaFree(ctx->shape_buf);
  cudaFree(ctx->q_pad);
  cudaFree(ctx->q_xpre);
  for (cudaEvent_t ev : ctx->q_ev)
    if (ev) cudaEventDestroy(ev);
  for (void *q : {(void *)ctx->g_pooled, (void *)ctx->g_logits, (void *)ctx->g_act, (void *)ctx->g_sel[0],
                  (void *)ctx->g_sel[1], (void *)ctx->g_count})
    cudaFree(q);
  for (void *q : {(void *)ctx->net_master, (void *)ctx->net_m, (void *)ctx->net_v, (void *)ctx->net_g,
                  (void *)ctx->net_loss, (void *)ctx->net_wb, (void *)ctx->net_work, (void *)ctx->d_loff,
                  (void *)ctx->d_ltw, (void *)ctx->d_lth})
    cudaFree(q);
  for (int i = 0; i < kf_ctx::kRing; ++i) {
    if (ctx->h_table[i]) cudaFreeHost(ctx->h_table[i]);
    if (ctx->table_ev[i]) cudaEventDestroy(ctx->table_ev[i]);
  }
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
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
  for (auto &d : tmp.designs) cudaFree(d.d_coef), cudaFree(d.d_bands), cudaFree(d.d_rowtaps);
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
  if (is_fir(type)) {
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
  if (ctx->q_chan < 0) ctx->q_times_valid = false;
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
  if (opts.response != KF_RESP_LAPLACIAN && opts.response != KF_RESP_HESSIAN)
    return fail(ctx, KF_EINVAL, "unknown response %d", opts.response);
  if (!(opts.offset_limit >= 0.f) || !std::isfinite(opts.offset_limit))
    return fail(ctx, KF_EINVAL, "offset_limit must be >= 0");
  // the derivative bank: R_H, or Threshold #2 with its eq (27) offsets
  const bool dbank = opts.response == KF_RESP_HESSIAN || opts.offset_limit > 0.f;
  if (dbank && opts.gate != KF_GATE_OFF)
    return fail(ctx, KF_EINVAL, "gating runs with the Laplacian response and no offset limit");
  if (opts.boundary != KF_BOUNDARY_HOLD && opts.boundary != KF_BOUNDARY_ZERO)
    return fail(ctx, KF_EINVAL, "unknown boundary %d", opts.boundary);
  if (opts.boundary == KF_BOUNDARY_ZERO && (!is_fir(type) || dbank || ctx->q_chan >= 0))
    return fail(ctx, KF_EINVAL,
                "the zero boundary applies to the FIR blurs (Filters A and C) with the Laplacian response and "
                "no offset limit");
  if (opts.neighbourhood != KF_NEIGH_ALL_SCALES && opts.neighbourhood != KF_NEIGH_ADJACENT)
    return fail(ctx, KF_EINVAL, "unknown neighbourhood %d", opts.neighbourhood);
  if (opts.storage != KF_DTYPE_F32 && opts.storage != KF_DTYPE_F16 && opts.storage != KF_DTYPE_BF16)
    return fail(ctx, KF_EINVAL, "storage must be f32, f16 or bf16");
  if (!(opts.threshold >= 0.0)) return fail(ctx, KF_EINVAL, "threshold must be >= 0");
  const int kmax_opt = opts.fir_kmax > 0 ? opts.fir_kmax : 96;
  if (kmax_opt > KF_MAX_FIR_K) return fail(ctx, KF_EINVAL, "fir_kmax must be <= %d", KF_MAX_FIR_K);
  if (opts.schedule != KF_SCHED_BATCHED && opts.schedule != KF_SCHED_PER_FRAME)
    return fail(ctx, KF_EINVAL, "unknown schedule %d", opts.schedule);
  const bool gate = opts.gate != KF_GATE_OFF;
  if (opts.gate != KF_GATE_OFF && opts.gate != KF_GATE_DILATED && opts.gate != KF_GATE_TILES)
    return fail(ctx, KF_EINVAL, "unknown gate mode %d", opts.gate);
  if (gate) {
    if (!ctx->net_ready) return fail(ctx, KF_EINVAL, "gating needs proposal weights (kf_proposal_set_weights)");
    if (nscales > KF_NET_CHANNELS) return fail(ctx, KF_EINVAL, "gating covers at most %d scales", KF_NET_CHANNELS);
    if (opts.schedule != KF_SCHED_BATCHED) return fail(ctx, KF_EINVAL, "gating runs with the batched schedule");
    if (!(opts.gate_threshold > 0.f && opts.gate_threshold < 1.f))
      return fail(ctx, KF_EINVAL, "gate_threshold must be in (0, 1)");
  }
  if (opts.gate_reuse != 0 && opts.gate_reuse != 1) return fail(ctx, KF_EINVAL, "gate_reuse must be 0 or 1");
  // what the tile marks of a gated call depend on
  std::vector<long long> gate_sig;
  if (gate) {
    long long thr;
    double gt = opts.gate_threshold;
    std::memcpy(&thr, &gt, sizeof thr);
    gate_sig = {nframes, nscales, opts.gate, thr, (long long)ctx->net_version};
    for (int f = 0; f < nframes; ++f) gate_sig.push_back(((long long)frames[f].width << 32) | frames[f].height);
    if (opts.gate_reuse && gate_sig != ctx->gate_sig)
      return fail(ctx, KF_EINVAL,
                  "gate_reuse: no earlier gated call with these frame sizes, scale count, gate mode, threshold "
                  "and weights");
  } else if (opts.gate_reuse) {
    return fail(ctx, KF_EINVAL, "gate_reuse needs gating");
  }
  long maxH = 0, maxPW = 0;
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
  }
  cudaError_t e;
  if ((e = cudaSetDevice(ctx->device)) != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  rc = ensure_design(ctx, type, order, scales, nscales, kmax_opt, ctx->q_ld);
  if (rc) return rc;
  int nstate = 0, kmax = 0;
  for (int s = 0; s < nscales; ++s) {
    nstate = std::max(nstate, ctx->cur->h_coef[s].K);
    kmax = std::max(kmax, ctx->cur->h_coef[s].K);
  }
  const bool iir = !is_fir(type);
  const int nfs = (type == KF_IIR_BUTTERWORTH) ? 2 * nstate : nstate;  // states per recursion
  // the FIR column pass on the tensor cores (f32 planes, all-scales
  // neighbourhood, <= 8 scales, detection); the other calls take the
  // mma.sync and FP32 passes
  long rows_all = 0;
  for (int f = 0; f < nframes; ++f) rows_all += (long)nscales * frames[f].height;
  const bool tcpass = !iir && ctx->cur->tc_ok &&
                      kf::fir_tc_applies(nscales, opts.storage, opts.neighbourhood, dbank || ctx->q_chan >= 0,
                                         maxPW, rows_all);
  // the single-read column pass of the recursive banks (calls whose tallest
  // frame's column strips fit on the GPU at once); else the segment passes
  const bool use_scan = iir && ctx->column_pass[type] == KF_COLUMN_SINGLE_READ &&
                        kf::iir_scan_fits(type, nstate, opts.storage, nscales, (int)maxH);
  // ---- layout: every frame resident in one plane row space of pitch PWb ----
  const long PWb = maxPW;
  std::vector<kf::FrameDev> fd(nframes);
  long prows = 0, roff = 0, aoff = 0, poff = 0, zoff = 0;
  size_t coff = 0;
  std::vector<long> g_poff(nframes), g_zoff(nframes);
  for (int f = 0; f < nframes; ++f) {
    const kf_frame &fr = frames[f];
    kf::FrameDev &d = fd[f];
    d.aoff = aoff;
    d.roff = roff;
    g_poff[f] = poff;
    g_zoff[f] = zoff;
    aoff += (long)((fr.height + 63) / 64) * ((fr.width + 63) / 64);
    poff += (long)((fr.height + 7) / 8) * ((fr.width + 7) / 8);
    zoff += (long)KF_NET_CHANNELS * ((fr.height + 63) / 64) * ((fr.width + 63) / 64);
    d.X = fr.data;
    d.resp = opts.responses ? opts.responses + roff : nullptr;
    d.rplane = 0;
    d.rpitch = d.rmx = d.rmy = 0;
    d.xpre = nullptr;
    if (ctx->q_chan >= 0) {  // D = 5 channel frame f: rows 2 .. H + 1 into out[s][f][H][W]
      const long hw = (long)ctx->q_H * ctx->q_W;
      d.resp = ctx->q_out + f * hw;
      d.rplane = kf::QUARTIC_NCH * hw;
      d.rpitch = ctx->q_W;
      d.rmy = 2;
      d.xpre = reinterpret_cast<const float4 *>(ctx->q_xpre) + (long)f * (ctx->q_H + 4);
    }
    d.xpitch = fr.pitch;
    d.prow = prows;
    d.eoff = (long)f * nscales * 2 * PWb;
    d.coff = (long)coff;
    d.dtype = fr.dtype;
    d.vscale = fr.value_scale == 0.0f ? 1.0f : fr.value_scale;
    d.H = fr.height;
    d.W = fr.width;
    d.nseg = (iir && !use_scan) ? kf::iir_segments(fr.height, ctx->seg_len[type]) : 0;
    d.index = f;
    prows += (long)nscales * fr.height;
    roff += (long)nscales * fr.height * fr.width;
    if (iir) coff += (size_t)nscales * d.nseg * 2 * nfs * PWb;
  }
  const size_t plane_floats = ((size_t)prows * PWb * kf::store_bytes(opts.storage) + 3) / 4;
  if ((rc = grow(ctx, &ctx->P, &ctx->P_floats, plane_floats, "planes"))) return rc;
  if ((rc = grow(ctx, &ctx->edge, &ctx->edge_floats, (size_t)nframes * nscales * 2 * PWb, "edge rows"))) return rc;
  if (iir && !use_scan && (rc = grow(ctx, &ctx->carry, &ctx->carry_floats, std::max(coff, (size_t)1), "carries")))
    return rc;
  if (use_scan) {
    long U = 0;
    for (int f = 0; f < nframes; ++f) U += kf::iir_scan_items(fd[f].H, fd[f].W);
    if (U > INT32_MAX / 4) return fail(ctx, KF_EINVAL, "too many column tiles in one call: split the batch");
    const size_t nb = kf::iir_scan_bytes(U, nscales, nfs);
    if ((rc = grow(ctx, &ctx->scan, &ctx->scan_floats, (nb + 3) / 4, "column-pass states"))) return rc;
  }
  // ---- work-item lists of the launches --------------------------------------
  struct L {
    int pass, nt, n, total;
    size_t fl, pre;  // offsets (ints) in the pool
  };
  std::vector<int> pool;
  std::vector<L> ls;
  constexpr int PASS_COMB = 99;  // the derivative bank's combine + detect launch
  constexpr int PASS_SCAN = 98;  // the single-read column pass of the recursive banks
  auto items = [&](int pass, int f) {
    if (pass == PASS_COMB) return kf::deriv_items(fd[f].H, fd[f].W);
    if (pass == PASS_SCAN) return kf::iir_scan_items(fd[f].H, fd[f].W);
    return iir ? kf::iir_items(pass, fd[f].H, fd[f].W, nscales, ctx->seg_len[type])
               : kf::fir_items(pass, fd[f].H, fd[f].W, nscales, opts.neighbourhood, tcpass);
  };
  auto add = [&](int pass, const std::vector<int> &fl, int nt) {
    L l{pass, nt, (int)fl.size(), 0, pool.size(), 0};
    pool.insert(pool.end(), fl.begin(), fl.end());
    l.pre = pool.size();
    long tot = 0;
    pool.push_back(0);
    for (int f : fl) {
      tot += items(pass, f);
      pool.push_back((int)std::min(tot, (long)INT32_MAX));
    }
    l.total = (int)std::min(tot, (long)INT32_MAX);
    ls.push_back(l);
    return tot <= INT32_MAX;
  };
  const std::vector<int> passes = iir ? std::vector<int>{kf::PASS_ROW, kf::PASS_SEG, kf::PASS_FOLD, kf::PASS_DET}
                                      : std::vector<int>{kf::PASS_ROW, kf::PASS_DET};
  bool fits = true;
  if (opts.schedule == KF_SCHED_PER_FRAME) {
    for (int p : passes)
      for (int f = 0; f < nframes; ++f)
        fits &= add(p, {f}, (iir && p == kf::PASS_ROW) ? kf::iir_row_threads(fd[f].W) : 0);
  } else {
    for (int p : passes) {
      if (iir && p == kf::PASS_ROW) {  // one launch per block width (width class)
        std::vector<int> nts;
        for (int f = 0; f < nframes; ++f) nts.push_back(kf::iir_row_threads(fd[f].W));
        std::vector<int> classes = nts;
        std::sort(classes.begin(), classes.end());
        classes.erase(std::unique(classes.begin(), classes.end()), classes.end());
        for (int nt : classes) {
          std::vector<int> fl;
          for (int f = 0; f < nframes; ++f)
            if (nts[f] == nt) fl.push_back(f);
          fits &= add(p, fl, nt);
        }
      } else {
        std::vector<int> fl(nframes);
        for (int f = 0; f < nframes; ++f) fl[f] = f;
        fits &= add(p, fl, 0);
      }
    }
  }
  if (dbank) {
    std::vector<int> fl(nframes);
    for (int f = 0; f < nframes; ++f) fl[f] = f;
    fits &= add(PASS_COMB, fl, 0);
  }
  if (use_scan) {
    if (opts.schedule == KF_SCHED_PER_FRAME) {
      for (int f = 0; f < nframes; ++f) fits &= add(PASS_SCAN, {f}, 0);
    } else {
      std::vector<int> fl(nframes);
      for (int f = 0; f < nframes; ++f) fl[f] = f;
      fits &= add(PASS_SCAN, fl, 0);
    }
  }
  if (!fits) return fail(ctx, KF_EINVAL, "too many work items in one call: split the batch");
  for (const L &l : ls)
    if (iir && l.pass == kf::PASS_ROW && l.nt == 0) return fail(ctx, KF_EINVAL, "frame too wide for the row pass");
  // ---- frame table: FrameDev[nframes] | int pool -----------------------------
  const size_t fd_bytes = sizeof(kf::FrameDev) * nframes;
  const size_t pool_off = (fd_bytes + 15) / 16 * 16;
  std::vector<unsigned char> table(pool_off + pool.size() * sizeof(int));
  std::memcpy(table.data(), fd.data(), fd_bytes);
  std::memcpy(table.data() + pool_off, pool.data(), pool.size() * sizeof(int));
  if ((rc = upload_table(ctx, table.data(), table.size()))) return rc;
  kf::Plan plan;
  plan.fr = reinterpret_cast<const kf::FrameDev *>(ctx->d_table);
  plan.nframes = nframes;
  plan.PWb = PWb;
  plan.prows = prows;
  plan.per_frame = opts.schedule == KF_SCHED_PER_FRAME;
  for (int p = 0; p < KF_NPASS; ++p) plan.mult[p] = ctx->grid_mult[type][p];
  plan.lc = ctx->seg_len[type];
  const int *dpool = reinterpret_cast<const int *>(ctx->d_table + pool_off);
  for (const L &l : ls) {
    kf::Launch x;
    x.it.fl = dpool + l.fl;
    x.it.pre = dpool + l.pre;
    x.it.n = l.n;
    x.it.total = l.total;
    x.nt = l.nt;
    if (l.pass == PASS_COMB) plan.comb = x;
    else if (l.pass == PASS_SCAN) plan.scan.push_back(x);
    else plan.pass[l.pass].push_back(x);
  }
  // ---- gating: buffers and the gated launches --------------------------------
  kf::Items full_det{}, full_row{};
  if (gate) {
    int ph = 1, pw = 1;
    for (int f = 0; f < nframes; ++f) {
      ph = std::max(ph, (frames[f].height + 7) / 8);
      pw = std::max(pw, (frames[f].width + 7) / 8);
    }
    if ((rc = grow(ctx, &ctx->g_pooled, &ctx->g_pooled_n, (size_t)std::max(poff, 1L), "gate pooled")) ||
        (rc = grow(ctx, &ctx->g_logits, &ctx->g_logits_n, (size_t)std::max(zoff, 1L), "gate logits")) ||
        (rc = grow(ctx, &ctx->g_act, &ctx->g_act_n, (size_t)std::max(aoff, 1L), "gate tiles")) ||
        (rc = grow(ctx, &ctx->g_count, &ctx->g_count_n, (size_t)2, "gate counts")) ||
        (rc = grow(ctx, &ctx->net_work, &ctx->net_work_floats, kf::net_work_floats(1, ph, pw), "network workspace")))
      return rc;
    full_det = plan.pass[kf::PASS_DET][0].it;
    if ((rc = grow(ctx, &ctx->g_sel[0], &ctx->g_sel_n[0], (size_t)std::max(full_det.total, 1), "gate items")))
      return rc;
    plan.pass[kf::PASS_DET][0].it.sel = ctx->g_sel[0];
    plan.pass[kf::PASS_DET][0].it.dcount = ctx->g_count;
    if (!iir) {
      full_row = plan.pass[kf::PASS_ROW][0].it;
      if ((rc = grow(ctx, &ctx->g_sel[1], &ctx->g_sel_n[1], (size_t)std::max(full_row.total, 1), "gate items")))
        return rc;
      plan.pass[kf::PASS_ROW][0].it.sel = ctx->g_sel[1];
      plan.pass[kf::PASS_ROW][0].it.dcount = ctx->g_count + 1;
    }
  }
  // pooling, logits and tile maps of every frame, then the selected items
  auto issue_gate = [&](cudaStream_t st, kf::Prof *prof) -> int {
    const float p = opts.gate_threshold, zthr = std::log(p / (1.f - p));
    prof->begin("gate", st);
    for (int f = 0; f < (opts.gate_reuse ? 0 : nframes); ++f) {
      const int H = frames[f].height, W = frames[f].width;
      const int ph = (H + 7) / 8, pw = (W + 7) / 8, th = (H + 63) / 64, tw = (W + 63) / 64;
      if (kf::net_pool_table(plan.fr, f, H, W, ctx->g_pooled + g_poff[f], st) ||
          kf::net_forward(ctx->g_pooled + g_poff[f], 1, ph, pw, ctx->net_wb, ctx->net_work, ctx->g_logits + g_zoff[f],
                          st) ||
          kf::gate_tiles(ctx->g_logits + g_zoff[f], nscales, th, tw, zthr, opts.gate == KF_GATE_DILATED ? 1 : 0,
                         ctx->g_act + fd[f].aoff, st))
        return cuda_fail(ctx, cudaGetLastError(), "gate");
    }
    cudaError_t ee;
    if ((ee = cudaMemsetAsync(ctx->g_count, 0, 2 * sizeof(int), st)) != cudaSuccess)
      return cuda_fail(ctx, ee, "gate counts");
    const int rows = iir ? ctx->seg_len[type]
                         : (tcpass ? kf::fir_tc_tile_rows(nscales) : kf::fir_tile_rows(opts.neighbourhood));
    if (!use_scan &&
        kf::gate_select_tiles(plan.fr, full_det, ctx->g_act, tcpass ? kf::fir_tc_tile_cols() : TW_COL, rows,
                              ctx->g_sel[0], ctx->g_count, st))
      return cuda_fail(ctx, cudaGetLastError(), "gate selection");
    if (!iir && kf::gate_select_rows(plan.fr, full_row, ctx->g_act, kf::fir_row_segment(), kf::fir_row_rows(),
                                     kf::fir_halo(kmax) + rows + 4,
                                     ctx->g_sel[1], ctx->g_count + 1, st))
      return cuda_fail(ctx, cudaGetLastError(), "gate selection");
    prof->end(st);
    return KF_OK;
  };
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
  a.scan = use_scan ? ctx->scan : nullptr;
  a.gate_act = gate ? ctx->g_act : nullptr;
  a.blobs = ctx->blobs;
  a.cap = ctx->blob_cap;
  a.status = ctx->status;
  a.wait_test = ctx->wait_test;
  a.zero = opts.boundary == KF_BOUNDARY_ZERO;
  if (!iir) {
    a.row_taps = ctx->cur->d_rowtaps;
    a.rg = ctx->cur->rg;
  }
  if (tcpass) {
    a.tc_bands = ctx->cur->d_bands;
    a.tc = ctx->cur->tc;
  }
  if (ctx->q_chan >= 0) {  // a channel of the D = 5 bank: raw planes, no detection
    a.chan = ctx->q_chan;
    a.raw = 1;
  }
  // the candidate ordering at the bank threshold runs at the end of the call
  const long nrows = (long)nframes * nscales * maxH;  // row buckets of the ordering
  if ((rc = ensure_sort(ctx, nrows))) return rc;
  long wmax = 0;
  for (int f = 0; f < nframes; ++f) wmax = std::max(wmax, (long)frames[f].width);
  const int keybits = sort_keybits(nframes, nscales, maxH, wmax);
  auto issue_sort = [&](cudaStream_t st, kf::Prof *prof) -> int {
    if (kf::launch_sort(ctx->blobs, ctx->blob_cap, &ctx->status->count, (float)opts.threshold, nscales, maxH, wmax,
                        keybits, nrows, ctx->sort_work, ctx->sorted, ctx->d_npass, prof, st))
      return cuda_fail(ctx, cudaGetLastError(), "candidate ordering launch");
    return KF_OK;
  };
  // status reset + all passes + ordering, on stream st
  auto issue = [&](cudaStream_t st, kf::Prof *prof) -> int {
    cudaError_t ee;
    if ((ee = cudaMemsetAsync(ctx->status, 0, sizeof(kf::DevStatus), st)) != cudaSuccess)
      return cuda_fail(ctx, ee, "reset status");
    a.prof = prof;
    if (gate)
      if (int grc = issue_gate(st, prof)) return grc;
    const int lr = iir ? kf::launch_iir(plan, a, st) : kf::launch_fir(plan, a, st);
    if (lr == -2) return fail(ctx, KF_EINVAL, "no kernel instance for order %d", order);
    if (lr) return cuda_fail(ctx, cudaGetLastError(), "filter-bank kernel launch");
    if (ctx->q_chan >= 0) return KF_OK;  // raw planes: no candidates to order
    return issue_sort(st, prof);
  };
  ctx->prof = kf::Prof{};
  ctx->prof.ev = nullptr;
  ctx->have_prof = true;
  if (opts.profile) {
    const int need = 2 * 256;
    while ((int)ctx->events.size() < need) {
      cudaEvent_t ev;
      if ((e = cudaEventCreate(&ev)) != cudaSuccess) return cuda_fail(ctx, e, "cudaEventCreate");
      ctx->events.push_back(ev);
    }
  }
  if (dbank) {
    // every needed derivative as its own channel (raw planes sigma^2 D), then
    // R and the detector; the frame table's response pointers select the
    // channel planes of each run (runs eagerly: one table per run)
    const int chans_h[5] = {kf::CH_U, kf::CH_V, kf::CH_W, kf::CH_DX, kf::CH_DY};
    const int nch = opts.offset_limit > 0.f ? 5 : 3;
    const size_t per = (size_t)std::max(roff, 1L);
    if ((rc = grow(ctx, &ctx->ch_buf, &ctx->ch_floats, per * nch, "derivative planes"))) return rc;
    if (opts.profile) {
      ctx->prof.ev = ctx->events.data();
      ctx->prof.cap = 256;
    }
    a.prof = &ctx->prof;
    if ((e = cudaMemsetAsync(ctx->status, 0, sizeof(kf::DevStatus), ctx->stream)) != cudaSuccess)
      return cuda_fail(ctx, e, "reset status");
    auto with_resp = [&](float *base) -> int {
      for (int f = 0; f < nframes; ++f) fd[f].resp = base ? base + fd[f].roff : nullptr;
      std::memcpy(table.data(), fd.data(), fd_bytes);
      return upload_table(ctx, table.data(), table.size());
    };
    for (int c = 0; c < nch; ++c) {
      if ((rc = with_resp(ctx->ch_buf + (size_t)c * per))) return rc;
      a.chan = chans_h[c];
      a.raw = 1;
      const int lr = iir ? kf::launch_iir(plan, a, ctx->stream) : kf::launch_fir(plan, a, ctx->stream);
      if (lr == -2) return fail(ctx, KF_EINVAL, "no kernel instance for order %d", order);
      if (lr) return cuda_fail(ctx, cudaGetLastError(), "derivative channel launch");
    }
    if ((rc = with_resp(opts.responses))) return rc;
    a.chan = kf::CH_LAP;
    a.raw = 0;
    const float *c20 = ctx->ch_buf, *c02 = ctx->ch_buf + per, *c11 = ctx->ch_buf + 2 * per;
    const float *c10 = nch == 5 ? ctx->ch_buf + 3 * per : nullptr, *c01 = nch == 5 ? ctx->ch_buf + 4 * per : nullptr;
    if (kf::launch_combine_detect(plan, plan.comb, a, opts.response == KF_RESP_HESSIAN, c20, c02, c11, c10, c01,
                                  opts.offset_limit, ctx->stream))
      return cuda_fail(ctx, cudaGetLastError(), "derivative bank detector");
    if ((rc = issue_sort(ctx->stream, &ctx->prof))) return rc;
    ctx->dplane_per = per;
    ctx->dlay.assign(3 * (size_t)nframes, 0);
    for (int f = 0; f < nframes; ++f) {
      ctx->dlay[3 * f] = fd[f].roff;
      ctx->dlay[3 * f + 1] = frames[f].height;
      ctx->dlay[3 * f + 2] = frames[f].width;
    }
  } else if (opts.graph && !opts.profile) {
    const std::vector<long long> key = call_key(ctx, frames, nframes, scales, nscales, type, order, kmax_opt, opts);
    kf_ctx::Graph *g = nullptr;
    for (auto &x : ctx->graphs)
      if (x.key == key) g = &x;
    if (!g) {  // first call of this geometry: run eagerly, remember it
      if (ctx->graphs.size() >= kGraphSlots) {
        auto lru = std::min_element(ctx->graphs.begin(), ctx->graphs.end(),
                                    [](const kf_ctx::Graph &p, const kf_ctx::Graph &q) { return p.used < q.used; });
        if (lru->exec) cudaGraphExecDestroy(lru->exec);
        ctx->graphs.erase(lru);
      }
      ctx->graphs.emplace_back();
      ctx->graphs.back().key = key;
      ctx->graphs.back().used = ++ctx->tick;
      if ((rc = issue(ctx->stream, &ctx->prof))) return rc;
    } else {
      g->used = ++ctx->tick;
      if (!g->exec) {  // second call: capture on the private stream, instantiate
        if (!ctx->cap_stream && (e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
          return cuda_fail(ctx, e, "cudaStreamCreate(capture)");
        kf::Prof cp{};
        cp.ev = nullptr;
        if ((e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
          return cuda_fail(ctx, e, "cudaStreamBeginCapture");
        const int irc = issue(ctx->cap_stream, &cp);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(ctx->cap_stream, &graph);
        if (irc || e != cudaSuccess) {
          if (graph) cudaGraphDestroy(graph);
          return irc ? irc : cuda_fail(ctx, e, "cudaStreamEndCapture");
        }
        e = cudaGraphInstantiate(&g->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
          g->exec = nullptr;
          return cuda_fail(ctx, e, "cudaGraphInstantiate");
        }
        g->prof = cp;
      }
      if ((e = cudaGraphLaunch(g->exec, ctx->stream)) != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphLaunch");
      ctx->prof = g->prof;
    }
  } else {
    if (opts.profile) {
      ctx->prof.ev = ctx->events.data();
      ctx->prof.cap = 256;
    }
    if ((rc = issue(ctx->stream, &ctx->prof))) return rc;
  }
  ctx->have_result = true;
  if (gate && !opts.gate_reuse) ctx->gate_sig = gate_sig;  // the marks a later call may reuse
  ctx->have_dplanes = dbank;
  ctx->sorted_valid = true;  // enqueued with the call
  ctx->sorted_thr = opts.threshold;
  ctx->npass_read = false;
  ctx->status_read = false;
  ctx->last_threshold = opts.threshold;
  ctx->last_S = nscales;
  ctx->last_nframes = nframes;
  ctx->last_hmax = maxH;
  ctx->last_wmax = wmax;
  ctx->last_H.resize(nframes);
  ctx->last_W.resize(nframes);
  for (int f = 0; f < nframes; ++f) ctx->last_H[f] = frames[f].height, ctx->last_W[f] = frames[f].width;
  return KF_OK;
}

int kf_set_launch_shape(kf_ctx *ctx, int type, int pass, int grid_mult) {
  if (!ctx) return fail(nullptr, KF_EINVAL, "kf_set_launch_shape: ctx is NULL");
  if (type < 0 || type >= KF_NTYPES) return fail(ctx, KF_EINVAL, "unknown filter type %d", type);
  if (pass < 0 || pass >= KF_NPASS) return fail(ctx, KF_EINVAL, "unknown pass %d", pass);
  if (grid_mult < -16 || grid_mult > 64) return fail(ctx, KF_EINVAL, "grid_mult must be -16..64");
  if (ctx->grid_mult[type][pass] != grid_mult) {
    drop_graphs(ctx);  // grid sizes are part of the captured launches
    ctx->grid_mult[type][pass] = grid_mult;
  }
  return KF_OK;
}

int kf_set_wait_limit(kf_ctx *ctx, int polls) {
  if (polls < 0 || polls > 1 << 20) return fail(ctx, KF_EINVAL, "kf_set_wait_limit: polls must be 0..2^20");
  if (!ctx) {
    kf::set_noalloc_wait_test((unsigned)polls);
    return KF_OK;
  }
  if (ctx->wait_test != (unsigned)polls) {
    drop_graphs(ctx);  // the limit is a launch argument of the captured passes
    ctx->wait_test = (unsigned)polls;
  }
  return KF_OK;
}

int kf_set_segment_length(kf_ctx *ctx, int type, int rows) {
  if (!ctx) return fail(nullptr, KF_EINVAL, "kf_set_segment_length: ctx is NULL");
  if (type != KF_IIR_REPEATED_POLE && type != KF_IIR_BUTTERWORTH)
    return fail(ctx, KF_EINVAL, "segment length applies to the recursive banks only");
  if (rows != 32 && rows != 64) return fail(ctx, KF_EINVAL, "segment length must be 32 or 64 rows");
  if (ctx->seg_len[type] != rows) {
    drop_graphs(ctx);
    ctx->seg_len[type] = rows;
  }
  ctx->seg_chosen[type] = true;
  return KF_OK;
}

int kf_set_column_pass(kf_ctx *ctx, int type, int mode) {
  if (!ctx) return fail(nullptr, KF_EINVAL, "kf_set_column_pass: ctx is NULL");
  if (type != KF_IIR_REPEATED_POLE && type != KF_IIR_BUTTERWORTH)
    return fail(ctx, KF_EINVAL, "the column pass applies to the recursive banks only");
  if (mode != KF_COLUMN_SINGLE_READ && mode != KF_COLUMN_SEGMENTS)
    return fail(ctx, KF_EINVAL, "unknown column pass %d", mode);
  if (ctx->column_pass[type] != mode) {
    drop_graphs(ctx);
    ctx->column_pass[type] = mode;
  }
  return KF_OK;
}

int kf_autotune(kf_ctx *ctx, const kf_frame *frames, int nframes, const double *scales, int nscales, int type,
                int order, const kf_bank_opts *opts_in, int32_t *chosen, float *ms_out) {
  if (!ctx) return fail(nullptr, KF_EINVAL, "kf_autotune: ctx is NULL");
  if (type < 0 || type >= KF_NTYPES) return fail(ctx, KF_EINVAL, "unknown filter type %d", type);
  kf_bank_opts o;
  if (opts_in) o = *opts_in;
  else kf_bank_opts_default(&o);
  o.profile = 1;
  o.graph = 0;
  constexpr int kCand[4] = {1, 2, 4, 0};
  const int saved[KF_NPASS] = {ctx->grid_mult[type][0], ctx->grid_mult[type][1], ctx->grid_mult[type][2],
                               ctx->grid_mult[type][3]};
  auto pass_of = [](const char *name) {
    const std::string n = name;
    if (n == "iir_row" || n == "fir_row") return (int)KF_PASS_ROW;
    if (n == "iir_colseg") return (int)KF_PASS_SEG;
    if (n == "iir_colfold") return (int)KF_PASS_FOLD;
    if (n == "iir_coldet" || n == "iir_colscan" || n == "fir_coldet") return (int)KF_PASS_DET;
    return -1;
  };
  cudaError_t e;
  const bool iir = !is_fir(type);
  const int saved_lc = ctx->seg_len[type], saved_col = ctx->column_pass[type];
  // per candidate (column pass: segments of 64 or 32 rows, or the
  // single-read pass (0); shape): per-pass time
  const int nlc = iir ? 3 : 1;
  const int lcs[3] = {64, 32, 0};
  float t[3][4][KF_NPASS];
  for (int l = 0; l < nlc; ++l) {
    if (iir) {
      ctx->seg_len[type] = lcs[l] ? lcs[l] : saved_lc;
      ctx->column_pass[type] = lcs[l] ? KF_COLUMN_SEGMENTS : KF_COLUMN_SINGLE_READ;
    }
    for (int c = 0; c < 4; ++c) {
      for (int p = 0; p < KF_NPASS; ++p) ctx->grid_mult[type][p] = kCand[c];
      float acc[KF_NPASS] = {0, 0, 0, 0};
      bool seen[KF_NPASS] = {false, false, false, false};
      for (int rep = 0; rep < 3; ++rep) {  // one warm-up, two timed
        int rc = kf_filter_bank(ctx, frames, nframes, scales, nscales, type, order, &o);
        if (rc) {
          for (int p = 0; p < KF_NPASS; ++p) ctx->grid_mult[type][p] = saved[p];
          ctx->seg_len[type] = saved_lc;
          ctx->column_pass[type] = saved_col;
          return rc;
        }
        if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return cuda_fail(ctx, e, "autotune");
        if (rep == 0) continue;
        const kf::Prof &pr = ctx->prof;
        for (int i = 0; i < pr.n && i < pr.cap; ++i) {
          const int p = pass_of(pr.names[i]);
          if (p < 0) continue;
          float dt = 0.f;
          if ((e = cudaEventElapsedTime(&dt, pr.ev[2 * i], pr.ev[2 * i + 1])) != cudaSuccess)
            return cuda_fail(ctx, e, "cudaEventElapsedTime");
          acc[p] += dt;
          seen[p] = true;
        }
      }
      for (int p = 0; p < KF_NPASS; ++p) t[l][c][p] = seen[p] ? acc[p] / 2.f : -1.f;
    }
  }
  // per segment length: the best shape of every pass and their summed time;
  // the segment length with the smaller sum wins (the row pass does not depend on it)
  int best_l = 0;
  float best_sum = -1.f;
  int best_c[3][KF_NPASS];
  for (int l = 0; l < nlc; ++l) {
    float sum = 0.f;
    for (int p = 0; p < KF_NPASS; ++p) {
      int b = -1;
      for (int c = 0; c < 4; ++c)
        if (t[l][c][p] >= 0.f && (b < 0 || t[l][c][p] < t[l][b][p])) b = c;
      best_c[l][p] = b;
      if (b >= 0) sum += t[l][b][p];
    }
    if (best_sum < 0.f || sum < best_sum) best_sum = sum, best_l = l;
  }
  if (iir) {
    ctx->seg_len[type] = lcs[best_l] ? lcs[best_l] : saved_lc;
    ctx->column_pass[type] = lcs[best_l] ? KF_COLUMN_SEGMENTS : KF_COLUMN_SINGLE_READ;
    if (lcs[best_l]) ctx->seg_chosen[type] = true;
  }
  for (int p = 0; p < KF_NPASS; ++p) {
    const int b = best_c[best_l][p];
    ctx->grid_mult[type][p] = b < 0 ? saved[p] : kCand[b];
    if (chosen) chosen[p] = b < 0 ? -1 : kCand[b];
    if (ms_out)
      for (int c = 0; c < 4; ++c) ms_out[p * 4 + c] = t[best_l][c][p];
  }
  if (chosen) chosen[KF_NPASS] = iir ? lcs[best_l] : -1;
  drop_graphs(ctx);
  return KF_OK;
}

// ---- proposal network --------------------------------------------------------

int kf_proposal_set_weights(kf_ctx *ctx, const float *weights) {
  if (!ctx) return fail(nullptr, KF_EINVAL, "kf_proposal_set_weights: ctx is NULL");
  if (!weights) return fail(ctx, KF_EINVAL, "kf_proposal_set_weights: weights is NULL");
  cudaError_t e;
  if ((e = cudaSetDevice(ctx->device)) != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  const size_t nb = sizeof(float) * kf::NET_NPARAM;
  if (!ctx->net_master) {
    for (float **q : {&ctx->net_master, &ctx->net_m, &ctx->net_v, &ctx->net_g})
      if ((e = cudaMalloc(q, nb)) != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(network)");
    if ((e = cudaMalloc(&ctx->net_loss, sizeof(float))) != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(loss)");
    if ((e = cudaMalloc(&ctx->net_wb, sizeof(__nv_bfloat16) * kf::NET_NPARAM)) != cudaSuccess)
      return cuda_fail(ctx, e, "cudaMalloc(network)");
  }
  if ((e = cudaMemcpyAsync(ctx->net_master, weights, nb, cudaMemcpyHostToDevice, ctx->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(ctx->net_m, 0, nb, ctx->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(ctx->net_v, 0, nb, ctx->stream)) != cudaSuccess)
    return cuda_fail(ctx, e, "set weights");
  if (kf::net_to_bf16(ctx->net_master, ctx->net_wb, ctx->stream)) return cuda_fail(ctx, cudaGetLastError(), "bf16");
  // the host array may be reused as soon as the copy has been made
  if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return cuda_fail(ctx, e, "set weights");
  ctx->net_step = 0;
  ctx->net_ready = true;
  ++ctx->net_version;
  drop_graphs(ctx);
  return KF_OK;
}

int kf_proposal_get_weights(kf_ctx *ctx, float *weights) {
  if (!ctx) return fail(nullptr, KF_EINVAL, "kf_proposal_get_weights: ctx is NULL");
  if (!weights || !ctx->net_ready) return fail(ctx, KF_EINVAL, "kf_proposal_get_weights: no weights / NULL output");
  cudaError_t e;
  if ((e = cudaMemcpyAsync(weights, ctx->net_master, sizeof(float) * kf::NET_NPARAM, cudaMemcpyDeviceToHost,
                           ctx->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess)
    return cuda_fail(ctx, e, "get weights");
  return KF_OK;
}

int kf_proposal_pool(kf_ctx *ctx, const kf_frame *frames, int nframes, float *pooled) {
  if (!ctx) return fail(nullptr, KF_EINVAL, "kf_proposal_pool: ctx is NULL");
  if (!frames || nframes < 1 || !pooled) return fail(ctx, KF_EINVAL, "kf_proposal_pool: bad arguments");
  long off = 0;
  for (int f = 0; f < nframes; ++f) {
    const kf_frame &fr = frames[f];
    if (!fr.data || fr.width < 1 || fr.height < 1 || fr.pitch < fr.width || fr.dtype < 0 || fr.dtype > 3)
      return fail(ctx, KF_EINVAL, "kf_proposal_pool: frame %d is invalid", f);
    if (kf::net_pool(fr.data, fr.dtype, fr.value_scale == 0.0f ? 1.0f : fr.value_scale, fr.pitch, fr.height,
                     fr.width, pooled + off, ctx->stream))
      return cuda_fail(ctx, cudaGetLastError(), "pool");
    off += (long)((fr.height + 7) / 8) * ((fr.width + 7) / 8);
  }
  return KF_OK;
}

namespace {
int net_check(kf_ctx *ctx, const float *pooled, int n, int h, int w, const char *who) {
  if (!ctx) return fail(nullptr, KF_EINVAL, "%s: ctx is NULL", who);
  if (!ctx->net_ready) return fail(ctx, KF_EINVAL, "%s: no weights set", who);
  if (!pooled || n < 1 || h < 1 || w < 1) return fail(ctx, KF_EINVAL, "%s: bad arguments", who);
  const size_t need = kf::net_work_floats(n, h, w);
  if (need > ctx->net_work_floats) {
    drop_graphs(ctx);  // gated graphs hold the workspace pointer
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->net_work);
    ctx->net_work = nullptr;
    ctx->net_work_floats = 0;
    const cudaError_t e = cudaMalloc(&ctx->net_work, need * sizeof(float));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(network workspace)");
    ctx->net_work_floats = need;
  }
  return KF_OK;
}
}  // namespace

int kf_proposal_logits(kf_ctx *ctx, const float *pooled, int n, int h, int w, float *logits) {
  if (int rc = net_check(ctx, pooled, n, h, w, "kf_proposal_logits")) return rc;
  if (!logits) return fail(ctx, KF_EINVAL, "kf_proposal_logits: logits is NULL");
  if (kf::net_forward(pooled, n, h, w, ctx->net_wb, ctx->net_work, logits, ctx->stream))
    return cuda_fail(ctx, cudaGetLastError(), "network forward");
  return KF_OK;
}

int kf_proposal_grad(kf_ctx *ctx, const float *pooled, const uint8_t *labels, int n, int h, int w,
                     float pos_weight, float *grad, float *loss) {
  if (int rc = net_check(ctx, pooled, n, h, w, "kf_proposal_grad")) return rc;
  if (!labels || !(pos_weight > 0.f)) return fail(ctx, KF_EINVAL, "kf_proposal_grad: bad labels / pos_weight");
  if (kf::net_grad(pooled, labels, n, h, w, pos_weight, ctx->net_wb, ctx->net_work, ctx->net_g, ctx->net_loss,
                   ctx->stream))
    return cuda_fail(ctx, cudaGetLastError(), "network gradient");
  cudaError_t e;
  if (grad && (e = cudaMemcpyAsync(grad, ctx->net_g, sizeof(float) * kf::NET_NPARAM, cudaMemcpyDeviceToHost,
                                   ctx->stream)) != cudaSuccess)
    return cuda_fail(ctx, e, "copy gradient");
  if (loss && (e = cudaMemcpyAsync(loss, ctx->net_loss, sizeof(float), cudaMemcpyDeviceToHost, ctx->stream)) !=
                  cudaSuccess)
    return cuda_fail(ctx, e, "copy loss");
  if ((grad || loss) && (e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return cuda_fail(ctx, e, "grad");
  return KF_OK;
}

int kf_proposal_train_step(kf_ctx *ctx, const float *pooled, const uint8_t *labels, int n, int h, int w,
                           float pos_weight, float lr, float *loss) {
  if (int rc = net_check(ctx, pooled, n, h, w, "kf_proposal_train_step")) return rc;
  if (!labels || !(pos_weight > 0.f) || !(lr > 0.f))
    return fail(ctx, KF_EINVAL, "kf_proposal_train_step: bad labels / pos_weight / lr");
  if (kf::net_grad(pooled, labels, n, h, w, pos_weight, ctx->net_wb, ctx->net_work, ctx->net_g, ctx->net_loss,
                   ctx->stream))
    return cuda_fail(ctx, cudaGetLastError(), "network gradient");
  ctx->net_step += 1;
  ++ctx->net_version;
  if (kf::net_adam(ctx->net_master, ctx->net_m, ctx->net_v, ctx->net_g, ctx->net_step, lr, ctx->net_wb, ctx->stream))
    return cuda_fail(ctx, cudaGetLastError(), "Adam");
  cudaError_t e;
  if (loss) {
    if ((e = cudaMemcpyAsync(loss, ctx->net_loss, sizeof(float), cudaMemcpyDeviceToHost, ctx->stream)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess)
      return cuda_fail(ctx, e, "copy loss");
  }
  return KF_OK;
}

int kf_proposal_labels(kf_ctx *ctx, double threshold, uint8_t *labels) {
  if (!ctx) return fail(nullptr, KF_EINVAL, "kf_proposal_labels: ctx is NULL");
  if (!labels || !ctx->have_result) return fail(ctx, KF_EINVAL, "kf_proposal_labels: no bank result / NULL output");
  if (!(threshold >= ctx->last_threshold))
    return fail(ctx, KF_EINVAL, "threshold %g is below the bank threshold %g", threshold, ctx->last_threshold);
  cudaError_t e;
  kf::DevStatus st;
  if ((e = cudaMemcpyAsync(&st, ctx->status, sizeof st, cudaMemcpyDeviceToHost, ctx->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess)
    return cuda_fail(ctx, e, "read status");
  if (st.error) return fail(ctx, KF_ETIMEOUT, "device wait gave up (code %d)", st.error);
  if (st.count > (unsigned long long)ctx->blob_cap)
    return fail(ctx, KF_ERERUN, "candidate list overflowed (%llu found): raise the capacity with kf_detect_blobs",
                (unsigned long long)st.count);
  const int nf = (int)ctx->last_H.size(), S = ctx->last_S;
  std::vector<long> loff(nf);
  std::vector<int> tw(nf), th(nf);
  long off = 0;
  for (int f = 0; f < nf; ++f) {
    th[f] = (ctx->last_H[f] + 63) / 64;
    tw[f] = (ctx->last_W[f] + 63) / 64;
    loff[f] = off;
    off += (long)S * th[f] * tw[f];
  }
  if (nf > ctx->lab_frames) {
    cudaFree(ctx->d_loff);
    cudaFree(ctx->d_ltw);
    cudaFree(ctx->d_lth);
    ctx->lab_frames = 0;
    if ((e = cudaMalloc(&ctx->d_loff, sizeof(long) * nf)) != cudaSuccess ||
        (e = cudaMalloc(&ctx->d_ltw, sizeof(int) * nf)) != cudaSuccess ||
        (e = cudaMalloc(&ctx->d_lth, sizeof(int) * nf)) != cudaSuccess)
      return cuda_fail(ctx, e, "cudaMalloc(labels)");
    ctx->lab_frames = nf;
  }
  if ((e = cudaMemcpyAsync(ctx->d_loff, loff.data(), sizeof(long) * nf, cudaMemcpyHostToDevice, ctx->stream)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(ctx->d_ltw, tw.data(), sizeof(int) * nf, cudaMemcpyHostToDevice, ctx->stream)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(ctx->d_lth, th.data(), sizeof(int) * nf, cudaMemcpyHostToDevice, ctx->stream)) !=
          cudaSuccess ||
      (e = cudaMemsetAsync(labels, 0, (size_t)off, ctx->stream)) != cudaSuccess)
    return cuda_fail(ctx, e, "labels");
  if (kf::net_labels(ctx->blobs, (long)st.count, (float)threshold, ctx->d_loff, ctx->d_ltw, ctx->d_lth, S, labels,
                     ctx->stream))
    return cuda_fail(ctx, cudaGetLastError(), "labels");
  // the host arrays above go out of scope: wait for their copies
  if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return cuda_fail(ctx, e, "labels");
  return KF_OK;
}

// add the launches (and, with events, the times) of the last bank call to the
// per-kernel lists; the stream must have been synchronised
static int collect_prof(kf_ctx *ctx, std::vector<std::string> &names, std::vector<int> &launches, std::vector<float> &ms) {
  cudaError_t e;
  const kf::Prof &p = ctx->prof;
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
  return KF_OK;
}

int kf_kernel_times(kf_ctx *ctx, kf_kernel_time *out, int cap, int *n) {
  if (!ctx) return fail(nullptr, KF_EINVAL, "kf_kernel_times: ctx is NULL");
  if (!n || cap < 0 || (cap > 0 && !out)) return fail(ctx, KF_EINVAL, "kf_kernel_times: bad outputs");
  if (!ctx->have_prof) return fail(ctx, KF_EINVAL, "kf_kernel_times: no bank call yet");
  cudaError_t e;
  if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return cuda_fail(ctx, e, "sync");
  std::vector<std::string> names;
  std::vector<int> launches;
  std::vector<float> ms;
  if (ctx->q_times_valid) {
    names = ctx->q_names;
    launches = ctx->q_launches;
    ms = ctx->q_ms;
  } else if (int rc = collect_prof(ctx, names, launches, ms)) {
    return rc;
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
  // A new threshold: order again (device-sized, enqueued without the count).
  if (!ctx->sorted_valid || ctx->sorted_thr != threshold) {
    int rc;
    const long nrows = (long)ctx->last_nframes * ctx->last_S * ctx->last_hmax;
    if ((rc = ensure_sort(ctx, nrows))) return rc;
    const int keybits = sort_keybits(ctx->last_nframes, ctx->last_S, ctx->last_hmax, ctx->last_wmax);
    kf::Prof none{};
    if (kf::launch_sort(ctx->blobs, ctx->blob_cap, &ctx->status->count, (float)threshold, ctx->last_S,
                        ctx->last_hmax, ctx->last_wmax, keybits, nrows, ctx->sort_work, ctx->sorted, ctx->d_npass,
                        &none,
                        ctx->stream))
      return cuda_fail(ctx, cudaGetLastError(), "sort launch");
    ctx->sorted_valid = true;
    ctx->sorted_thr = threshold;
    ctx->npass_read = false;
  }
  // One synchronisation for the status, the count and the records: until the
  // count is known, the first min(capacity, count_hint) records are copied
  // with them; a longer list is completed by a second copy.
  kf_ctx::HostRead *hr = ctx->h_read;
  if (!ctx->status_read &&
      (e = cudaMemcpyAsync(&hr->st, ctx->status, sizeof hr->st, cudaMemcpyDeviceToHost, ctx->stream)) != cudaSuccess)
    return cuda_fail(ctx, e, "read status");
  if (!ctx->npass_read && (e = cudaMemcpyAsync(&hr->npass, ctx->d_npass, sizeof hr->npass, cudaMemcpyDeviceToHost,
                                               ctx->stream)) != cudaSuccess)
    return cuda_fail(ctx, e, "read count");
  const int64_t first = std::min<int64_t>({capacity, ctx->npass_read ? (int64_t)ctx->sorted_n : ctx->count_hint,
                                           (int64_t)ctx->sorted_cap});
  static_assert(sizeof(kf_blob) == sizeof(kf::Blob), "record layout");
  if (first > 0 && (e = cudaMemcpyAsync(out, ctx->sorted, sizeof(kf::Blob) * first, cudaMemcpyDeviceToHost,
                                        ctx->stream)) != cudaSuccess)
    return cuda_fail(ctx, e, "copy blobs");
  if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return cuda_fail(ctx, e, "filter bank / ordering");
  if (!ctx->status_read) {
    ctx->last_status = hr->st;
    ctx->status_read = true;
  }
  const kf::DevStatus &st = ctx->last_status;
  if (st.error) return fail(ctx, KF_ETIMEOUT, "device wait gave up (code %d)", st.error);
  if (st.range)
    return fail(ctx, KF_ERANGE,
                "a stored plane value exceeded the f16 range: scale the input (value_scale) or use bf16/f32 storage");
  if (st.count > (unsigned long long)ctx->blob_cap) {
    *count = (int64_t)st.count;
    // grow for the next call; this call's list is incomplete
    drop_graphs(ctx);
    cudaFree(ctx->blobs);
    ctx->blobs = nullptr;
    long ncap = (long)st.count + (long)st.count / 4 + 1024;
    if ((e = cudaMalloc(&ctx->blobs, sizeof(kf::Blob) * ncap)) != cudaSuccess) {
      ctx->blob_cap = 0;
      return cuda_fail(ctx, e, "cudaMalloc(blobs)");
    }
    ctx->blob_cap = ncap;
    ctx->have_result = false;
    ctx->sorted_valid = false;
    return fail(ctx, KF_ERERUN,
                "candidate list overflowed (%llu found); capacity raised, run the bank again",
                (unsigned long long)st.count);
  }
  if (!ctx->npass_read) {
    ctx->sorted_n = (long)hr->npass;
    ctx->npass_read = true;
    ctx->count_hint = ctx->sorted_n + ctx->sorted_n / 8 + 1024;
  }
  *count = (int64_t)ctx->sorted_n;
  const int64_t all = std::min<int64_t>(capacity, ctx->sorted_n);
  if (all > first) {
    if ((e = cudaMemcpyAsync(out + first, ctx->sorted + first, sizeof(kf::Blob) * (all - first),
                             cudaMemcpyDeviceToHost, ctx->stream)) != cudaSuccess)
      return cuda_fail(ctx, e, "copy blobs");
    if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return cuda_fail(ctx, e, "copy blobs");
  }
  if (ctx->sorted_n > capacity)
    return fail(ctx, KF_EOVERFLOW, "capacity %lld < %lld blobs", (long long)capacity,
                (long long)ctx->sorted_n);
  return KF_OK;
}

int kf_quartic_bank(kf_ctx *ctx, const kf_frame *frame, const double *scales, int nscales, int type,
                    int order, float *out, int profile) {
  if (!ctx) return fail(nullptr, KF_EINVAL, "kf_quartic_bank: ctx is NULL");
  if (!frame || !out) return fail(ctx, KF_EINVAL, "kf_quartic_bank: frame and out must not be NULL");
  if (!scales || nscales < 1 || nscales > KF_MAX_SCALES)
    return fail(ctx, KF_EINVAL, "nscales must be 1..%d", KF_MAX_SCALES);
  // blurs flat at dc to order 4 (L_D = 2)
  if (type == KF_IIR_REPEATED_POLE) {
    if (order < 3 || order > 6)
      return fail(ctx, KF_EINVAL, "the D = 5 bank's repeated-pole order (L_D + Lbar_pi) must be 3..6 (got %d)", order);
  } else if (type == KF_IIR_BUTTERWORTH) {
    if (order < 3 || order > 6)
      return fail(ctx, KF_EINVAL, "the D = 5 bank's Butterworth order (L_B / 2) must be 3..6 (got %d)", order);
  } else if (type == KF_FIR_COLORED_SG) {
    if (order != 2) return fail(ctx, KF_EINVAL, "the D = 5 bank's colored SG blur needs L_D = 2 (got %d)", order);
  } else {
    return fail(ctx, KF_EINVAL, "the D = 5 bank needs a blur with vanishing moments (types 0, 1, 2; got %d)", type);
  }
  const int W = frame->width, H = frame->height;
  if (!frame->data || W < 1 || H < 1 || frame->pitch < W)
    return fail(ctx, KF_EINVAL, "kf_quartic_bank: bad frame %dx%d pitch %lld", W, H, (long long)frame->pitch);
  if (W > 8192) return fail(ctx, KF_EINVAL, "kf_quartic_bank: width > 8192");
  if (H > 65535) return fail(ctx, KF_EINVAL, "kf_quartic_bank: height > 65535");
  if (frame->dtype < KF_DTYPE_F32 || frame->dtype > KF_DTYPE_U16)
    return fail(ctx, KF_EINVAL, "kf_quartic_bank: unknown dtype %d", frame->dtype);
  if (!std::isfinite(frame->value_scale)) return fail(ctx, KF_EINVAL, "kf_quartic_bank: value_scale is not finite");
  if ((reinterpret_cast<uintptr_t>(frame->data) & (uintptr_t)(kf::in_bytes(frame->dtype) - 1)) != 0)
    return fail(ctx, KF_EINVAL, "kf_quartic_bank: data is not aligned to its element size");
  cudaError_t e;
  if ((e = cudaSetDevice(ctx->device)) != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  const int Hp = H + 4;
  const size_t npad = (size_t)W * Hp;
  int rc;
  if ((rc = grow(ctx, &ctx->q_pad, &ctx->q_pad_floats, npad * kf::QUARTIC_NCH, "D = 5 channel planes")))
    return rc;
  if ((rc = grow(ctx, &ctx->q_xpre, &ctx->q_xpre_floats, (size_t)4 * Hp * kf::QUARTIC_NCH, "D = 5 pre-rolls")))
    return rc;
  // recursive blurs: 32-row column segments unless the caller chose a length
  // (at the bank's few scales per call the shorter segments fit more blocks
  // per SM: 1.81 against 1.90 ms on a 2048^2 frame at four scales)
  struct Restore {
    kf_ctx *c;
    int type, lc;
    ~Restore() {
      c->q_chan = -1;
      c->q_ld = 1;
      c->q_out = nullptr;
      if (type >= 0) c->seg_len[type] = lc;
    }
  } restore{ctx, -1, 0};
  if ((type == KF_IIR_REPEATED_POLE || type == KF_IIR_BUTTERWORTH) && !ctx->seg_chosen[type] &&
      ctx->seg_len[type] != 32) {
    restore.type = type;
    restore.lc = ctx->seg_len[type];
    ctx->seg_len[type] = 32;
  }
  ctx->q_ld = type == KF_IIR_REPEATED_POLE ? 2 : 1;
  const float vs = frame->value_scale == 0.f ? 1.f : frame->value_scale;
  // the 15 channel planes are the frames of one bank call (one launch per pass)
  kf_frame pf[kf::QUARTIC_NCH];
  for (int c = 0; c < kf::QUARTIC_NCH; ++c) {
    pf[c] = kf_frame{};
    pf[c].data = ctx->q_pad + (size_t)c * npad;
    pf[c].width = W;
    pf[c].height = Hp;
    pf[c].pitch = W;
    pf[c].dtype = KF_DTYPE_F32;
    pf[c].value_scale = 1.f;
  }
  kf_bank_opts o;
  kf_bank_opts_default(&o);
  o.storage = KF_DTYPE_F32;
  o.graph = 0;
  o.gate = KF_GATE_OFF;
  // FIR blur: the FP32-FMA column pass (the one of the adjacent-scale
  // neighbourhood; raw planes are not detected, so the neighbourhood has no
  // other effect).  The tensor-core pass's three TF32 products carry about
  // 2^-21 of each tap product, and the fourth differences of a textured frame
  // are up to a thousand times larger than their blurred output.
  if (type == KF_FIR_COLORED_SG) o.neighbourhood = KF_NEIGH_ADJACENT;
  // profiling: every launch between a pair of events, the stream synchronised
  // after each, times summed per kernel over the channels
  ctx->q_times_valid = false;
  ctx->q_names.clear();
  ctx->q_launches.clear();
  ctx->q_ms.clear();
  o.profile = profile ? 1 : 0;
  if (profile)
    for (cudaEvent_t &ev : ctx->q_ev)
      if (!ev && (e = cudaEventCreate(&ev)) != cudaSuccess) return cuda_fail(ctx, e, "cudaEventCreate");
  auto timed = [&](const char *name, auto &&launch) -> int {
    if (profile) cudaEventRecord(ctx->q_ev[0], ctx->stream);
    if (launch()) return cuda_fail(ctx, cudaGetLastError(), name);
    if (!profile) return KF_OK;
    cudaEventRecord(ctx->q_ev[1], ctx->stream);
    float t = 0.f;
    if ((e = cudaEventSynchronize(ctx->q_ev[1])) != cudaSuccess ||
        (e = cudaEventElapsedTime(&t, ctx->q_ev[0], ctx->q_ev[1])) != cudaSuccess)
      return cuda_fail(ctx, e, "profile events");
    size_t k = std::find(ctx->q_names.begin(), ctx->q_names.end(), std::string(name)) - ctx->q_names.begin();
    if (k == ctx->q_names.size()) {
      ctx->q_names.push_back(name);
      ctx->q_launches.push_back(0);
      ctx->q_ms.push_back(0.f);
    }
    ctx->q_launches[k] += 1;
    ctx->q_ms[k] += t;
    return KF_OK;
  };
  if ((rc = timed("quartic_hpf", [&] {
         return kf::launch_hpf5(frame->data, frame->dtype, vs, (long)frame->pitch, W, H, ctx->q_pad, ctx->q_xpre,
                                ctx->stream);
       })))
    return rc;
  // the column passes write D (the identity channel carries no sigma^2)
  // straight into out, without the two padding rows at each end
  ctx->q_chan = kf::CH_ID;
  ctx->q_out = out;
  ctx->q_H = H;
  ctx->q_W = W;
  if ((rc = kf_filter_bank(ctx, pf, kf::QUARTIC_NCH, scales, nscales, type, order, &o))) return rc;
  if (profile) {
    if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return cuda_fail(ctx, e, "sync");
    if ((rc = collect_prof(ctx, ctx->q_names, ctx->q_launches, ctx->q_ms))) return rc;
  }
  ctx->have_result = false;  // the bank ran raw planes: no blob list
  ctx->q_times_valid = profile != 0;
  return KF_OK;
}

int kf_quartic_steer(kf_ctx *ctx, const float *in, int64_t npix, int nsets, double phi, float *out) {
  if (!ctx) return fail(nullptr, KF_EINVAL, "kf_quartic_steer: ctx is NULL");
  if (!in || !out || npix < 1 || nsets < 1 || !std::isfinite(phi))
    return fail(ctx, KF_EINVAL, "kf_quartic_steer: bad arguments");
  // Per order n: the coefficient of x^(n-a) y^a in the expansion of
  // (x cos + y sin)^(n-b) (-x sin + y cos)^b, as polynomials in y with x
  // implied, scaled from beta to D by (n-a)! a! / ((n-b)! b!).
  const double cph = std::cos(phi), sph = std::sin(phi);
  float m55[55];
  int mb = 0;
  for (int n = 0; n <= 4; ++n) {
    for (int b = 0; b <= n; ++b) {
      double poly[5] = {1.0, 0.0, 0.0, 0.0, 0.0};  // coefficient of y^k
      int deg = 0;
      auto times = [&](double cx, double cy) {  // poly *= (cx x + cy y)
        for (int k = deg + 1; k >= 0; --k) poly[k] = cx * poly[k] + (k > 0 ? cy * poly[k - 1] : 0.0);
        ++deg;
      };
      for (int i = 0; i < n - b; ++i) times(cph, sph);
      for (int i = 0; i < b; ++i) times(-sph, cph);
      for (int a = 0; a <= n; ++a) {
        double fa = 1.0, fb = 1.0;
        for (int k = 2; k <= n - a; ++k) fa *= k;
        for (int k = 2; k <= a; ++k) fa *= k;
        for (int k = 2; k <= n - b; ++k) fb *= k;
        for (int k = 2; k <= b; ++k) fb *= k;
        m55[mb + a * (n + 1) + b] = (float)(poly[a] * fa / fb);
      }
    }
    mb += (n + 1) * (n + 1);
  }
  cudaError_t e;
  if ((e = cudaSetDevice(ctx->device)) != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  if (kf::launch_steer(in, (long)npix, nsets, m55, out, ctx->stream))
    return cuda_fail(ctx, cudaGetLastError(), "steering launch");
  return KF_OK;
}

int kf_blob_shapes(kf_ctx *ctx, double threshold, kf_blob_shape *out, int64_t capacity, int64_t *count) {
  if (!ctx) return fail(nullptr, KF_EINVAL, "kf_blob_shapes: ctx is NULL");
  if (!count || capacity < 0 || (capacity > 0 && !out))
    return fail(ctx, KF_EINVAL, "kf_blob_shapes: bad output arguments");
  if (!ctx->have_result || !ctx->have_dplanes)
    return fail(ctx, KF_EINVAL,
                "kf_blob_shapes: the last bank call did not run the derivative bank (KF_RESP_HESSIAN or offset_limit)");
  // the ordered list at this threshold and its count (no records copied)
  int64_t n = 0;
  int rc = kf_detect_blobs(ctx, threshold, nullptr, 0, &n);
  if (rc != KF_OK && rc != KF_EOVERFLOW) return rc;
  *count = n;
  if (n == 0) return KF_OK;
  cudaError_t e;
  if (ctx->d_dlay_n < ctx->dlay.size()) {
    cudaFree(ctx->d_dlay);
    ctx->d_dlay = nullptr;
    ctx->d_dlay_n = 0;
    if ((e = cudaMalloc(&ctx->d_dlay, sizeof(long) * ctx->dlay.size())) != cudaSuccess)
      return cuda_fail(ctx, e, "cudaMalloc(shape layout)");
    ctx->d_dlay_n = ctx->dlay.size();
  }
  if ((rc = grow(ctx, &ctx->shape_buf, &ctx->shape_floats, (size_t)4 * ctx->blob_cap, "shapes"))) return rc;
  if ((e = cudaMemcpyAsync(ctx->d_dlay, ctx->dlay.data(), sizeof(long) * ctx->dlay.size(), cudaMemcpyHostToDevice,
                           ctx->stream)) != cudaSuccess)
    return cuda_fail(ctx, e, "shape layout");
  const float *c20 = ctx->ch_buf, *c02 = ctx->ch_buf + ctx->dplane_per, *c11 = ctx->ch_buf + 2 * ctx->dplane_per;
  if (kf::launch_shapes(ctx->sorted, (long)n, c20, c02, c11, ctx->d_dlay, ctx->cur->d_coef, ctx->shape_buf,
                        ctx->stream))
    return cuda_fail(ctx, cudaGetLastError(), "shape launch");
  static_assert(sizeof(kf_blob_shape) == 4 * sizeof(float), "shape record layout");
  const int64_t ncopy = std::min<int64_t>(capacity, n);
  if (ncopy > 0 && (e = cudaMemcpyAsync(out, ctx->shape_buf, sizeof(kf_blob_shape) * ncopy, cudaMemcpyDeviceToHost,
                                        ctx->stream)) != cudaSuccess)
    return cuda_fail(ctx, e, "copy shapes");
  if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return cuda_fail(ctx, e, "shapes");
  if (n > capacity) return fail(ctx, KF_EOVERFLOW, "capacity %lld < %lld shapes", (long long)capacity, (long long)n);
  return KF_OK;
}

}  // extern "C"
