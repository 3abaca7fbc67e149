// kf_internal.h -- host-side declarations shared by the library's translation
// units (launchers of the CUDA kernels).  Not part of the C ABI.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <vector>

#include "kf_batch.cuh"
#include "kf_common.cuh"

namespace kf {

// FP64 design of S scales into d_out (device array of S Coef).  d_work holds
// S * 2 (Nmax^2 + Nmax) doubles (double-double KKT matrix and right-hand side
// of the colored-SG design).  ld: L_D of a Filter D design (1: the D = 3
// bank; 2: D = 5); the other types take L_D from `order`.
int launch_design(int type, int order, const double *d_lambdas, int S, int fir_kmax, Coef *d_out,
                  double *d_work, int Nmax, cudaStream_t st, int ld = 1);

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

// Tensor-core FIR column pass (kf_fir_tc.cu): per scale (<= 8) the taps as a
// banded Toeplitz operand for MMAs of NR output rows; K half-length, Kp = K
// rounded up to 4, Kd = NR + 2 Kp input rows, G band chunks of 128 bytes
// (per hi and lo part), boff the float offset of the scale's hi band in the
// band buffer (its lo band follows G x 32 floats later).
constexpr int TC_MAXS = 8;
struct TcGeom {
  int S = 0;
  int NR = 64;  // output rows per tile (64 for <= 6 scales, else 32)
  int K[TC_MAXS] = {}, Kp[TC_MAXS] = {}, Kd[TC_MAXS] = {}, G[TC_MAXS] = {};
  long boff[TC_MAXS] = {};
  int gmax = 0;
  long floats = 0;
};

// FIR row pass: the call's scales ordered by half-length (largest first) in
// groups of three that share the pair sums x(j - k) + x(j + k), and the
// grouped tap table: entry g * TK + k holds h_k of the group's three scales
// (four floats, the fourth zero; zero beyond a scale's K).  Built on the host
// from the design (kf_fir.cu).
constexpr int ROW_GS = 3;
constexpr int ROW_MAXS = 16;
struct RowGroups {
  int S = 0, NG = 0, TK = 0;
  int ord[ROW_MAXS] = {};       // scales by K, largest first (stable)
  int K[ROW_MAXS + 2] = {};     // half-length of group slot i (-1: empty)
};
// fills g and the table (4 x NG x TK floats); returns its length in floats
long row_groups(const Coef *h_coef, int S, RowGroups *g, std::vector<float> *table);

struct BankArgs {
  const Coef *coef;      // device, S entries
  int S;
  int type, nstate;      // filter type; D: chain length, E: number of modes
  int kmax;              // FIR: largest half-length over the scales
  float threshold;
  int neigh;
  void *P;               // the plane row space: prows x PWb, element type `storage`
  int storage;           // ST_F32 / ST_F16 / ST_BF16
  float *edge;           // per frame S x 2 x PWb: one-sided rows for the column boundary
  float *carry;          // per frame S x nseg x 2 x NF x PWb (IIR column carries)
  Blob *blobs;
  long cap;
  DevStatus *status;
  Prof *prof;            // launch bookkeeping (never null)
  int chan = CH_LAP;     // derivative channel of the row pass (CH_*)
  int raw = 0;           // 1: column passes write +sigma^2 D of the channel, no detection
  float *raw_out = nullptr;  // raw channel planes (per frame S x H x W at the frame's response offset)
  // failure-detection test hook (kf_set_wait_limit): > 0, the column pass
  // issues no copy to its load barrier and gives up after this many polls
  unsigned wait_test = 0;
  // FIR banks: 1 for the zero boundary (the frame extended by zeros: the
  // Laplacian is nonzero one pixel beyond the edges, the column passes take
  // the blurred first / last input row one row beyond and zero further out);
  // 0 for the hold boundary
  int zero = 0;
  // tensor-core FIR column pass: the design's taps as band operands (device)
  // and their geometry; null: the pass does not apply to this call
  const float *tc_bands = nullptr;
  TcGeom tc;
  // FIR row pass: the design's grouped tap table (device) and its groups
  const float *row_taps = nullptr;
  RowGroups rg;
  // single-read IIR column pass (k_colscan): scratch of the launch (ticket,
  // publication flags, the super-tiles' end states and carries); null: the
  // segment passes (k_colseg, k_colfold, k_coldet) run instead
  void *scan = nullptr;
  // gated calls: the active-tile maps of the frames (FrameDev.aoff); null
  // otherwise
  const unsigned char *gate_act = nullptr;
};

// Passes of the banks.  IIR: row (with the two edge rows per frame), column
// segment states, carry fold, column pass + detector.  FIR: row, column +
// detector.
enum Pass { PASS_ROW = 0, PASS_SEG = 1, PASS_FOLD = 2, PASS_DET = 3, NPASS = 4 };

// one launch of a pass: its frames and items (device pointers into the call's
// table) and, for the IIR row pass, the threads per block of its width class
struct Launch {
  Items it;
  int nt = 0;
};

struct Plan {
  const FrameDev *fr = nullptr;  // device frame table
  int nframes = 0;
  long PWb = 0;                  // plane pitch (elements)
  long prows = 0;                // rows of the plane row space
  int maxW = 0, maxH = 0;
  bool per_frame = false;        // launch every pass frame by frame
  int mult[NPASS] = {0, 0, 0, 0}; // launch shape per pass (see persistent_blocks)
  Launch comb;                    // derivative bank: the combine + detect launch
  int lc = 64;                    // IIR column segment length (32 or 64 rows)
  std::vector<Launch> pass[NPASS];
  std::vector<Launch> scan;       // IIR single-read column pass: one launch (per frame, if per_frame)
};

// work items of one frame in a pass (the kernels' decomposition)
int iir_items(int pass, int H, int W, int S, int lc);
int iir_row_threads(int W);    // threads per block of the IIR row pass (0: too wide)
int fir_items(int pass, int H, int W, int S, int neigh, bool tc = false);  // tc: the tensor-core column pass
// tensor-core FIR column pass (kf_fir_tc.cu): whether it serves a call (f32
// planes, all-scales neighbourhood, <= 8 scales, detection, a plane row
// space of at least 68 x 32 elements), its tiles' interior width, the band geometry of a design (floats of the band buffer,
// -1 if it does not apply), the band builder and the launch
bool fir_tc_applies(int S, int storage, int neigh, int raw, long PWb, long prows);
int fir_tc_tile_cols();
int fir_tc_tile_rows(int S);
long tc_geometry(const int *K, int S, TcGeom *g);
int launch_tc_bands(const Coef *d_coef, const TcGeom &g, float sgn, float *d_bands, cudaStream_t st);
int launch_colfir_tc(const Plan &p, const Launch &l, const BankArgs &a, const struct DetectArgs &da,
                     cudaStream_t st);
int iir_segments(int H, int lc);  // IIR column segments of a frame (segment length lc)
// single-read IIR column pass: super-tiles of a frame, bytes of the launch
// scratch for U super-tiles, and whether the pass can serve a call (every
// super-tile of the tallest frame's strips resident at once)
int iir_scan_items(int H, int W);
size_t iir_scan_bytes(long U, int S, int nf);
bool iir_scan_fits(int type, int nstate, int storage, int S, int maxH);

int launch_iir(const Plan &p, const BankArgs &a, cudaStream_t st);
// derivative bank: tiles of 30 x 30 per frame; R (R_H or R_L) from the
// channel planes and the detector (kf_deriv.cu)
int deriv_items(int H, int W);
int launch_combine_detect(const Plan &p, const Launch &l, const BankArgs &a, int hessian, const float *c20,
                          const float *c02, const float *c11, const float *c10, const float *c01, float limit2,
                          cudaStream_t st);
int launch_fir(const Plan &p, const BankArgs &a, cudaStream_t st);

// 2-D tensor map over the plane row space (x, plane row), element type
// `storage`, box boxw x boxh (kf_fir.cu)
int encode_plane_map(CUtensorMap *m, void *P, int storage, long PWb, long prows, int boxw, int boxh);

// blocks of a launch over `items` work items: mult = 0, one block per item;
// mult = k >= 1, at most k x the blocks of this kernel and block shape that are
// resident on the whole GPU at once (each block loops over items); mult = -b,
// b blocks per SM (at most the resident limit) so that kernels of other
// streams keep the rest of every SM
int persistent_blocks(const void *kernel, int threads, size_t smem, int items, int mult);

// proposal network (kf_proposal.cu): flat parameters W1 b1 W2 b2 W3 b3
constexpr int NET_NPARAM = 3640;
size_t net_work_floats(int N, int h, int w);
int net_pool(const void *X, int dtype, float vs, long xpitch, int H, int W, float *out, cudaStream_t st);
int net_forward(const float *x, int N, int h, int w, const __nv_bfloat16 *wb, float *work, float *z_out,
                cudaStream_t st);
int net_grad(const float *x, const unsigned char *t, int N, int h, int w, float pw, const __nv_bfloat16 *wb,
             float *work, float *g, float *loss_dev, cudaStream_t st);
int net_adam(float *master, float *m, float *v, const float *g, int step, float lr, __nv_bfloat16 *wb,
             cudaStream_t st);
int net_to_bf16(const float *x, __nv_bfloat16 *y, cudaStream_t st);
int net_labels(const Blob *b, long n, float thr, const long *loff, const int *ltw, const int *lth, int S,
               unsigned char *lab, cudaStream_t st);
// gating: active-tile map of one frame from its logits; selection of the
// items of a column pass (interior tiles tw x th) or of the FIR row pass
int net_pool_table(const FrameDev *fr, int f, int H, int W, float *out, cudaStream_t st);
int gate_tiles(const float *z, int S, int th, int tw, float zthr, int dilate, unsigned char *act,
               cudaStream_t st);
int gate_select_tiles(const FrameDev *fr, const Items &full, const unsigned char *act, int tw, int th, int2 *sel,
                      int *count, cudaStream_t st);
int gate_select_rows(const FrameDev *fr, const Items &full, const unsigned char *act, int rseg, int rrows,
                     int reach, int2 *sel, int *count, cudaStream_t st);
// geometry of the gated passes
int fir_row_segment();         // outputs per row of a FIR row item
int fir_row_rows();            // rows of a FIR row item (items past the frame rows: its two U-only edge rows)
int fir_tile_rows(int neigh);  // interior rows of a FIR column tile
int fir_halo(int kmax);        // rows a FIR column tile reads beyond its 128 (or 64) rows

// shape descriptors of an ordered blob list from the derivative-bank planes
// (kf_deriv.cu); lay: per frame (plane offset, H, W); out: n float4 records
// (p1, p2, theta, |H|)
int launch_shapes(const Blob *b, long n, const float *c20, const float *c02, const float *c11, const long *lay,
                  const Coef *coef, void *out, cudaStream_t st);

// D = 5 derivative bank (kf_quartic.cu): the 15 differentiated channels of a
// frame on the frame padded by 2 rows (f32 planes of pitch W and H + 4 rows,
// one after the other) and, per plane row, the values 2 and 1 pixels before
// and 1 and 2 after the row (xpre, 4 floats); the steering of 15-channel sets (m55: per order n =
// 0..4 an (n+1) x (n+1) row-major block)
int launch_hpf5(const void *X, int dtype, float vs, long pitch, int W, int H, float *out, float *xpre,
                cudaStream_t st);
int launch_steer(const float *in, long npix, int nsets, const float *m55, float *out, cudaStream_t st);

// failure-detection test hook of kf_responses_noalloc (kf_noalloc.cu)
void set_noalloc_wait_test(unsigned polls);

// candidate ordering (kf_sort.cu)
size_t sort_workspace_bytes(long cap, long nrows);
int launch_sort(const Blob *blobs, long cap, const unsigned long long *count, float thr, int nscales, long hmax,
                long wmax, int keybits, long nrows, void *work, Blob *out, unsigned *d_npass, Prof *prof,
                cudaStream_t st);

}  // namespace kf
