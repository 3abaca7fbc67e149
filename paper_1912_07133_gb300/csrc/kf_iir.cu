// kf_iir.cu -- host side of the recursive banks: work items of the passes and
// the dispatch to the Filter D (kf_iir_d.cu) and Filter E (kf_iir_e.cu)
// instances of the kernels in kf_iir_kernels.cuh.
#include "kf_common.cuh"
#include "kf_internal.h"

namespace kf {

int run_iir_chain(int K, const Plan &p, const BankArgs &a, cudaStream_t st);  // kf_iir_d.cu
int run_iir_modes(int NM, const Plan &p, const BankArgs &a, cudaStream_t st);  // kf_iir_e.cu
bool iir_scan_fits_chain(int K, int storage, int S, int maxH);                 // kf_iir_d.cu
bool iir_scan_fits_modes(int NM, int storage, int S, int maxH);                // kf_iir_e.cu

int iir_segments(int H, int lc) { return (H + lc - 1) / lc; }

int iir_row_threads(int W) {
  const int nt = ((W + CH - 1) / CH + 31) / 32 * 32;
  return nt <= 256 ? nt : 0;
}

int iir_items(int pass, int H, int W, int S, int lc) {
  const int nxb = (W + 127) / 128, nseg = iir_segments(H, lc);
  switch (pass) {
    case PASS_ROW: return H + 2;
    case PASS_SEG: return nxb * nseg * S;
    case PASS_FOLD: return nxb * S * 2;
    case PASS_DET: return ((W + TW - 1) / TW) * nseg;
    default: return 0;
  }
}

// single-read column pass (k_colscan in kf_iir_kernels.cuh): super-tiles of
// 8 tiles of 32 rows in strips of 30 interior columns
int iir_scan_items(int H, int W) {
  const int nt = (H + 31) / 32;
  return ((W + TW - 1) / TW) * ((nt + 7) / 8);
}

// ticket (32 ints) and flags (2 per super-tile), then per super-tile and
// direction its zero-state end state (nf x S x 32 floats)
size_t iir_scan_bytes(long U, int S, int nf) {
  const size_t head = ((32 + 2 * (size_t)U) * 4 + 255) / 256 * 256;
  return head + (size_t)U * 2 * nf * S * 32 * sizeof(float);
}

bool iir_scan_fits(int type, int nstate, int storage, int S, int maxH) {
  if (S < 1 || S > MAXS) return false;
  if (type == T_D) return iir_scan_fits_chain(nstate, storage, S, maxH);
  if (type == T_E) return iir_scan_fits_modes(nstate, storage, S, maxH);
  return false;
}

int launch_iir(const Plan &p, const BankArgs &a, cudaStream_t st) {
  if (a.type == T_D) return run_iir_chain(a.nstate, p, a, st);
  if (a.type == T_E) return run_iir_modes(a.nstate, p, a, st);
  return -2;
}

}  // namespace kf
