// kf_iir.cu -- host side of the recursive banks: work items of the passes and
// the dispatch to the Filter D (kf_iir_d.cu) and Filter E (kf_iir_e.cu)
// instances of the kernels in kf_iir_kernels.cuh.
#include "kf_common.cuh"
#include "kf_internal.h"

namespace kf {

int run_iir_chain(int K, const Plan &p, const BankArgs &a, cudaStream_t st);  // kf_iir_d.cu
int run_iir_modes(int NM, const Plan &p, const BankArgs &a, cudaStream_t st);  // kf_iir_e.cu

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

int launch_iir(const Plan &p, const BankArgs &a, cudaStream_t st) {
  if (a.type == T_D) return run_iir_chain(a.nstate, p, a, st);
  if (a.type == T_E) return run_iir_modes(a.nstate, p, a, st);
  return -2;
}

}  // namespace kf
