// kf_iir_e.cu -- Filter E (discrete Butterworth, Sec. 4.4): the recursive-bank
// kernels instantiated for 1..3 complex one-pole modes.
#include "kf_iir_kernels.cuh"

namespace kf {

int run_iir_modes(int NM, const Plan &p, const BankArgs &a, cudaStream_t st) {
  switch (NM) {
    case 1: return run_iir<Modes<1>>(p, a, st);
    case 2: return run_iir<Modes<2>>(p, a, st);
    case 3: return run_iir<Modes<3>>(p, a, st);
    default: return -2;
  }
}

bool iir_scan_fits_modes(int NM, int storage, int S, int maxH) {
  switch (NM) {
    case 1: return colscan_fits_st<Modes<1>>(storage, S, maxH);
    case 2: return colscan_fits_st<Modes<2>>(storage, S, maxH);
    case 3: return colscan_fits_st<Modes<3>>(storage, S, maxH);
    default: return false;
  }
}

}  // namespace kf
