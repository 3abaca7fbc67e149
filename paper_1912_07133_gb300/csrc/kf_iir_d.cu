// kf_iir_d.cu -- Filter D (repeated pole, Sec. 4.3): the recursive-bank
// kernels instantiated for first-order-section chains of 2..6 stages.
#include "kf_iir_kernels.cuh"

namespace kf {

int run_iir_chain(int K, const Plan &p, const BankArgs &a, cudaStream_t st) {
  switch (K) {
    case 2: return run_iir<Chain<2>>(p, a, st);
    case 3: return run_iir<Chain<3>>(p, a, st);
    case 4: return run_iir<Chain<4>>(p, a, st);
    case 5: return run_iir<Chain<5>>(p, a, st);
    case 6: return run_iir<Chain<6>>(p, a, st);
    default: return -2;
  }
}

bool iir_scan_fits_chain(int K, int storage, int S, int maxH) {
  switch (K) {
    case 2: return colscan_fits_st<Chain<2>>(storage, S, maxH);
    case 3: return colscan_fits_st<Chain<3>>(storage, S, maxH);
    case 4: return colscan_fits_st<Chain<4>>(storage, S, maxH);
    case 5: return colscan_fits_st<Chain<5>>(storage, S, maxH);
    case 6: return colscan_fits_st<Chain<6>>(storage, S, maxH);
    default: return false;
  }
}

}  // namespace kf
