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

}  // namespace kf
