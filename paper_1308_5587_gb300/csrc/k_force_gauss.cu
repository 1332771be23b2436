// k_force_gauss.cu -- the Gaussian instances of the pair-force gather (k_force.cuh).
#include "k_force.cuh"

namespace gbmd {

void* k_force_variant_gauss(int prec, int tpp, int mt, int mode) {
  return k_force_variant<EVAL_GAUSS>(prec, tpp, mt, mode);
}

}  // namespace gbmd
