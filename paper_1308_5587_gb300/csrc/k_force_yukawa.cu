// k_force_yukawa.cu -- the Yukawa instances of the pair-force gather (k_force.cuh).
#include "k_force.cuh"

namespace gbmd {

void* k_force_variant_yukawa(int prec, int tpp, int mt, int mode) {
  return k_force_variant<EVAL_YUKAWA>(prec, tpp, mt, mode);
}

}  // namespace gbmd
