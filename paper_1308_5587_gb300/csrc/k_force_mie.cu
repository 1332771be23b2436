// k_force_mie.cu -- the Mie instances of the pair-force gather (k_force.cuh).
#include "k_force.cuh"

namespace gbmd {

void* k_force_variant_mie(int prec, int tpp, int mt, int mode) {
  return k_force_variant<EVAL_MIE>(prec, tpp, mt, mode);
}

}  // namespace gbmd
