// Gradient-epilogue instantiations of the tensor-core level kernel (the two
// GEMMs per p of maxprod_pnorm_backward), on one CTA or a CTA pair per tile.
#include "pn_gemm_kernel.cuh"

namespace pn {

int launch_gemm_grad(const Common& cm, const Level& lv, int sms, void* stream) {
  if (cm.cg == 2) {  // CTA pairs on 256 x 256 tiles
    if (cm.BN != 256) return cudaErrorInvalidValue;
    switch (cm.mode) {
      case MODE_3XTF32: return gemm::launch_pair_t<MODE_3XTF32, 256, 1>(cm, lv, sms, stream);
      case MODE_TF32: return gemm::launch_pair_t<MODE_TF32, 256, 1>(cm, lv, sms, stream);
      case MODE_BF16: return gemm::launch_pair_t<MODE_BF16, 256, 1>(cm, lv, sms, stream);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (cm.mode) {
    case MODE_3XTF32: return gemm::launch_t<MODE_3XTF32, 128, 1>(cm, lv, sms, stream);
    case MODE_TF32:
      return cm.BN == 256 ? gemm::launch_t<MODE_TF32, 256, 1>(cm, lv, sms, stream)
                          : gemm::launch_t<MODE_TF32, 128, 1>(cm, lv, sms, stream);
    case MODE_BF16:
      return cm.BN == 256 ? gemm::launch_t<MODE_BF16, 256, 1>(cm, lv, sms, stream)
                          : gemm::launch_t<MODE_BF16, 128, 1>(cm, lv, sms, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pn
