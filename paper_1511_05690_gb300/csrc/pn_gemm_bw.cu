// Gradient-epilogue instantiations of the tensor-core level kernel (the two
// GEMMs per p of maxprod_pnorm_backward).
#include "pn_gemm_kernel.cuh"

namespace pn {

int launch_gemm_grad(const Common& cm, const Level& lv, int sms, void* stream) {
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
