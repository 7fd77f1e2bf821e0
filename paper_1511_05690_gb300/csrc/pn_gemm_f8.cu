// FP8 E4M3 operand instantiations of the tensor-core level kernel.
#include "pn_gemm_kernel.cuh"

namespace pn {

int gemm_launch_f8(int mode, int BN, const Common& cm, const Level& lv, int sms, void* stream) {
  (void)mode;
  if (cm.cg == 2)
    return BN == 256 ? gemm::launch_pair_t<MODE_E4M3, 256>(cm, lv, sms, stream)
                     : gemm::launch_pair_t<MODE_E4M3, 128>(cm, lv, sms, stream);
  return BN == 256 ? gemm::launch_t<MODE_E4M3, 256>(cm, lv, sms, stream)
                   : gemm::launch_t<MODE_E4M3, 128>(cm, lv, sms, stream);
}

}  // namespace pn
