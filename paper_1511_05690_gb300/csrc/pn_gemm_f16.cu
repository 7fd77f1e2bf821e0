// BF16 / FP16 operand instantiations of the tensor-core level kernel.
#include "pn_gemm_kernel.cuh"

namespace pn {

int gemm_launch_f16(int mode, int BN, const Common& cm, const Level& lv, int sms, void* stream) {
  if (cm.cg == 2)
    return mode == MODE_BF16
               ? (BN == 256 ? gemm::launch_pair_t<MODE_BF16, 256>(cm, lv, sms, stream)
                            : gemm::launch_pair_t<MODE_BF16, 128>(cm, lv, sms, stream))
               : (BN == 256 ? gemm::launch_pair_t<MODE_F16, 256>(cm, lv, sms, stream)
                            : gemm::launch_pair_t<MODE_F16, 128>(cm, lv, sms, stream));
  if (mode == MODE_BF16)
    return BN == 256 ? gemm::launch_t<MODE_BF16, 256>(cm, lv, sms, stream)
                     : gemm::launch_t<MODE_BF16, 128>(cm, lv, sms, stream);
  return BN == 256 ? gemm::launch_t<MODE_F16, 256>(cm, lv, sms, stream)
                   : gemm::launch_t<MODE_F16, 128>(cm, lv, sms, stream);
}

}  // namespace pn
