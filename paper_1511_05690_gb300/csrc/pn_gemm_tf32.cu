// TF32 and 3xTF32 (FP32-accurate) operand instantiations of the tensor-core
// level kernel.  3xTF32 carries a second (lo) operand plane and only fits
// 128-wide tiles.
#include "pn_gemm_kernel.cuh"

namespace pn {

int gemm_launch_tf32(int mode, int BN, const Common& cm, const Level& lv, int sms, void* stream) {
  if (cm.cg == 2)
    return mode == MODE_3XTF32
               ? (BN == 256 ? gemm::launch_pair_t<MODE_3XTF32, 256>(cm, lv, sms, stream)
                            : gemm::launch_pair_t<MODE_3XTF32, 128>(cm, lv, sms, stream))
               : (BN == 256 ? gemm::launch_pair_t<MODE_TF32, 256>(cm, lv, sms, stream)
                            : gemm::launch_pair_t<MODE_TF32, 128>(cm, lv, sms, stream));
  if (mode == MODE_3XTF32) return gemm::launch_t<MODE_3XTF32, 128>(cm, lv, sms, stream);
  return BN == 256 ? gemm::launch_t<MODE_TF32, 256>(cm, lv, sms, stream)
                   : gemm::launch_t<MODE_TF32, 128>(cm, lv, sms, stream);
}

}  // namespace pn
