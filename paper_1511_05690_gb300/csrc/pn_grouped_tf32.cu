// TF32 / 3xTF32 instantiations of the persistent grouped kernel.
#include "pn_grouped_kernel.cuh"

namespace pn {

int grouped_persist_tf32(const Common& cm, const GroupedRun& gr, int sms, void* stream) {
  if (cm.mode == MODE_3XTF32) return gemm::launch_grouped_persist_t<MODE_3XTF32, 128>(cm, gr, sms, stream, gr.plain != 0);
  return cm.BN == 256 ? gemm::launch_grouped_persist_t<MODE_TF32, 256>(cm, gr, sms, stream, gr.plain != 0)
                      : gemm::launch_grouped_persist_t<MODE_TF32, 128>(cm, gr, sms, stream, gr.plain != 0);
}

}  // namespace pn
