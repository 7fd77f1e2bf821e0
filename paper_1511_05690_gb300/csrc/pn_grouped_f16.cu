// BF16 / FP16 instantiations of the persistent grouped kernel.
#include "pn_grouped_kernel.cuh"

namespace pn {

int grouped_persist_f16(const Common& cm, const GroupedRun& gr, int sms, void* stream) {
  if (cm.mode == MODE_BF16)
    return cm.BN == 256 ? gemm::launch_grouped_persist_t<MODE_BF16, 256>(cm, gr, sms, stream, gr.plain != 0)
                        : gemm::launch_grouped_persist_t<MODE_BF16, 128>(cm, gr, sms, stream, gr.plain != 0);
  return cm.BN == 256 ? gemm::launch_grouped_persist_t<MODE_F16, 256>(cm, gr, sms, stream, gr.plain != 0)
                      : gemm::launch_grouped_persist_t<MODE_F16, 128>(cm, gr, sms, stream, gr.plain != 0);
}

}  // namespace pn
