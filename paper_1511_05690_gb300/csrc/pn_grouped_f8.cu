// FP8 E4M3 instantiations of the persistent grouped kernel.
#include "pn_grouped_kernel.cuh"

namespace pn {

int grouped_persist_f8(const Common& cm, const GroupedRun& gr, int sms, void* stream) {
  return cm.BN == 256 ? gemm::launch_grouped_persist_t<MODE_E4M3, 256>(cm, gr, sms, stream, gr.plain != 0)
                      : gemm::launch_grouped_persist_t<MODE_E4M3, 128>(cm, gr, sms, stream, gr.plain != 0);
}

}  // namespace pn
