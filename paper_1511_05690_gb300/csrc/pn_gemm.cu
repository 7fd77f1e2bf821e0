// Ring GEMM H of the p-norm product (Alg. 5: H^(p) = A'^p B'^p, here a
// tcgen05 tensor-core GEMM) with the stable-p estimate fused into the
// epilogue (Alg. 5 second loop; Sec. 2.1, plain
// estimateMaxFromNormPowerSequence).
//
// One launch handles one p of the family, largest p first.  Because every
// scaled term is <= 1, S^(p) is non-increasing in p, so the stable set of an
// entry is a prefix of P and its largest stable p is the first p, going
// down, with S^(p) >= tau.  The top launch computes every output tile; an
// entry that is stable there is final.  A tile that still has unstable
// entries is pushed to the next lower level's work list together with a bit
// mask of its resolved entries, and only those tiles are recomputed at the
// next p.  The smallest p resolves whatever is left (flagged unstable).
//
// Kernel structure (one persistent CTA per SM, 10 warps; or a CTA pair per
// 256 x BN tile, cta_group::2):
//   warp 0      one thread issues copies of pre-swizzled 16 KB operand tile
//               images into a STAGES-deep shared-memory ring (192 KB): 1-D
//               bulk copies, or for a pair 2-D tensor copies completing on
//               rank 0's barrier;
//   warp 1      allocates TMEM (all 512 columns: 512 / BN accumulators of
//               128 x BN FP32) and one thread issues tcgen05.mma (M = 128,
//               or 256 over a pair; N = BN; 32 bytes of K each);
//   warps 2-9   epilogue: tcgen05.ld of the accumulator (lane = output row),
//               tau test, root, un-scaling, and stores staged through a 4 KB
//               shared buffer per warp so that global writes are whole
//               128-byte rows.  Where the epilogue bounds a tile (grouped
//               problems, short contractions) the eight warps form two
//               groups that finish alternate tiles, one per accumulator;
//               otherwise all eight finish every tile on half the columns
//               each.  The projection estimators (Sec. 2.1) park sums in C
//               and the workspace and finish them at a lower level, walking
//               each warp's 32 x 32 block row by row.
// The accumulators rotate so the epilogue of one tile overlaps the MMAs of
// the next ones.  Every wait is bounded (PN_ETIMEOUT on expiry).
#include "pn_gemm_kernel.cuh"

namespace pn {

// Per-format instantiations live in pn_gemm_f16.cu, pn_gemm_tf32.cu and
// pn_gemm_f8.cu so that they compile in parallel.
int gemm_launch_f16(int mode, int BN, const Common& cm, const Level& lv, int sms, void* stream);
int gemm_launch_tf32(int mode, int BN, const Common& cm, const Level& lv, int sms, void* stream);
int gemm_launch_f8(int mode, int BN, const Common& cm, const Level& lv, int sms, void* stream);

int gemm_smem_bytes(int mode, int BN) { return gemm::smem_total(mode, BN); }
int gemm_stages(int mode, int BN) { return gemm::num_stages(mode, BN); }

int launch_gemm_level(const Common& cm, const Level& lv, int num_sms, void* stream) {
  if (cm.BN != 128 && cm.BN != 256) return cudaErrorInvalidValue;
  switch (cm.mode) {
    case MODE_BF16:
    case MODE_F16: return gemm_launch_f16(cm.mode, cm.BN, cm, lv, num_sms, stream);
    case MODE_TF32:
    case MODE_3XTF32: return gemm_launch_tf32(cm.mode, cm.BN, cm, lv, num_sms, stream);
    case MODE_E4M3: return gemm_launch_f8(cm.mode, cm.BN, cm, lv, num_sms, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pn
