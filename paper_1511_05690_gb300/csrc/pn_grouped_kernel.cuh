// Persistent grouped kernel: every (problem, p, tile) work item of a group of
// independent products in ONE launch (the p rings and the problems
// parallelise coarsely, Sec. 4; Alg. 5 per problem).
//
// One CTA per SM (cooperative launch, so every CTA is resident): the copy
// producer, the MMA issuer and grouped_ng(BN) epilogue groups of four warps
// (three at 128-wide tiles: the epilogues of small problems, not the MMAs,
// bound the launch, and TMEM holds four 128-column accumulators).
// For each slot of the level schedule (largest p first):
//   1. operand blocks -- warps 2-9 build the powered images of the blocks
//      this level needs: below the top level only the blocks of pushed
//      tiles.  The top level's images (every block of every problem) are
//      either written before the launch by the strip kernel (top_built), or
//      built here (a test mode), reading each block once for its row /
//      column maxima (domain test, power-of-two scales) and once more, from
//      L2, for the images.  Each block is published with a release store of
//      its ready flag (slot + 1).
//   2. tiles -- the tensor-core roles of the level kernel (copy producer,
//      MMA issuer, the epilogue groups) over the slot's tiles; the producer
//      waits, bounded, for a tile's two ready flags before copying its
//      images, and the epilogue acquires them before reading the scales.
//   3. a bounded grid-wide barrier (a counter per slot): once every CTA has
//      finished the slot, the next slot's work list is complete; an empty
//      list ends the launch on every CTA.
// The ring positions and the accumulator count carry over between slots, so
// the pipeline never restarts.  Every wait is bounded (PN_ETIMEOUT).
#pragma once
#include "pn_gemm_kernel.cuh"
#include "pn_image.cuh"

namespace pn {
namespace gemm {

constexpr int IMG_BAR = 15;  // named barrier of the block builders (warps 2-9)

constexpr int GROUPED_NG_PLAIN_128 = 3;  // epilogue groups of the plain flavour at 128-wide tiles
__host__ __device__ constexpr int grouped_ng(int BN, bool plain) {
  return BN == 128 ? (plain ? GROUPED_NG_PLAIN_128 : 3) : 2;
}
__host__ __device__ constexpr int grouped_threads(int BN, bool plain) {
  return 64 + 128 * grouped_ng(BN, plain);
}

template <int MODE, int BN, bool PLAIN>
__global__ void __launch_bounds__(grouped_threads(BN, PLAIN), 1)
    k_grouped_persist(const __grid_constant__ Common cm, const __grid_constant__ GroupedRun gr) {
  constexpr int NG = grouped_ng(BN, PLAIN);
  static_assert(num_stages(MODE, BN, 1, NG) >= 2, "operand ring too small");
  static_assert(mode_bk(MODE) * 129 * 4 + 8 * TILE_M * 4 <=
                    num_stages(MODE, BN, 1, NG) * stage_bytes(MODE, BN),
                "block builders' staging does not fit the ring");
  __shared__ int32_t s_count;
  // tiles rotate over the epilogue groups
  const Ctx cx = ctx_setup<MODE, BN, 1, NG>(true, cm.timeout_ns);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  ProdState ps{};
  for (int s = 0; s < 8; ++s) ps.pend[s] = -1;
  ps.first = true;
  MmaState ms{};
  int it0 = 0;  // tiles this CTA processed in earlier slots
  bool bad = false;
  for (int t = 0; t < gr.n_slots; ++t) {
    const Level& lv = gr.lv[t];
    int count = cm.total_tiles;
    if (t > 0) {
      if (threadIdx.x == 0) {
        const bool ok = wait_flag_geq(gr.level_done + (t - 1), static_cast<int32_t>(gridDim.x),
                                      cx.tmo, cx.abort_flag);
        if (!ok) {
          *cx.abort_flag = 1;
          set_status(cm.status, PN_ETIMEOUT);
        }
        s_count = ok ? ld_acquire_gpu(lv.work_count) : 0;
      }
      __syncthreads();
      count = s_count;
      if (count == 0 || *cx.abort_flag) break;  // uniform
    }
    // ---------------------------------------------------- operand blocks ---
    const bool built = t == 0 && gr.top_built;
    if (warp >= 2 && warp < 10 && !built) {  // PRO_THREADS builder threads
      const int ti = threadIdx.x - 64;
      float* stile = reinterpret_cast<float*>(cx.smem);  // the ring is idle between slots
      uint32_t* red = reinterpret_cast<uint32_t*>(cx.smem + mode_bk(MODE) * 129 * 4);
      const bool mx = lv.is_top && gr.maxima;
      const int n_items = gr.n_a + gr.n_b;
      for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const bool is_b = item >= gr.n_a;
        const int id = is_b ? item - gr.n_a : item;
        if (!lv.is_top && !(is_b ? lv.cflag[id] : lv.rflag[id])) continue;  // block-uniform
        const int g = find_prob(cm, id, is_b ? 4 : 3);
        const Prob& P = prob_at(cm, g);
        if (!is_b) {
          bad |= a_block_fused<MODE>(cm, lv, g, P, id - P.tm_base, mx, ti, IMG_BAR);
        } else {
#pragma unroll 1
          for (int h = 0; h < BN / TILE_M; ++h)
            bad |= b_block_fused<MODE>(cm, lv, g, P, (id - P.tn_base) * (BN / TILE_M) + h, mx,
                                       stile, red, ti, IMG_BAR);
        }
        // publish: every writer orders its image stores before the bulk
        // copies of other CTAs, then one release store of the flag
        fence_proxy_async_global();
        bar_sync_named(IMG_BAR, PRO_THREADS);
        if (ti == 0) {
          __threadfence();
          st_release_gpu(gr.ready + item, t + 1);
        }
      }
      // the staging writes to the ring's shared memory precede the next bulk
      // copies into it (async proxy)
      fence_proxy_async_smem();
    }
    __syncthreads();
    // ------------------------------------------------------------- tiles ---
    const Ready rd{built ? nullptr : gr.ready, t + 1, gr.n_a};
    if (warp == 0) {
      if (lane == 0) run_producer<MODE, BN, 1, NG>(cm, lv, cx, count, ps, rd);
      __syncwarp();
    } else if (warp == 1) {
      if (lane == 0) run_mma<MODE, BN, 1, NG>(cm, lv, cx, count, it0, ms);
      __syncwarp();
    } else {
      run_epilogue<MODE, BN, 0, 1, NG, PLAIN>(cm, lv, cx, count, true, it0, rd);
    }
    if (count > static_cast<int>(blockIdx.x)) it0 += (count - 1 - static_cast<int>(blockIdx.x)) / static_cast<int>(gridDim.x) + 1;
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(gr.level_done + t, 1);
    }
  }
  if (bad) set_status(cm.status, PN_EDOMAIN);
  ctx_teardown<BN>(cx);
}

template <int MODE, int BN, bool PLAIN>
inline int launch_grouped_persist_k(const Common& cm, const GroupedRun& gr, int num_sms,
                                    void* stream) {
  static int attr_done = 0;
  if (!attr_done) {
    const cudaError_t e = cudaFuncSetAttribute(k_grouped_persist<MODE, BN, PLAIN>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               smem_total(MODE, BN, 1, grouped_ng(BN, PLAIN)));
    if (e != cudaSuccess) return e;
    attr_done = 1;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(num_sms));
  cfg.blockDim = dim3(grouped_threads(BN, PLAIN));
  cfg.dynamicSmemBytes = smem_total(MODE, BN, 1, grouped_ng(BN, PLAIN));
  cfg.stream = static_cast<cudaStream_t>(stream);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // every CTA resident: the flags and the
  attr[0].val.cooperative = 1;                  // level barrier wait on other CTAs
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_grouped_persist<MODE, BN, PLAIN>, cm, gr);
  return e != cudaSuccess ? e : cudaGetLastError();
}

// The plain flavour for the plain estimator (no projection state).
template <int MODE, int BN>
inline int launch_grouped_persist_t(const Common& cm, const GroupedRun& gr, int num_sms,
                                    void* stream, bool plain) {
  return plain ? launch_grouped_persist_k<MODE, BN, true>(cm, gr, num_sms, stream)
               : launch_grouped_persist_k<MODE, BN, false>(cm, gr, num_sms, stream);
}

}  // namespace gemm
}  // namespace pn
