// Prologue of the p-norm product (Alg. 5, first loop, with the scaled H' of
// Sec. 2.1): per-row maxima of A and per-column maxima of B, power-of-two
// scales, and the scaled operands raised to the power p of one level and cast
// to the tensor-core operand format.
//
// Operands are written as "tile images": for every block of 128 output rows
// (rows of A, or columns of B) and every 128 bytes of K, a 16 KB block holding
// exactly the shared-memory image the tensor cores read (K-major, 128-byte
// swizzle).  The GEMM then moves each tile with one 1-D bulk copy.  Rows past
// M (N) and K past K are zero in the image, so the GEMM needs no tail logic.
#include <cstring>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "pn_image.cuh"

namespace pn {

namespace {

__global__ void __launch_bounds__(PRO_THREADS) k_maxes(const __grid_constant__ Common cm) {
  pdl_wait();
  pdl_trigger();
  __shared__ uint32_t red[8][128];
  __shared__ float blk_max[PRO_THREADS / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int id = blockIdx.x;
  const bool is_b = id >= cm.total_ma;
  if (is_b) id -= cm.total_ma;
  const int g = find_prob(cm, id, is_b ? 6 : 5);
  const Prob& P = prob_at(cm, g);
  bool bad = false;
  float bmax = 0.0f;
  if (!is_b) {
    const int local = id - P.ma_base;
    const int rb = local / P.KMA, seg = local - rb * P.KMA;
    const int k0 = seg * MAXSEG_A;
    const bool vec = ((P.lda & 3) == 0) && ((reinterpret_cast<uintptr_t>(P.A) & 15) == 0);
    const int seg_len = P.K - k0 < MAXSEG_A ? P.K - k0 : MAXSEG_A;  // values in this segment
    const float* base = P.A + k0;
    // the row maximum from each lane's bits (all <= DOMAIN_MAX_BITS here)
    auto commit_row = [&](int row, uint32_t u) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) u = max(u, __shfl_xor_sync(0xffffffffu, u, o));
      if (lane == 0 && u > 0u) atomicMax(cm.rmax + P.rc_r + row, u);
      bmax = fmaxf(bmax, __uint_as_float(u));
    };
    if (vec && seg_len == MAXSEG_A) {
      // whole aligned segment: 16-byte loads, 8 in flight per lane per row
      for (int rr = 0; rr < 16; ++rr) {
        const int row = rb * TILE_M + warp * 16 + rr;
        if (row >= P.M) break;  // warp-uniform; later rows are past M too
        const float* src = base + (int64_t)row * P.lda;
        uint4 t[MAXSEG_A / 128];
#pragma unroll
        for (int it = 0; it < MAXSEG_A / 128; ++it)
          t[it] = __ldg(reinterpret_cast<const uint4*>(src + it * 128 + lane * 4));
        uint32_t u = 0u;
#pragma unroll
        for (int it = 0; it < MAXSEG_A / 128; ++it)
          u = umax3(u, max(t[it].x, t[it].y), max(t[it].z, t[it].w));
        if (u > DOMAIN_MAX_BITS) {
          uint32_t e = 0u;
          for (int q = 0; q < 4; ++q)
            e = max(e, take_exact(exact_max_bits(src + lane * 4 + q, 128, MAXSEG_A / 128), bad));
          u = e;
        }
        commit_row(row, u);
      }
    } else {
      // four rows at a time, lane reading columns lane + 32 t: 16 loads in
      // flight per lane, each load instruction one contiguous row segment.
      // The loads are unconditional: a column past the segment reads the
      // segment's last value (already part of the row maximum) and a row past
      // M reads row M - 1 (never committed).
      for (int rr = 0; rr < 16; rr += 4) {
        const int row0 = rb * TILE_M + warp * 16 + rr;
        if (row0 >= P.M) break;  // warp-uniform
        uint32_t u[4] = {0u, 0u, 0u, 0u};
        for (int kk0 = lane; kk0 < seg_len; kk0 += 128) {
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const float* src = base + (int64_t)min(row0 + r, P.M - 1) * P.lda;
#pragma unroll
            for (int q = 0; q < 4; ++q)
              u[r] = max(u[r], __float_as_uint(__ldg(src + min(kk0 + 32 * q, seg_len - 1))));
          }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int row = row0 + r;
          if (row < P.M) {  // warp-uniform
            if (u[r] > DOMAIN_MAX_BITS) {
              const int cnt = lane < seg_len ? (seg_len - 1 - lane) / 32 + 1 : 0;
              u[r] = take_exact(exact_max_bits(base + (int64_t)row * P.lda + lane, 32, cnt), bad);
            }
            commit_row(row, u[r]);
          }
        }
      }
    }
  } else {
    const int local = id - P.mb_base;
    const int rb = local / P.KMB, seg = local - rb * P.KMB;
    const int k0 = seg * MAXSEG_B;
    const int n4 = rb * TILE_M + lane * 4;
    const int nl = rb * TILE_M + lane;
    const bool vec = ((P.ldb & 3) == 0) && ((reinterpret_cast<uintptr_t>(P.B) & 15) == 0);
    uint32_t u4[4] = {0u, 0u, 0u, 0u};
    // whole aligned segment: thread = columns 4 lane .. 4 lane + 3, 16-byte
    // loads; otherwise thread = columns lane + 32 c, so that each load
    // instruction reads one contiguous 128-byte row segment, 16 in flight
    const bool full_vec = vec && rb * TILE_M + TILE_M <= P.N && k0 + MAXSEG_B <= P.K;
    if (full_vec) {
#pragma unroll 8
      for (int it = 0; it < MAXSEG_B / 8; ++it) {
        const int k = k0 + warp + 8 * it;
        const uint4 t = __ldg(reinterpret_cast<const uint4*>(P.B + (int64_t)k * P.ldb + n4));
        u4[0] = max(u4[0], t.x); u4[1] = max(u4[1], t.y);
        u4[2] = max(u4[2], t.z); u4[3] = max(u4[3], t.w);
      }
    } else {
      // unconditional loads: a row past K reads row K - 1 of the same column
      // (part of this segment), a column past N reads column N - 1 (its
      // maximum is never committed)
      int ncol[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) ncol[c] = min(nl + 32 * c, P.N - 1);
      for (int it0 = 0; it0 < MAXSEG_B / 8; it0 += 4) {
        if (k0 + warp + 8 * it0 >= P.K) break;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float* src = P.B + (int64_t)min(k0 + warp + 8 * (it0 + q), P.K - 1) * P.ldb;
#pragma unroll
          for (int c = 0; c < 4; ++c) u4[c] = max(u4[c], __float_as_uint(__ldg(src + ncol[c])));
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int n = full_vec ? n4 + c : nl + 32 * c;
      if (n >= P.N) u4[c] = 0u;
      if (u4[c] > DOMAIN_MAX_BITS) {
        // rows k0 + warp + 8 t < K of column n (n < N: other columns stay 0)
        const int rows = P.K - k0 < MAXSEG_B ? P.K - k0 : MAXSEG_B;
        const int cnt = warp < rows ? (rows - 1 - warp) / 8 + 1 : 0;
        u4[c] = take_exact(exact_max_bits(P.B + (int64_t)(k0 + warp) * P.ldb + n, 8 * P.ldb, cnt),
                           bad);
      }
      red[warp][full_vec ? lane * 4 + c : lane + 32 * c] = u4[c];
    }
    __syncthreads();
    if (tid < 128) {
      uint32_t m = red[0][tid];
#pragma unroll
      for (int w = 1; w < 8; ++w) m = max(m, red[w][tid]);
      const int n = rb * TILE_M + tid;
      if (n < P.N && m > 0u) atomicMax(cm.cmax + P.rc_c + n, m);
      bmax = __uint_as_float(m);
    }
  }
  if (__syncthreads_or(bad) && tid == 0) set_status(cm.status, PN_EDOMAIN);
  if (cm.scaling == 1) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bmax = fmaxf(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
    if (lane == 0) blk_max[warp] = bmax;
    __syncthreads();
    if (tid == 0) {
      float m = 0.0f;
      for (int w = 0; w < PRO_THREADS / 32; ++w) m = fmaxf(m, blk_max[w]);
      if (m > 0.0f) atomicMax(cm.gmax + 2 * g + (is_b ? 1 : 0), __float_as_uint(m));
    }
  }
}

// Top level without a tensor map (k_image_tma below): one block per operand
// tile.  Lower levels: the same operand-tile ids strided over a grid of a few
// blocks per SM; a tile is rebuilt only if a pushed output tile needs its row
// block (few at most levels, every one when the r = 1 projection sends every
// tile to the level p*/2).
// Resident blocks per SM for the image kernels: as many as the registers of
// the format's loads allow without heavy spilling -- more blocks keep more
// loads in flight (the max pass, at HBM speed, keeps about 200 KB per SM).
// Lower levels: block b owns the operand-tile ids b, b + gridDim.x, ...; the
// threads test PRO_THREADS of them at once (one flag load each, in parallel)
// and the block then builds the flagged ones in order.  `needed(id)` and
// `body(id)` must be block-uniform in effect (body may synchronise the block).
template <typename Need, typename Body>
__device__ __forceinline__ void for_flagged_ids(int total, const Need& needed, const Body& body) {
  __shared__ uint32_t mask[PRO_THREADS / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_ids = blockIdx.x < total ? (total - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  for (int j0 = 0; j0 < n_ids; j0 += PRO_THREADS) {
    const int j = j0 + threadIdx.x;
    const bool need = j < n_ids && needed((int)blockIdx.x + j * (int)gridDim.x);
    const uint32_t b = __ballot_sync(0xffffffffu, need);
    if (lane == 0) mask[warp] = b;
    __syncthreads();
    for (int w = 0; w < PRO_THREADS / 32; ++w) {
      uint32_t m = mask[w];
      while (m) {
        const int bit = __ffs(m) - 1;
        m &= m - 1;
        body((int)blockIdx.x + (j0 + w * 32 + bit) * (int)gridDim.x);
      }
    }
    __syncthreads();  // mask is rewritten by the next round
  }
}

template <int MODE>
constexpr int img_min_blocks() {
  return MODE == MODE_E4M3 ? 3 : (MODE == MODE_BF16 || MODE == MODE_F16) ? 4 : 5;
}

template <int MODE>
__global__ void __launch_bounds__(PRO_THREADS, img_min_blocks<MODE>())
    k_power_a(const __grid_constant__ Common cm, const __grid_constant__ Level lv) {
  pdl_wait();
  pdl_trigger();
  if (lv.is_top) {
    const int id = blockIdx.x;
    const int g = find_prob(cm, id, 1);
    const Prob& P = prob_at(cm, g);
    const int local = id - P.xa_base;
    const int rb = local / P.KB;
    power_a_tile<MODE>(cm, lv, g, P, rb, local - rb * P.KB, threadIdx.x);
    return;
  }
  if (*lv.work_count == 0) return;  // no tile pushed to this level (uniform)
  for_flagged_ids(
      cm.total_xa,
      [&](int id) {
        const Prob& P = prob_at(cm, find_prob(cm, id, 1));
        return lv.rflag[P.tm_base + (id - P.xa_base) / P.KB] != 0;
      },
      [&](int id) {
        const int g = find_prob(cm, id, 1);
        const Prob& P = prob_at(cm, g);
        const int local = id - P.xa_base;
        const int rb = local / P.KB;
        power_a_tile<MODE>(cm, lv, g, P, rb, local - rb * P.KB, threadIdx.x);
      });
}

// Top level without a tensor map: one block per operand tile.  Lower levels:
// as for A, a tile is rebuilt only if a pushed output tile needs its tile
// column.
template <int MODE>
__global__ void __launch_bounds__(PRO_THREADS, img_min_blocks<MODE>())
    k_power_b(const __grid_constant__ Common cm, const __grid_constant__ Level lv) {
  extern __shared__ float stile[];  // [BK][129]
  pdl_wait();
  pdl_trigger();
  if (lv.is_top) {
    const int id = blockIdx.x;
    const int g = find_prob(cm, id, 2);
    const Prob& P = prob_at(cm, g);
    const int local = id - P.xb_base;
    const int rb = local / P.KB;
    power_b_tile<MODE>(cm, lv, g, P, rb, local - rb * P.KB, stile, threadIdx.x, 0);
    return;
  }
  if (*lv.work_count == 0) return;  // no tile pushed to this level (uniform)
  const int per_tile = cm.BN / TILE_M;
  for_flagged_ids(
      cm.total_xb,
      [&](int id) {
        const Prob& P = prob_at(cm, find_prob(cm, id, 2));
        return lv.cflag[P.tn_base + (id - P.xb_base) / P.KB / per_tile] != 0;
      },
      [&](int id) {
        const int g = find_prob(cm, id, 2);
        const Prob& P = prob_at(cm, g);
        const int local = id - P.xb_base;
        const int rb = local / P.KB;
        power_b_tile<MODE>(cm, lv, g, P, rb, local - rb * P.KB, stile, threadIdx.x, 0);
      });
}

// ------------------------------------------------ TMA top-level images ---
// The top level of a single product builds every operand tile once.
// Persistent CTAs (two per SM, 256 threads each: while one waits at its
// block barrier the other computes) walk the tile ids blockIdx.x,
// blockIdx.x + gridDim.x, ... and keep the FP32 sources of their next NST
// stages in flight in a shared-memory ring (a stage is a tile, or half of
// the K values of a tile whose source exceeds 32 KB: E4M3); one thread
// issues a 2-D tensor copy per stage (an A tile
// is 128 rows x BK values, a B tile BK rows x 128 values; the copy fills
// zeros past M, N and K), completion counted in bytes on the stage's mbarrier,
// while all warps power and pack the current tile.  A images leave with
// coalesced 16-byte stores; B^T images are transposed into a double-buffered
// shared 16 KB image and written with one bulk copy per tile.
constexpr int TMA_CTAS_32K = 2;  // resident CTAs per SM with stages of at most 32 KB (every format)
constexpr int TMA_MAX_OWNED = 4096;  // tiles per SM the tensor-copy kernel takes

// Source values of K per stage: an image tile whose FP32 source exceeds 32 KB
// (E4M3: 128 x 128 values) arrives as two halves of K, so that every format
// keeps 32 KB stages and two CTAs per SM.
__host__ __device__ constexpr int tma_halves(int mode) {
  return mode_bk(mode) * TILE_M * 4 > 32768 ? 2 : 1;
}
__host__ __device__ constexpr int tma_src_bk(int mode) { return mode_bk(mode) / tma_halves(mode); }

template <int MODE, bool IS_B>
struct TmaCfg {
  static constexpr int BK = mode_bk(MODE);
  static constexpr int HALVES = tma_halves(MODE);
  static constexpr int SBK = tma_src_bk(MODE);   // K values per stage
  static constexpr int CPR = 8 / HALVES;         // 16-byte image chunks per image row and stage
  static constexpr int ROWS = IS_B ? SBK : TILE_M;  // source rows per stage
  static constexpr int COLS = IS_B ? TILE_M : SBK;  // source values per row
  static constexpr int STAGE_BYTES = ROWS * COLS * 4;
  static constexpr int PLANES = MODE == MODE_3XTF32 ? 2 : 1;
  static constexpr int OUT_BYTES = IS_B ? 2 * PLANES * IMG_BYTES : 0;
  static constexpr int CTAS = STAGE_BYTES <= 32768 ? TMA_CTAS_32K : 1;
  static constexpr int THREADS = 512 / CTAS;
  static constexpr int MAX_OWNED = TMA_MAX_OWNED / CTAS;
  static constexpr int RING_BUDGET = 200 * 1024 / CTAS - OUT_BYTES;
  static constexpr int NST = RING_BUDGET / STAGE_BYTES > 8 ? 8 : RING_BUDGET / STAGE_BYTES;
  static constexpr int SMEM = 1024 + NST * STAGE_BYTES + OUT_BYTES + 8 * NST + 16;
  static_assert(NST >= 2, "ring too small");
};

// Q float4 chunks of a staged row starting at src, read in the rotated order
// (q + rot) mod Q (so that the 8 threads of a quarter warp, rot = cc Q / 8,
// hit distinct banks) and returned in natural order.
template <int Q>
__device__ __forceinline__ void lds_rotated(const float* src, int rot, float* v) {
  float4 t[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) t[q] = *reinterpret_cast<const float4*>(src + 4 * ((q + rot) & (Q - 1)));
#pragma unroll
  for (int c = 0; c < Q; ++c) {
    float4 x = t[0];
#pragma unroll
    for (int q = 1; q < Q; ++q)
      if (((q + rot) & (Q - 1)) == c) x = t[q];
    v[4 * c] = x.x; v[4 * c + 1] = x.y; v[4 * c + 2] = x.z; v[4 * c + 3] = x.w;
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst_smem, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
      "%3}], [%4];" ::"r"(dst_smem),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

template <int MODE, bool IS_B>
__global__ void __launch_bounds__(TmaCfg<MODE, IS_B>::THREADS, TmaCfg<MODE, IS_B>::CTAS)
    k_image_tma(const __grid_constant__ Common cm, const __grid_constant__ Level lv,
                const __grid_constant__ CUtensorMap map) {
  pdl_wait();
  pdl_trigger();
  using CF = TmaCfg<MODE, IS_B>;
  using PK = Packer<MODE>;
  constexpr int EPC = PK::EPC;
  constexpr int BK = CF::BK, NST = CF::NST, H = CF::HALVES, SBK = CF::SBK, CPR = CF::CPR;
  constexpr int TMA_THREADS = CF::THREADS;
  constexpr int U = TILE_M * CPR / TMA_THREADS;  // 16-byte image chunks per thread and stage
  extern __shared__ uint8_t smem_dyn[];
  const uint32_t raw = smem_u32(smem_dyn);
  uint8_t* smem = smem_dyn + (((raw + 1023u) & ~1023u) - raw);
  float* ring = reinterpret_cast<float*>(smem);
  uint8_t* outimg = smem + NST * CF::STAGE_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(outimg + CF::OUT_BYTES);
  volatile int32_t* abort_flag = reinterpret_cast<volatile int32_t*>(full + NST);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const Prob& P = cm.single;
  const int total = IS_B ? cm.total_xb : cm.total_xa;
  const int owned = (int)blockIdx.x < total ? (total - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  if (owned == 0) return;  // uniform
  if (!lv.is_top && *lv.work_count == 0) return;  // no tile pushed to this level (uniform)
  // This CTA's tiles: ids blockIdx.x + k * gridDim.x, k < owned; below the top
  // level only those whose row block (A) or tile column (B) is flagged,
  // compacted into tile_k[] (the launcher bounds owned by CF::MAX_OWNED).
  __shared__ int32_t tile_k[CF::MAX_OWNED];
  __shared__ int32_t n_tiles;
  if (tid == 0) {
    for (int s = 0; s < NST; ++s) mbar_init(&full[s], 1);
    *abort_flag = 0;
    n_tiles = 0;
    fence_barrier_init();
  }
  __syncthreads();
  if (lv.is_top) {
    for (int k = tid; k < owned; k += TMA_THREADS) tile_k[k] = k;
    if (tid == 0) n_tiles = owned;
  } else {
    const int per_tile = cm.BN / TILE_M;
    for (int k0 = 0; k0 < owned; k0 += TMA_THREADS) {
      const int k = k0 + tid;
      bool need = false;
      if (k < owned) {
        const int rb = ((int)blockIdx.x + k * (int)gridDim.x) / P.KB;
        need = IS_B ? lv.cflag[rb / per_tile] != 0 : lv.rflag[rb] != 0;
      }
      const uint32_t bal = __ballot_sync(0xffffffffu, need);
      int base = 0;
      if (lane == 0 && bal) base = atomicAdd(&n_tiles, __popc(bal));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (need) tile_k[base + __popc(bal & ((1u << lane) - 1u))] = k;
      __syncthreads();  // n_tiles complete before the next round's adds are read
    }
  }
  __syncthreads();
  const int mine = n_tiles;
  if (mine == 0) return;  // uniform

  // thread 0: the tensor copy of this CTA's j-th stage (tile j / H, half
  // j % H of its K values) into ring slot j % NST
  auto issue = [&](int j) {
    const int id = (int)blockIdx.x + tile_k[j / H] * (int)gridDim.x;
    const int rb = id / P.KB, kb = id - rb * P.KB;
    const int k0 = kb * BK + (j % H) * SBK;
    uint64_t* bar = &full[j % NST];
    mbar_arrive_expect_tx(bar, CF::STAGE_BYTES);
    // test hook (debug_flags bit 1): the first tile's bytes are announced but
    // never copied, so the bounded wait for them runs out
    if ((cm.debug_flags & 2) && j == 0) return;
    const uint32_t dst = smem_u32(ring) + (j % NST) * CF::STAGE_BYTES;
    if constexpr (!IS_B)
      tma_load_2d(dst, &map, k0, rb * TILE_M, bar);
    else
      tma_load_2d(dst, &map, rb * TILE_M, k0, bar);
  };

  // A: thread = image chunks (row tid / CPR + (128 / U) u, slot tid % CPR of
  // the stage's CPR).  B: warp w = slot w % CPR of image rows nr = lane + 32
  // (U (w / CPR) + u), i.e. contraction indices (w % CPR) EPC + e of column
  // rb 128 + nr.  The slot's chunk of the image row is ccl + CPR h for the
  // stage's half h.
  const int ccl = IS_B ? (warp % CPR) : (tid % CPR);
  auto line = [&](int u) {  // this thread's image row of chunk u
    return IS_B ? lane + 32 * (U * (warp / CPR) + u) : tid / CPR + (TILE_M / U) * u;
  };
  // shared-memory reads of a staged A row: the 8 threads of a quarter warp
  // (8 / CPR rows, CPR slots) rotate their float4 order so that they hit
  // distinct banks
  const int rot = (ccl * (EPC / 4) / 8 + (tid / CPR) % (8 / CPR) * (EPC / 4) * CPR / 8) &
                  (EPC / 4 - 1);
  // the maxima behind this thread's U row (A) or column (B) scales of tile
  // j, loaded one tile ahead of their use
  uint32_t pre[U];
  auto prefetch = [&](int jj) {
    const int rbj = ((int)blockIdx.x + tile_k[jj] * (int)gridDim.x) / P.KB;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = rbj * TILE_M + line(u);
      pre[u] = idx < (IS_B ? P.N : P.M)
                   ? scale_bits(cm, IS_B ? cm.cmax : cm.rmax, (IS_B ? P.rc_c : P.rc_r) + idx, 0,
                                IS_B ? 1 : 0)
                   : 0u;
    }
  };

  const uint64_t tmo = cm.timeout_ns;
  const int nj = mine * H;  // stages of this CTA
  if (tid == 0)
    for (int j = 0; j < NST && j < nj; ++j) issue(j);
  prefetch(0);
  const float opscale = ldexpf(1.0f, cm.s_op);
  float sc[U];
  int j = 0;
  for (; j < nj; ++j) {
    const int s = j % NST;
    if (tid == 0 && !mbar_wait(&full[s], (j / NST) & 1, tmo, abort_flag)) {
      *abort_flag = 1;
      set_status(cm.status, PN_ETIMEOUT);
    }
    __syncthreads();  // also: the shared B image ((j / H) & 1) is free again
    if (*abort_flag) break;
    const int tj = j / H, h = j % H;
    const int id = (int)blockIdx.x + tile_k[tj] * (int)gridDim.x;
    const int rb = id / P.KB, kb = id - rb * P.KB;
    const int cc = ccl + CPR * h;  // this thread's chunk of the image row
    const float* st = ring + s * (CF::STAGE_BYTES / 4);
    if (h == 0) {
#pragma unroll
      for (int u = 0; u < U; ++u) sc[u] = scale_from_bits(cm, pre[u]);
      if (tj + 1 < mine) prefetch(tj + 1);
    }
    float v[U][EPC];  // the copy filled zeros past M, N and K
    if constexpr (!IS_B) {
#pragma unroll
      for (int u = 0; u < U; ++u) lds_rotated<EPC / 4>(st + line(u) * SBK + ccl * EPC, rot, v[u]);
      // power_a_store's mapping (row t / 8 + (128 / U) u, chunk t % 8) for
      // this thread's rows and chunk
      power_a_store<MODE, U>(cm, lv, P, rb, kb, v, sc, (tid / CPR) * 8 + cc);
    } else {
      uint8_t* ob = outimg + (tj & 1) * CF::PLANES * IMG_BYTES;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int nr = line(u);
#pragma unroll
        for (int e = 0; e < EPC; ++e) v[u][e] = st[(ccl * EPC + e) * TILE_M + nr];
        if (lv.is_top && kb == 0 && cc == 0 && rb * TILE_M + nr < P.N)
          cm.c[P.rc_c + rb * TILE_M + nr] = sc[u];
      }
      div_scales(v, sc);
      power_all(v, lv.plog, lv.half, opscale);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int nr = line(u);
        uint4 hi, lo;
        PK::pack(v[u], hi, lo);
        const uint32_t off = sw128_offset(nr, cc * 16);
        *reinterpret_cast<uint4*>(ob + off) = hi;
        if constexpr (CF::PLANES == 2) *reinterpret_cast<uint4*>(ob + IMG_BYTES + off) = lo;
      }
      fence_proxy_async_smem();
    }
    __syncthreads();  // stage s is consumed; the shared B image is complete
    if (tid == 0) {
      if constexpr (IS_B) {
        if (h == H - 1) {
          uint8_t* dst = lv.b_level + P.b_img + ((int64_t)(rb * P.KB + kb) << 14);
          const uint32_t src = smem_u32(outimg + (tj & 1) * CF::PLANES * IMG_BYTES);
          bulk_s2g(dst, src, IMG_BYTES);
          if constexpr (CF::PLANES == 2) bulk_s2g(dst + P.b_plane, src + IMG_BYTES, IMG_BYTES);
          bulk_commit();
          bulk_wait_read<1>();  // the image of tile tj - 1 has been read out
        }
      }
      if (j + NST < nj) issue(j + NST);
    }
  }
  if (tid == 0) {
    if (j < nj) {  // gave up: let the copies in flight land before exiting
      int32_t never = 0;
      const int last = nj < j + NST ? nj : j + NST;
      for (int t = j; t < last; ++t) mbar_wait(&full[t % NST], (t / NST) & 1, tmo, &never);
    }
    if constexpr (IS_B) bulk_wait_all();
  }
}

// ------------------------------------------------------------ K == 0 ---
// Empty contraction: every S^(p) is 0, so p* is the smallest p (unstable)
// and the estimate is the exact empty max, 0.
__global__ void k_fill_empty(const __grid_constant__ Common cm, int plog0) {
  pdl_wait();
  pdl_trigger();
  const Prob& P = cm.single;
  const int64_t total = (int64_t)P.M * P.N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / P.N, j = e - i * P.N;
    P.C[i * P.ldc + j] = 0.0f;
    if (P.psel) P.psel[i * P.ldaux + j] = static_cast<uint8_t>(0x80 | plog0);
    if (P.Ssel) P.Ssel[i * P.ldaux + j] = 0.0f;
  }
}

// ---------------------------------------------------------------- APSP ---
// x = exp(-w) (Sec. 2.2), +inf -> 0; weights must be >= 0 or +inf.
__global__ void k_apsp_init(int64_t n, const float* __restrict__ W, int64_t ldw,
                            float* __restrict__ X, int diag, int32_t* status) {
  pdl_wait();
  pdl_trigger();
  const int64_t total = n * n;
  bool bad = false;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e - i * n;
    const float w = W[i * ldw + j];
    bad |= !(w >= 0.0f);  // negative or NaN
    float x = (w == INFINITY) ? 0.0f : expf(-w);
    if (diag && i == j) x = 1.0f;
    X[e] = x;
  }
  if (bad) set_status(status, PN_EDOMAIN);
}

// d = -log x; x = 0 (no path) -> +inf.
__global__ void k_apsp_final(int64_t n, const float* X, int64_t ldx, float* D, int64_t ldd) {
  pdl_wait();
  pdl_trigger();
  const int64_t total = n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e - i * n;
    const float x = X[i * ldx + j];
    D[i * ldd + j] = x > 0.0f ? -logf(x) : INFINITY;
  }
}

int sm_count();

// Lower-level image grids: two waves of the resident blocks on every SM.
int lower_grid(int total, int per_sm) {
  const int g = 2 * sm_count() * per_sm;
  return total < g ? total : g;
}

int sm_count() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      sms = v;
    else
      return 152;
  }
  return sms;
}

template <int MODE, bool IS_B>
int launch_tma_t(const Common& cm, const Level& lv, void* stream, const TensorMapBytes& map) {
  using CF = TmaCfg<MODE, IS_B>;
  static bool attr_done = false;
  if (!attr_done) {
    const cudaError_t e = cudaFuncSetAttribute(
        k_image_tma<MODE, IS_B>, cudaFuncAttributeMaxDynamicSharedMemorySize, CF::SMEM);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  const int total = IS_B ? cm.total_xb : cm.total_xa;
  const int grid = total < CF::CTAS * sm_count() ? total : CF::CTAS * sm_count();
  const cudaError_t e = launch_pdl(k_image_tma<MODE, IS_B>, dim3(grid), dim3(CF::THREADS), CF::SMEM,
                                   stream, cm, lv, *reinterpret_cast<const CUtensorMap*>(&map));
  return e != cudaSuccess ? e : cudaGetLastError();
}

// The tensor-copy kernel takes at most TMA_MAX_OWNED tiles per SM.
bool tma_fits(int total) { return total <= TMA_MAX_OWNED * sm_count(); }

template <bool IS_B>
int launch_tma(const Common& cm, const Level& lv, void* stream, const TensorMapBytes& map) {
  switch (cm.mode) {
    case MODE_3XTF32: return launch_tma_t<MODE_3XTF32, IS_B>(cm, lv, stream, map);
    case MODE_TF32: return launch_tma_t<MODE_TF32, IS_B>(cm, lv, stream, map);
    case MODE_BF16: return launch_tma_t<MODE_BF16, IS_B>(cm, lv, stream, map);
    case MODE_F16: return launch_tma_t<MODE_F16, IS_B>(cm, lv, stream, map);
    case MODE_E4M3: return launch_tma_t<MODE_E4M3, IS_B>(cm, lv, stream, map);
    default: return cudaErrorInvalidValue;
  }
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// Row-major FP32 matrix of rows x cols with row pitch ld (elements) as a 2-D
// tensor map with box box_rows x box_cols, zeros outside the matrix.
bool encode_fp32_2d(TensorMapBytes& out, const float* base, int64_t rows, int64_t cols, int64_t ld,
                    int box_rows, int box_cols) {
  const EncodeTiledFn fn = encode_tiled();
  if (!fn || !base || rows < 1 || cols < 1 || ld < cols) return false;
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || (ld & 3) != 0) return false;
  if (rows > (int64_t(1) << 31) || cols > (int64_t(1) << 31) || ld * 4 >= (int64_t(1) << 40))
    return false;
  const cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * 4};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(box_cols), static_cast<cuuint32_t>(box_rows)};
  const cuuint32_t estr[2] = {1, 1};
  return fn(reinterpret_cast<CUtensorMap*>(&out), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
            const_cast<float*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int MODE>
int launch_power_b_t(const Common& cm, const Level& lv, void* stream) {
  const int smem = mode_bk(MODE) * 129 * 4;
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(k_power_b<MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  const int grid = lv.is_top ? cm.total_xb : lower_grid(cm.total_xb, img_min_blocks<MODE>());
  const cudaError_t e = launch_pdl(k_power_b<MODE>, dim3(grid), dim3(PRO_THREADS), smem, stream, cm, lv);
  return e != cudaSuccess ? e : cudaGetLastError();
}

int grid_for(int64_t total, int threads) {
  int64_t b = (total + threads - 1) / threads;
  if (b > 152 * 32) b = 152 * 32;
  return static_cast<int>(b > 0 ? b : 1);
}

// Grouped products, top level: the maxima (domain test), scales and powered
// images of every operand block, in strips of 32 rows of A or 32 columns of
// B, one strip per CTA.  A strip is read once from memory for its maxima and
// once more for its images, from L2 (at most 32 K floats per CTA, so the
// strips in flight fit in it); every load instruction of a warp reads one
// contiguous row segment, and shared memory regroups the values into the
// image layout.  The arithmetic per value is that of power_a_store /
// power_b_tile (same scales, same operation order), so the images are
// bit-identical to theirs.
constexpr int STRIP_ROWS = 32;

// A rows 128 rb + 32 s .. + 31 of problem P.  Warp w owns rows 4w .. 4w + 3
// of the strip: their maxima stay in registers, and its shared area `sm`
// (4 rows of BK floats, 4 floats of padding after every 32) stages them.
template <int MODE>
__device__ __forceinline__ bool a_strip(const Common& cm, const Level& lv, const Prob& P, int rb,
                                        int s, float* sm) {
  using PK = Packer<MODE>;
  constexpr int EPC = PK::EPC;
  constexpr int BK = mode_bk(MODE);
  constexpr int LDS = BK + BK / 8;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rloc = s * STRIP_ROWS + warp * 4;  // first row of the warp within the block
  const int row0 = rb * TILE_M + rloc;
  bool bad = false;
  uint32_t u[4] = {0u, 0u, 0u, 0u};
  // the warp's rows (a row past M reads row M - 1 and is never committed)
  const float* src[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) src[r] = P.A + (int64_t)min(row0 + r, P.M - 1) * P.lda;
  if (row0 < P.M) {  // warp-uniform
    int kk0 = lane;
    for (; kk0 + 96 < P.K; kk0 += 128) {  // whole 128-column steps: no clamps
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) u[r] = max(u[r], __float_as_uint(__ldg(src[r] + kk0 + 32 * q)));
    }
    if (kk0 < P.K) {
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          u[r] = max(u[r], __float_as_uint(__ldg(src[r] + min(kk0 + 32 * q, P.K - 1))));
    }
  }
  float rs[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int row = row0 + r;
    rs[r] = 1.0f;
    if (row < P.M) {  // warp-uniform
      if (u[r] > DOMAIN_MAX_BITS) {
        const int cnt = lane < P.K ? (P.K - 1 - lane) / 32 + 1 : 0;
        u[r] = take_exact(exact_max_bits(P.A + (int64_t)row * P.lda + lane, 32, cnt), bad);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) u[r] = max(u[r], __shfl_xor_sync(0xffffffffu, u[r], o));
      rs[r] = scale_from_bits(cm, u[r]);
      if (lane == 0) {
        cm.rmax[P.rc_r + row] = u[r];
        if (lv.is_top) cm.r[P.rc_r + row] = rs[r];
      }
    }
  }
  const float opscale = ldexpf(1.0f, cm.s_op);
  float* wsm = sm + warp * 4 * LDS;
  const int jr = lane >> 3, cc = lane & 7;
  const float rsj[1] = {jr == 0 ? rs[0] : jr == 1 ? rs[1] : jr == 2 ? rs[2] : rs[3]};
  const float* rp = wsm + jr * LDS + cc * EPC + ((cc * EPC) >> 5) * 4;
  const bool rows_in = row0 + 3 < P.M;  // warp-uniform: all four rows exist
  for (int kb = 0; kb < P.KB; ++kb) {
    float t[4][BK / 32];
    if (rows_in && (kb + 1) * BK <= P.K) {  // warp-uniform: no clamps, no zeros
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int h = 0; h < BK / 32; ++h) t[r][h] = __ldg(src[r] + kb * BK + 32 * h + lane);
    } else {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const bool rok = row0 + r < P.M;
#pragma unroll
        for (int h = 0; h < BK / 32; ++h) {
          const int k = kb * BK + 32 * h + lane;
          const float x = __ldg(src[r] + min(k, P.K - 1));
          t[r][h] = (rok && k < P.K) ? x : 0.0f;
        }
      }
    }
    __syncwarp();  // the previous k-block's reads of wsm are done
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int h = 0; h < BK / 32; ++h) wsm[r * LDS + 36 * h + lane] = t[r][h];
    __syncwarp();
    float v[1][EPC];
#pragma unroll
    for (int e = 0; e < EPC; e += 4) {
      const float4 f = *reinterpret_cast<const float4*>(rp + e);
      v[0][e] = f.x; v[0][e + 1] = f.y; v[0][e + 2] = f.z; v[0][e + 3] = f.w;
    }
    div_scales(v, rsj);
    power_all(v, lv.plog, lv.half, opscale);
    uint4 hi, lo;
    PK::pack(v[0], hi, lo);
    uint8_t* dst = lv.a_level + P.a_img + ((int64_t)(rb * P.KB + kb) << 14);
    const uint32_t off = sw128_offset(static_cast<uint32_t>(rloc + jr), cc * 16);
    *reinterpret_cast<uint4*>(dst + off) = hi;
    if constexpr (MODE == MODE_3XTF32) *reinterpret_cast<uint4*>(dst + P.a_plane + off) = lo;
  }
  return bad;
}

// B columns 128 cb + 32 s .. + 31 of problem P (rows of the B^T image).
// Lane l owns column l of the strip for the maxima and the staging; warp w
// writes image rows 4w .. 4w + 3.  `sm` holds two staged k-blocks (BK x 33
// floats each), `red` 288 words.
template <int MODE>
__device__ __forceinline__ bool b_strip(const Common& cm, const Level& lv, const Prob& P, int cb,
                                        int s, float* sm, uint32_t* red) {
  using PK = Packer<MODE>;
  constexpr int EPC = PK::EPC;
  constexpr int BK = mode_bk(MODE);
  constexpr int TS = 33;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int col0 = cb * TILE_M + s * STRIP_ROWS;
  const int col = col0 + lane;
  const int colc = min(col, P.N - 1);
  bool bad = false;
  uint32_t u = 0u;
  const int64_t ld8 = 8 * P.ldb;
  if (col0 < P.N) {  // block-uniform
    int k0 = warp;
    const float* p = P.B + (int64_t)warp * P.ldb + colc;
    for (; k0 + 8 * 15 < P.K; k0 += 128, p += 16 * ld8) {  // 16 whole rows: no clamps
#pragma unroll
      for (int q = 0; q < 16; ++q) u = max(u, __float_as_uint(__ldg(p + q * ld8)));
    }
    if (k0 < P.K) {
#pragma unroll
      for (int q = 0; q < 16; ++q)
        u = max(u, __float_as_uint(__ldg(P.B + (int64_t)min(k0 + 8 * q, P.K - 1) * P.ldb + colc)));
    }
    if (col >= P.N) u = 0u;
    if (u > DOMAIN_MAX_BITS) {
      const int cnt = warp < P.K ? (P.K - 1 - warp) / 8 + 1 : 0;
      u = take_exact(exact_max_bits(P.B + (int64_t)warp * P.ldb + col, 8 * P.ldb, cnt), bad);
    }
  }
  red[warp * 32 + lane] = u;
  __syncthreads();
  if (warp == 0) {
    uint32_t m = red[lane];
#pragma unroll
    for (int w = 1; w < PRO_THREADS / 32; ++w) m = max(m, red[w * 32 + lane]);
    const float cs = col < P.N ? scale_from_bits(cm, m) : 1.0f;
    if (col < P.N) {
      cm.cmax[P.rc_c + col] = m;
      if (lv.is_top) cm.c[P.rc_c + col] = cs;
    }
    red[256 + lane] = __float_as_uint(cs);
  }
  __syncthreads();
  const float cs_l = __uint_as_float(red[256 + lane]);
  const float inv = 1.0f / cs_l;
  const bool inv_ok = recip_exact(cs_l);
  const float opscale = ldexpf(1.0f, cm.s_op);
  const int jr = lane >> 3, cc = lane & 7;
  const int irow = s * STRIP_ROWS + warp * 4 + jr;  // image row within the block
  for (int kb = 0; kb < P.KB; ++kb) {
    float* st = sm + (kb & 1) * (BK * TS);
    float t[BK / 8];
    if ((kb + 1) * BK <= P.K) {  // block-uniform: whole rows, no clamps
      const float* p = P.B + (int64_t)(kb * BK + warp) * P.ldb + colc;
#pragma unroll
      for (int i = 0; i < BK / 8; ++i) t[i] = __ldg(p + i * ld8);
#pragma unroll
      for (int i = 0; i < BK / 8; ++i) t[i] = col < P.N ? t[i] : 0.0f;
    } else {
#pragma unroll
      for (int i = 0; i < BK / 8; ++i) {
        const int k = kb * BK + warp + 8 * i;
        const float x = __ldg(P.B + (int64_t)min(k, P.K - 1) * P.ldb + colc);
        t[i] = (k < P.K && col < P.N) ? x : 0.0f;
      }
    }
#pragma unroll
    for (int i = 0; i < BK / 8; ++i)
      st[(warp + 8 * i) * TS + lane] = div_pow2(t[i], cs_l, inv, inv_ok);
    __syncthreads();  // (two buffers: the reads of k-block kb - 1 ended before)
    float v[1][EPC];
#pragma unroll
    for (int e = 0; e < EPC; ++e) v[0][e] = st[(cc * EPC + e) * TS + warp * 4 + jr];
    power_all(v, lv.plog, lv.half, opscale);
    uint4 hi, lo;
    PK::pack(v[0], hi, lo);
    uint8_t* dst = lv.b_level + P.b_img + ((int64_t)(cb * P.KB + kb) << 14);
    const uint32_t off = sw128_offset(static_cast<uint32_t>(irow), cc * 16);
    *reinterpret_cast<uint4*>(dst + off) = hi;
    if constexpr (MODE == MODE_3XTF32) *reinterpret_cast<uint4*>(dst + P.b_plane + off) = lo;
  }
  return bad;
}

template <int MODE>
__host__ __device__ constexpr int strip_smem() {
  constexpr int a = 8 * 4 * (mode_bk(MODE) + mode_bk(MODE) / 8) * 4;
  constexpr int b = 2 * mode_bk(MODE) * 33 * 4;
  return (a > b ? a : b) + 288 * 4;
}

// One CTA per strip: A strips (4 per row block) first, then B strips (4 per
// 128-column block, BN / 128 blocks per tile column).
template <int MODE>
__global__ void __launch_bounds__(PRO_THREADS)
    k_strips(const __grid_constant__ Common cm, const __grid_constant__ Level lv, int n_a) {
  extern __shared__ __align__(16) float sm_strip[];
  pdl_wait();
  pdl_trigger();
  const int unit = static_cast<int>(blockIdx.x);
  constexpr int SM_FLOATS = strip_smem<MODE>() / 4 - 288;
  uint32_t* red = reinterpret_cast<uint32_t*>(sm_strip + SM_FLOATS);
  bool bad;
  if (unit < n_a) {
    const int g = find_prob(cm, unit >> 2, 3);
    const Prob& P = prob_at(cm, g);
    bad = a_strip<MODE>(cm, lv, P, (unit >> 2) - P.tm_base, unit & 3, sm_strip);
  } else {
    const int bpt = cm.BN / TILE_M;
    const int cbg = (unit - n_a) >> 2;
    const int g = find_prob(cm, cbg / bpt, 4);
    const Prob& P = prob_at(cm, g);
    bad = b_strip<MODE>(cm, lv, P, cbg - P.tn_base * bpt, (unit - n_a) & 3, sm_strip, red);
  }
  if (bad) set_status(cm.status, PN_EDOMAIN);
}

template <int MODE>
int launch_strips_t(const Common& cm, const Level& lv, void* stream) {
  constexpr int smem = strip_smem<MODE>();
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e =
        cudaFuncSetAttribute(k_strips<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  const int n_a = 4 * cm.total_tm;
  const int grid = n_a + 4 * cm.total_tn * (cm.BN / TILE_M);
  const cudaError_t e = launch_pdl(k_strips<MODE>, dim3(grid), dim3(PRO_THREADS), smem, stream, cm,
                                   lv, n_a);
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace

int launch_strips(const Common& cm, const Level& lv, void* stream) {
  if (cm.total_tm + cm.total_tn <= 0) return 0;
  if (cm.scaling == 1 || !lv.is_top) return cudaErrorInvalidValue;  // per-row / column scales only
  switch (cm.mode) {
    case MODE_3XTF32: return launch_strips_t<MODE_3XTF32>(cm, lv, stream);
    case MODE_TF32: return launch_strips_t<MODE_TF32>(cm, lv, stream);
    case MODE_BF16: return launch_strips_t<MODE_BF16>(cm, lv, stream);
    case MODE_F16: return launch_strips_t<MODE_F16>(cm, lv, stream);
    case MODE_E4M3: return launch_strips_t<MODE_E4M3>(cm, lv, stream);
    default: return cudaErrorInvalidValue;
  }
}

int launch_maxes(const Common& cm, void* stream) {
  const int blocks = cm.total_ma + cm.total_mb;
  if (blocks <= 0) return 0;
  const cudaError_t e = launch_pdl(k_maxes, dim3(blocks), dim3(PRO_THREADS), 0, stream, cm);
  return e != cudaSuccess ? e : cudaGetLastError();
}

bool encode_img_rows(TensorMapBytes& out, const void* base, int64_t bytes, int box_rows) {
  const EncodeTiledFn fn = encode_tiled();
  if (!fn || !base || bytes < 128 * 128 || (bytes & 127) != 0) return false;
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || (bytes >> 7) > (int64_t(1) << 31))
    return false;
  const cuuint64_t dims[2] = {128, static_cast<cuuint64_t>(bytes >> 7)};
  const cuuint64_t strides[1] = {128};
  if (box_rows < 8 || box_rows > 256) return false;
  const cuuint32_t box[2] = {128, static_cast<cuuint32_t>(box_rows)};
  const cuuint32_t estr[2] = {1, 1};
  return fn(reinterpret_cast<CUtensorMap*>(&out), CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
            const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void make_operand_maps(const Common& cm, OperandMaps& maps) {
  std::memset(&maps, 0, sizeof(maps));
  if (cm.nprob != 1) return;
  const Prob& P = cm.single;
  const int bk = tma_src_bk(cm.mode);  // K values per stage of the tensor-copy kernel
  maps.has_a = encode_fp32_2d(maps.a, P.A, P.M, P.K, P.lda, TILE_M, bk) ? 1 : 0;
  maps.has_b = encode_fp32_2d(maps.b, P.B, P.K, P.N, P.ldb, bk, TILE_M) ? 1 : 0;
}

int launch_power_a(const Common& cm, const Level& lv, void* stream, const OperandMaps* maps) {
  if (cm.total_xa <= 0) return 0;
  if (maps && maps->has_a && tma_fits(cm.total_xa)) return launch_tma<false>(cm, lv, stream, maps->a);
  auto grid = [&](int per_sm) { return lv.is_top ? cm.total_xa : lower_grid(cm.total_xa, per_sm); };
  cudaError_t e = cudaSuccess;
  switch (cm.mode) {
    case MODE_3XTF32:
      e = launch_pdl(k_power_a<MODE_3XTF32>, dim3(grid(img_min_blocks<MODE_3XTF32>())), dim3(PRO_THREADS), 0,
                     stream, cm, lv);
      break;
    case MODE_TF32:
      e = launch_pdl(k_power_a<MODE_TF32>, dim3(grid(img_min_blocks<MODE_TF32>())), dim3(PRO_THREADS), 0,
                     stream, cm, lv);
      break;
    case MODE_BF16:
      e = launch_pdl(k_power_a<MODE_BF16>, dim3(grid(img_min_blocks<MODE_BF16>())), dim3(PRO_THREADS), 0,
                     stream, cm, lv);
      break;
    case MODE_F16:
      e = launch_pdl(k_power_a<MODE_F16>, dim3(grid(img_min_blocks<MODE_F16>())), dim3(PRO_THREADS), 0,
                     stream, cm, lv);
      break;
    case MODE_E4M3:
      e = launch_pdl(k_power_a<MODE_E4M3>, dim3(grid(img_min_blocks<MODE_E4M3>())), dim3(PRO_THREADS), 0,
                     stream, cm, lv);
      break;
    default: return cudaErrorInvalidValue;
  }
  return e != cudaSuccess ? e : cudaGetLastError();
}

int launch_power_b(const Common& cm, const Level& lv, void* stream, const OperandMaps* maps) {
  if (cm.total_xb <= 0) return 0;
  if (maps && maps->has_b && tma_fits(cm.total_xb)) return launch_tma<true>(cm, lv, stream, maps->b);
  switch (cm.mode) {
    case MODE_3XTF32: return launch_power_b_t<MODE_3XTF32>(cm, lv, stream);
    case MODE_TF32: return launch_power_b_t<MODE_TF32>(cm, lv, stream);
    case MODE_BF16: return launch_power_b_t<MODE_BF16>(cm, lv, stream);
    case MODE_F16: return launch_power_b_t<MODE_F16>(cm, lv, stream);
    case MODE_E4M3: return launch_power_b_t<MODE_E4M3>(cm, lv, stream);
    default: return cudaErrorInvalidValue;
  }
}

int launch_fill_empty(const Common& cm, int plog0, void* stream) {
  const int64_t total = (int64_t)cm.single.M * cm.single.N;
  if (total <= 0) return 0;
  const cudaError_t e =
      launch_pdl(k_fill_empty, dim3(grid_for(total, 256)), dim3(256), 0, stream, cm, plog0);
  return e != cudaSuccess ? e : cudaGetLastError();
}

int launch_apsp_init(int64_t n, const float* W, int64_t ldw, float* X, int diag, int32_t* status,
                     void* stream) {
  if (n <= 0) return 0;
  const cudaError_t e = launch_pdl(k_apsp_init, dim3(grid_for(n * n, 256)), dim3(256), 0, stream, n,
                                   W, ldw, X, diag, status);
  return e != cudaSuccess ? e : cudaGetLastError();
}

int launch_apsp_final(int64_t n, const float* X, int64_t ldx, float* D, int64_t ldd,
                      void* stream) {
  if (n <= 0) return 0;
  const cudaError_t e = launch_pdl(k_apsp_final, dim3(grid_for(n * n, 256)), dim3(256), 0, stream,
                                   n, X, ldx, D, ldd);
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace pn
