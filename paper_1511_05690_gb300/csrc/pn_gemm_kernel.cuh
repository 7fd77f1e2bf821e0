// Tensor-core level kernel of the p-norm product (template; instantiated per
// operand format in pn_gemm_*.cu).  See pn_gemm.cu for the design notes.
#pragma once
#include <cfloat>
#include <type_traits>

#include "pn_device.cuh"

namespace pn {
namespace gemm {

// Epilogue warps: NG groups of four, one warp per TMEM lane quarter each.
// The level kernel runs two groups; the persistent grouped kernel three at
// 128-wide tiles (its epilogue, not the MMA, bounds the small problems).
constexpr int EPI_WARPS = 8;
constexpr int EPI_THREADS = EPI_WARPS * 32;
constexpr int GEMM_THREADS = 64 + EPI_THREADS;     // producer, MMA, epilogue
constexpr int SMEM_STAGE_BUDGET = 196608;  // bytes of the operand ring with two epilogue groups
constexpr int STG_BYTES = 4096;  // per epilogue warp: a 32 x 32 FP32 block for the transposed stores

// Bytes of one ring stage: the A image tile and this CTA's B image tiles of
// 128 rows each (CG = 2: a CTA pair, each CTA holding half of the BN rows of
// B^T), per operand plane.
__host__ __device__ constexpr inline int stage_bytes(int mode, int BN, int CG = 1) {
  return mode_planes(mode) * (IMG_BYTES + IMG_BYTES * (BN / TILE_M) / CG);
}
// Ring stages: each epilogue group beyond two takes its staging buffers
// from the ring's budget.
__host__ __device__ constexpr int num_stages(int mode, int BN, int CG = 1, int NG = 2) {
  return (SMEM_STAGE_BUDGET - (NG - 2) * 4 * STG_BYTES) / stage_bytes(mode, BN, CG) > 8
             ? 8
             : (SMEM_STAGE_BUDGET - (NG - 2) * 4 * STG_BYTES) / stage_bytes(mode, BN, CG);
}
// TMEM accumulator buffers: all 512 columns, so 128-wide tiles get four.
// With the epilogue slower than the MMAs (short contractions), the MMA issuer
// then fills the next buffers while both epilogue groups are still busy,
// instead of waiting for a buffer to be released before each tile.
__host__ __device__ constexpr int acc_bufs(int BN) { return 512 / BN; }
__host__ __device__ constexpr int smem_total(int mode, int BN, int CG = 1, int NG = 2) {
  return num_stages(mode, BN, CG, NG) * stage_bytes(mode, BN, CG) + 1024 /*align*/ +
         256 /*barriers*/ + 4 * NG * STG_BYTES;
}
__host__ __device__ constexpr int mma_kind(int mode) {
  return (mode == MODE_BF16 || mode == MODE_F16) ? KIND_F16 : mode == MODE_E4M3 ? KIND_F8 : KIND_TF32;
}
// A/B format codes of the instruction descriptor.
__host__ __device__ constexpr uint32_t ab_format(int mode) {
  return mode == MODE_BF16 ? 1u : (mode == MODE_TF32 || mode == MODE_3XTF32) ? 2u : 0u;
}

// Waits without looking at the abort flag (used while draining after an abort).
__device__ __forceinline__ bool mbar_wait_drain(uint64_t* bar, uint32_t parity, uint64_t timeout_ns) {
  int32_t never = 0;
  return mbar_wait(bar, parity, timeout_ns, &never);
}

// Stores a warp's 32 x 32 block of FP32 results through shared memory so that
// the global writes are row-contiguous: lane l holds row l (v[c] for column
// j0 + c) and mask bit c of lane l selects the entries of row l to write; row
// r starts at base + r * ld.  stg is the warp's 4 KB buffer, float4 groups
// XOR-swizzled by row (conflict-free both ways).  When every mask is full and
// rows are 16-byte aligned, each instruction writes four whole 128-byte rows;
// otherwise one row per instruction (rows with no entry are skipped).  The
// call must be warp-uniform; base + r * ld is only formed for rows written.
__device__ __forceinline__ void warp_store_f32(float* stg, const float (&v)[32], uint32_t mask,
                                               float* base, int64_t ld, bool vec, int lane) {
#pragma unroll
  for (int g = 0; g < 8; ++g)
    *reinterpret_cast<float4*>(stg + lane * 32 + ((g ^ (lane & 7)) << 2)) =
        make_float4(v[4 * g], v[4 * g + 1], v[4 * g + 2], v[4 * g + 3]);
  __syncwarp();
  if (__all_sync(0xffffffffu, mask == 0xffffffffu) && vec) {
    const int g = lane & 7;
#pragma unroll
    for (int r0 = 0; r0 < 32; r0 += 4) {
      const int r = r0 + (lane >> 3);
      const float4 t = *reinterpret_cast<const float4*>(stg + r * 32 + ((g ^ (r & 7)) << 2));
      *reinterpret_cast<float4*>(base + r * ld + 4 * g) = t;
    }
  } else if (__all_sync(0xffffffffu, mask == 0xffffffffu)) {
    // a whole block, rows not 16-byte aligned: one row per instruction (a
    // contiguous 128-byte run), every row unrolled so that the shared-memory
    // loads and global stores of several rows overlap.  (Aligned float4 runs
    // plus head and tail floats per row measured slower: four-way divergence
    // and address arithmetic per row.)
    float* p = base + lane;
    const int c4 = lane >> 2, c1 = lane & 3;
#pragma unroll 8
    for (int r = 0; r < 32; ++r) p[r * ld] = stg[r * 32 + ((c4 ^ (r & 7)) << 2) + c1];
  } else {
#pragma unroll 4
    for (int r = 0; r < 32; ++r) {
      const uint32_t m = __shfl_sync(0xffffffffu, mask, r);
      if (m == 0u) continue;
      if ((m >> lane) & 1u)
        base[r * ld + lane] = stg[r * 32 + (((lane >> 2) ^ (r & 7)) << 2) + (lane & 3)];
    }
  }
  __syncwarp();
}

// The same for a 32 x 32 block of bytes held as eight words per lane (w[q]
// holds columns 4q..4q+3); the two 16-byte halves of row l are swapped when
// bit 2 of l is set (conflict-free both ways).
__device__ __forceinline__ void warp_store_u8(uint32_t* stg, const uint32_t (&w)[8], uint32_t mask,
                                              uint8_t* base, int64_t ld, bool vec, int lane) {
  const int sw = (lane >> 2) & 1;
  *reinterpret_cast<uint4*>(stg + lane * 8 + (sw << 2)) = make_uint4(w[0], w[1], w[2], w[3]);
  *reinterpret_cast<uint4*>(stg + lane * 8 + ((sw ^ 1) << 2)) = make_uint4(w[4], w[5], w[6], w[7]);
  __syncwarp();
  if (__all_sync(0xffffffffu, mask == 0xffffffffu) && vec) {
    const int h = lane & 1;
#pragma unroll
    for (int r0 = 0; r0 < 32; r0 += 16) {
      const int r = r0 + (lane >> 1);
      const uint4 t = *reinterpret_cast<const uint4*>(stg + r * 8 + ((h ^ ((r >> 2) & 1)) << 2));
      *reinterpret_cast<uint4*>(base + r * ld + 16 * h) = t;
    }
  } else {
    const uint8_t* sb = reinterpret_cast<const uint8_t*>(stg);
#pragma unroll 4
    for (int r = 0; r < 32; ++r) {
      const uint32_t m = __shfl_sync(0xffffffffu, mask, r);
      if (m == 0u) continue;
      if ((m >> lane) & 1u)
        base[r * ld + lane] = sb[r * 32 + (((lane >> 4) ^ ((r >> 2) & 1)) << 4) + (lane & 15)];
    }
  }
  __syncwarp();
}

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// r = 2 projection (Sec. 2.1) of the sums s_m = S^(m p'), m = 1..4, returned
// as alpha^p': the larger root of gamma_0 + gamma_1 a + gamma_2 a^2 with
// gamma = (s2 s4 - s3^2, s2 s3 - s1 s4, s1 s3 - s2^2), the cross product of
// the Hankel rows [s1 s2 s3] and [s2 s3 s4].  Computed in FP32 on the sums
// normalised by lam = s2 / s1 (t_m = s_m / (s1 lam^(m-1)), so t1 = t2 = 1
// and every term is O(1)): a = lam * b with b the larger root of
// (t4 - t3^2) + (t3 - t4) b + (t3 - 1) b^2.  The roots are the 2-point Gauss
// nodes of the measure with moments s1..s4, so the larger lies between the
// r = 1 value lam and the plain norm s4^(1/4); it is clamped there (never
// binding for exact sums, bounding the effect of rounded ones).  Sums that
// do not resolve a second value (gamma_2 <= eta s2^2, i.e. t3 - 1 <= eta) or
// a root that is not positive give lam; a negative discriminant counts as 0.
// Reciprocals and square roots are the hardware approximations (about one
// ulp): the sums' own errors are orders of magnitude larger.
__device__ __forceinline__ float r2_project(float s1, float s2, float s3, float s4, float eta) {
  const float i1 = rcp_approx(s1), i2 = rcp_approx(s2);
  const float lam = s2 * i1;
  const float q = s1 * i2;
  const float t3 = (s3 * i2) * q;
  const float t4 = (s4 * i2) * q * q;
  const float g2 = t3 - 1.0f;
  if (!(g2 > eta)) return lam;
  const float g1 = t3 - t4;
  const float g0 = fmaf(-t3, t3, t4);
  const float disc = fmaxf(fmaf(g1, g1, -4.0f * g0 * g2), 0.0f);
  const float b = (sqrt_approx(disc) - g1) * rcp_approx(2.0f * g2);
  if (!(b > 0.0f)) return lam;
  return fminf(fmaxf(lam * b, lam), sqrt_approx(sqrt_approx(s4)));
}

// Finishes the r = 2 projection for the entries w3 of a warp's 32 x 32 block
// (lane l holds row l: x = this level's S^(p*/4), rs its row scale): the
// block is staged in stg and walked row by row, lane l taking column l, so
// that the three parked sums are read and C is written as whole 128-byte
// rows.  Row r's sums: S^(p*/2) at s2row + r ldp, S^(3p*/4) at s3row + r ldp,
// S^(p*) in C at crow + r ldc; cs_lane is column l's scale.  The root is
// plog correctly rounded square roots (FP32-accurate mode) or 2^(log2(a) / p').
// Called by the whole warp.
template <bool SQRT_ROOT>
__device__ __forceinline__ void r2_finish_block(float* stg, const float (&x)[32], uint32_t w3,
                                                float rs, const float* s2row, const float* s3row,
                                                int64_t ldp, float* crow, int64_t ldc,
                                                float cs_lane, float eta, int plog, float inv_p,
                                                int lane) {
#pragma unroll
  for (int g = 0; g < 8; ++g)
    *reinterpret_cast<float4*>(stg + lane * 32 + ((g ^ (lane & 7)) << 2)) =
        make_float4(x[4 * g], x[4 * g + 1], x[4 * g + 2], x[4 * g + 3]);
  __syncwarp();
  auto finish = [&](float s1, float s2, float s3, float s0, float rsr) {
    float a = r2_project(s1, s2, s3, s0, eta);
    if constexpr (SQRT_ROOT) {
      for (int t = 0; t < plog; ++t) a = sqrtf(a);
    } else if (plog > 0) {
      a = ex2_approx(lg2_approx(a) * inv_p);
    }
    return a * rsr * cs_lane;
  };
  if (__all_sync(0xffffffffu, w3 == 0xffffffffu)) {
    // a whole block: the sums of four rows (two parked, C) are loaded
    // before any is used, so their latencies overlap
#pragma unroll 1
    for (int r0 = 0; r0 < 32; r0 += 4) {
      float s2[4], s3[4], s0[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        s2[i] = __ldg(s2row + (r0 + i) * ldp + lane);  // parked at earlier levels
        s3[i] = __ldg(s3row + (r0 + i) * ldp + lane);
        s0[i] = crow[(r0 + i) * ldc + lane];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = r0 + i;
        const float rsr = __shfl_sync(0xffffffffu, rs, r);
        const float s1 = stg[r * 32 + (((lane >> 2) ^ (r & 7)) << 2) + (lane & 3)];
        crow[r * ldc + lane] = finish(s1, s2[i], s3[i], s0[i], rsr);
      }
    }
  } else {
#pragma unroll 4
    for (int r = 0; r < 32; ++r) {
      const uint32_t m = __shfl_sync(0xffffffffu, w3, r);
      const float rsr = __shfl_sync(0xffffffffu, rs, r);
      if (m == 0u) continue;
      if ((m >> lane) & 1u) {
        const float s1 = stg[r * 32 + (((lane >> 2) ^ (r & 7)) << 2) + (lane & 3)];
        const float s2 = __ldg(s2row + r * ldp + lane);  // parked at earlier levels
        const float s3 = __ldg(s3row + r * ldp + lane);
        float* c = crow + r * ldc + lane;
        *c = finish(s1, s2, s3, *c, rsr);
      }
    }
  }
  __syncwarp();
}

// Finishes the r = 1 projection for the entries `pend` of a warp's 32 x 32
// block (lane l holds row l: x = this level's S^(p), rs its row scale; C
// holds S^(2p) of these entries): (S^(2p) / S^(p))^(1/p), the ratio clamped
// to <= 1 (S is non-increasing in p), then the affine line (pa, pb) when
// `affine`, the scales, and the write-back to C -- row by row, lane l on
// column l, so that C is read and written as 128-byte rows.  Called by the
// whole warp.
template <bool SQRT_ROOT>
__device__ __forceinline__ void r1_finish_block(float* stg, const float (&x)[32], uint32_t pend,
                                                float rs, float* crow, int64_t ldc, float cs_lane,
                                                int plog, float inv_p, bool affine, float pa,
                                                float pb, int lane) {
#pragma unroll
  for (int g = 0; g < 8; ++g)
    *reinterpret_cast<float4*>(stg + lane * 32 + ((g ^ (lane & 7)) << 2)) =
        make_float4(x[4 * g], x[4 * g + 1], x[4 * g + 2], x[4 * g + 3]);
  __syncwarp();
  auto finish = [&](float s1, float s2, float rsr) {
    float y = s2 / fmaxf(s1, s2);
    if constexpr (SQRT_ROOT) {
      for (int t = 0; t < plog; ++t) y = sqrtf(y);
    } else if (plog > 0) {
      y = ex2_approx(lg2_approx(y) * inv_p);
    }
    if (affine) y = fmaf(pa, y, pb);
    return y * (rsr * cs_lane);
  };
  if (__all_sync(0xffffffffu, pend == 0xffffffffu)) {
    // a whole block: the stored sums of eight rows are loaded before any is
    // used, so their latencies overlap
    float* c0 = crow + lane;
#pragma unroll 1
    for (int r0 = 0; r0 < 32; r0 += 8) {
      float s2[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) s2[i] = c0[(r0 + i) * ldc];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int r = r0 + i;
        const float rsr = __shfl_sync(0xffffffffu, rs, r);
        const float s1 = stg[r * 32 + (((lane >> 2) ^ (r & 7)) << 2) + (lane & 3)];
        c0[r * ldc] = finish(s1, s2[i], rsr);
      }
    }
  } else {
#pragma unroll 4
    for (int r = 0; r < 32; ++r) {
      const uint32_t m = __shfl_sync(0xffffffffu, pend, r);
      const float rsr = __shfl_sync(0xffffffffu, rs, r);
      if (m == 0u) continue;
      if ((m >> lane) & 1u) {
        const float s1 = stg[r * 32 + (((lane >> 2) ^ (r & 7)) << 2) + (lane & 3)];
        float* c = crow + r * ldc + lane;
        *c = finish(s1, *c, rsr);
      }
    }
  }
  __syncwarp();
}

// ------------------------------------------------------------ roles ---
// The kernel's three roles as functions of a CTA context, so that the
// single-level kernel runs them once and the persistent grouped kernel once
// per level, with the ring positions and the tile count carried over.

// Output tile (tile row tm of 128 rows, tile column tn of BN columns) of
// list entry t: single CTAs walk the tiles in grouped raster order; a CTA
// pair walks pairs of tile rows (256 rows), rank r taking tile row 2 TM + r.
template <int CG>
__device__ __forceinline__ void tile_coords(const Prob& P, int t, uint32_t rank, int& tm, int& tn) {
  if constexpr (CG == 1) {
    raster(t - P.tile_base, P.tiles_m, P.tiles_n, tm, tn);
  } else {
    int TM;
    raster(t - P.tile_base, (P.tiles_m + 1) >> 1, P.tiles_n, TM, tn, RASTER_GM / 2);
    tm = 2 * TM + static_cast<int>(rank);
  }
}

// Shared memory, barriers and TMEM of one CTA.
struct Ctx {
  uint8_t* smem;
  uint64_t* full;
  uint64_t* empty;
  uint64_t* acc_full;
  uint64_t* acc_empty;
  uint64_t* drain;
  uint32_t* tmem_slot;
  volatile int32_t* abort_flag;
  volatile int32_t* ok_flag;  // [2 NG], epilogue item hand-off (2 per group)
  uint32_t tmem_base;
  uint64_t tmo;
  uint32_t rank;              // CTA pair: rank in the cluster (0 issues the MMAs); else 0
  int32_t wid, wstride;       // work index and stride: the cluster (pair) or the CTA
};

// Operand blocks built earlier in the same launch: flags[tile row] (A) and
// flags[b_off + tile column] (B) reach `need` once the level's images of the
// block are written.  flags == nullptr: the images come from earlier launches.
struct Ready {
  const int32_t* flags;
  int32_t need;
  int32_t b_off;
};

// Copy producer state (ring position, copies in flight per stage).
struct ProdState {
  int stage;
  uint32_t phase;
  bool first;
  bool aborted;
  int8_t pend[8];
};
// MMA issuer state (ring position).
struct MmaState {
  int stage;
  uint32_t phase;
  bool aborted;
};

// Lays out shared memory, initialises the barriers, allocates TMEM (warp 1)
// and synchronises the block.  timeout_ns limits every bounded wait of the
// roles.  Called by every thread.
template <int MODE, int BN, int CG = 1, int NG = 2>
__device__ __forceinline__ Ctx ctx_setup(bool by_tile, uint64_t timeout_ns) {
  constexpr int STAGE_BYTES = stage_bytes(MODE, BN, CG);
  constexpr int STAGES = num_stages(MODE, BN, CG, NG);
  constexpr uint32_t TMEM_COLS = acc_bufs(BN) * BN;
  extern __shared__ uint8_t smem_raw[];
  Ctx cx{};
  const uint32_t raw_addr = smem_u32(smem_raw);
  cx.smem = smem_raw + (((raw_addr + 1023u) & ~1023u) - raw_addr);
  cx.full = reinterpret_cast<uint64_t*>(cx.smem + STAGES * STAGE_BYTES);
  cx.empty = cx.full + STAGES;
  cx.acc_full = cx.empty + STAGES;
  cx.acc_empty = cx.acc_full + 4;
  cx.drain = cx.acc_empty + 4;
  cx.tmem_slot = reinterpret_cast<uint32_t*>(cx.drain + 1);
  cx.abort_flag = reinterpret_cast<volatile int32_t*>(cx.tmem_slot + 1);
  cx.ok_flag = cx.abort_flag + 1;
  cx.tmo = timeout_ns;
  if constexpr (CG == 2) {
    cx.rank = cluster_ctarank();
    cx.wid = static_cast<int32_t>(cluster_id_x());
    cx.wstride = static_cast<int32_t>(nclusters_x());
  } else {
    cx.rank = 0;
    cx.wid = static_cast<int32_t>(blockIdx.x);
    cx.wstride = static_cast<int32_t>(gridDim.x);
  }
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      // a pair: rank 0's full barrier counts both CTAs' copies (rank 1's stay unused)
      mbar_init(&cx.full[s], 1);
      mbar_init(&cx.empty[s], 1);
    }
    for (int b = 0; b < acc_bufs(BN); ++b) {
      mbar_init(&cx.acc_full[b], 1);
      // single CTA: every epilogue thread of the group arrives; a pair: one
      // lane per epilogue warp of both CTAs, on rank 0's barrier
      mbar_init(&cx.acc_empty[b], CG == 2 ? 2 * (by_tile ? 4 : 4 * NG)
                                          : (by_tile ? 128 : 128 * NG));
    }
    mbar_init(cx.drain, 1);
    *cx.abort_flag = 0;
    for (int i = 0; i < 2 * NG; ++i) cx.ok_flag[i] = 0;
    fence_barrier_init();
  }
  if (warp == 1) {
    if constexpr (CG == 2) {
      tmem_alloc_pair(cx.tmem_slot, TMEM_COLS);
      tmem_relinquish_pair();
    } else {
      tmem_alloc(cx.tmem_slot, TMEM_COLS);
      tmem_relinquish();
    }
  }
  tc_fence_before();
  if constexpr (CG == 2)
    cluster_sync_all();  // both CTAs' barriers and TMEM ready before any remote use
  else
    __syncthreads();
  tc_fence_after();
  cx.tmem_base = *cx.tmem_slot;
  return cx;
}

// Frees TMEM once every role is done (a pair: once both CTAs are done, so
// that no MMA of the pair still reads this CTA's shared memory or writes its
// TMEM).  Called by every thread.
template <int BN, int CG = 1>
__device__ __forceinline__ void ctx_teardown(const Ctx& cx) {
  if constexpr (CG == 2) {
    tc_fence_before();
    cluster_sync_all();
  } else {
    __syncthreads();
  }
  if ((threadIdx.x >> 5) == 1) {
    tc_fence_after();
    if constexpr (CG == 2)
      tmem_dealloc_pair(cx.tmem_base, acc_bufs(BN) * BN);
    else
      tmem_dealloc(cx.tmem_base, acc_bufs(BN) * BN);
  }
}

// Producer (one thread): bulk copies of the operand images of this CTA's
// tiles blockIdx.x, blockIdx.x + gridDim.x, ... < count into the ring.
template <int MODE, int BN, int CG = 1, int NG = 2>
__device__ __forceinline__ void run_producer(const Common& cm, const Level& lv, const Ctx& cx,
                                             int count, ProdState& ps, const Ready& rd,
                                             const ImgMaps* maps = nullptr) {
  constexpr int PLANES = mode_planes(MODE);
  constexpr int A_BYTES = IMG_BYTES;
  constexpr int B_BYTES = IMG_BYTES * (BN / TILE_M) / CG;
  constexpr int STAGE_BYTES = stage_bytes(MODE, BN, CG);
  constexpr int STAGES = num_stages(MODE, BN, CG, NG);
  constexpr int KIND = mma_kind(MODE);
  constexpr uint32_t IDESC = idesc_make(ab_format(MODE), TILE_M * CG, BN);
  constexpr int CHUNKS = BN / 32;
  (void)PLANES; (void)A_BYTES; (void)B_BYTES; (void)STAGE_BYTES; (void)STAGES; (void)KIND;
  (void)IDESC; (void)CHUNKS;
  uint8_t* smem = cx.smem;
  uint64_t* full = cx.full;
  uint64_t* empty = cx.empty;
  uint64_t* acc_full = cx.acc_full;
  uint64_t* acc_empty = cx.acc_empty;
  uint64_t* drain = cx.drain;
  volatile int32_t* abort_flag = cx.abort_flag;
  volatile int32_t* ok_flag = cx.ok_flag;
  const uint32_t tmem_base = cx.tmem_base;
  const uint64_t tmo = cx.tmo;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  (void)smem; (void)full; (void)empty; (void)acc_full; (void)acc_empty; (void)drain;
  (void)abort_flag; (void)ok_flag; (void)tmem_base; (void)tmo; (void)warp; (void)lane;
  if (ps.aborted) return;
    int stage = ps.stage;
      uint32_t phase = ps.phase;
      int8_t* pend = ps.pend;
      bool aborted = false;
      bool first = ps.first;
      const uint64_t pol = policy_evict_last();
      for (int idx = cx.wid; idx < count && !aborted; idx += cx.wstride) {
        const int t = lv.is_top ? idx : lv.work[idx];
        const Prob& P = prob_at(cm, find_prob(cm, t, 0));
        int tm, tn;
        tile_coords<CG>(P, t, cx.rank, tm, tn);
        if (rd.flags) {
          // operand blocks built earlier in this launch (persistent grouped
          // kernel): wait until both are ready for this level, then order
          // their generic-proxy writes before the bulk copies read them
          if (!wait_flag_geq(rd.flags + P.tm_base + tm, rd.need, tmo, abort_flag) ||
              !wait_flag_geq(rd.flags + rd.b_off + P.tn_base + tn, rd.need, tmo, abort_flag)) {
            aborted = true;
            break;
          }
          fence_proxy_async_global();
        }
        const uint8_t* a_src = lv.a_level + P.a_img + (int64_t)tm * P.KB * IMG_BYTES;
        // a single CTA's B^T blocks: all BN / 128 of the column tile (a pair
        // addresses its half through the tensor map)
        const uint8_t* b_src =
            lv.b_level + P.b_img + (int64_t)tn * (BN / TILE_M) * P.KB * IMG_BYTES;
        for (int kb = 0; kb < P.KB; ++kb) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, tmo, abort_flag)) {
            aborted = true;
            break;
          }
          pend[stage] = -1;
          const bool drop = (cm.debug_flags & 1) && first && kb == 0;
          if constexpr (CG == 2) {
            // a pair: both CTAs copy their own halves into their own ring,
            // completing on rank 0's full barrier, which rank 0 arms with the
            // bytes of both (rank 1's copies may land before it is armed: the
            // transaction count goes below zero until then).  Rank 1 may
            // only refill a stage after rank 0's MMAs freed it, so its copies
            // always count toward the phase rank 0 waits for next.
            if (!drop) {
              const uint32_t fb = cx.rank == 0 ? smem_u32(&full[stage])
                                               : mapa_shared(smem_u32(&full[stage]), 0);
              if (cx.rank == 0) mbar_arrive_expect_tx(&full[stage], 2 * STAGE_BYTES);
              const uint32_t sa = smem_u32(smem + stage * STAGE_BYTES);
#pragma unroll
              for (int pl = 0; pl < PLANES; ++pl) {
                const uint32_t base = sa + pl * (A_BYTES + B_BYTES);
                const int64_t ya = (pl * P.a_plane + ((int64_t)tm * P.KB + kb) * IMG_BYTES) >> 7;
                // this CTA's half of the B^T column tile: BN / 2 rows from
                // row tn BN + rank BN / 2 (a whole 128-row block, or half of one)
                const int brow = tn * BN + static_cast<int>(cx.rank) * (BN / 2);
                const int64_t yb =
                    ((pl * P.b_plane + ((int64_t)(brow >> 7) * P.KB + kb) * IMG_BYTES) >> 7) +
                    (brow & 127);
                tma_load_2d_pair(base, &maps->a, 0, static_cast<int>(ya), fb, pol);
                tma_load_2d_pair(base + A_BYTES, &maps->b, 0, static_cast<int>(yb), fb, pol);
              }
              pend[stage] = static_cast<int8_t>(phase);
            }
          } else if (!drop) {
            mbar_arrive_expect_tx(&full[stage], STAGE_BYTES);
            const uint32_t sa = smem_u32(smem + stage * STAGE_BYTES);
#pragma unroll
            for (int pl = 0; pl < PLANES; ++pl) {
              const uint32_t base = sa + pl * (A_BYTES + B_BYTES);
              bulk_g2s_hint(base, a_src + pl * P.a_plane + (int64_t)kb * IMG_BYTES, IMG_BYTES,
                            &full[stage], pol);
#pragma unroll
              for (int h = 0; h < BN / TILE_M / CG; ++h)
                bulk_g2s_hint(base + A_BYTES + h * IMG_BYTES,
                              b_src + pl * P.b_plane + ((int64_t)h * P.KB + kb) * IMG_BYTES,
                              IMG_BYTES, &full[stage], pol);
            }
            pend[stage] = static_cast<int8_t>(phase);
          }
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
        first = false;
      }
      ps.stage = stage;
      ps.phase = phase;
      ps.first = first;
      if (aborted) {
        ps.aborted = true;
        *abort_flag = 1;
        set_status(cm.status, PN_ETIMEOUT);
        // let every copy still in flight land before the CTA exits
        if (CG == 2 && cx.rank == 1) {
          // its copies complete on rank 0's barriers: a bounded grace period
          // (a 16 KB copy lands within microseconds)
          bool any = false;
          for (int s = 0; s < STAGES; ++s) any |= pend[s] >= 0;
          if (any) {
            const uint64_t t0 = globaltimer_ns();
            while (globaltimer_ns() - t0 < 200000ull) __nanosleep(1000);
          }
        } else {
          for (int s = 0; s < STAGES; ++s)
            if (pend[s] >= 0) mbar_wait_drain(&full[s], static_cast<uint32_t>(pend[s]), tmo);
        }
      }
}

// MMA issuer (one thread): the tensor-core K loop of each tile into the
// accumulator buffer it mod acc_bufs(BN), it = it0, it0 + 1, ... counting
// this CTA's tiles over the whole launch.
template <int MODE, int BN, int CG = 1, int NG = 2>
__device__ __forceinline__ void run_mma(const Common& cm, const Level& lv, const Ctx& cx,
                                        int count, int it0, MmaState& ms) {
  constexpr int PLANES = mode_planes(MODE);
  constexpr int A_BYTES = IMG_BYTES;
  constexpr int B_BYTES = IMG_BYTES * (BN / TILE_M) / CG;
  constexpr int STAGE_BYTES = stage_bytes(MODE, BN, CG);
  constexpr int STAGES = num_stages(MODE, BN, CG, NG);
  constexpr int KIND = mma_kind(MODE);
  constexpr uint32_t IDESC = idesc_make(ab_format(MODE), TILE_M * CG, BN);
  constexpr int CHUNKS = BN / 32;
  (void)PLANES; (void)A_BYTES; (void)B_BYTES; (void)STAGE_BYTES; (void)STAGES; (void)KIND;
  (void)IDESC; (void)CHUNKS;
  uint8_t* smem = cx.smem;
  uint64_t* full = cx.full;
  uint64_t* empty = cx.empty;
  uint64_t* acc_full = cx.acc_full;
  uint64_t* acc_empty = cx.acc_empty;
  uint64_t* drain = cx.drain;
  volatile int32_t* abort_flag = cx.abort_flag;
  volatile int32_t* ok_flag = cx.ok_flag;
  const uint32_t tmem_base = cx.tmem_base;
  const uint64_t tmo = cx.tmo;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  (void)smem; (void)full; (void)empty; (void)acc_full; (void)acc_empty; (void)drain;
  (void)abort_flag; (void)ok_flag; (void)tmem_base; (void)tmo; (void)warp; (void)lane;
  if (ms.aborted) return;
  if constexpr (CG == 2) {
    if (cx.rank == 1) return;  // rank 0 issues the pair's MMAs
  }
    int stage = ms.stage;
      uint32_t phase = ms.phase;
      bool aborted = false;
      int it = it0;
      for (int idx = cx.wid; idx < count && !aborted; idx += cx.wstride, ++it) {
        const int t = lv.is_top ? idx : lv.work[idx];
        const Prob& P = prob_at(cm, find_prob(cm, t, 0));
        constexpr int NB = acc_bufs(BN);
        const int buf = it & (NB - 1);
        // a pair: the epilogues of both CTAs release the accumulator
        if (!mbar_wait(&acc_empty[buf], ((it / NB) & 1) ^ 1u, tmo, abort_flag)) {
          aborted = true;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem_base + buf * BN;
        for (int kb = 0; kb < P.KB; ++kb) {
          // a pair: rank 0's barrier completes once both CTAs' copies landed
          if (!mbar_wait(&full[stage], phase, tmo, abort_flag)) {
            aborted = true;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + stage * STAGE_BYTES);
          const uint32_t sb = sa + A_BYTES;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t ad = sdesc_sw128(sa + kk * 32);
            const uint64_t bd = sdesc_sw128(sb + kk * 32);
            const uint32_t acc = (kb | kk) != 0;
            if constexpr (CG == 2) {
              // M = 256 over both CTAs' A halves, N = BN over both B halves
              if constexpr (PLANES == 1) {
                mma_pair<KIND>(d, ad, bd, IDESC, acc);
              } else {
                const uint32_t sa_lo = sa + A_BYTES + B_BYTES, sb_lo = sa_lo + A_BYTES;
                const uint64_t adl = sdesc_sw128(sa_lo + kk * 32);
                const uint64_t bdl = sdesc_sw128(sb_lo + kk * 32);
                mma_pair<KIND>(d, adl, bd, IDESC, acc);  // small terms first
                mma_pair<KIND>(d, ad, bdl, IDESC, 1u);
                mma_pair<KIND>(d, ad, bd, IDESC, 1u);
              }
            } else if constexpr (PLANES == 1) {
              mma_ss<KIND>(d, ad, bd, IDESC, acc);
            } else {
              const uint32_t sa_lo = sa + A_BYTES + B_BYTES, sb_lo = sa_lo + A_BYTES;
              const uint64_t adl = sdesc_sw128(sa_lo + kk * 32);
              const uint64_t bdl = sdesc_sw128(sb_lo + kk * 32);
              mma_ss<KIND>(d, adl, bd, IDESC, acc);  // small terms first
              mma_ss<KIND>(d, ad, bdl, IDESC, 1u);
              mma_ss<KIND>(d, ad, bd, IDESC, 1u);
            }
          }
          if constexpr (CG == 2)
            mma_commit_pair(&empty[stage], 0x3);  // frees the stage in both CTAs
          else
            mma_commit(&empty[stage]);
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (aborted) break;
        if constexpr (CG == 2)
          mma_commit_pair(&acc_full[buf], 0x3);  // both CTAs' accumulators are complete
        else
          mma_commit(&acc_full[buf]);
      }
      ms.stage = stage;
      ms.phase = phase;
      if (aborted) {
        ms.aborted = true;
        *abort_flag = 1;
        set_status(cm.status, PN_ETIMEOUT);
        if constexpr (CG == 2)
          mma_commit_pair(drain, 0x1);  // completes once every issued MMA has finished
        else
          mma_commit(drain);  // completes once every issued MMA has finished
        mbar_wait_drain(drain, 0, tmo);
      }
}

// Epilogue (warps 2-9).  EPI 0: p-norm epilogue (tau test, root, un-scaling,
// p_sel / S_sel, work lists).  EPI 1: gradient epilogue of the adjoint,
// out (+)= acc * x'^(p-1) / s with x the source element at the output position
// and s its row (grad_axis 0) or column (1) scale; the first p present
// overwrites, later ones add.
// PLAIN: the plain estimator only (no projection state, no parked sums, no
// affine line), compiled without those paths for launches that never take them.
template <int MODE, int BN, int EPI, int CG = 1, int NG = 2, bool PLAIN = false>
__device__ __forceinline__ void run_epilogue(const Common& cm, const Level& lv, const Ctx& cx,
                                             int count, bool by_tile, int it0, const Ready& rd) {
  constexpr int PLANES = mode_planes(MODE);
  constexpr int A_BYTES = IMG_BYTES;
  constexpr int B_BYTES = IMG_BYTES * (BN / TILE_M) / CG;
  constexpr int STAGE_BYTES = stage_bytes(MODE, BN, CG);
  constexpr int STAGES = num_stages(MODE, BN, CG, NG);
  constexpr int KIND = mma_kind(MODE);
  constexpr uint32_t IDESC = idesc_make(ab_format(MODE), TILE_M * CG, BN);
  constexpr int CHUNKS = BN / 32;
  (void)PLANES; (void)A_BYTES; (void)B_BYTES; (void)STAGE_BYTES; (void)STAGES; (void)KIND;
  (void)IDESC; (void)CHUNKS;
  uint8_t* smem = cx.smem;
  uint64_t* full = cx.full;
  uint64_t* empty = cx.empty;
  uint64_t* acc_full = cx.acc_full;
  uint64_t* acc_empty = cx.acc_empty;
  uint64_t* drain = cx.drain;
  volatile int32_t* abort_flag = cx.abort_flag;
  volatile int32_t* ok_flag = cx.ok_flag;
  const uint32_t tmem_base = cx.tmem_base;
  const uint64_t tmo = cx.tmo;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  (void)smem; (void)full; (void)empty; (void)acc_full; (void)acc_empty; (void)drain;
  (void)abort_flag; (void)ok_flag; (void)tmem_base; (void)tmo; (void)warp; (void)lane;
    // Warp w may only read TMEM lanes 32*(w%4)..+31 (one output row each).
    // With several tiles per CTA (by_tile) the epilogue warps form two groups
    // of four, one warp per lane quarter each; group g finishes every other
    // tile (it = g mod 2; accumulator buffers g, g + 2, ... of the
    // acc_bufs(BN)), so two tiles' epilogues overlap their latencies.  With few tiles all eight warps
    // finish every tile, the two warps of a lane quarter taking one half of
    // the columns each, which shortens the last tile's epilogue.
    const int ew = warp - 2;
    const int quarter = warp & 3;
    const int grp = by_tile ? ew >> 2 : 0;
    // (more than two groups only with by_tile)
    const int nch = by_tile ? CHUNKS : CHUNKS / NG;  // 32-column chunks per warp
    const int ch0 = by_tile ? 0 : (ew >> 2) * nch;
    const int gthreads = by_tile ? 128 : 128 * NG;
    const int et = (threadIdx.x - 64) & (gthreads - 1);  // thread of the group
    float* stg = reinterpret_cast<float*>(smem + STAGES * STAGE_BYTES + 256 + ew * STG_BYTES);
    const int step = by_tile ? NG : 1;
    for (int j = by_tile ? ((grp - it0) % NG + NG) % NG : 0;; j += step) {
      const int idx = cx.wid + j * cx.wstride;
      if (idx >= count) break;
      const int it = it0 + j;
      const int t = lv.is_top ? idx : lv.work[idx];
      const int g = find_prob(cm, t, 0);
      const Prob& P = prob_at(cm, g);
      // the fields the chunk loop uses, held in registers: through the
      // reference into the grouped table every store to C could alias them
      const int PN = P.N;
      const float Ptau = P.tau;
      float* const PC = P.C;
      const int64_t Pldc = P.ldc;
      const bool Pvec = P.vec_c != 0;
      uint8_t* const Ppsel = P.psel;
      float* const PSsel = P.Ssel;
      const int64_t Pldaux = P.ldaux;
      const int64_t Prc_c = P.rc_c;
      int tm, tn;
      tile_coords<CG>(P, t, cx.rank, tm, tn);
      constexpr int NB = acc_bufs(BN);
      const int buf = it & (NB - 1);
      const int okslot = 2 * grp + ((it / NG) & 1);
      if (et == 0) {
        const bool ok = mbar_wait(&acc_full[buf], (it / NB) & 1, tmo, abort_flag);
        if (!ok) {
          *abort_flag = 1;
          set_status(cm.status, PN_ETIMEOUT);
        }
        // operand blocks built in this launch: acquire their flags, so that
        // the scales written with them are visible to the whole group after
        // the barrier below
        if (ok && rd.flags) {
          ld_acquire_gpu(rd.flags + P.tm_base + tm);
          ld_acquire_gpu(rd.flags + rd.b_off + P.tn_base + tn);
        }
        ok_flag[okslot] = ok ? 1 : 0;
      }
      bar_sync_named(1 + grp, gthreads);
      if (!ok_flag[okslot]) break;
      tc_fence_after();

      const int i = tm * TILE_M + quarter * 32 + lane;
      const bool row_ok = i < P.M;
      // row scale: the p-norm epilogue, or the dA gradient (grad_axis 0)
      const bool use_rs = row_ok && (EPI == 0 || cm.grad_axis == 0);
      const float rs = use_rs ? cm.r[P.rc_r + i] : 0.0f;
      const int64_t st_idx = P.state_off + (int64_t)i * P.state_ld + tn * CHUNKS + ch0;
      const uint32_t* st_row = cm.state + st_idx;
      const float inv_p = __uint_as_float((127u - (uint32_t)lv.plog) << 23);  // 2^-plog
      // bias correction of this level's estimates (scaled space): K^(-1/p),
      // or the affine line of this level's class
      float corr_a = 1.0f, corr_b = 0.0f;
      if (EPI == 0 && cm.corr == 1) corr_a = exp2f(-log2f(static_cast<float>(P.K)) * inv_p);
      if (EPI == 0 && !PLAIN && cm.corr == 2) {
        corr_a = cm.coef[2 * lv.q];
        corr_b = cm.coef[2 * lv.q + 1];
      }
      uint32_t res_all[CHUNKS], pend_all[CHUNKS], pend2_all[CHUNKS];
      bool any_left = false;
      bool new_chain = false;  // r = 2: an entry of the tile resolved here
      // the warp's chunks that hold outputs: none when its 32 rows all lie
      // past M (a padded tile of a small problem), else those starting
      // before N; the others are neither read from TMEM nor processed
      const int jw = PN - (tn * BN + ch0 * 32);
      const int nv = (tm * TILE_M + quarter * 32 >= P.M || jw <= 0) ? 0
                     : ((jw + 31) >> 5) < nch                        ? ((jw + 31) >> 5)
                                                                     : nch;
      // hands the accumulator back once this warp's last TMEM load completed
      auto release = [&]() {
        tc_fence_before();
        if constexpr (CG == 2) {
          // one lane per warp, on rank 0's barrier (the MMA issuer's)
          __syncwarp();
          if (lane == 0) {
            if (cx.rank == 0)
              mbar_arrive(&acc_empty[buf]);
            else
              mbar_arrive_peer(mapa_shared(smem_u32(&acc_empty[buf]), 0));
          }
        } else {
          mbar_arrive(&acc_empty[buf]);
        }
      };
      if (nv == 0) release();
#pragma unroll 1
      for (int hc = 0; hc < nv; ++hc) {
        const int ch = ch0 + hc;
        uint32_t v[32];
        tmem_ld_32x32b_x32(tmem_base + ((uint32_t)(quarter * 32) << 16) + buf * BN + ch * 32, v);
        tmem_ld_wait();
        if (hc == nv - 1) release();
        const int j0 = tn * BN + ch * 32;
        uint32_t res = 0;
        pend_all[hc] = 0;
        pend2_all[hc] = 0;
        if constexpr (EPI == 1) {
          if (row_ok && j0 < PN) {
            const int jn = PN - j0 < 32 ? PN - j0 : 32;
            const float* erow = P.A + (int64_t)i * P.lda + j0;
            float* orow = PC + (int64_t)i * Pldc + j0;
            const bool vec = jn == 32 && Pvec;
            const bool first = (*lv.pmask >> (lv.q + 1)) == 0u;
            float x[32], sv[32];
            if (vec) {
#pragma unroll
              for (int e = 0; e < 32; e += 4) {
                const float4 t4 = __ldg(reinterpret_cast<const float4*>(erow + e));
                x[e] = t4.x; x[e + 1] = t4.y; x[e + 2] = t4.z; x[e + 3] = t4.w;
              }
            } else {
#pragma unroll
              for (int e = 0; e < 32; ++e) x[e] = e < jn ? __ldg(erow + e) : 0.0f;
            }
            if (cm.grad_axis == 0) {
#pragma unroll
              for (int e = 0; e < 32; ++e) sv[e] = rs;
            } else {
              const float* cs = cm.c + Prc_c + j0;
#pragma unroll
              for (int e = 0; e < 32; ++e) sv[e] = e < jn ? __ldg(cs + e) : 1.0f;
            }
#pragma unroll
            for (int e = 0; e < 32; ++e) x[e] = grad_factor(__uint_as_float(v[e]), x[e], sv[e], lv.plog);
            if (!first) {
              if (vec) {
#pragma unroll
                for (int e = 0; e < 32; e += 4) {
                  const float4 o4 = *reinterpret_cast<const float4*>(orow + e);
                  x[e] += o4.x; x[e + 1] += o4.y; x[e + 2] += o4.z; x[e + 3] += o4.w;
                }
              } else {
#pragma unroll
                for (int e = 0; e < 32; ++e)
                  if (e < jn) x[e] += orow[e];
              }
            }
            if (vec) {
#pragma unroll
              for (int e = 0; e < 32; e += 4)
                *reinterpret_cast<float4*>(orow + e) = make_float4(x[e], x[e + 1], x[e + 2], x[e + 3]);
            } else {
#pragma unroll
              for (int e = 0; e < 32; ++e)
                if (e < jn) orow[e] = x[e];
            }
          }
        } else if (j0 < PN) {  // warp-uniform: rows past M resolve nothing
          if (!row_ok) res = 0xffffffffu;
          else if (!lv.is_top) res = st_row[hc];
          const int jn = PN - j0 < 32 ? PN - j0 : 32;
          const uint32_t inrange = jn == 32 ? 0xffffffffu : ((1u << jn) - 1u);
          // entries to resolve at this p: not yet resolved, in range, and stable
          // (or the smallest p, which takes whatever is left)
          uint32_t stable = 0, near = 0;
          float x[32];
          float mn = FLT_MAX;
#pragma unroll
          for (int e = 0; e < 32; ++e) {
            x[e] = mode_op_shift(MODE) ? __uint_as_float(v[e]) * cm.unscale : __uint_as_float(v[e]);
            mn = fminf(mn, x[e]);
          }
          if (jn == 32 && mn >= 10.0f * Ptau) {
            // the common case: every entry of the lane's chunk is stable, none
            // within a decade of tau (no per-entry masks to build)
            stable = 0xffffffffu;
          } else {
#pragma unroll
            for (int e = 0; e < 32; ++e) {
              stable |= (x[e] >= Ptau ? 1u : 0u) << e;
              near |= (x[e] < 10.0f * Ptau ? 1u : 0u) << e;
            }
          }
          const uint32_t open = inrange & ~res;
          // a half level (r = 2) resolves nothing: its p is not in P
          const uint32_t cand = lv.half ? 0u : lv.is_bottom ? open : (open & stable);
          any_left |= (open & ~cand) != 0u;
          // FP64 near tau only for the FP32-range formats (the host's fp64_near rule)
          constexpr bool FP64_NEAR = MODE == MODE_3XTF32 || MODE == MODE_TF32 || MODE == MODE_BF16;
          near &= cand & (FP64_NEAR && cm.fp64_near ? 0xffffffffu : 0u);
          // r = 1 projection (Sec. 2.1): entries resolved at 2p hold S^(2p) in C;
          // with S^(p) from this level the estimate is (S^(2p) / S^(p))^(1/p).
          // The ratio is clamped to <= 1 (S is non-increasing in p).
          const uint32_t pend = !PLAIN && lv.proj_here && row_ok ? cm.pend[st_idx + hc] : 0u;
          if (!PLAIN && lv.proj_here && __any_sync(0xffffffffu, pend != 0u)) {
            const float cs_lane = lane < PN - j0 ? __ldg(cm.c + Prc_c + j0 + lane) : 0.0f;
            // the affine line of p*'s class (the level above)
            const bool affine = cm.corr == 2;
            const float pa = affine ? cm.coef[2 * (lv.q + 1)] : 1.0f;
            const float pb = affine ? cm.coef[2 * (lv.q + 1) + 1] : 0.0f;
            r1_finish_block<MODE == MODE_3XTF32>(
                stg, x, pend, rs, PC + ((int64_t)tm * TILE_M + quarter * 32) * Pldc + j0, Pldc,
                cs_lane, lv.plog, inv_p, affine, pa, pb, lane);
          }
          if (!PLAIN && lv.proj_next) {
            any_left |= cand != 0u;  // their S^(p/2) comes from the next level
            pend_all[hc] = cand;
          }
          // r = 2 projection (Sec. 2.1): entries resolved at p* wait, in stages
          // 1..3, for S^(3p*/4) (half level), S^(p*/2) and S^(p*/4); C keeps
          // S^(p*), the two middle sums are parked in the workspace
          if (!PLAIN && (lv.r2_state || lv.r2_new)) {
            uint32_t b0 = 0, b1 = 0;
            if (lv.r2_state && row_ok) {
              b0 = cm.pend[st_idx + hc];
              b1 = cm.pend2[st_idx + hc];
            }
            // rows of this warp's block in the parked arrays and in C
            const int64_t ibr = (int64_t)tm * TILE_M + quarter * 32;
            float* park3 = cm.park + ibr * PN + j0;        // S^(3p*/4)
            float* park2 = park3 + (int64_t)P.M * PN;      // S^(p*/2)
            if (lv.half) {
              const uint32_t w1 = b0 & ~b1;
              if (__any_sync(0xffffffffu, w1 != 0u))
                warp_store_f32(stg, x, w1, park3, PN, Pvec, lane);
              b0 &= ~w1;
              b1 |= w1;
            } else if (lv.r2_state) {
              const uint32_t w2 = b1 & ~b0, w3 = b0 & b1;
              if (__any_sync(0xffffffffu, w2 != 0u))
                warp_store_f32(stg, x, w2, park2, PN, Pvec, lane);
              if (__any_sync(0xffffffffu, w3 != 0u)) {
                // this level's S is S^(p'), p' = p*/4: finish the projection
                const float cs_lane = lane < PN - j0 ? __ldg(cm.c + Prc_c + j0 + lane) : 0.0f;
                r2_finish_block<MODE == MODE_3XTF32>(stg, x, w3, rs, park2, park3, PN,
                                                     PC + ibr * Pldc + j0, Pldc, cs_lane,
                                                     cm.r2_eta, lv.plog, inv_p, lane);
              }
              b0 = (b0 | w2) & ~w3;
              b1 &= ~w3;
            }
            if (lv.r2_new) {
              b0 |= cand;  // stage 1: their S^(3p*/4) comes next
              new_chain |= cand != 0u;
            }
            pend_all[hc] = b0;
            pend2_all[hc] = b1;
            any_left |= (b0 | b1) != 0u;
          }
          if (__any_sync(0xffffffffu, cand != 0u)) {
            const uint32_t pbits = lv.plog * 0x01010101u;
            uint32_t pw[8];
            if (Ppsel) {
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                const uint32_t nb = (~stable >> (4 * q)) & 0xfu;  // unstable bytes
                const uint32_t flag =
                    (nb & 1u) | ((nb & 2u) << 7) | ((nb & 4u) << 14) | ((nb & 8u) << 21);
                pw[q] = pbits | (flag << 7);
              }
            }
            // rows of this warp's block start at ibase
            const int64_t ibase = (int64_t)tm * TILE_M + quarter * 32;
            // S_sel before x is overwritten by the root
            if (PSsel)
              warp_store_f32(stg, x, cand, PSsel + ibase * Pldaux + j0, Pldaux, Pvec, lane);
            // a projection still to come (r = 1: level p/2 below; r = 2: the
            // chain down to p/4): C keeps S^(p) until then
            if (PLAIN || (!lv.proj_next && !lv.r2_new)) {
              if constexpr (MODE == MODE_3XTF32) {
                // FP32-accurate mode: (S^(p))^(1/p) for p = 2^plog as plog correctly
                // rounded square roots (about one ulp in total); repeated APSP
                // squarings double any bias each step, so no approximation here
                for (int s2 = 0; s2 < lv.plog; ++s2) {
#pragma unroll
                  for (int e = 0; e < 32; ++e) x[e] = sqrtf(x[e]);
                }
              } else if (lv.plog > 0) {
                // (S^(p))^(1/p) = 2^(log2(S) / p): two MUFU operations, relative
                // error ~2^-22, far below the operand rounding of these formats
#pragma unroll
                for (int e = 0; e < 32; ++e) x[e] = ex2_approx(lg2_approx(x[e]) * inv_p);
              }
              if (FP64_NEAR && near) {
                // within a decade of tau, which for these formats sits near the
                // FP32 underflow range: root in FP64
#pragma unroll
                for (int e = 0; e < 32; ++e) {
                  if ((near >> e) & 1u) {
                    double dr = static_cast<double>(__uint_as_float(v[e]) * cm.unscale);
                    for (int s2 = 0; s2 < lv.plog; ++s2) dr = sqrt(dr);
                    x[e] = static_cast<float>(dr);
                  }
                }
              }
              if (cm.corr) {
#pragma unroll
                for (int e = 0; e < 32; ++e) x[e] = fmaf(corr_a, x[e], corr_b);
              }
              const float* cs = cm.c + Prc_c + j0;
              if (jn == 32 && Pvec) {
#pragma unroll
                for (int e = 0; e < 32; e += 4) {
                  const float4 cv = __ldg(reinterpret_cast<const float4*>(cs + e));
                  x[e] *= rs * cv.x; x[e + 1] *= rs * cv.y; x[e + 2] *= rs * cv.z; x[e + 3] *= rs * cv.w;
                }
              } else {
                // one load per lane, broadcast by shuffles (the same products)
                const float cl = lane < jn ? __ldg(cs + lane) : 0.0f;
#pragma unroll
                for (int e = 0; e < 32; ++e) x[e] *= rs * __shfl_sync(0xffffffffu, cl, e);
              }
              if (cm.post) {
                // APSP squaring: distances are >= 0 (x <= 1) and d_ii = 0 (x_ii = 1)
                if (cm.post == 2) {
#pragma unroll
                  for (int e = 0; e < 32; ++e) x[e] = fminf(x[e], 1.0f);
                }
#pragma unroll
                for (int e = 0; e < 32; ++e)
                  if (j0 + e == i) x[e] = 1.0f;
              }
            }
            warp_store_f32(stg, x, cand, PC + ibase * Pldc + j0, Pldc, Pvec, lane);
            if (Ppsel)
              warp_store_u8(reinterpret_cast<uint32_t*>(stg), pw, cand,
                            Ppsel + ibase * Pldaux + j0, Pldaux, Pvec, lane);
            res |= cand;
          }
        }
        res_all[hc] = res;
      }
      if (EPI == 0 && !lv.is_bottom) {
        const bool tile_left = bar_red_or(any_left, 1 + NG + grp, gthreads);
        // a pair's tile goes down if either half has entries left, so each
        // half's state is written whenever it could be needed
        if (tile_left || CG == 2) {
          if (row_ok) {
            uint32_t* st_w = cm.state + st_idx;
#pragma unroll
            for (int hc = 0; hc < CHUNKS; ++hc)
              if (hc < nv) st_w[hc] = res_all[hc];
            if (!PLAIN && cm.pend) {
#pragma unroll
              for (int hc = 0; hc < CHUNKS; ++hc)
                if (hc < nv) cm.pend[st_idx + hc] = pend_all[hc];
            }
            if (!PLAIN && cm.pend2) {
#pragma unroll
              for (int hc = 0; hc < CHUNKS; ++hc)
                if (hc < nv) cm.pend2[st_idx + hc] = pend2_all[hc];
            }
          }
          // r = 2: a tile that starts no chain here skips the half level
          const bool chain = !PLAIN && lv.skip_work && bar_red_or(new_chain, 1 + NG + grp, gthreads);
          bool skip = lv.skip_work && !chain;
          bool push = et == 0 && tile_left;
          if constexpr (CG == 2) {
            // a pair's tile is pushed once, with both halves' decisions: each
            // half adds its bits (entries left, a chain started) in its own
            // field and one arrival; the second to arrive pushes if either
            // half has entries left, to the half level if either started a
            // chain
            push = false;
            if (et == 0) {
              const uint32_t mine = (tile_left ? 1u : 0u) | (chain ? 2u : 0u);
              const uint32_t old =
                  atomicAdd(lv.pair_pushed + t, (1u << 8) | (mine << (2 * cx.rank)));
              if ((old >> 8) != 0u) {
                const uint32_t both = mine | ((old >> (2 * (cx.rank ^ 1u))) & 3u);
                push = (both & 1u) != 0u;
                skip = lv.skip_work && (both & 2u) == 0u;
              }
            }
          }
          if (push) {
            int32_t* cnt = skip ? lv.skip_count : lv.next_count;
            const int slot = atomicAdd(cnt, 1);
            (skip ? lv.skip_work : lv.next_work)[slot] = t;
            (skip ? lv.skip_rflag : lv.next_rflag)[P.tm_base + tm] = 1;
            if constexpr (CG == 2) (skip ? lv.skip_rflag : lv.next_rflag)[P.tm_base + (tm ^ 1)] = 1;
            (skip ? lv.skip_cflag : lv.next_cflag)[P.tn_base + tn] = 1;
          }
        }
      }
    }
}

// One p level: every CTA processes tiles blockIdx.x, blockIdx.x + gridDim.x,
// ... of the level's tile list (the whole problem at the top level).
template <int CG>
using MapsArg = typename std::conditional<CG == 2, ImgMaps, NoMaps>::type;

template <int MODE, int BN, int EPI, int CG = 1>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
    k_gemm_level(const __grid_constant__ Common cm, const __grid_constant__ Level lv,
                 const __grid_constant__ MapsArg<CG> maps) {
  static_assert(num_stages(MODE, BN, CG) >= 2, "operand ring too small");
  pdl_wait();
  pdl_trigger();
  if constexpr (EPI == 1) {
    if (!((*lv.pmask >> lv.q) & 1u)) return;  // no entry selected this p
  }
  const int count = lv.is_top ? cm.total_tiles : *lv.work_count;
  // uniform: nothing for this CTA (a pair: for this cluster, both CTAs alike)
  const int wid = CG == 2 ? static_cast<int>(cluster_id_x()) : static_cast<int>(blockIdx.x);
  if (wid >= count) return;
  // epilogue split: tile per warp group where the epilogue, not the MMA,
  // bounds a tile (grouped problems, or short contractions)
  const bool by_tile = count >= 4 * static_cast<int>(gridDim.x) / CG &&
                       (cm.nprob > 1 || cm.single.KB * mode_planes(MODE) <= 32);
  const Ctx cx = ctx_setup<MODE, BN, CG>(by_tile, cm.timeout_ns);
  const Ready none{nullptr, 0, 0};
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    if (lane == 0) {
      ProdState ps{};
      for (int s = 0; s < 8; ++s) ps.pend[s] = -1;
      ps.first = true;
      if constexpr (CG == 2)
        run_producer<MODE, BN, CG>(cm, lv, cx, count, ps, none, &maps);
      else
        run_producer<MODE, BN, CG>(cm, lv, cx, count, ps, none);
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      MmaState ms{};
      run_mma<MODE, BN, CG>(cm, lv, cx, count, 0, ms);
    }
    __syncwarp();
  } else {
    run_epilogue<MODE, BN, EPI, CG>(cm, lv, cx, count, by_tile, 0, none);
  }
  ctx_teardown<BN, CG>(cx);
}

template <int MODE, int BN, int EPI, int CG = 1>
inline int set_attr_t() {
  static int done = 0;
  if (done) return 0;
  const cudaError_t e = cudaFuncSetAttribute(k_gemm_level<MODE, BN, EPI, CG>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             smem_total(MODE, BN, CG));
  if (e == cudaSuccess) done = 1;
  return e;
}

template <int MODE, int BN, int EPI = 0>
inline int launch_t(const Common& cm, const Level& lv, int num_sms, void* stream) {
  const int e = set_attr_t<MODE, BN, EPI>();
  if (e) return e;
  int grid = cm.total_tiles < num_sms ? cm.total_tiles : num_sms;
  if (grid < 1) return 0;
  const cudaError_t le = launch_pdl(k_gemm_level<MODE, BN, EPI>, dim3(grid), dim3(GEMM_THREADS),
                                    smem_total(MODE, BN), stream, cm, lv, NoMaps{});
  return le != cudaSuccess ? le : cudaGetLastError();
}

// A CTA pair per 256 x BN output tile (cta_group::2): clusters of two CTAs,
// one cluster per pair of SMs (cm.total_tiles counts pair tiles).  EPI as for
// k_gemm_level.
template <int MODE, int BN, int EPI = 0>
inline int launch_pair_t(const Common& cm, const Level& lv, int num_sms, void* stream) {
  const int e = set_attr_t<MODE, BN, EPI, 2>();
  if (e) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(GEMM_THREADS);
  cfg.dynamicSmemBytes = smem_total(MODE, BN, 2);
  cfg.stream = static_cast<cudaStream_t>(stream);
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;  // see launch_pdl
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;  // the occupancy query below sees the cluster shape only
  // A pair needs two SMs of one GPC; with an odd number of SMs in a GPC fewer
  // than num_sms / 2 pairs fit at once.  The tile walk is persistent (each
  // pair strides over the tiles), so a pair that is not resident would start
  // its whole share after the others end: launch only resident pairs.
  int dev = 0;
  cudaGetDevice(&dev);
  static int resident[64] = {0};
  int pairs = num_sms / 2;
  if (dev >= 0 && dev < 64) {
    if (resident[dev] == 0) {
      cfg.gridDim = dim3(static_cast<unsigned>(2 * pairs));
      int n = 0;
      if (cudaOccupancyMaxActiveClusters(&n, k_gemm_level<MODE, BN, EPI, 2>, &cfg) != cudaSuccess ||
          n < 1) {
        cudaGetLastError();
        n = pairs;
      }
      resident[dev] = n;
    }
    if (resident[dev] < pairs) pairs = resident[dev];
  }
  const int clusters = cm.total_tiles < pairs ? cm.total_tiles : pairs;
  if (clusters < 1) return 0;
  cfg.gridDim = dim3(static_cast<unsigned>(2 * clusters));
  cfg.numAttrs = 2;
  // the operand-image regions as tensors of 128-byte rows (the pair's copies
  // complete on rank 0's barriers, which only tensor copies can address)
  ImgMaps maps;
  const Prob& P = cm.single;
  constexpr int PL = mode_planes(MODE);
  if (cm.nprob != 1 ||
      !encode_img_rows(maps.a, lv.a_level + P.a_img, P.a_plane * PL) ||
      !encode_img_rows(maps.b, lv.b_level + P.b_img, P.b_plane * PL, BN / 2))
    return cudaErrorNotSupported;
  const cudaError_t le = cudaLaunchKernelEx(&cfg, k_gemm_level<MODE, BN, EPI, 2>, cm, lv, maps);
  return le != cudaSuccess ? le : cudaGetLastError();
}

}  // namespace gemm
}  // namespace pn
