// Operand-image building blocks shared by the prologue kernels and the
// persistent grouped kernel: the domain test and maxima on raw float bits,
// the power-of-two scales (Sec. 2.1, H'), and the per-tile powered images
// (Alg. 5, first loop) written in the tensor cores' swizzled K-major layout.
// The image functions are run by PRO_THREADS threads; `t` is the calling
// thread's index among them and `bar` the barrier that synchronises them
// (0: the whole block, else a named barrier of PRO_THREADS threads).
#pragma once
#include "pn_pack.cuh"

namespace pn {
namespace {

constexpr int PRO_THREADS = 256;

__device__ __forceinline__ bool in_domain(float x) {
  // R+ with every power-of-two scale representable: 0 <= x <= 2^127.
  return x >= 0.0f && x <= 1.7014118346046923e38f;
}

__device__ __forceinline__ float nonneg_bits_max(float m) { return m > 0.0f ? m : 0.0f; }

// ------------------------------------------------------------- maxima ---
// A unit: 128 rows x 1024 columns of A; each warp reduces 16 rows.  B unit:
// 128 columns x 256 rows of B; each thread keeps the maxima of 4 columns over
// 32 rows, then the 8 row groups are combined in shared memory.  One
// atomicMax per row / column per unit.
//
// Non-negative floats order like their bit patterns, and every value of the
// domain [0, 2^127] has bits <= DOMAIN_MAX_BITS, so the maxima run on the raw
// bits: one unsigned max per value gives both the maximum and the domain
// test.  A thread whose running maximum is above DOMAIN_MAX_BITS (one of its
// values is negative, -0, +inf, NaN or above 2^127) goes over its values again
// with the exact test, which flags the error and yields the maximum of the
// non-negative values.
constexpr uint32_t DOMAIN_MAX_BITS = 0x7F000000u;  // bits of 2^127

__device__ __forceinline__ uint32_t umax3(uint32_t a, uint32_t b, uint32_t c) {
  return max(a, max(b, c));
}

// Exact pass over len values src[0], src[step], ...: the maximum of the
// non-negative values as bits (at most those of +inf), with bit 31 set if any
// value is outside the domain.
__device__ __forceinline__ uint32_t exact_max_bits(const float* src, int64_t step, int len) {
  float m = 0.0f;
  bool bad = false;
  for (int t = 0; t < len; ++t) {
    const float x = __ldg(src + t * step);
    bad |= !in_domain(x);
    m = fmaxf(m, x);
  }
  return __float_as_uint(nonneg_bits_max(m)) | (bad ? 0x80000000u : 0u);
}

// Folds the error bit of exact_max_bits into bad and returns the maximum.
__device__ __forceinline__ uint32_t take_exact(uint32_t e, bool& bad) {
  bad |= (e >> 31) != 0u;
  return e & 0x7FFFFFFFu;
}

__device__ __forceinline__ void img_sync(int bar) {
  if (bar == 0)
    __syncthreads();
  else
    bar_sync_named(static_cast<uint32_t>(bar), PRO_THREADS);
}

// The maximum behind a row / column scale (its bits; 0 gives the scale 1),
// and the power-of-two scale from it.
__device__ __forceinline__ uint32_t scale_bits(const Common& cm, const uint32_t* mx, int64_t idx,
                                               int g, int which) {
  if (cm.scaling == 0) return 0u;
  return cm.scaling == 1 ? cm.gmax[2 * g + which] : mx[idx];
}
__device__ __forceinline__ float scale_from_bits(const Common& cm, uint32_t bits) {
  return cm.scaling == 0 ? 1.0f : pow2_ceil_f(__uint_as_float(bits));
}
__device__ __forceinline__ float scale_of(const Common& cm, const uint32_t* mx, int64_t idx,
                                          int g, int which) {
  return scale_from_bits(cm, scale_bits(cm, mx, idx, g, which));
}

// v[u][e] <- v[u][e] / s[u] for power-of-two scales s[u]; a multiply by the
// exact reciprocal whenever every scale of the warp has a normal one (called
// by whole warps).
template <int U, int EPC>
__device__ __forceinline__ void div_scales(float (&v)[U][EPC], const float (&s)[U]) {
  float inv[U];
  bool ok = true;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    inv[u] = 1.0f / s[u];
    ok = ok && recip_exact(s[u]);
  }
  if (__all_sync(0xffffffffu, ok)) {
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int e = 0; e < EPC; ++e) v[u][e] *= inv[u];
  } else {
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int e = 0; e < EPC; ++e) v[u][e] = div_pow2(v[u][e], s[u], inv[u], recip_exact(s[u]));
  }
}

// v <- v^p * opscale with p = 2^plog, or p = 1.5 * 2^plog for a half level
// (y * sqrt(y), y = v^(2^plog)); the squarings of all U x EPC values
// interleaved (independent chains; the same products as pow2k value by value).
template <int U, int EPC>
__device__ __forceinline__ void power_all(float (&v)[U][EPC], int plog, int half, float opscale) {
#pragma unroll 1
  for (int t = 0; t < plog; ++t) {
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int e = 0; e < EPC; ++e) v[u][e] *= v[u][e];
  }
  if (half) {
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int e = 0; e < EPC; ++e) v[u][e] *= sqrtf(v[u][e]);
  }
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int e = 0; e < EPC; ++e) v[u][e] *= opscale;
}

// ----------------------------------------------------------- A images ---
// Second half of an A image tile built by 1024 / U threads: thread t holds
// the source values of image chunks (row (t >> 3) + (128 / U) u, 16-byte slot
// t & 7), u < U (zero past M), and their row scales rs[u] (1 past M);
// scales, powers, packs and stores them (a warp writes four whole 128-byte
// image rows).
template <int MODE, int U>
__device__ __forceinline__ void power_a_store(const Common& cm, const Level& lv, const Prob& P,
                                              int rb, int kb, float (&v)[U][Packer<MODE>::EPC],
                                              const float (&rs)[U], int t) {
  using PK = Packer<MODE>;
  constexpr int RSTEP = TILE_M / U;
  const float opscale = ldexpf(1.0f, cm.s_op);
  uint8_t* dst = lv.a_level + P.a_img + ((int64_t)(rb * P.KB + kb) << 14);
  const int cc = t & 7;
  if (lv.is_top && kb == 0 && cc == 0) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int row = rb * TILE_M + (t >> 3) + RSTEP * u;
      if (row < P.M) cm.r[P.rc_r + row] = rs[u];
    }
  }
  div_scales(v, rs);
  power_all(v, lv.plog, lv.half, opscale);
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int rr = (t >> 3) + RSTEP * u;
    uint4 hi, lo;
    PK::pack(v[u], hi, lo);
    const uint32_t off = sw128_offset(rr, cc * 16);
    *reinterpret_cast<uint4*>(dst + off) = hi;
    if constexpr (MODE == MODE_3XTF32) *reinterpret_cast<uint4*>(dst + P.a_plane + off) = lo;
  }
}

template <int MODE>
__device__ __forceinline__ void power_a_tile(const Common& cm, const Level& lv, int g,
                                             const Prob& P, int rb, int kb, int t) {
  using PK = Packer<MODE>;
  constexpr int EPC = PK::EPC;
  constexpr int BK = mode_bk(MODE);
  const bool vec = ((P.lda & 3) == 0) && ((reinterpret_cast<uintptr_t>(P.A) & 15) == 0);
  // 1024 16-byte output chunks per tile, 4 per thread: chunk = tid + 256 u,
  // row = chunk / 8 (8 threads cover one 128-byte image row), 16-byte slot
  // = chunk % 8.  All loads are issued, unconditionally, before any
  // arithmetic: rows past M and columns past K read the clamped (in-bounds)
  // index and are zeroed afterwards.
  float v[4][EPC];
  const int cc = t & 7;
  const int k0 = kb * BK + cc * EPC;
  const bool vec_k = vec && k0 + EPC <= P.K;  // this thread's columns are whole 16-byte groups
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int row = rb * TILE_M + (t >> 3) + 32 * u;
    const float* srow = P.A + (int64_t)min(row, P.M - 1) * P.lda;
    if (vec_k) {
#pragma unroll
      for (int e = 0; e < EPC; e += 4) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(srow + k0 + e));
        v[u][e] = t.x; v[u][e + 1] = t.y; v[u][e + 2] = t.z; v[u][e + 3] = t.w;
      }
    } else {
#pragma unroll
      for (int e = 0; e < EPC; ++e) v[u][e] = __ldg(srow + min(k0 + e, P.K - 1));
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const bool row_in = rb * TILE_M + (t >> 3) + 32 * u < P.M;
#pragma unroll
    for (int e = 0; e < EPC; ++e) v[u][e] = (row_in && k0 + e < P.K) ? v[u][e] : 0.0f;
  }
  float rs[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int row = rb * TILE_M + (t >> 3) + 32 * u;
    rs[u] = row < P.M ? scale_of(cm, cm.rmax, P.rc_r + row, g, 0) : 1.0f;
  }
  power_a_store<MODE, 4>(cm, lv, P, rb, kb, v, rs, t);
}


// ----------------------------------------------------------- B images ---
// The B image holds B^T: image row n, K along the 128-byte row.  The tile of
// B (BK rows of K x 128 columns) is staged in shared memory and transposed.
template <int MODE>
__device__ __forceinline__ void power_b_tile(const Common& cm, const Level& lv, int g,
                                             const Prob& P, int rb, int kb, float* stile, int t,
                                             int bar) {
  using PK = Packer<MODE>;
  constexpr int EPC = PK::EPC;
  constexpr int BK = mode_bk(MODE);
  const float opscale = ldexpf(1.0f, cm.s_op);
  img_sync(bar);  // stile reuse across consecutive tiles
  {
    // BK rows of K x 128 columns, staged in chunks of up to 64 rows (below).
    // 16-byte aligned rows: thread = (row group tid/32, columns 4 lane ..
    // 4 lane + 3), float4 loads.  Otherwise thread = (row group, columns
    // lane + 32 c), so that each load instruction reads one contiguous
    // 128-byte row segment.
    const int lane = t & 31, rg = t >> 5;
    const int n0 = rb * TILE_M;
    const bool vec = ((P.ldb & 3) == 0) && ((reinterpret_cast<uintptr_t>(P.B) & 15) == 0) &&
                     n0 + TILE_M <= P.N;
    float cs[4], inv[4];
    bool inv_ok[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int n = vec ? n0 + lane * 4 + c : n0 + lane + 32 * c;
      cs[c] = n < P.N ? scale_of(cm, cm.cmax, P.rc_c + n, g, 1) : 1.0f;
      inv[c] = 1.0f / cs[c];
      inv_ok[c] = cs[c] >= 1.1754944e-38f && cs[c] <= 8.507059e37f;
      if (lv.is_top && kb == 0 && rg == 0 && n < P.N) cm.c[P.rc_c + n] = cs[c];
    }
    // Loads in chunks of up to 8 row groups (64 rows), all of a chunk
    // issued, unconditionally, before its values are used: rows past K and
    // columns past N read the clamped (in-bounds) index and are zeroed after.
    constexpr int CH = BK / 8 < 8 ? BK / 8 : 8;
    const int nlast = P.N - 1 - n0;  // last column of the tile block in bounds
#pragma unroll
    for (int it0 = 0; it0 < BK / 8; it0 += CH) {
      float4 t[CH];
#pragma unroll
      for (int i = 0; i < CH; ++i) {
        const int k = kb * BK + rg + 8 * (it0 + i);
        const float* srow = P.B + (int64_t)min(k, P.K - 1) * P.ldb + n0;
        if (vec) {
          t[i] = __ldg(reinterpret_cast<const float4*>(srow + lane * 4));
        } else {
          t[i].x = __ldg(srow + min(lane, nlast));
          t[i].y = __ldg(srow + min(lane + 32, nlast));
          t[i].z = __ldg(srow + min(lane + 64, nlast));
          t[i].w = __ldg(srow + min(lane + 96, nlast));
        }
      }
#pragma unroll
      for (int i = 0; i < CH; ++i) {
        const bool kin = kb * BK + rg + 8 * (it0 + i) < P.K;
        if (vec) {
          t[i] = kin ? t[i] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        } else {
          t[i].x = (kin && lane <= nlast) ? t[i].x : 0.0f;
          t[i].y = (kin && lane + 32 <= nlast) ? t[i].y : 0.0f;
          t[i].z = (kin && lane + 64 <= nlast) ? t[i].z : 0.0f;
          t[i].w = (kin && lane + 96 <= nlast) ? t[i].w : 0.0f;
        }
        float* rowp = stile + (rg + 8 * (it0 + i)) * 129;
        const int c0 = vec ? lane * 4 : lane, cst = vec ? 1 : 32;
        rowp[c0] = div_pow2(t[i].x, cs[0], inv[0], inv_ok[0]);
        rowp[c0 + cst] = div_pow2(t[i].y, cs[1], inv[1], inv_ok[1]);
        rowp[c0 + 2 * cst] = div_pow2(t[i].z, cs[2], inv[2], inv_ok[2]);
        rowp[c0 + 3 * cst] = div_pow2(t[i].w, cs[3], inv[3], inv_ok[3]);
      }
    }
  }
  img_sync(bar);
  uint8_t* dst = lv.b_level + P.b_img + ((int64_t)(rb * P.KB + kb) << 14);
  float v[4][EPC];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int ch = t + PRO_THREADS * u;
    const int nr = ch >> 3, cc = ch & 7;
#pragma unroll
    for (int e = 0; e < EPC; ++e) v[u][e] = stile[(cc * EPC + e) * 129 + nr];
  }
  power_all(v, lv.plog, lv.half, opscale);
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int ch = t + PRO_THREADS * u;
    const int nr = ch >> 3, cc = ch & 7;
    uint4 hi, lo;
    PK::pack(v[u], hi, lo);
    const uint32_t off = sw128_offset(nr, cc * 16);
    *reinterpret_cast<uint4*>(dst + off) = hi;
    if constexpr (MODE == MODE_3XTF32) *reinterpret_cast<uint4*>(dst + P.b_plane + off) = lo;
  }
}


// ------------------------------------------------ fused operand blocks ---
// A row block rb of problem P (rows 128 rb .. 128 rb + 127, all of K): the
// row maxima on raw bits with the domain test (written to cm.rmax, which this
// block owns: no atomics) when `maxima`, then the powered images of every
// k-block for level lv (power_a_tile, which also writes the row scales at the
// top level).  Run by PRO_THREADS threads (index t, barrier bar); returns
// true if a value outside the domain was seen by this thread.
template <int MODE>
__device__ __forceinline__ bool a_block_fused(const Common& cm, const Level& lv, int g,
                                              const Prob& P, int rb, bool maxima, int t,
                                              int bar) {
  bool bad = false;
  if (maxima) {
    const int lane = t & 31, warp = t >> 5;
    // warp w: rows 16 w .. 16 w + 15 of the block, four at a time, lanes
    // over K with 16 loads in flight (clamped indexes; a row past M is never
    // committed, a column past K re-reads the row's last value)
    for (int rr = 0; rr < 16; rr += 4) {
      const int row0 = rb * TILE_M + warp * 16 + rr;
      if (row0 >= P.M) break;  // warp-uniform
      uint32_t u[4] = {0u, 0u, 0u, 0u};
      for (int kk0 = lane; kk0 < P.K; kk0 += 128) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const float* src = P.A + (int64_t)min(row0 + r, P.M - 1) * P.lda;
#pragma unroll
          for (int q = 0; q < 4; ++q)
            u[r] = max(u[r], __float_as_uint(__ldg(src + min(kk0 + 32 * q, P.K - 1))));
        }
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int row = row0 + r;
        if (row < P.M) {  // warp-uniform
          if (u[r] > DOMAIN_MAX_BITS) {
            const int cnt = lane < P.K ? (P.K - 1 - lane) / 32 + 1 : 0;
            u[r] = take_exact(exact_max_bits(P.A + (int64_t)row * P.lda + lane, 32, cnt), bad);
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) u[r] = max(u[r], __shfl_xor_sync(0xffffffffu, u[r], o));
          if (lane == 0) cm.rmax[P.rc_r + row] = u[r];
        }
      }
    }
    img_sync(bar);  // the row maxima before the scales are formed from them
  }
  for (int kb = 0; kb < P.KB; ++kb) power_a_tile<MODE>(cm, lv, g, P, rb, kb, t);
  return bad;
}

// B column block cb of problem P (columns 128 cb .. 128 cb + 127 = rows of
// the B^T image, all of K): column maxima on raw bits with the domain test
// (written to cm.cmax) when `maxima`, then the powered B^T images of every
// k-block (power_b_tile, staging in `stile`).  `red` is shared scratch of
// 8 x 128 words.  Run by PRO_THREADS threads (t, bar); returns true if a
// value outside the domain was seen by this thread.
template <int MODE>
__device__ __forceinline__ bool b_block_fused(const Common& cm, const Level& lv, int g,
                                              const Prob& P, int cb, bool maxima, float* stile,
                                              uint32_t* red, int t, int bar) {
  bool bad = false;
  if (maxima) {
    const int lane = t & 31, warp = t >> 5;
    const int nl = cb * TILE_M + lane;
    int ncol[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) ncol[c] = min(nl + 32 * c, P.N - 1);
    uint32_t u4[4] = {0u, 0u, 0u, 0u};
    // warp w: rows w, w + 8, ..., four at a time; lane: columns lane + 32 c,
    // so that each load instruction reads one contiguous 128-byte row segment
    for (int k0 = warp; k0 < P.K; k0 += 32) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float* src = P.B + (int64_t)min(k0 + 8 * q, P.K - 1) * P.ldb;
#pragma unroll
        for (int c = 0; c < 4; ++c) u4[c] = max(u4[c], __float_as_uint(__ldg(src + ncol[c])));
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int n = nl + 32 * c;
      if (n >= P.N) u4[c] = 0u;
      if (u4[c] > DOMAIN_MAX_BITS) {
        const int cnt = warp < P.K ? (P.K - 1 - warp) / 8 + 1 : 0;
        u4[c] = take_exact(exact_max_bits(P.B + (int64_t)warp * P.ldb + n, 8 * P.ldb, cnt), bad);
      }
      red[warp * TILE_M + lane + 32 * c] = u4[c];
    }
    img_sync(bar);
    if (t < TILE_M) {
      uint32_t m = red[t];
#pragma unroll
      for (int w = 1; w < PRO_THREADS / 32; ++w) m = max(m, red[w * TILE_M + t]);
      const int n = cb * TILE_M + t;
      if (n < P.N) cm.cmax[P.rc_c + n] = m;
    }
    img_sync(bar);  // the column maxima before the scales are formed from them
  }
  for (int kb = 0; kb < P.KB; ++kb) power_b_tile<MODE>(cm, lv, g, P, cb, kb, stile, t, bar);
  return bad;
}

}  // namespace
}  // namespace pn
