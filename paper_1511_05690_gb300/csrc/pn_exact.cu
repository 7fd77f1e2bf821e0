// Exact semiring products on the CUDA cores (the plain comparison):
//   (x,max): C_ij = max_k a_ik * b_kj   (Alg. 2, F'_APSP)
//   (+,min): C_ij = min_k a_ik + b_kj   (Alg. 1, F_APSP)
// Register-tiled like an SGEMM: a 128 x 128 output tile per 256-thread
// block, 8 x 8 outputs per thread, K staged through shared memory 16 at a
// time with a register prefetch of the next slice; two blocks per SM (128
// registers a thread) so that one block's barrier wait is covered by the other.  Each product (sum) is one
// correctly rounded FP32 operation and max (min) is exact, so the result is
// bit-identical to any sequential evaluation.
//
// Variant 1 pairs consecutive k: one mul.rn.f32x2 forms a_ik*b_kj and
// a_i(k+1)*b_(k+1)j, and one 3-input max folds both into the accumulator,
// i.e. one instruction per semiring operation instead of two.  Variant 2 (the
// default) issues the same instructions in a software-pipelined order.
// Issue bound: a paired multiply and a 3-input max each issue at 2 warp
// instructions per clock per SM alone but only about 2.3 together, so the
// instruction mix caps the kernel near 1.15 x 64 semiring operations per clock
// per SM.
#include <cstdint>

#include "pn_device.cuh"

namespace pn {

namespace {

#ifndef PN_EXACT_BK
#define PN_EXACT_BK 16
#endif
#ifndef PN_EXACT_MIN_BLOCKS
#define PN_EXACT_MIN_BLOCKS 2
#endif
constexpr int EX_BM = 128, EX_BN = 128, EX_BK = PN_EXACT_BK, EX_THREADS = 256;
static_assert(EX_BK == 8 || EX_BK == 16, "slice depth: 8 or 16");

template <int SEMI>
__device__ __forceinline__ float ident() {
  return SEMI == 0 ? 0.0f : __int_as_float(0x7f800000);
}

template <int SEMI>
__device__ __forceinline__ float op1(float acc, float a, float b) {
  if constexpr (SEMI == 0) return fmaxf(acc, a * b);
  else return fminf(acc, a + b);
}

// Variant 2 splits op2 into its two instructions, each a volatile asm so that
// the order written in the source is kept: the paired products of one output
// are formed LAG outputs ahead of the 3-input max that consumes them, which
// alternates FMA-pipe and ALU-pipe work instead of grouping it.
template <int SEMI>
__device__ __forceinline__ uint64_t pair_op(uint64_t a2, uint64_t b2) {
  uint64_t p;
  if constexpr (SEMI == 0) asm volatile("mul.rn.f32x2 %0, %1, %2;" : "=l"(p) : "l"(a2), "l"(b2));
  else asm volatile("add.rn.f32x2 %0, %1, %2;" : "=l"(p) : "l"(a2), "l"(b2));
  return p;
}

template <int SEMI>
__device__ __forceinline__ float fold3(float acc, uint64_t p) {
  float r;
  if constexpr (SEMI == 0)
    asm volatile("max.f32 %0, %1, %2, %3;"
                 : "=f"(r)
                 : "f"(acc), "f"(__uint_as_float(static_cast<uint32_t>(p))),
                   "f"(__uint_as_float(static_cast<uint32_t>(p >> 32))));
  else
    asm volatile("min.f32 %0, %1, %2, %3;"
                 : "=f"(r)
                 : "f"(acc), "f"(__uint_as_float(static_cast<uint32_t>(p))),
                   "f"(__uint_as_float(static_cast<uint32_t>(p >> 32))));
  return r;
}

#ifndef PN_EXACT_LAG
#define PN_EXACT_LAG 4
#endif

template <int SEMI>
__device__ __forceinline__ float op2(float acc, uint64_t a2, uint64_t b2) {
  uint64_t p;
  float r;
  if constexpr (SEMI == 0) {
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(p) : "l"(a2), "l"(b2));
    asm("max.f32 %0, %1, %2, %3;"
        : "=f"(r)
        : "f"(acc), "f"(__uint_as_float(static_cast<uint32_t>(p))),
          "f"(__uint_as_float(static_cast<uint32_t>(p >> 32))));
  } else {
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(p) : "l"(a2), "l"(b2));
    asm("min.f32 %0, %1, %2, %3;"
        : "=f"(r)
        : "f"(acc), "f"(__uint_as_float(static_cast<uint32_t>(p))),
          "f"(__uint_as_float(static_cast<uint32_t>(p >> 32))));
  }
  return r;
}

// Shared-memory layout, both variants: element (k, x) of the A^T (or B) slice
// sits at [k/2][x][k%2], so a k-pair of one row/column is one 8-byte word.
template <int SEMI, int VARIANT>
__global__ void __launch_bounds__(EX_THREADS, PN_EXACT_MIN_BLOCKS)
    k_exact(int M, int N, int K, const float* __restrict__ A, int64_t lda,
            const float* __restrict__ B, int64_t ldb, float* __restrict__ C, int64_t ldc,
            int vec_a, int vec_b) {
  __shared__ __align__(16) float As[2][EX_BK / 2][EX_BM][2];
  __shared__ __align__(16) float Bs[2][EX_BK / 2][EX_BN][2];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * EX_BM, n0 = blockIdx.x * EX_BN;
  const float pad = ident<SEMI>();

  // global -> register slice loaders: 128 rows x EX_BK of A, EX_BK x 128 of B,
  // EX_BK / 4 float4 per thread each
  constexpr int LPT = EX_BK / 8;  // float4 loads per thread per operand
  float ra[LPT][4], rb[LPT][4];
  auto load_slice = [&](int k0) {
#pragma unroll
    for (int l = 0; l < LPT; ++l) {
      const int idx = tid + l * EX_THREADS;
      const int a_row = idx / (EX_BK / 4), a_k = (idx % (EX_BK / 4)) * 4;
      const int gm = m0 + a_row, gk = k0 + a_k;
      if (vec_a && gm < M && gk + 4 <= K) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(A + (int64_t)gm * lda + gk));
        ra[l][0] = t.x; ra[l][1] = t.y; ra[l][2] = t.z; ra[l][3] = t.w;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          ra[l][e] = (gm < M && gk + e < K) ? __ldg(A + (int64_t)gm * lda + gk + e) : pad;
      }
      const int b_k = idx >> 5, b_col = (idx & 31) * 4;
      const int bk = k0 + b_k, bn = n0 + b_col;
      if (vec_b && bk < K && bn + 4 <= N) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(B + (int64_t)bk * ldb + bn));
        rb[l][0] = t.x; rb[l][1] = t.y; rb[l][2] = t.z; rb[l][3] = t.w;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          rb[l][e] = (bk < K && bn + e < N) ? __ldg(B + (int64_t)bk * ldb + bn + e) : pad;
      }
    }
  };
  auto store_slice = [&](int buf) {
#pragma unroll
    for (int l = 0; l < LPT; ++l) {
      const int idx = tid + l * EX_THREADS;
      const int a_row = idx / (EX_BK / 4), a_k = (idx % (EX_BK / 4)) * 4;
#pragma unroll
      for (int e = 0; e < 4; ++e) As[buf][(a_k + e) >> 1][a_row][(a_k + e) & 1] = ra[l][e];
      const int b_k = idx >> 5, b_col = (idx & 31) * 4;
#pragma unroll
      for (int e = 0; e < 4; ++e) Bs[buf][b_k >> 1][b_col + e][b_k & 1] = rb[l][e];
    }
  };

  float acc[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = pad;

  const int nslices = (K + EX_BK - 1) / EX_BK;
  if (nslices > 0) {
    load_slice(0);
    store_slice(0);
  }
  __syncthreads();
  for (int s = 0; s < nslices; ++s) {
    const int buf = s & 1;
    if (s + 1 < nslices) load_slice((s + 1) * EX_BK);
#pragma unroll
    for (int kp = 0; kp < EX_BK / 2; ++kp) {
      uint64_t a2[8], b2[8];
      const ulonglong2* ap0 = reinterpret_cast<const ulonglong2*>(&As[buf][kp][ty * 4][0]);
      const ulonglong2* ap1 = reinterpret_cast<const ulonglong2*>(&As[buf][kp][64 + ty * 4][0]);
      const ulonglong2* bp0 = reinterpret_cast<const ulonglong2*>(&Bs[buf][kp][tx * 4][0]);
      const ulonglong2* bp1 = reinterpret_cast<const ulonglong2*>(&Bs[buf][kp][64 + tx * 4][0]);
      {
        ulonglong2 t;
        t = ap0[0]; a2[0] = t.x; a2[1] = t.y;
        t = ap0[1]; a2[2] = t.x; a2[3] = t.y;
        t = ap1[0]; a2[4] = t.x; a2[5] = t.y;
        t = ap1[1]; a2[6] = t.x; a2[7] = t.y;
        t = bp0[0]; b2[0] = t.x; b2[1] = t.y;
        t = bp0[1]; b2[2] = t.x; b2[3] = t.y;
        t = bp1[0]; b2[4] = t.x; b2[5] = t.y;
        t = bp1[1]; b2[6] = t.x; b2[7] = t.y;
      }
      if constexpr (VARIANT == 1) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
          for (int c = 0; c < 8; ++c) acc[r][c] = op2<SEMI>(acc[r][c], a2[r], b2[c]);
      } else if constexpr (VARIANT == 2) {
        constexpr int LAG = PN_EXACT_LAG;
        uint64_t pr[LAG];
#pragma unroll
        for (int t = 0; t < 64 + LAG; ++t) {
          if (t >= LAG) {
            const int u = t - LAG;
            acc[u >> 3][u & 7] = fold3<SEMI>(acc[u >> 3][u & 7], pr[u % LAG]);
          }
          if (t < 64) pr[t % LAG] = pair_op<SEMI>(a2[t >> 3], b2[t & 7]);
        }
      } else {
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            const float a = __uint_as_float(static_cast<uint32_t>(a2[r] >> (32 * h)));
#pragma unroll
            for (int c = 0; c < 8; ++c)
              acc[r][c] = op1<SEMI>(acc[r][c], a,
                                    __uint_as_float(static_cast<uint32_t>(b2[c] >> (32 * h))));
          }
      }
    }
    if (s + 1 < nslices) store_slice(buf ^ 1);
    __syncthreads();
  }

  const bool vec_c = ((ldc & 3) == 0) && ((reinterpret_cast<uintptr_t>(C) & 15) == 0);
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int gm = m0 + (r < 4 ? ty * 4 + r : 64 + ty * 4 + (r - 4));
    if (gm >= M) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int gn = n0 + h * 64 + tx * 4;
      float* dst = C + (int64_t)gm * ldc + gn;
      if (vec_c && gn + 4 <= N) {
        *reinterpret_cast<float4*>(dst) =
            make_float4(acc[r][4 * h], acc[r][4 * h + 1], acc[r][4 * h + 2], acc[r][4 * h + 3]);
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (gn + e < N) dst[e] = acc[r][4 * h + e];
      }
    }
  }
}

template <int SEMI, int VARIANT>
int launch_exact_t(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, const float* B,
                   int64_t ldb, float* C, int64_t ldc, void* stream) {
  const dim3 grid(static_cast<unsigned>((N + EX_BN - 1) / EX_BN),
                  static_cast<unsigned>((M + EX_BM - 1) / EX_BM));
  const int vec_a = ((lda & 3) == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
  const int vec_b = ((ldb & 3) == 0) && ((reinterpret_cast<uintptr_t>(B) & 15) == 0);
  k_exact<SEMI, VARIANT><<<grid, EX_THREADS, 0, static_cast<cudaStream_t>(stream)>>>(
      static_cast<int>(M), static_cast<int>(N), static_cast<int>(K), A, lda, B, ldb, C, ldc, vec_a,
      vec_b);
  return cudaGetLastError();
}

}  // namespace

int launch_exact(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, const float* B,
                 int64_t ldb, float* C, int64_t ldc, int semiring, int variant, void* stream) {
  if (M <= 0 || N <= 0) return 0;
  if (semiring == 0)
    return variant == 2   ? launch_exact_t<0, 2>(M, N, K, A, lda, B, ldb, C, ldc, stream)
           : variant == 1 ? launch_exact_t<0, 1>(M, N, K, A, lda, B, ldb, C, ldc, stream)
                          : launch_exact_t<0, 0>(M, N, K, A, lda, B, ldb, C, ldc, stream);
  return variant == 2   ? launch_exact_t<1, 2>(M, N, K, A, lda, B, ldb, C, ldc, stream)
         : variant == 1 ? launch_exact_t<1, 1>(M, N, K, A, lda, B, ldb, C, ldc, stream)
                        : launch_exact_t<1, 0>(M, N, K, A, lda, B, ldb, C, ldc, stream);
}

}  // namespace pn
