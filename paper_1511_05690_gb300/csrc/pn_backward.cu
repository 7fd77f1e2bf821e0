// Device side of the adjoint of the p-norm product (maxprod_pnorm_backward).
//
// With p = p*_ij held fixed per entry, C_ij = (sum_k (a_ik b_kj)^p)^(1/p) is
// differentiable (the p-norm rings are, Sec. 4), and in the forward's scaled
// variables a' = a / r_i, b' = b / c_j, S = sum_k (a'_ik b'_kj)^p:
//   dC_ij / da_ik = (C_ij / S_ij) (a'_ik^(p-1) / r_i) b'_kj^p.
// Hence, with W_ij = dC_ij C_ij / S_ij and W^(p) = W masked to p*_ij = p,
//   dA = sum_p (a'^(p-1) / r) (.) (W^(p) B'^p^T),
//   dB = sum_p (b'^(p-1) / c) (.) (A'^p^T W^(p)),
// two ring GEMMs per p that occurs in p_sel.  This file builds their operand
// images (recomputed from A, B, C, S_sel, p_sel rather than stored) and the
// mask of the p values that occur; the GEMMs are the tensor-core level kernel
// with its gradient epilogue.
#include "pn_pack.cuh"

namespace pn {

namespace {

constexpr int BW_THREADS = 256;

// Bit q of *mask is set when some entry of p_sel selected p = 2^plog_list[q].
struct PList {
  int32_t n_p;
  int32_t plog[PN_MAX_P];
};

__global__ void k_bw_mask(const uint8_t* __restrict__ psel, int64_t count, PList pl,
                          uint32_t* mask) {
  pdl_wait();
  pdl_trigger();
  uint32_t bits = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int lp = psel[e] & 0x7F;
    for (int q = 0; q < pl.n_p; ++q)
      if (pl.plog[q] == lp) bits |= 1u << q;
  }
  bits = __reduce_or_sync(0xffffffffu, bits);
  if ((threadIdx.x & 31) == 0 && bits) atomicOr(mask, bits);
}

// Row and column scales from the maxima (same rule as the forward).
__global__ void k_scales(const __grid_constant__ Common cm) {
  pdl_wait();
  pdl_trigger();
  const Prob& P = cm.single;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)P.M + P.N;
       e += (int64_t)gridDim.x * blockDim.x) {
    const bool col = e >= P.M;
    const int64_t idx = col ? e - P.M : e;
    float s = 1.0f;
    if (cm.scaling != 0) {
      const uint32_t bits = cm.scaling == 1 ? cm.gmax[col ? 1 : 0] : (col ? cm.cmax : cm.rmax)[idx];
      s = pow2_ceil_f(__uint_as_float(bits));
    }
    (col ? cm.c : cm.r)[idx] = s;
  }
}

template <int KIND>
__device__ __forceinline__ float bw_value(const BwImage& im, int64_t srow, int64_t scol) {
  // element (srow, scol) of the source, in range
  if constexpr (KIND == 1) {
    const int64_t e = srow * im.scols + scol;
    if ((im.psel[e] & 0x7F) != im.plog) return 0.0f;
    const float S = __ldg(im.S + e);
    return S > 0.0f ? __ldg(im.dC + e) * __ldg(im.Cv + e) / S : 0.0f;
  } else {
    const float s = __ldg(im.scale + (im.trans ? srow : scol));
    return pow2k(__ldg(im.src + srow * im.lds + scol) / s, im.plog);
  }
}

// One 16 KB tile image (128 image rows x 128 bytes of contraction) per block.
template <int MODE, int TRANS, int KIND>
__global__ void __launch_bounds__(BW_THREADS) k_bw_image(const __grid_constant__ BwImage im) {
  pdl_wait();
  pdl_trigger();
  using PK = Packer<MODE>;
  constexpr int EPC = PK::EPC;
  constexpr int BK = mode_bk(MODE);
  if (!((*im.pmask >> im.q) & 1u)) return;  // no entry selected this p
  extern __shared__ float stile[];          // [BK][129] (TRANS only)
  const int rb = blockIdx.x / im.KB, kb = blockIdx.x - rb * im.KB;
  const int64_t img_rows = TRANS ? im.scols : im.srows;
  const int64_t img_cont = TRANS ? im.srows : im.scols;
  uint8_t* dst = im.dst + ((int64_t)(rb * im.KB + kb) << 14);
  if constexpr (TRANS) {
    // stage source rows kb*BK.. (contraction) x columns rb*128.. (image rows)
    const int nl = threadIdx.x & 127;
    const int64_t r = (int64_t)rb * TILE_M + nl;
    for (int kk = threadIdx.x >> 7; kk < BK; kk += 2) {
      const int64_t c = (int64_t)kb * BK + kk;
      stile[kk * 129 + nl] = (r < img_rows && c < img_cont) ? bw_value<KIND>(im, c, r) : 0.0f;
    }
    __syncthreads();
  }
#pragma unroll 1
  for (int u = 0; u < 4; ++u) {
    const int ch = threadIdx.x + BW_THREADS * u;
    const int rr = ch >> 3, cc = ch & 7;
    const int64_t r = (int64_t)rb * TILE_M + rr;
    float v[EPC];
#pragma unroll
    for (int e = 0; e < EPC; ++e) {
      if constexpr (TRANS) {
        v[e] = stile[(cc * EPC + e) * 129 + rr];
      } else {
        const int64_t c = (int64_t)kb * BK + cc * EPC + e;
        v[e] = (r < img_rows && c < img_cont) ? bw_value<KIND>(im, r, c) : 0.0f;
      }
    }
    uint4 hi, lo;
    PK::pack(v, hi, lo);
    const uint32_t off = sw128_offset(rr, cc * 16);
    *reinterpret_cast<uint4*>(dst + off) = hi;
    if constexpr (MODE == MODE_3XTF32) *reinterpret_cast<uint4*>(dst + im.plane + off) = lo;
  }
}

template <int MODE, int TRANS, int KIND>
int launch_img_t(const BwImage& im, void* stream) {
  const int smem = TRANS ? mode_bk(MODE) * 129 * 4 : 0;
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(k_bw_image<MODE, TRANS, KIND>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  const int blocks = im.RB * im.KB;
  if (blocks <= 0) return 0;
  const cudaError_t e = launch_pdl(k_bw_image<MODE, TRANS, KIND>, dim3(blocks), dim3(BW_THREADS),
                                   smem, stream, im);
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <int MODE>
int launch_img_mode(const BwImage& im, void* stream) {
  if (im.trans)
    return im.kind ? launch_img_t<MODE, 1, 1>(im, stream) : launch_img_t<MODE, 1, 0>(im, stream);
  return im.kind ? launch_img_t<MODE, 0, 1>(im, stream) : launch_img_t<MODE, 0, 0>(im, stream);
}

}  // namespace

int launch_bw_mask(const uint8_t* psel, int64_t count, const int32_t* plog_list, int n_p,
                   uint32_t* mask, void* stream) {
  if (count <= 0) return 0;
  PList pl{};
  pl.n_p = n_p;
  for (int q = 0; q < n_p; ++q) pl.plog[q] = plog_list[q];
  int64_t blocks = (count + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  const cudaError_t e = launch_pdl(k_bw_mask, dim3(static_cast<unsigned>(blocks)), dim3(256), 0,
                                   stream, psel, count, pl, mask);
  return e != cudaSuccess ? e : cudaGetLastError();
}

int launch_scales(const Common& cm, void* stream) {
  const int64_t total = (int64_t)cm.single.M + cm.single.N;
  if (total <= 0) return 0;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  const cudaError_t e = launch_pdl(k_scales, dim3(static_cast<unsigned>(blocks)), dim3(256), 0,
                                   stream, cm);
  return e != cudaSuccess ? e : cudaGetLastError();
}

int launch_bw_image(int mode, const BwImage& im, void* stream) {
  switch (mode) {
    case MODE_3XTF32: return launch_img_mode<MODE_3XTF32>(im, stream);
    case MODE_TF32: return launch_img_mode<MODE_TF32>(im, stream);
    case MODE_BF16: return launch_img_mode<MODE_BF16>(im, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pn
