// Bias corrections of the p-norm estimate.
//
// correction 1 (Sec. 2.1, the envelope ||u||_inf <= ||u||_p <= K^(1/p) ||u||_inf):
//   the estimate divided by K^(1/p*), applied in the GEMM epilogue.
// correction 2 (Discussion: an affine model fitted to a few exact
//   sub-solutions): at caller-chosen sample entries the exact max and the
//   estimate are computed directly here; a least-squares line
//   exact = a_q * est + b_q per p* class q, in the scaled space
//   (value / (r_i c_j)), is applied to every entry by the GEMM epilogue.
#include <cstdint>

#include "pn_device.cuh"

namespace pn {

namespace {

constexpr int FIT_THREADS = 256;  // one block per sample

// One block per sample entry (i, j): u_k = (a_ik / r_i)(b_kj / c_j) in FP32,
// the exact max over k and the p-sums S^(p) for every p of P (each thread a
// strided part of k, then warp and block reductions), the sample's own p* and
// estimate (the same rule as the epilogue); the sample's record (estimate,
// exact value, class) goes to its own slot, so that the class sums can be
// formed in a fixed order (deterministic results).
__global__ void __launch_bounds__(FIT_THREADS)
    k_fit_samples(const __grid_constant__ Common cm, const __grid_constant__ FitArgs fa) {
  __shared__ float red[FIT_THREADS / 32][PN_MAX_P + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int s = blockIdx.x;
  const Prob& P = cm.single;
  const int i = fa.fi[s], j = fa.fj[s];
  if (i < 0 || i >= P.M || j < 0 || j >= P.N) {
    if (threadIdx.x == 0) {
      set_status(cm.status, PN_EINVAL);
      fa.scls[s] = -1;
    }
    return;
  }
  const float ri = cm.r[P.rc_r + i], cj = cm.c[P.rc_c + j];
  float mx = 0.0f;
  float S[PN_MAX_P];
#pragma unroll
  for (int q = 0; q < PN_MAX_P; ++q) S[q] = 0.0f;
  const float* arow = P.A + (int64_t)i * P.lda;
  for (int k = threadIdx.x; k < P.K; k += FIT_THREADS) {
    const float u = (__ldg(arow + k) / ri) * (__ldg(P.B + (int64_t)k * P.ldb + j) / cj);
    mx = fmaxf(mx, u);
    float t = u;
    int lg = 0;
#pragma unroll
    for (int q = 0; q < PN_MAX_P; ++q) {
      if (q < fa.n_p) {
        while (lg < fa.p_log2[q]) {
          t = t * t;
          ++lg;
        }
        S[q] += t;
      }
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
#pragma unroll
    for (int q = 0; q < PN_MAX_P; ++q) S[q] += __shfl_xor_sync(0xffffffffu, S[q], off);
  }
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < PN_MAX_P; ++q) red[warp][q] = S[q];
    red[warp][PN_MAX_P] = mx;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
#pragma unroll
  for (int q = 0; q < PN_MAX_P; ++q) {
    S[q] = 0.0f;
    for (int w = 0; w < FIT_THREADS / 32; ++w) S[q] += red[w][q];
  }
  mx = 0.0f;
  for (int w = 0; w < FIT_THREADS / 32; ++w) mx = fmaxf(mx, red[w][PN_MAX_P]);
  int qs = -1;
  for (int q = fa.n_p - 1; q >= 0; --q) {
    float sq = 0.0f;
#pragma unroll
    for (int t = 0; t < PN_MAX_P; ++t)
      if (t == q) sq = S[t];
    if (sq >= P.tau) {
      qs = q;
      break;
    }
  }
  const bool unstable = qs < 0;
  if (unstable) qs = 0;
  float s_sel = 0.0f, s_half = 0.0f;
#pragma unroll
  for (int t = 0; t < PN_MAX_P; ++t) {
    if (t == qs) s_sel = S[t];
    if (t == qs - 1) s_half = S[t];
  }
  const double p = ldexp(1.0, fa.p_log2[qs]);
  double est = s_sel > 0.0f ? pow(static_cast<double>(s_sel), 1.0 / p) : 0.0;
  if (fa.estimator == 1 && !unstable && qs > 0 && fa.p_log2[qs - 1] == fa.p_log2[qs] - 1) {
    // r = 1 projection, with the epilogue's clamp of the ratio to <= 1
    const double ratio = static_cast<double>(s_sel) / fmax(static_cast<double>(s_half),
                                                           static_cast<double>(s_sel));
    est = pow(ratio, 2.0 / p);
  }
  fa.samp[2 * s] = est;
  fa.samp[2 * s + 1] = static_cast<double>(mx);
  fa.scls[s] = qs;
}

// One warp per class q: the FP64 sums n, x, y, x^2, x y over the samples of
// the class (x = estimate, y = exact value), lane l taking samples l, l + 32,
// ... in order and a fixed butterfly combining the lanes, so the sums and the
// line are the same on every run; then the least-squares line (the oracle's
// rule, including the degenerate cases).
__global__ void k_fit_solve(const __grid_constant__ FitArgs fa) {
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (q >= fa.n_p) return;
  double c5[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int s = lane; s < fa.n_fit; s += 32) {
    if (fa.scls[s] != q) continue;
    const double x = fa.samp[2 * s], y = fa.samp[2 * s + 1];
    c5[0] += 1.0;
    c5[1] += x;
    c5[2] += y;
    c5[3] += x * x;
    c5[4] += x * y;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
#pragma unroll
    for (int t = 0; t < 5; ++t) c5[t] += __shfl_xor_sync(0xffffffffu, c5[t], off);
  if (lane != 0) return;
  const double n = c5[0], sx = c5[1], sy = c5[2], sxx = c5[3], sxy = c5[4];
  double a = 1.0, b = 0.0;
  if (n >= 2.0 && sxx - sx * sx / n > 1e-12 * sxx) {
    a = (sxy - sx * sy / n) / (sxx - sx * sx / n);
    b = (sy - a * sx) / n;
  } else if (n >= 1.0 && sx > 0.0) {
    a = sy / sx;
  }
  fa.coef[2 * q] = static_cast<float>(a);
  fa.coef[2 * q + 1] = static_cast<float>(b);
  if (fa.user_coef) {
    fa.user_coef[2 * q] = static_cast<float>(a);
    fa.user_coef[2 * q + 1] = static_cast<float>(b);
  }
}

}  // namespace

int launch_fit(const Common& cm, const FitArgs& fa, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (fa.n_fit > 0) {
    k_fit_samples<<<fa.n_fit, FIT_THREADS, 0, s>>>(cm, fa);
    const int e = cudaGetLastError();
    if (e) return e;
  }
  k_fit_solve<<<1, 32 * PN_MAX_P, 0, s>>>(fa);
  return cudaGetLastError();
}

}  // namespace pn
