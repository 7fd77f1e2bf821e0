// Max-convolution z_m = max_i x_i y_(m-i) (Sec. 1) and its p-norm estimate
// with H = FFT convolution (Sec. 1; the scaled H' and the threshold tau of
// Sec. 2.1).
//
// k_maxconv_fft: one CTA per problem, everything in shared memory.  Per p
// (largest first): x' = x / max x and y' = y / max y raised to p in FP64, packed
// as one complex sequence a = x'^p + i y'^p and transformed by one radix-2 FFT
// (bit-reversed load, decimation in time); the spectra X, Y are separated from
// A by Hermitian symmetry, Z = X Y, and the inverse FFT gives the ring
// convolution S^(p) = x'^p * y'^p.  Each index m takes the first p with
// S^(p)_m >= tau; z_m = max x max y (S^(p*)_m)^(1/p*).  The CTA stops as soon
// as every index is resolved.  The transforms run in FP64: the FFT's absolute
// error is about log2(N) 2^-53 times the norms of the powered vectors, which
// is what the paper's tau = 1e-12 guards (GB300 issues FP64 at 1/64 of the
// FP32 rate, so everything that needs no FP64 is kept out of it: the powers
// x'^p are formed in FP32, relative error (p - 1) 2^-24, and the roots of
// S >= 1e-30 by FP32 square roots).  When the indices still open after
// a level hold few terms in total (typically the edges of the convolution),
// their p-sums for every remaining p are summed directly in FP64 (the naive
// ring convolution, which the FFT only reproduces) instead of running more
// FFT levels.
//
// k_maxconv_exact: the exact comparison on the CUDA cores, one CTA per 1792
// outputs and 8192 terms of one problem, 7 consecutive outputs per thread;
// each FP32 product is correctly rounded and the max is exact, so the result
// is bit-identical to any sequential evaluation.
#include <cstdint>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "pn_device.cuh"

namespace pn {

namespace {

constexpr int FFT_THREADS = 512;
constexpr int FFT_LOG_NMAX = MAXCONV_LOG_NMAX;
constexpr int FFT_NMAX = 1 << FFT_LOG_NMAX;

// exp(-2 pi i k / NMAX), k < NMAX / 2; a transform of length N uses every
// (NMAX / N)-th entry.
__device__ double2 g_twiddle[FFT_NMAX / 2];

__global__ void k_twiddle_init() {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= FFT_NMAX / 2) return;
  double s, c;
  sincospi(-2.0 * static_cast<double>(k) / FFT_NMAX, &s, &c);
  g_twiddle[k] = make_double2(c, s);
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

// conj(a) * b
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.x, b.y, -a.y * b.x));
}

// In-place radix-2 decimation-in-time FFT of a[0..L) (L = 2^logL) held in
// bit-reversed order; natural order on return; unscaled.  INV selects the
// inverse (conjugate twiddles).  tw[k * tws] = exp(-2 pi i k / L).  The first
// two stages (twiddles 1 and -+i) run as one multiply-free radix-4 pass.
template <bool INV>
__device__ void fft_dit(double2* a, const double2* tw, int logL, int tws) {
  const int L = 1 << logL;
  int s0 = 0;
  if (logL >= 2) {
    for (int g = threadIdx.x; g < (L >> 2); g += FFT_THREADS) {
      double2* q = a + 4 * g;
      const double2 a0 = q[0], a1 = q[1], a2 = q[2], a3 = q[3];
      const double2 b0 = make_double2(a0.x + a1.x, a0.y + a1.y);
      const double2 b1 = make_double2(a0.x - a1.x, a0.y - a1.y);
      const double2 b2 = make_double2(a2.x + a3.x, a2.y + a3.y);
      const double2 b3 = make_double2(a2.x - a3.x, a2.y - a3.y);
      // forward: t = -i b3; inverse: t = +i b3
      const double2 t = INV ? make_double2(-b3.y, b3.x) : make_double2(b3.y, -b3.x);
      q[0] = make_double2(b0.x + b2.x, b0.y + b2.y);
      q[2] = make_double2(b0.x - b2.x, b0.y - b2.y);
      q[1] = make_double2(b1.x + t.x, b1.y + t.y);
      q[3] = make_double2(b1.x - t.x, b1.y - t.y);
    }
    __syncthreads();
    s0 = 2;
  }
  for (int s = s0; s < logL; ++s) {
    const int h = 1 << s;                     // half span
    const int step = ((L >> 1) >> s) * tws;   // twiddle stride: L / (2h)
    for (int b = threadIdx.x; b < (L >> 1); b += FFT_THREADS) {
      const int j = b & (h - 1);
      const int i0 = ((b >> s) << (s + 1)) + j;
      const int i1 = i0 + h;
      const double2 w = tw[j * step];
      const double2 t = INV ? cmulc(w, a[i1]) : cmul(w, a[i1]);
      const double2 u = a[i0];
      a[i0] = make_double2(u.x + t.x, u.y + t.y);
      a[i1] = make_double2(u.x - t.x, u.y - t.y);
    }
    __syncthreads();
  }
}

// (S)^(1/2^plog): plog correctly rounded FP32 square roots of float(S) for
// S >= 1e-30 (the output is FP32; relative error about (plog + 1) 2^-24),
// FP64 square roots below that (only unstable indices at the smallest p).
__device__ __forceinline__ double root_pow2(double S, int plog) {
  if (S >= 1e-30) {
    float r = static_cast<float>(S);
    for (int s = 0; s < plog; ++s) r = sqrtf(r);
    return r;
  }
  double r = S > 0.0 ? S : 0.0;
  for (int s = 0; s < plog; ++s) r = sqrt(r);
  return r;
}

// Number of terms x_i y_(m-i) of output m.
__device__ __forceinline__ int terms_of(int m, int nx, int ny) {
  const int lo = m - ny + 1 > 0 ? m - ny + 1 : 0;
  const int hi = m < nx - 1 ? m : nx - 1;
  return hi - lo + 1;
}

// Index m still open after level q: its p-sums for levels q-1 .. 0 summed
// directly, sum_i (x'_i y'_(m-i))^p in FP64, then the selection rule.
__device__ void direct_levels(const MaxconvArgs& ma, const float* x, const float* y, double isx,
                              double isy, double sxy, int m, int q, float* z, uint8_t* res) {
  double S[PN_MAX_P];
#pragma unroll
  for (int t = 0; t < PN_MAX_P; ++t) S[t] = 0.0;
  const int lo = m - ma.ny + 1 > 0 ? m - ma.ny + 1 : 0;
  const int hi = m < ma.nx - 1 ? m : ma.nx - 1;
  for (int i = lo; i <= hi; ++i) {
    double t = (static_cast<double>(x[i]) * isx) * (static_cast<double>(y[m - i]) * isy);
    int lg = 0;
#pragma unroll
    for (int u = 0; u < PN_MAX_P; ++u) {
      if (u < q) {
        while (lg < ma.p_log2[u]) {
          t *= t;
          ++lg;
        }
        S[u] += t;
      }
    }
  }
  int qs = -1;
  double s_sel = 0.0;
#pragma unroll
  for (int u = PN_MAX_P - 1; u >= 0; --u) {
    if (u < q && qs < 0 && S[u] >= ma.tau) {
      qs = u;
      s_sel = S[u];
    }
  }
  const bool stable = qs >= 0;
  if (!stable) {
    qs = 0;
    s_sel = S[0];
  }
  z[m] = static_cast<float>(sxy * root_pow2(s_sel, ma.p_log2[qs]));
  res[m] = static_cast<uint8_t>(ma.p_log2[qs] | (stable ? 0 : 0x80));
}

// In-place radix-2 decimation-in-frequency FFT of a[0..L) in natural order;
// bit-reversed order on return; unscaled; INV: conjugate twiddles.
template <bool INV>
__device__ void fft_dif(double2* a, const double2* tw, int logL, int tws) {
  const int L = 1 << logL;
  for (int s = logL - 1; s >= 0; --s) {
    const int h = 1 << s;
    const int step = ((L >> 1) >> s) * tws;
    for (int b = threadIdx.x; b < (L >> 1); b += FFT_THREADS) {
      const int j = b & (h - 1);
      const int i0 = ((b >> s) << (s + 1)) + j;
      const int i1 = i0 + h;
      const double2 u = a[i0], v = a[i1];
      const double2 d = make_double2(u.x - v.x, u.y - v.y);
      a[i0] = make_double2(u.x + v.x, u.y + v.y);
      const double2 w = tw[j * step];
      a[i1] = INV ? cmulc(w, d) : cmul(w, d);
    }
    __syncthreads();
  }
}

// Z_k from A_k and A_(N-k) (the spectra of the packed real pair).
__device__ __forceinline__ double2 spec_z(double2 ak, double2 an) {
  const double2 X = make_double2(0.5 * (ak.x + an.x), 0.5 * (ak.y - an.y));
  const double2 Y = make_double2(0.5 * (ak.y + an.y), -0.5 * (ak.x - an.x));
  return cmul(X, Y);
}

// V_k = (Z_k + conj Z_(M-k)) / 2 + i conj(W^k) (Z_k - conj Z_(M-k)) / 2, w = W^k.
__device__ __forceinline__ double2 spec_v(double2 zk, double2 zmk, double2 w) {
  const double2 e = make_double2(0.5 * (zk.x + zmk.x), 0.5 * (zk.y - zmk.y));
  const double2 d = make_double2(0.5 * (zk.x - zmk.x), 0.5 * (zk.y + zmk.y));
  const double2 o = cmulc(w, d);  // O_k = conj(W^k) d
  return make_double2(e.x - o.y, e.y + o.x);
}

__device__ __forceinline__ int bitrev(int k, int logN) {
  return logN == 0 ? 0 : static_cast<int>(__brev(static_cast<unsigned>(k)) >> (32 - logN));
}

// One level of the FFT convolution in shared memory: a = x'^p + i y'^p (zero
// padded; powers in FP32, or in FP64 with POW64, which the NormQueue needs:
// it subtracts the popped term's p-th power from the sums, so their error
// must stay far below the next term's; y_rev reads y backwards), forward FFT
// of length N,
// the spectrum of the ring convolution, inverse at half length.  On return
// S_m = (m odd ? a[m/2].y : a[m/2].x) * 2 / N.
//
// The spectrum: X_k = (A_k + conj A_(N-k)) / 2, Y_k = (A_k - conj A_(N-k)) /
// (2i), Z = X Y (Hermitian: the convolution is real).  Its inverse runs at
// half length M = N / 2: with E, O the length-M DFTs of the even and odd
// samples of S, Z_k = E_k + W^k O_k and Z_(k+M) = conj Z_(M-k) = E_k - W^k O_k
// (W = exp(-2 pi i / N)), so
// V_k = E_k + i O_k = (Z_k + conj Z_(M-k)) / 2 + i W^-k (Z_k - conj Z_(M-k)) / 2
// is the DFT of v_j = S_2j + i S_(2j+1).  Thread work: k and M - k together
// (reads A at k, N - k, M - k, M + k).
template <bool POW64>
__device__ void conv_level(double2* a, const double2* tw, const MaxconvArgs& ma, const float* x,
                           const float* y, double isx, double isy, int plog, bool y_rev) {
  const int N = 1 << ma.logN;
  const int tid = threadIdx.x;
  using T = typename std::conditional<POW64, double, float>::type;
  for (int k = tid; k < N; k += FFT_THREADS) {
    T xr = 0, yr = 0;
    if (k < ma.nx) {
      xr = static_cast<T>(x[k]) * static_cast<T>(isx);
      for (int s = 0; s < plog; ++s) xr *= xr;
    }
    if (k < ma.ny) {
      yr = static_cast<T>(y[y_rev ? ma.ny - 1 - k : k]) * static_cast<T>(isy);
      for (int s = 0; s < plog; ++s) yr *= yr;
    }
    a[bitrev(k, ma.logN)] = make_double2(static_cast<double>(xr), static_cast<double>(yr));
  }
  __syncthreads();
  fft_dit<false>(a, tw, ma.logN, 1);
  const int M = N >> 1;
  constexpr int QUADS = FFT_NMAX / 4 / FFT_THREADS + 1;
  double2 vk[QUADS], vm[QUADS];
  for (int u = 0; u < QUADS; ++u) {
    const int k = tid + u * FFT_THREADS;
    if (k <= (M >> 1)) {
      const double2 zk = spec_z(a[k], a[(N - k) & (N - 1)]);
      const double2 zm = spec_z(a[M - k], a[M + k]);
      vk[u] = spec_v(zk, zm, tw[k]);
      vm[u] = spec_v(zm, zk, (M - k) < M ? tw[M - k] : make_double2(1.0, 0.0));
    }
  }
  __syncthreads();
  for (int u = 0; u < QUADS; ++u) {
    const int k = tid + u * FFT_THREADS;
    if (k <= (M >> 1)) {
      a[bitrev(k, ma.logN - 1)] = vk[u];
      if (k != 0 && (M - k) != k) a[bitrev(M - k, ma.logN - 1)] = vm[u];
    }
  }
  __syncthreads();
  fft_dit<true>(a, tw, ma.logN - 1, 2);
}

__global__ void __launch_bounds__(FFT_THREADS, 1)
    k_maxconv_fft(const __grid_constant__ MaxconvArgs ma) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int N = 1 << ma.logN;
  double2* a = reinterpret_cast<double2*>(smem);
  double2* tw = a + N;
  uint8_t* res = reinterpret_cast<uint8_t*>(tw + (N >> 1));  // p_sel, 0xFF = open
  __shared__ double red[2][FFT_THREADS / 32];
  const int b = blockIdx.x;
  const float* x = ma.x + (int64_t)b * ma.ldx;
  const float* y = ma.y + (int64_t)b * ma.ldy;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (int k = tid; k < (N >> 1); k += FFT_THREADS) tw[k] = g_twiddle[k << (FFT_LOG_NMAX - ma.logN)];
  // maxima and domain (R+, finite)
  float mx = 0.0f, my = 0.0f;
  bool bad = false;
  for (int k = tid; k < ma.nx; k += FFT_THREADS) {
    const float v = x[k];
    bad |= !(v >= 0.0f && v <= 3.4028235e38f);
    mx = fmaxf(mx, v);
  }
  for (int k = tid; k < ma.ny; k += FFT_THREADS) {
    const float v = y[k];
    bad |= !(v >= 0.0f && v <= 3.4028235e38f);
    my = fmaxf(my, v);
  }
  if (__syncthreads_or(bad)) {
    if (tid == 0) set_status(ma.status, PN_EDOMAIN);
    return;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    my = fmaxf(my, __shfl_xor_sync(0xffffffffu, my, off));
  }
  if (lane == 0) {
    red[0][warp] = mx;
    red[1][warp] = my;
  }
  for (int m = tid; m < ma.nz; m += FFT_THREADS) res[m] = 0xFF;
  __syncthreads();
  double sx = 0.0, sy = 0.0;
  for (int w = 0; w < FFT_THREADS / 32; ++w) {
    sx = fmax(sx, red[0][w]);
    sy = fmax(sy, red[1][w]);
  }
  if (sx == 0.0) sx = 1.0;  // a zero vector keeps scale 1
  if (sy == 0.0) sy = 1.0;
  const double invM = 2.0 / N;
  const float isx_f = static_cast<float>(1.0 / sx), isy_f = static_cast<float>(1.0 / sy);
  const double sxy = sx * sy;
  float* z = ma.z + (int64_t)b * ma.ldz;
  __shared__ unsigned long long open_terms;
  __shared__ int n_open;

  for (int q = ma.n_p - 1; q >= 0; --q) {
    const int plog = ma.p_log2[q];
    conv_level<false>(a, tw, ma, x, y, isx_f, isy_f, plog, false);
    // selection: first (largest) p with S >= tau; the smallest p takes the rest
    if (tid == 0) {
      open_terms = 0ull;
      n_open = 0;
    }
    __syncthreads();
    unsigned long long my_terms = 0ull;
    for (int m = tid; m < ma.nz; m += FFT_THREADS) {
      if (res[m] != 0xFF) continue;
      const double S = ((m & 1) ? a[m >> 1].y : a[m >> 1].x) * invM;
      const bool stable = S >= ma.tau;
      if (stable || q == 0) {
        z[m] = static_cast<float>(sxy * root_pow2(S, plog));
        res[m] = static_cast<uint8_t>(plog | (stable ? 0 : 0x80));
      } else {
        my_terms += static_cast<unsigned long long>(terms_of(m, ma.nx, ma.ny));
      }
    }
    if (my_terms) atomicAdd(&open_terms, my_terms);
    __syncthreads();
    const unsigned long long W = open_terms;
    if (W == 0ull) break;
    // few open terms: sum the remaining p directly (cost ~ W (8 + 2q) FP64
    // operations against ~10 N log2 N for one more FFT level)
    if (W * static_cast<unsigned long long>(8 + 2 * q) <=
        10ull * static_cast<unsigned long long>(N) * static_cast<unsigned long long>(ma.logN)) {
      // compact list of the open indices (the FFT buffer is free now)
      int* list = reinterpret_cast<int*>(a);
      for (int m = tid; m < ma.nz; m += FFT_THREADS)
        if (res[m] == 0xFF) list[atomicAdd(&n_open, 1)] = m;
      __syncthreads();
      const int cnt = n_open;
      for (int e = tid; e < cnt; e += FFT_THREADS)
        direct_levels(ma, x, y, static_cast<double>(isx_f), static_cast<double>(isy_f), sxy,
                      list[e], q, z, res);
      break;
    }
  }
  __syncthreads();
  if (ma.psel) {
    uint8_t* ps = ma.psel + (int64_t)b * ma.ldp;
    for (int m = tid; m < ma.nz; m += FFT_THREADS) ps[m] = res[m];
  }
}

// ---------------------------------------------------------------- exact ---
constexpr int MCX_THREADS = 256;
constexpr int MCX_OUT = 7;                              // outputs per thread
constexpr int MCX_SPAN = MCX_THREADS * MCX_OUT;         // outputs per CTA
constexpr int MCX_IB = 8192;                            // terms i per CTA

// z_m for m in [m0, m0 + MCX_SPAN), terms i in [i0, i0 + MCX_IB), problems
// blockIdx.z, + gridDim.z, ...  Shared memory holds x[i0 .. i0 + IB + 8) and
// the y values those terms reach, zero outside [0, ny), so invalid terms
// contribute 0 (every product is >= 0, and the max over the nonempty set of
// valid terms is unchanged; terms counted by two CTAs are harmless for a max).
// Thread t owns outputs m0 + 7t .. m0 + 7t + 6: 7 is coprime with the 32
// banks, so the threads of a warp read their y windows without conflicts,
// and the warp walks one common range of i, so x is read by broadcast.
// Several i-blocks combine by atomicMax on the float bits (non-negative
// floats order like their bit patterns; z is zeroed first).
__global__ void __launch_bounds__(MCX_THREADS)
    k_maxconv_exact(const __grid_constant__ MaxconvArgs ma) {
  extern __shared__ __align__(16) float sm[];
  const int m0 = blockIdx.x * MCX_SPAN;
  const int i0 = blockIdx.y * MCX_IB;
  const int warp = threadIdx.x >> 5;
  float* xs = sm;                        // MCX_IB + 8 values: x[i0 + k]
  float* ys = sm + MCX_IB + 8;           // MCX_SPAN + MCX_IB + 16 values: y[tb + u]
  const int tb = m0 - i0 - MCX_IB - 8;   // y index of ys[0]
  const bool atomic = gridDim.y > 1;
  // terms of this CTA: i in [max(i0, m0 - ny + 1), min(i0 + IB, m0 + SPAN, nx))
  const int c_lo = max(i0, m0 - ma.ny + 1);
  const int c_hi = min(min(i0 + MCX_IB, m0 + MCX_SPAN), ma.nx);
  if (c_lo >= c_hi || m0 >= ma.nz) return;
  // the warp's outputs and terms
  const int mw = m0 + warp * 32 * MCX_OUT;
  const int w_lo = max(c_lo, mw - ma.ny + 1);
  const int w_hi = min(c_hi, mw + 32 * MCX_OUT);
  const int mt = m0 + threadIdx.x * MCX_OUT;
  for (int64_t b = blockIdx.z; b < ma.batch; b += gridDim.z) {
    __syncthreads();  // the previous problem's reads are done
    const float* x = ma.x + b * ma.ldx;
    const float* y = ma.y + b * ma.ldy;
    for (int k = threadIdx.x; k < MCX_IB + 8; k += MCX_THREADS)
      xs[k] = (i0 + k < ma.nx) ? x[i0 + k] : 0.0f;
    for (int u = threadIdx.x; u < MCX_SPAN + MCX_IB + 16; u += MCX_THREADS) {
      const int t = tb + u;
      ys[u] = (t >= 0 && t < ma.ny) ? y[t] : 0.0f;
    }
    __syncthreads();
    float acc[MCX_OUT];
#pragma unroll
    for (int r = 0; r < MCX_OUT; ++r) acc[r] = 0.0f;
#pragma unroll 1
    for (int i = w_lo; i < w_hi; i += 8) {
      const int k = i - i0;
      float xv[8], yv[MCX_OUT + 7];
#pragma unroll
      for (int e = 0; e < 8; ++e) xv[e] = xs[k + e];
      // yv[u] = y_(mt - i - 7 + u), i.e. ys[(mt - i - 7 + u) - tb]
      const float* yp = ys + (mt - i - 7 - tb);
#pragma unroll
      for (int u = 0; u < MCX_OUT + 7; ++u) yv[u] = yp[u];
#pragma unroll
      for (int r = 0; r < MCX_OUT; ++r) {
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
          // terms i+e and i+e+1 of output mt + r
          const float p0 = xv[e] * yv[r - e + 7];
          const float p1 = xv[e + 1] * yv[r - e + 6];
          float t;
          asm("max.f32 %0, %1, %2, %3;" : "=f"(t) : "f"(acc[r]), "f"(p0), "f"(p1));
          acc[r] = t;
        }
      }
    }
    float* z = ma.z + b * ma.ldz;
#pragma unroll
    for (int r = 0; r < MCX_OUT; ++r) {
      const int m = mt + r;
      if (m >= ma.nz) continue;
      if (atomic) {
        if (acc[r] > 0.0f) atomicMax(reinterpret_cast<unsigned int*>(z + m), __float_as_uint(acc[r]));
      } else {
        z[m] = acc[r];
      }
    }
  }
}

// ------------------------------------------------------- long problems ---
// One max-convolution of any length up to N = 2^22 (nz = nx + ny - 1 <= N),
// four-step FFT over the N1 x N2 view of the length-N buffer (index
// n = N2 n1 + n2, N1 = 2^min(10, floor(log2 N / 2))):
//   forward  A[k1 + N1 k2] = sum_n2 W_N2^(n2 k2) [W_N^(n2 k1) sum_n1 a[n] W_N1^(n1 k1)]
//   inverse  s[n] = sum_k1 W_N1^-(n1 k1) [W_N^-(n2 k1) sum_k2 Z[k1 + N1 k2] W_N2^-(n2 k2)]
// Three kernels per level: columns forward (the powered inputs are formed on
// the fly), row pairs (forward rows, spectrum, inverse rows: row k1 holds the
// partners N - k of row N1 - k1), columns inverse with the selection.  A
// fourth kernel ends the level loop (nothing open) or sums the remaining
// levels directly for few open terms.  All kernels of a finished call return
// at once (device flag), so every launch is issued unconditionally.
constexpr int LONG_CC = 8;   // columns per CTA of the column kernels

struct LongArgs {
  const float* x;
  const float* y;
  float* z;
  uint8_t* res;            // p_sel, 0xFF while open
  int32_t nx, ny, nz;
  int32_t logN, l1, l2;    // N = 2^logN = N1 N2
  int32_t n_p;
  int32_t p_log2[PN_MAX_P];
  double tau;
  int32_t* status;
  double2* buf;            // N complex
  const double2* tlo;      // W_N^m, m < 2048
  const double2* thi;      // W_N^(2048 m), m < N / 2048
  unsigned long long* open_terms;  // per level
  int32_t* done;
  uint32_t* mxy;           // max x, max y (float bits)
};

__device__ __forceinline__ double2 w_n(const LongArgs& la, int m) {
  return cmul(la.thi[m >> 11], la.tlo[m & 2047]);
}

__global__ void k_long_tables(double2* tlo, double2* thi, int logN) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const double N = static_cast<double>(1 << logN);
  double s, c;
  if (k < 2048) {
    sincospi(-2.0 * k / N, &s, &c);
    tlo[k] = make_double2(c, s);
  }
  if (k < ((1 << logN) >> 11)) {
    sincospi(-2.0 * (2048.0 * k) / N, &s, &c);
    thi[k] = make_double2(c, s);
  }
}

__global__ void k_long_max(const __grid_constant__ LongArgs la) {
  float mx = 0.0f, my = 0.0f;
  bool bad = false;
  const int stride = gridDim.x * blockDim.x;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < la.nx; k += stride) {
    const float v = la.x[k];
    bad |= !(v >= 0.0f && v <= 3.4028235e38f);
    mx = fmaxf(mx, v);
  }
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < la.ny; k += stride) {
    const float v = la.y[k];
    bad |= !(v >= 0.0f && v <= 3.4028235e38f);
    my = fmaxf(my, v);
  }
  if (bad) {
    set_status(la.status, PN_EDOMAIN);
    *la.done = 1;  // nothing more runs
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    my = fmaxf(my, __shfl_xor_sync(0xffffffffu, my, off));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(la.mxy, __float_as_uint(mx));
    atomicMax(la.mxy + 1, __float_as_uint(my));
  }
}

__device__ __forceinline__ void long_scales(const LongArgs& la, double& sx, double& sy) {
  sx = __uint_as_float(la.mxy[0]);
  sy = __uint_as_float(la.mxy[1]);
  if (sx == 0.0) sx = 1.0;
  if (sy == 0.0) sy = 1.0;
}

// columns [c0, c0 + CC): a[N2 n1 + n2] = x'^p + i y'^p, DFT over n1 (length
// N1), times W_N^(n2 k1), stored row-major as buf[k1 N2 + n2].
__global__ void __launch_bounds__(FFT_THREADS, 1)
    k_long_col_fwd(const __grid_constant__ LongArgs la, int q) {
  if (*la.done) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int N1 = 1 << la.l1, N2 = 1 << la.l2;
  double2* col = reinterpret_cast<double2*>(smem);   // [CC][N1]
  double2* tw = col + LONG_CC * N1;                   // N1 / 2
  const int tid = threadIdx.x;
  for (int k = tid; k < (N1 >> 1); k += FFT_THREADS) tw[k] = g_twiddle[k << (FFT_LOG_NMAX - la.l1)];
  double sx, sy;
  long_scales(la, sx, sy);
  const float isx = static_cast<float>(1.0 / sx), isy = static_cast<float>(1.0 / sy);
  const int plog = la.p_log2[q];
  const int c0 = blockIdx.x * LONG_CC;
  for (int e = tid; e < LONG_CC * N1; e += FFT_THREADS) {
    const int n1 = e / LONG_CC, c = e % LONG_CC;
    const int n = n1 * N2 + c0 + c;
    float xr = 0.0f, yr = 0.0f;
    if (n < la.nx) {
      xr = la.x[n] * isx;
      for (int s = 0; s < plog; ++s) xr *= xr;
    }
    if (n < la.ny) {
      yr = la.y[n] * isy;
      for (int s = 0; s < plog; ++s) yr *= yr;
    }
    col[c * N1 + bitrev(n1, la.l1)] = make_double2(xr, yr);
  }
  __syncthreads();
  for (int c = 0; c < LONG_CC; ++c) fft_dit<false>(col + c * N1, tw, la.l1, 1);
  for (int e = tid; e < LONG_CC * N1; e += FFT_THREADS) {
    const int k1 = e / LONG_CC, c = e % LONG_CC;
    const int n2 = c0 + c;
    la.buf[(int64_t)k1 * N2 + n2] = cmul(w_n(la, n2 * k1), col[c * N1 + k1]);
  }
}

// Z from a spectrum value and its partner (the packed real pair).
__device__ __forceinline__ void pair_z(double2& a, double2& b) {
  const double2 za = spec_z(a, b), zb = spec_z(b, a);
  a = za;
  b = zb;
}

// rows k1 and N1 - k1 (blockIdx.x = k1 in [0, N1/2]; rows 0 and N1/2 alone)
__global__ void __launch_bounds__(FFT_THREADS, 1)
    k_long_rows(const __grid_constant__ LongArgs la) {
  if (*la.done) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int N1 = 1 << la.l1, N2 = 1 << la.l2;
  double2* r0 = reinterpret_cast<double2*>(smem);  // row k1
  double2* r1 = r0 + N2;                            // row N1 - k1
  double2* tw = r1 + N2;                            // N2 / 2
  const int tid = threadIdx.x;
  const int k1 = blockIdx.x, k1b = N1 - k1;
  const bool two = k1 != 0 && k1 != (N1 >> 1);
  for (int k = tid; k < (N2 >> 1); k += FFT_THREADS) tw[k] = g_twiddle[k << (FFT_LOG_NMAX - la.l2)];
  for (int k = tid; k < N2; k += FFT_THREADS) {
    r0[bitrev(k, la.l2)] = la.buf[(int64_t)k1 * N2 + k];
    if (two) r1[bitrev(k, la.l2)] = la.buf[(int64_t)k1b * N2 + k];
  }
  __syncthreads();
  fft_dit<false>(r0, tw, la.l2, 1);
  if (two) fft_dit<false>(r1, tw, la.l2, 1);
  // spectrum in place: the partner of (k1, k2) is (N1 - k1, N2 - 1 - k2),
  // of (0, k2) it is (0, (N2 - k2) mod N2)
  if (two) {
    for (int k2 = tid; k2 < N2; k2 += FFT_THREADS) pair_z(r0[k2], r1[N2 - 1 - k2]);
  } else if (k1 == 0) {
    for (int k2 = tid; k2 <= (N2 >> 1); k2 += FFT_THREADS) {
      const int p2 = (N2 - k2) & (N2 - 1);
      if (p2 == k2) r0[k2] = spec_z(r0[k2], r0[k2]);
      else pair_z(r0[k2], r0[p2]);
    }
  } else {
    for (int k2 = tid; k2 < (N2 >> 1); k2 += FFT_THREADS) pair_z(r0[k2], r0[N2 - 1 - k2]);
  }
  __syncthreads();
  fft_dif<true>(r0, tw, la.l2, 1);
  if (two) fft_dif<true>(r1, tw, la.l2, 1);
  // bit-reversed rows; times conj W_N^(n2 k1)
  for (int n2 = tid; n2 < N2; n2 += FFT_THREADS) {
    la.buf[(int64_t)k1 * N2 + n2] = cmulc(w_n(la, n2 * k1), r0[bitrev(n2, la.l2)]);
    if (two) la.buf[(int64_t)k1b * N2 + n2] = cmulc(w_n(la, n2 * k1b), r1[bitrev(n2, la.l2)]);
  }
}

// columns [c0, c0 + CC): inverse DFT over k1 gives s[N2 n1 + n2]; the
// selection of level q for every open index; open terms counted for the
// direct-sum decision.
__global__ void __launch_bounds__(FFT_THREADS, 1)
    k_long_col_inv(const __grid_constant__ LongArgs la, int q) {
  if (*la.done) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int N1 = 1 << la.l1, N2 = 1 << la.l2;
  double2* col = reinterpret_cast<double2*>(smem);
  double2* tw = col + LONG_CC * N1;
  const int tid = threadIdx.x;
  for (int k = tid; k < (N1 >> 1); k += FFT_THREADS) tw[k] = g_twiddle[k << (FFT_LOG_NMAX - la.l1)];
  const int c0 = blockIdx.x * LONG_CC;
  for (int e = tid; e < LONG_CC * N1; e += FFT_THREADS) {
    const int k1 = e / LONG_CC, c = e % LONG_CC;
    col[c * N1 + bitrev(k1, la.l1)] = la.buf[(int64_t)k1 * N2 + c0 + c];
  }
  __syncthreads();
  for (int c = 0; c < LONG_CC; ++c) fft_dit<true>(col + c * N1, tw, la.l1, 1);
  double sx, sy;
  long_scales(la, sx, sy);
  const double sxy = sx * sy, invN = 1.0 / static_cast<double>(1 << la.logN);
  const int plog = la.p_log2[q];
  unsigned long long terms = 0ull;
  for (int e = tid; e < LONG_CC * N1; e += FFT_THREADS) {
    const int n1 = e / LONG_CC, c = e % LONG_CC;
    const int m = n1 * N2 + c0 + c;
    if (m >= la.nz || la.res[m] != 0xFF) continue;
    const double S = col[c * N1 + n1].x * invN;
    const bool stable = S >= la.tau;
    if (stable || q == 0) {
      la.z[m] = static_cast<float>(sxy * root_pow2(S, plog));
      la.res[m] = static_cast<uint8_t>(plog | (stable ? 0 : 0x80));
    } else {
      terms += static_cast<unsigned long long>(terms_of(m, la.nx, la.ny));
    }
  }
  if (terms) atomicAdd(la.open_terms + q, terms);
}

// After level q: nothing open ends the call; few open terms are summed
// directly for every remaining level (then the call ends); otherwise the
// next level runs.
__global__ void k_long_direct(const __grid_constant__ LongArgs la, int q) {
  if (*la.done) return;
  const unsigned long long W = la.open_terms[q];
  const int N = 1 << la.logN;
  if (W == 0ull || q == 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *la.done = 1;
    return;
  }
  if (W * static_cast<unsigned long long>(8 + 2 * q) >
      10ull * static_cast<unsigned long long>(N) * static_cast<unsigned long long>(la.logN))
    return;
  double sx, sy;
  long_scales(la, sx, sy);
  MaxconvArgs ma;
  ma.nx = la.nx;
  ma.ny = la.ny;
  ma.tau = la.tau;
  for (int t = 0; t < PN_MAX_P; ++t) ma.p_log2[t] = la.p_log2[t];
  const double isx = static_cast<double>(static_cast<float>(1.0 / sx));
  const double isy = static_cast<double>(static_cast<float>(1.0 / sy));
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < la.nz; m += gridDim.x * blockDim.x)
    if (la.res[m] == 0xFF) direct_levels(ma, la.x, la.y, isx, isy, sx * sy, m, q, la.z, la.res);
  if (blockIdx.x == 0 && threadIdx.x == 0) *la.done = 1;  // read by the next launches only
}

// ------------------------------------------------------------ top-k x y ---
// Approximate top-k of the products x_i y_j (Alg. 9 with the NormQueue), for
// `batch` independent pairs of length n (2n - 1 <= 8192), each run twice (y,
// and y reversed for the index recovery):
//   k_topk_sums  one CTA per (problem, direction): the p-sums of every p of P
//                for every diagonal m = i + j (the FFT level above), and the
//                first estimate psi_m;
//   k_topk_pop   one warp per (problem, direction): k NormQueue pops -- the
//                diagonal with the largest psi (two-level argmax over blocks
//                of 32 diagonals), its value, the subtraction of psi^p from
//                every p-sum of that diagonal, the re-estimate clamped to the
//                value just popped; a diagonal is exhausted after as many
//                pops as it has terms;
//   k_topk_index i = (m1 + m2 - n + 1) / 2, j = m1 - i from the diagonals of
//                the two calls' pops of equal rank, kept when x_i y_j agrees
//                with the popped value within TOPK_VERIFY.
constexpr double TOPK_VERIFY = 1e-2;

struct TopkArgs {
  const float* x;
  const float* y;
  int64_t ldx, ldy;
  int32_t batch, n, nz, logN, n_p, k;
  int32_t p_log2[PN_MAX_P];
  double tau;
  double* sig;     // [batch][2][n_p][nz]
  double* psi0;    // [batch][2][nz] estimates (the first, then kept by the pops)
  double* bmax0;   // [batch][2][nb] the largest estimate of each block of 32 diagonals
  uint16_t* left;  // [batch][2][nz] terms of each diagonal not yet popped
  double* scale;   // [batch] max x * max y
  int32_t* diag;   // [batch][2][k]
  float* vals;     // [batch][ldk]
  int32_t* out_i;
  int32_t* out_j;
  int64_t ldk;
  int32_t* status;
};

// sigma^(1/2^plog) in FP64: FP32 square roots, then two Newton steps on
// r^p = sigma (sigma >= tau > 0 is in the FP32 range for the default tau).
__device__ double root_fp64(double sig, int plog) {
  if (!(sig > 0.0)) return 0.0;
  float rf = static_cast<float>(sig);
  for (int s = 0; s < plog; ++s) rf = sqrtf(rf);
  double r = rf;
  if (!(r > 0.0)) {  // below the FP32 range: FP64 square roots
    r = sig;
    for (int s = 0; s < plog; ++s) r = sqrt(r);
    return r;
  }
  const double p = ldexp(1.0, plog);
  for (int it = 0; it < 2; ++it) {
    double rp = r;
    for (int s = 0; s < plog; ++s) rp *= rp;
    r = r * (1.0 + (sig / rp - 1.0) / p);
  }
  return r;
}

__device__ __forceinline__ double pow_pow2(double a, int plog) {
  for (int s = 0; s < plog; ++s) a *= a;
  return a;
}

__global__ void __launch_bounds__(FFT_THREADS, 1)
    k_topk_sums(const __grid_constant__ TopkArgs ta) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int N = 1 << ta.logN;
  double2* a = reinterpret_cast<double2*>(smem);
  double2* tw = a + N;
  __shared__ float red[2][FFT_THREADS / 32];
  const int b = blockIdx.x >> 1, dir = blockIdx.x & 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float* x = ta.x + (int64_t)b * ta.ldx;
  const float* y = ta.y + (int64_t)b * ta.ldy;
  for (int k = tid; k < (N >> 1); k += FFT_THREADS) tw[k] = g_twiddle[k << (FFT_LOG_NMAX - ta.logN)];
  float mx = 0.0f, my = 0.0f;
  bool bad = false;
  for (int k = tid; k < ta.n; k += FFT_THREADS) {
    const float u = x[k], v = y[k];
    bad |= !(u >= 0.0f && u <= 3.4028235e38f) || !(v >= 0.0f && v <= 3.4028235e38f);
    mx = fmaxf(mx, u);
    my = fmaxf(my, v);
  }
  if (__syncthreads_or(bad)) {
    if (tid == 0) set_status(ta.status, PN_EDOMAIN);
    return;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    my = fmaxf(my, __shfl_xor_sync(0xffffffffu, my, off));
  }
  if (lane == 0) {
    red[0][warp] = mx;
    red[1][warp] = my;
  }
  __syncthreads();
  double sx = 0.0, sy = 0.0;
  for (int w = 0; w < FFT_THREADS / 32; ++w) {
    sx = fmax(sx, static_cast<double>(red[0][w]));
    sy = fmax(sy, static_cast<double>(red[1][w]));
  }
  if (sx == 0.0) sx = 1.0;
  if (sy == 0.0) sy = 1.0;
  if (tid == 0 && dir == 0) ta.scale[b] = sx * sy;
  MaxconvArgs ma;
  ma.nx = ta.n;
  ma.ny = ta.n;
  ma.logN = ta.logN;
  const double invM = 2.0 / N;
  double* sig = ta.sig + (int64_t)blockIdx.x * ta.n_p * ta.nz;
  for (int q = 0; q < ta.n_p; ++q) {
    conv_level<true>(a, tw, ma, x, y, 1.0 / sx, 1.0 / sy, ta.p_log2[q], dir == 1);
    for (int m = tid; m < ta.nz; m += FFT_THREADS)
      sig[(int64_t)q * ta.nz + m] = ((m & 1) ? a[m >> 1].y : a[m >> 1].x) * invM;
    __syncthreads();
  }
  // first estimates: the largest p with sigma >= tau (none: 0)
  double* psi = ta.psi0 + (int64_t)blockIdx.x * ta.nz;
  uint16_t* left = ta.left + (int64_t)blockIdx.x * ta.nz;
  for (int m = tid; m < ta.nz; m += FFT_THREADS) {
    double e = 0.0;
    for (int q = ta.n_p - 1; q >= 0; --q) {
      const double v = sig[(int64_t)q * ta.nz + m];
      if (v >= ta.tau) {
        e = root_fp64(v, ta.p_log2[q]);
        break;
      }
    }
    psi[m] = e;
    left[m] = static_cast<uint16_t>(terms_of(m, ta.n, ta.n));
  }
  __syncthreads();
  // the largest estimate of each block of 32 diagonals (-1 past the last)
  const int nb = (ta.nz + 31) >> 5;
  double* bmax = ta.bmax0 + (int64_t)blockIdx.x * nb;
  for (int blk = warp; blk < nb; blk += FFT_THREADS / 32) {
    const int m = blk * 32 + lane;
    double v = m < ta.nz ? psi[m] : -1.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
    if (lane == 0) bmax[blk] = v;
  }
}

// (value, index) argmax across a warp: larger value, then smaller index.
__device__ __forceinline__ void warp_argmax(double& v, int& i) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, off);
    const int oi = __shfl_xor_sync(0xffffffffu, i, off);
    if (ov > v || (ov == v && oi < i)) {
      v = ov;
      i = oi;
    }
  }
}

// One warp per (problem, direction).  The estimates psi and the counts of
// terms left live in the workspace; shared memory holds only the largest
// estimate of each block of 32 diagonals, so every warp of the launch is
// resident at once.  A pop reads the chosen block's 32 estimates with one
// coalesced load.
__global__ void __launch_bounds__(32) k_topk_pop(const __grid_constant__ TopkArgs ta) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int nb = (ta.nz + 31) >> 5;
  double* bmax = reinterpret_cast<double*>(smem);  // nb
  const int lane = threadIdx.x;
  const int b = blockIdx.x >> 1, dir = blockIdx.x & 1;
  double* sig = ta.sig + (int64_t)blockIdx.x * ta.n_p * ta.nz;
  double* psi = ta.psi0 + (int64_t)blockIdx.x * ta.nz;
  uint16_t* left = ta.left + (int64_t)blockIdx.x * ta.nz;
  int32_t* diag = ta.diag + (int64_t)blockIdx.x * ta.k;
  const double* bmax0 = ta.bmax0 + (int64_t)blockIdx.x * nb;
  for (int blk = lane; blk < nb; blk += 32) bmax[blk] = bmax0[blk];
  __syncwarp();
  const double scale = dir == 0 ? ta.scale[b] : 0.0;
  for (int t = 0; t < ta.k; ++t) {
    // the block, then the diagonal, with the largest psi
    double v = -2.0;
    int bi = 0x7fffffff;
    for (int blk = lane; blk < nb; blk += 32) {
      const double w = bmax[blk];
      if (w > v) {
        v = w;
        bi = blk;
      }
    }
    warp_argmax(v, bi);
    const int mcand = bi * 32 + lane;
    double pv = mcand < ta.nz ? psi[mcand] : -1.0;
    const int lf = mcand < ta.nz ? left[mcand] : 0;
    double pm = pv;
    int m = mcand;
    warp_argmax(pm, m);
    if (!(pm > 0.0)) {  // every diagonal exhausted or without a stable p
      for (int r = t + lane; r < ta.k; r += 32) {
        diag[r] = -1;
        if (dir == 0) ta.vals[(int64_t)b * ta.ldk + r] = 0.0f;
      }
      break;
    }
    const double alpha = pm;
    if (lane == 0) {
      diag[t] = m;
      if (dir == 0) ta.vals[(int64_t)b * ta.ldk + t] = static_cast<float>(alpha * scale);
    }
    const int mi = m - bi * 32;  // the popped diagonal's lane
    const int rem = __shfl_sync(0xffffffffu, lf, mi) - 1;
    // NormQueue pop: sigma^(p)_m -= alpha^p for every p (one lane per p)
    double sq = 0.0;
    if (lane < ta.n_p) {
      const int64_t at = (int64_t)lane * ta.nz + m;
      sq = sig[at] - pow_pow2(alpha, ta.p_log2[lane]);
      sig[at] = sq;
    }
    // re-estimate: the largest p whose sigma is >= tau, clamped to alpha
    const unsigned stable = __ballot_sync(0xffffffffu, lane < ta.n_p && sq >= ta.tau);
    double e = 0.0;
    if (rem > 0 && stable) {
      const int qs = 31 - __clz(stable);
      const double sv = __shfl_sync(0xffffffffu, sq, qs);
      e = fmin(root_fp64(sv, ta.p_log2[qs]), alpha);
    }
    if (lane == mi) {
      pv = e;
      psi[m] = e;
      left[m] = static_cast<uint16_t>(rem);
    }
    double w = pv;
    int wi = lane;
    warp_argmax(w, wi);
    if (lane == 0) bmax[bi] = w;
    __syncwarp();
  }
}

__global__ void k_topk_index(const __grid_constant__ TopkArgs ta) {
  const int b = blockIdx.x;
  const int32_t* d1 = ta.diag + (int64_t)(2 * b) * ta.k;
  const int32_t* d2 = ta.diag + (int64_t)(2 * b + 1) * ta.k;
  const float* x = ta.x + (int64_t)b * ta.ldx;
  const float* y = ta.y + (int64_t)b * ta.ldy;
  for (int t = threadIdx.x; t < ta.k; t += blockDim.x) {
    int i = -1, j = -1;
    const int m1 = d1[t], m2 = d2[t];
    const int s = m1 + m2 - ta.n + 1;
    if (m1 >= 0 && m2 >= 0 && (s & 1) == 0) {
      const int ii = s >> 1, jj = m1 - ii;
      if (ii >= 0 && ii < ta.n && jj >= 0 && jj < ta.n) {
        const double v = ta.vals[(int64_t)b * ta.ldk + t];
        const double prod = static_cast<double>(x[ii]) * static_cast<double>(y[jj]);
        if (fabs(prod - v) <= TOPK_VERIFY * v) {
          i = ii;
          j = jj;
        }
      }
    }
    if (ta.out_i) ta.out_i[(int64_t)b * ta.ldk + t] = i;
    if (ta.out_j) ta.out_j[(int64_t)b * ta.ldk + t] = j;
  }
}

std::mutex g_tw_mu;
bool g_tw_ready[64];

}  // namespace

int maxconv_fft_smem_bytes(int logN) {
  const int N = 1 << logN;
  return N * 16 + (N / 2) * 16 + N;  // data, twiddles, p_sel of up to N indices
}

// The device's table of FFT twiddle factors, filled on the first use.
int ensure_twiddles(cudaStream_t s) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_tw_mu);
  if (!g_tw_ready[dev]) {
    k_twiddle_init<<<(FFT_NMAX / 2 + 255) / 256, 256, 0, s>>>();
    const int e = cudaGetLastError();
    if (e) return e;
    g_tw_ready[dev] = true;
  }
  return 0;
}

int launch_maxconv_fft(const MaxconvArgs& ma, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int te = ensure_twiddles(s);
  if (te) return te;
  const int smem = maxconv_fft_smem_bytes(ma.logN);
  const cudaError_t e = cudaFuncSetAttribute(k_maxconv_fft,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  k_maxconv_fft<<<static_cast<unsigned>(ma.batch), FFT_THREADS, smem, s>>>(ma);
  return cudaGetLastError();
}

int maxconv_exact_smem_bytes() {
  return static_cast<int>(sizeof(float)) * (MCX_IB + 8 + MCX_SPAN + MCX_IB + 16);
}

int launch_maxconv_exact(const MaxconvArgs& ma, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int smem = maxconv_exact_smem_bytes();
  const cudaError_t e = cudaFuncSetAttribute(k_maxconv_exact,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int iblocks = (ma.nx + MCX_IB - 1) / MCX_IB;
  if (iblocks > 1) {  // partial maxima meet in z by atomicMax: start from 0
    const cudaError_t me = cudaMemset2DAsync(ma.z, sizeof(float) * ma.ldz, 0,
                                             sizeof(float) * ma.nz, ma.batch, s);
    if (me != cudaSuccess) return me;
  }
  const dim3 grid(static_cast<unsigned>((ma.nz + MCX_SPAN - 1) / MCX_SPAN),
                  static_cast<unsigned>(iblocks),
                  static_cast<unsigned>(ma.batch < 65535 ? ma.batch : 65535));
  k_maxconv_exact<<<grid, MCX_THREADS, smem, s>>>(ma);
  return cudaGetLastError();
}

// Workspace of a long problem: control words, the W_N^m tables, the
// complex buffer of N, and p_sel when the caller passes none.
struct LongLayout {
  size_t off_ctrl = 0, off_tlo = 0, off_thi = 0, off_buf = 0, off_res = 0, total = 0;
};

LongLayout long_layout(int64_t nz, int logN, bool own_res) {
  LongLayout L;
  size_t off = 0;
  L.off_ctrl = off; off += 256;  // open_terms[16] (128 B), done, max x, max y
  L.off_tlo = off; off += 2048 * sizeof(double2);
  L.off_thi = off; off += 2048 * sizeof(double2);
  L.off_buf = off; off += (size_t(1) << logN) * sizeof(double2);
  if (own_res) { L.off_res = off; off += (static_cast<size_t>(nz) + 255) & ~size_t(255); }
  L.total = off;
  return L;
}

int long_logN(int64_t nz) {
  int logN = 1;
  while ((int64_t(1) << logN) < nz) ++logN;
  return logN < 14 ? 14 : logN;
}

int launch_maxconv_long(const pn_opts* o, int64_t nx, const float* x, int64_t ny, const float* y,
                        float* z, uint8_t* p_sel, uint8_t* ws, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int e = ensure_twiddles(s);
  if (e) return e;
  const int64_t nz = nx + ny - 1;
  LongArgs la;
  std::memset(&la, 0, sizeof(la));
  la.logN = long_logN(nz);
  la.l1 = la.logN / 2 < 10 ? la.logN / 2 : 10;
  la.l2 = la.logN - la.l1;
  const LongLayout L = long_layout(nz, la.logN, p_sel == nullptr);
  la.x = x; la.y = y; la.z = z;
  la.res = p_sel ? p_sel : ws + L.off_res;
  la.nx = static_cast<int32_t>(nx);
  la.ny = static_cast<int32_t>(ny);
  la.nz = static_cast<int32_t>(nz);
  la.n_p = o->n_p;
  for (int q = 0; q < o->n_p; ++q) la.p_log2[q] = o->p_log2[q];
  la.tau = o->tau > 0.0 ? o->tau : 1e-12;
  la.status = o->dev_status;
  la.buf = reinterpret_cast<double2*>(ws + L.off_buf);
  la.tlo = reinterpret_cast<const double2*>(ws + L.off_tlo);
  la.thi = reinterpret_cast<const double2*>(ws + L.off_thi);
  la.open_terms = reinterpret_cast<unsigned long long*>(ws + L.off_ctrl);
  la.done = reinterpret_cast<int32_t*>(ws + L.off_ctrl + 128);
  la.mxy = reinterpret_cast<uint32_t*>(ws + L.off_ctrl + 136);
  if ((e = cudaMemsetAsync(ws + L.off_ctrl, 0, 256, s))) return e;
  if ((e = cudaMemsetAsync(la.res, 0xFF, static_cast<size_t>(nz), s))) return e;
  k_long_tables<<<8, 256, 0, s>>>(reinterpret_cast<double2*>(ws + L.off_tlo),
                                  reinterpret_cast<double2*>(ws + L.off_thi), la.logN);
  k_long_max<<<152 * 4, 256, 0, s>>>(la);
  const int N1 = 1 << la.l1, N2 = 1 << la.l2;
  const int smem_col = (LONG_CC * N1 + N1 / 2) * static_cast<int>(sizeof(double2));
  const int smem_row = (2 * N2 + N2 / 2) * static_cast<int>(sizeof(double2));
  if ((e = cudaFuncSetAttribute(k_long_col_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_col)))
    return e;
  if ((e = cudaFuncSetAttribute(k_long_col_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_col)))
    return e;
  if ((e = cudaFuncSetAttribute(k_long_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_row)))
    return e;
  for (int q = o->n_p - 1; q >= 0; --q) {
    k_long_col_fwd<<<N2 / LONG_CC, FFT_THREADS, smem_col, s>>>(la, q);
    k_long_rows<<<N1 / 2 + 1, FFT_THREADS, smem_row, s>>>(la);
    k_long_col_inv<<<N2 / LONG_CC, FFT_THREADS, smem_col, s>>>(la, q);
    k_long_direct<<<152 * 4, 256, 0, s>>>(la, q);
  }
  return cudaGetLastError();
}

struct TopkLayout {
  size_t off_sig = 0, off_psi = 0, off_bmax = 0, off_left = 0, off_scale = 0, off_diag = 0,
         total = 0;
};

TopkLayout topk_layout(int64_t batch, int64_t n, int64_t k, int n_p) {
  TopkLayout L;
  const int64_t nz = 2 * n - 1;
  size_t off = 0;
  L.off_sig = off; off += static_cast<size_t>(batch) * 2 * n_p * nz * sizeof(double);
  off = (off + 255) & ~size_t(255);
  L.off_psi = off; off += static_cast<size_t>(batch) * 2 * nz * sizeof(double);
  off = (off + 255) & ~size_t(255);
  L.off_bmax = off; off += static_cast<size_t>(batch) * 2 * ((nz + 31) / 32) * sizeof(double);
  off = (off + 255) & ~size_t(255);
  L.off_left = off; off += static_cast<size_t>(batch) * 2 * nz * sizeof(uint16_t);
  off = (off + 255) & ~size_t(255);
  L.off_scale = off; off += static_cast<size_t>(batch) * sizeof(double);
  off = (off + 255) & ~size_t(255);
  L.off_diag = off; off += static_cast<size_t>(batch) * 2 * k * sizeof(int32_t);
  L.total = (off + 255) & ~size_t(255);
  return L;
}

int launch_topk(const TopkArgs& ta0, uint8_t* ws, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int e = ensure_twiddles(s);
  if (e) return e;
  TopkArgs ta = ta0;
  const TopkLayout L = topk_layout(ta.batch, ta.n, ta.k, ta.n_p);
  ta.sig = reinterpret_cast<double*>(ws + L.off_sig);
  ta.psi0 = reinterpret_cast<double*>(ws + L.off_psi);
  ta.bmax0 = reinterpret_cast<double*>(ws + L.off_bmax);
  ta.left = reinterpret_cast<uint16_t*>(ws + L.off_left);
  ta.scale = reinterpret_cast<double*>(ws + L.off_scale);
  ta.diag = reinterpret_cast<int32_t*>(ws + L.off_diag);
  const int N = 1 << ta.logN;
  const int smem_sums = (N + N / 2) * static_cast<int>(sizeof(double2));
  if ((e = cudaFuncSetAttribute(k_topk_sums, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_sums)))
    return e;
  const int nb = (ta.nz + 31) / 32;
  const int smem_pop = nb * 8;
  if ((e = cudaFuncSetAttribute(k_topk_pop, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_pop)))
    return e;
  k_topk_sums<<<2 * ta.batch, FFT_THREADS, smem_sums, s>>>(ta);
  k_topk_pop<<<2 * ta.batch, 32, smem_pop, s>>>(ta);
  k_topk_index<<<ta.batch, 256, 0, s>>>(ta);
  return cudaGetLastError();
}

}  // namespace pn

using namespace pn;

extern "C" {

size_t pn_topk_xy_workspace_size(int64_t batch, int64_t n, int64_t k, const pn_opts* opts) {
  if (!host_opts_valid(opts) || batch < 1 || n < 1 || 2 * n - 1 > (int64_t(1) << MAXCONV_LOG_NMAX) ||
      k < 1 || batch > (1 << 20) || k > (int64_t(1) << 30))
    return 0;
  return topk_layout(batch, n, k, opts->n_p).total;
}

pn_status topk_xy(int64_t batch, int64_t n, const float* x, int64_t ldx, const float* y,
                  int64_t ldy, int64_t k, float* vals, int32_t* idx_i, int32_t* idx_j,
                  int64_t ldk, const pn_opts* opts, void* ws, size_t ws_bytes, void* stream) {
  if (!host_opts_valid(opts)) return PN_EINVAL;
  if (opts->estimator != 0 || opts->correction != 0) return PN_EUNSUPPORTED;
  if (batch < 0 || n < 1 || k < 1) return PN_EINVAL;
  if (batch == 0) return PN_OK;
  if (2 * n - 1 > (int64_t(1) << MAXCONV_LOG_NMAX) || batch > (1 << 20) || k > (int64_t(1) << 30))
    return PN_EUNSUPPORTED;
  if (!x || !y || !vals || ldx < n || ldy < n || ldk < k) return PN_EINVAL;
  const size_t need = pn_topk_xy_workspace_size(batch, n, k, opts);
  if (!ws || ws_bytes < need) return PN_EWORKSPACE;
  if (reinterpret_cast<uintptr_t>(ws) % 256) return PN_EALIGN;
  if (host_device_sms() <= 0) return PN_EUNSUPPORTED;
  TopkArgs ta;
  std::memset(&ta, 0, sizeof(ta));
  ta.x = x; ta.y = y; ta.ldx = ldx; ta.ldy = ldy;
  ta.batch = static_cast<int32_t>(batch);
  ta.n = static_cast<int32_t>(n);
  ta.nz = static_cast<int32_t>(2 * n - 1);
  int logN = 1;
  while ((int64_t(1) << logN) < 2 * n - 1) ++logN;
  ta.logN = logN;
  ta.n_p = opts->n_p;
  for (int q = 0; q < opts->n_p; ++q) ta.p_log2[q] = opts->p_log2[q];
  ta.tau = opts->tau > 0.0 ? opts->tau : pn_maxconv_default_tau();
  ta.k = static_cast<int32_t>(k);
  ta.vals = vals; ta.out_i = idx_i; ta.out_j = idx_j; ta.ldk = ldk;
  ta.status = opts->dev_status;
  return launch_topk(ta, static_cast<uint8_t*>(ws), stream) == 0 ? PN_OK : PN_ECUDA;
}


size_t pn_maxconv_long_workspace_size(int64_t nx, int64_t ny, int32_t with_p_sel) {
  if (nx < 1 || ny < 1 || nx + ny - 1 > (int64_t(1) << 22)) return 0;
  const int64_t nz = nx + ny - 1;
  return long_layout(nz, long_logN(nz), with_p_sel == 0).total;
}

pn_status maxconv_pnorm_long(int64_t nx, const float* x, int64_t ny, const float* y, float* z,
                             uint8_t* p_sel, const pn_opts* opts, void* ws, size_t ws_bytes,
                             void* stream) {
  if (!host_opts_valid(opts)) return PN_EINVAL;
  if (opts->estimator != 0 || opts->correction != 0) return PN_EUNSUPPORTED;
  if (nx < 1 || ny < 1) return PN_EINVAL;
  if (nx + ny - 1 > (int64_t(1) << 22)) return PN_EUNSUPPORTED;
  if (!x || !y || !z) return PN_EINVAL;
  const size_t need = pn_maxconv_long_workspace_size(nx, ny, p_sel != nullptr);
  if (!ws || ws_bytes < need) return PN_EWORKSPACE;
  if (reinterpret_cast<uintptr_t>(ws) % 256) return PN_EALIGN;
  if (host_device_sms() <= 0) return PN_EUNSUPPORTED;
  return launch_maxconv_long(opts, nx, x, ny, y, z, p_sel, static_cast<uint8_t*>(ws), stream) == 0
             ? PN_OK
             : PN_ECUDA;
}


double pn_maxconv_default_tau(void) { return 1e-12; }

pn_status maxconv_pnorm(int64_t batch, int64_t nx, const float* x, int64_t ldx, int64_t ny,
                        const float* y, int64_t ldy, float* z, int64_t ldz, uint8_t* p_sel,
                        int64_t ldp, const pn_opts* opts, void* stream) {
  if (!host_opts_valid(opts)) return PN_EINVAL;
  if (opts->estimator != 0 || opts->correction != 0) return PN_EUNSUPPORTED;
  if (batch < 0 || batch > 0x7fffffff || nx < 1 || ny < 1) return PN_EINVAL;
  if (batch == 0) return PN_OK;
  const int64_t nz = nx + ny - 1;
  if (nz > (int64_t(1) << MAXCONV_LOG_NMAX)) return PN_EUNSUPPORTED;
  if (!x || !y || !z || ldx < nx || ldy < ny || ldz < nz || (p_sel && ldp < nz)) return PN_EINVAL;
  if (host_device_sms() <= 0) return PN_EUNSUPPORTED;
  MaxconvArgs ma;
  std::memset(&ma, 0, sizeof(ma));
  ma.x = x; ma.y = y; ma.z = z; ma.psel = p_sel;
  ma.ldx = ldx; ma.ldy = ldy; ma.ldz = ldz; ma.ldp = ldp;
  ma.batch = batch;
  ma.nx = static_cast<int32_t>(nx);
  ma.ny = static_cast<int32_t>(ny);
  ma.nz = static_cast<int32_t>(nz);
  int logN = 1;
  while ((int64_t(1) << logN) < nz) ++logN;
  ma.logN = logN;
  ma.n_p = opts->n_p;
  for (int q = 0; q < opts->n_p; ++q) ma.p_log2[q] = opts->p_log2[q];
  ma.tau = opts->tau > 0.0 ? opts->tau : pn_maxconv_default_tau();
  ma.status = opts->dev_status;
  return launch_maxconv_fft(ma, stream) == 0 ? PN_OK : PN_ECUDA;
}

pn_status maxconv_exact(int64_t batch, int64_t nx, const float* x, int64_t ldx, int64_t ny,
                        const float* y, int64_t ldy, float* z, int64_t ldz, void* stream) {
  if (batch < 0 || nx < 1 || ny < 1) return PN_EINVAL;
  if (batch == 0) return PN_OK;
  if (nx + ny > (int64_t(1) << 30)) return PN_EUNSUPPORTED;
  const int64_t nz = nx + ny - 1;
  if (!x || !y || !z || ldx < nx || ldy < ny || ldz < nz) return PN_EINVAL;
  if (host_device_sms() <= 0) return PN_EUNSUPPORTED;
  MaxconvArgs ma;
  std::memset(&ma, 0, sizeof(ma));
  ma.x = x; ma.y = y; ma.z = z;
  ma.ldx = ldx; ma.ldy = ldy; ma.ldz = ldz;
  ma.batch = batch;
  ma.nx = static_cast<int32_t>(nx);
  ma.ny = static_cast<int32_t>(ny);
  ma.nz = static_cast<int32_t>(nz);
  return launch_maxconv_exact(ma, stream) == 0 ? PN_OK : PN_ECUDA;
}

}  // extern "C"
