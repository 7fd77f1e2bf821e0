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
// k_maxconv_exact: the exact comparison on the CUDA cores, one CTA per 2048
// outputs of one problem, x and zero-padded y in shared memory, 8 consecutive
// outputs per thread; each FP32 product is correctly rounded and the max is
// exact, so the result is bit-identical to any sequential evaluation.
#include <cstdint>
#include <cstring>
#include <mutex>

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

// In-place radix-2 decimation-in-time FFT of a[0..N) held in bit-reversed
// order; natural order on return.  sign = -1 forward, +1 inverse (unscaled).
__device__ void fft_dit(double2* a, const double2* tw, int logN, double sign) {
  const int N = 1 << logN;
  for (int s = 0; s < logN; ++s) {
    const int h = 1 << s;                  // half span
    const int step = (N >> 1) >> s;        // twiddle stride: N / (2h)
    for (int b = threadIdx.x; b < (N >> 1); b += FFT_THREADS) {
      const int j = b & (h - 1);
      const int i0 = ((b >> s) << (s + 1)) + j;
      const int i1 = i0 + h;
      double2 w = tw[j * step];
      w.y *= -sign;                         // table holds the forward sign
      const double2 t = cmul(w, a[i1]);
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

__device__ __forceinline__ int bitrev(int k, int logN) {
  return logN == 0 ? 0 : static_cast<int>(__brev(static_cast<unsigned>(k)) >> (32 - logN));
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
  const double invN = 1.0 / N;
  const float isx_f = static_cast<float>(1.0 / sx), isy_f = static_cast<float>(1.0 / sy);
  const double sxy = sx * sy;
  float* z = ma.z + (int64_t)b * ma.ldz;
  __shared__ unsigned long long open_terms;
  __shared__ int n_open;

  for (int q = ma.n_p - 1; q >= 0; --q) {
    const int plog = ma.p_log2[q];
    // a = x'^p + i y'^p, zero padded, in bit-reversed order (powers in FP32)
    for (int k = tid; k < N; k += FFT_THREADS) {
      float xr = 0.0f, yr = 0.0f;
      if (k < ma.nx) {
        xr = x[k] * isx_f;
        for (int s = 0; s < plog; ++s) xr *= xr;
      }
      if (k < ma.ny) {
        yr = y[k] * isy_f;
        for (int s = 0; s < plog; ++s) yr *= yr;
      }
      a[bitrev(k, ma.logN)] = make_double2(xr, yr);
    }
    __syncthreads();
    fft_dit(a, tw, ma.logN, -1.0);
    // X_k = (A_k + conj A_(N-k)) / 2, Y_k = (A_k - conj A_(N-k)) / (2i),
    // Z = X Y (Hermitian), written back in bit-reversed order
    constexpr int PAIRS = FFT_NMAX / 2 / FFT_THREADS;
    double2 zk[PAIRS];
    for (int u = 0; u < PAIRS; ++u) {
      const int k = tid + u * FFT_THREADS;
      if (k <= (N >> 1)) {
        const double2 ak = a[k], an = a[(N - k) & (N - 1)];
        const double2 X = make_double2(0.5 * (ak.x + an.x), 0.5 * (ak.y - an.y));
        const double2 Y = make_double2(0.5 * (ak.y + an.y), -0.5 * (ak.x - an.x));
        zk[u] = cmul(X, Y);
      }
    }
    double2 zmid = make_double2(0.0, 0.0);  // k = N/2 when it falls past the pairs
    if (tid == 0 && (N >> 1) >= PAIRS * FFT_THREADS) {
      const double2 ak = a[N >> 1];
      zmid = make_double2(ak.x * ak.y, 0.0);
    }
    __syncthreads();
    for (int u = 0; u < PAIRS; ++u) {
      const int k = tid + u * FFT_THREADS;
      if (k <= (N >> 1)) {
        a[bitrev(k, ma.logN)] = zk[u];
        if (k != 0 && k != (N >> 1))
          a[bitrev(N - k, ma.logN)] = make_double2(zk[u].x, -zk[u].y);
      }
    }
    if (tid == 0 && (N >> 1) >= PAIRS * FFT_THREADS) a[bitrev(N >> 1, ma.logN)] = zmid;
    __syncthreads();
    fft_dit(a, tw, ma.logN, 1.0);
    // selection: first (largest) p with S >= tau; the smallest p takes the rest
    if (tid == 0) {
      open_terms = 0ull;
      n_open = 0;
    }
    __syncthreads();
    unsigned long long my_terms = 0ull;
    for (int m = tid; m < ma.nz; m += FFT_THREADS) {
      if (res[m] != 0xFF) continue;
      const double S = a[m].x * invN;
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
constexpr int MCX_OUT = 8;                              // outputs per thread
constexpr int MCX_SPAN = MCX_THREADS * MCX_OUT;         // outputs per CTA

// z_m for m in [m0, m0 + MCX_SPAN) of problems blockIdx.y, + gridDim.y, ...
// Shared memory:
// x[0..nx) and y padded with zeros so that y[t] for t in (-SPAN, ny + 8)
// reads 0 outside [0, ny) (every product is >= 0, so zeros never change a
// max over a nonempty set of valid terms).
__global__ void __launch_bounds__(MCX_THREADS)
    k_maxconv_exact(const __grid_constant__ MaxconvArgs ma) {
  extern __shared__ __align__(16) float sm[];
  const int m0 = blockIdx.x * MCX_SPAN;
  const int ypad = MCX_SPAN + 8;
  float* xs = sm;                        // nx (+8 slack)
  float* ys = sm + ma.nx + 8 + ypad;     // ys[t] = y_t, valid for t in [-ypad, ny + ypad)
  for (int64_t b = blockIdx.y; b < ma.batch; b += gridDim.y) {
    __syncthreads();  // the previous problem's reads are done
    const float* x = ma.x + (int64_t)b * ma.ldx;
    const float* y = ma.y + (int64_t)b * ma.ldy;
    for (int k = threadIdx.x; k < ma.nx + 8; k += MCX_THREADS) xs[k] = k < ma.nx ? x[k] : 0.0f;
    for (int t = threadIdx.x - ypad; t < ma.ny + ypad; t += MCX_THREADS)
      ys[t] = (t >= 0 && t < ma.ny) ? y[t] : 0.0f;
    __syncthreads();
    const int mt = m0 + threadIdx.x * MCX_OUT;  // this thread's first output
    float acc[MCX_OUT];
#pragma unroll
    for (int r = 0; r < MCX_OUT; ++r) acc[r] = 0.0f;
    // valid i for some output of the thread: mt - ny + 1 <= i <= mt + 7, 0 <= i < nx
    int ilo = mt - ma.ny + 1;
    ilo = ilo < 0 ? 0 : ilo;
    ilo &= ~1;
    int ihi = mt + MCX_OUT - 1;
    ihi = ihi > ma.nx - 1 ? ma.nx - 1 : ihi;
    if (mt < ma.nz) {
#pragma unroll 1
      for (int i = ilo; i <= ihi; i += 8) {
        float xv[8], yv[MCX_OUT + 8];
#pragma unroll
        for (int e = 0; e < 8; ++e) xv[e] = xs[i + e];  // zero past nx
        // yv[u] = y_(mt - i - 7 + u), u in [0, 15)
#pragma unroll
        for (int u = 0; u < MCX_OUT + 7; ++u) yv[u] = ys[mt - i - 7 + u];
#pragma unroll
        for (int r = 0; r < MCX_OUT; ++r) {
#pragma unroll
          for (int e = 0; e < 8; e += 2) {
            // terms i+e and i+e+1 of output mt + r: y index mt + r - i - e (- 1)
            const float p0 = xv[e] * yv[r - e + 7];
            const float p1 = xv[e + 1] * yv[r - e + 6];
            float t;
            asm("max.f32 %0, %1, %2, %3;" : "=f"(t) : "f"(acc[r]), "f"(p0), "f"(p1));
            acc[r] = t;
          }
        }
      }
    }
    float* z = ma.z + (int64_t)b * ma.ldz;
#pragma unroll
    for (int r = 0; r < MCX_OUT; ++r)
      if (mt + r < ma.nz) z[mt + r] = acc[r];
  }
}

std::mutex g_tw_mu;
bool g_tw_ready[64];

}  // namespace

int maxconv_fft_smem_bytes(int logN) {
  const int N = 1 << logN;
  return N * 16 + (N / 2) * 16 + N;  // data, twiddles, p_sel of up to N indices
}

int launch_maxconv_fft(const MaxconvArgs& ma, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  {
    std::lock_guard<std::mutex> lk(g_tw_mu);
    if (!g_tw_ready[dev]) {
      k_twiddle_init<<<(FFT_NMAX / 2 + 255) / 256, 256, 0, s>>>();
      const int e = cudaGetLastError();
      if (e) return e;
      g_tw_ready[dev] = true;
    }
  }
  const int smem = maxconv_fft_smem_bytes(ma.logN);
  const cudaError_t e = cudaFuncSetAttribute(k_maxconv_fft,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  k_maxconv_fft<<<static_cast<unsigned>(ma.batch), FFT_THREADS, smem, s>>>(ma);
  return cudaGetLastError();
}

int maxconv_exact_smem_bytes(int nx, int ny) {
  return static_cast<int>(sizeof(float)) * (nx + 8 + 2 * (MCX_SPAN + 8) + ny);
}

int launch_maxconv_exact(const MaxconvArgs& ma, void* stream) {
  const int smem = maxconv_exact_smem_bytes(ma.nx, ma.ny);
  const cudaError_t e = cudaFuncSetAttribute(k_maxconv_exact,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const dim3 grid(static_cast<unsigned>((ma.nz + MCX_SPAN - 1) / MCX_SPAN),
                  static_cast<unsigned>(ma.batch < 65535 ? ma.batch : 65535));
  k_maxconv_exact<<<grid, MCX_THREADS, smem, static_cast<cudaStream_t>(stream)>>>(ma);
  return cudaGetLastError();
}

}  // namespace pn

using namespace pn;

extern "C" {

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
  if (nx + ny > 50000) return PN_EUNSUPPORTED;
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
