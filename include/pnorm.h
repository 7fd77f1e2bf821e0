/*
 * pnorm.h -- C ABI of the GB300 (sm_103a) p-norm semiring product library.
 *
 * The library estimates products on the semiring (x, max) over nonnegative
 * reals with a small family of p-norm rings, following O. Serang, "Fast
 * Computation on Semirings Isomorphic to (x, max) on R+" (arXiv 1511.05690):
 * for each p in P the operands are scaled into [0, 1], raised elementwise to
 * the power p, multiplied with an ordinary (x, +) GEMM on the tensor cores,
 * and per output entry the largest numerically stable p gives the estimate
 * (S^(p*))^(1/p*), which is then un-scaled (Sec. 2.1; Alg. 5).  Through
 * x = exp(-w) the same product gives (+, min) shortest-path squarings
 * (Sec. 2.2).
 *
 * Conventions shared by every call:
 *  - Matrices are row-major FP32 with an explicit leading dimension (in
 *    elements) unless a call says otherwise.  All matrix pointers are DEVICE
 *    pointers owned by the caller; the library never allocates device or
 *    host memory and keeps no state between calls except a per-device cache
 *    of device properties and tile choices (thread-safe).
 *  - `stream` is a cudaStream_t (passed as void*; NULL = legacy default
 *    stream).  Calls only enqueue work: they return before the GPU finishes,
 *    they do not synchronise, and they are safe to capture in a CUDA graph.
 *  - The return value reports errors the host can see (bad sizes, pointers,
 *    options, workspace).  Errors found on the device (inputs outside the
 *    domain, a bounded wait that ran out) are written, first error wins, to
 *    the optional device word `opts->dev_status` as a pn_status value; the
 *    caller reads it after synchronising.  The word must be zeroed by the
 *    caller before the call if it is to be read.
 *  - M, N or K equal to 0 is legal.  No call falls back to the CPU and no
 *    C++ exception crosses this boundary.
 */
#ifndef PNORM_H
#define PNORM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define PN_API __attribute__((visibility("default")))
#else
#define PN_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pn_status {
  PN_OK = 0,
  PN_EINVAL = 1,        /* invalid size, stride, pointer or option */
  PN_EALIGN = 2,        /* workspace not 256-byte aligned */
  PN_EWORKSPACE = 3,    /* workspace smaller than the *_workspace_size query */
  PN_EDOMAIN = 4,       /* (device) input NaN, negative, +inf, or > 2^127 */
  PN_ECUDA = 5,         /* a CUDA runtime call failed (launch, attribute, ...) */
  PN_ETIMEOUT = 6,      /* (device) a bounded wait inside a kernel ran out */
  PN_EUNSUPPORTED = 7   /* no GB300-class device, or an unsupported mode */
} pn_status;

/* Arithmetic of the powered operands fed to the tensor cores (the ring
 * GEMM H of Sec. 2.1).  Accumulation is always FP32. */
typedef enum pn_compute {
  PN_F32_EXACT = 0, /* FP32 operands as a 3xTF32 split: a = hi + lo, hi*hi+hi*lo+lo*hi */
  PN_TF32 = 1,      /* TF32 operands (10-bit mantissa) */
  PN_BF16 = 2,      /* BF16 operands */
  PN_F16 = 3,       /* FP16 operands, powered values mapped to [0, 2^15] */
  PN_E4M3 = 4       /* FP8 E4M3 operands, powered values mapped to [0, 2^8] */
} pn_compute;

#define PN_MAX_P 16

/* Options of every p-norm call.  Fill with pn_default_opts() first. */
typedef struct pn_opts {
  /* The p family P = { 2^p_log2[0] < 2^p_log2[1] < ... } (Sec. 1, the
   * piecewise family {1, 2, 4, ..., p_max}).  1 <= n_p <= 16, p_log2 strictly
   * ascending, each in [0, 15]. */
  int32_t n_p;
  int32_t p_log2[PN_MAX_P];
  /* Stability threshold tau (Sec. 2.1): p is stable for an entry when the
   * scaled p-sum S^(p) >= tau.  <= 0 selects pn_default_tau(K, compute). */
  double tau;
  int32_t compute;     /* pn_compute */
  /* Operand scaling (Sec. 2.1, H'): 2 = per-row (A) / per-column (B) powers
   * of two (default); 1 = one global power of two per operand; 0 = none. */
  int32_t scaling;
  /* APSP only (reading of Sec. 2.2; the paper is silent): 1 = set the
   * diagonal to x = 1 (distance 0) after the transform and after each
   * squaring; 2 (default) = that, and clamp every entry to x <= 1 (distance
   * >= 0); 0 = neither.  Both are exact facts for nonnegative weights, and
   * since the p-norm estimate only overestimates x, the clamped estimate still
   * lies between the exact x and the unclamped one.  Without the clamp,
   * overestimated entries above 1 form cycles whose value grows with every
   * squaring. */
  int32_t diag_policy;
  /* Output tile width of the tensor-core kernel: 0 = automatic (the
   * autotuner's choice, else a size rule), else 128 or 256 (PN_F32_EXACT on
   * one CTA always uses 128; see tile_m for CTA pairs). */
  int32_t tile_n;
  /* Optional device int32 receiving device-side errors (see above). */
  int32_t* dev_status;
  /* Optional cudaEvent_t pair recorded on `stream` immediately before and
   * after the first (largest-p) tensor-core launch, for timing it (the
   * persistent grouped launch: before and after that whole launch). */
  void* ev_gemm_begin;
  void* ev_gemm_end;
  /* Limit of every bounded device-side wait, in nanoseconds; 0 = 2e9. */
  int64_t timeout_ns;
  /* Test hooks, 0 in normal use.  Bit 0: the tensor-core kernel's copy
   * producer skips one stage so that the consumer's bounded wait runs out
   * (PN_ETIMEOUT).  Bit 1: the tensor-copy image kernel announces its first
   * tile's bytes without copying them, with the same effect.  Bit 2: the
   * grouped call runs one launch sequence per p level instead of its single
   * persistent launch (same results; for comparing the two).  Bit 3: the
   * persistent grouped launch also builds the top level's operand images
   * itself instead of taking them from the image kernels launched before it
   * (same results). */
  int32_t debug_flags;
  /* Estimate of max_k u_k from the p-sums (Sec. 2.1):
   *   0 (default) = plain, (S^(p*))^(1/p*), an overestimate by at most
   *       K^(1/p*);
   *   1 = multiset projection with r = 1 from the two evenly spaced sums at
   *       p* / 2 and p*: (S^(p*) / S^(p* / 2))^(2/p*), an underestimate by at most
   *       the factor (2/(sqrt(K)+1))^(2/p*).  Entries whose p* / 2 is not in P
   *       (p* = min P, or a gap in P) and unstable entries keep the plain
   *       estimate.  p_sel and S_sel still report p* and S^(p*).  The level
   *       p* / 2 is then evaluated for every tile holding an entry resolved at
   *       p*, about one more tensor-core pass in total.  maxprod_pnorm,
   *       maxprod_pnorm_static and the grouped call accept it (the grouped
   *       table is built for one value); apsp_pnorm and
   *       maxprod_pnorm_backward return PN_EUNSUPPORTED for 1;
   *   2 = multiset projection with r = 2 (the estimator of the paper's
   *       experiments) from the four evenly spaced sums s_m at m p* / 4,
   *       m = 1..4: the larger root a of gamma_0 + gamma_1 a + gamma_2 a^2,
   *       gamma = (s2 s4 - s3^2, s2 s3 - s1 s4, s1 s3 - s2^2), to the power
   *       4/p*; it never exceeds the exact max and never falls below the
   *       r = 1 value.  The sums at 3p* / 4 come from extra levels
   *       p = 1.5 * 2^k; entries whose p* / 2 and p* / 4 are not the two p
   *       below p* in P (and unstable entries) keep the plain estimate; sums
   *       that the operand format's rounding leaves unresolved
   *       (s1 s3 - s2^2 <= eta s2^2, eta = 32 u of the powered-operand
   *       format: 2^-16 PN_F32_EXACT, 2^-6 PN_TF32 / PN_F16, 2^-3 PN_BF16,
   *       2 PN_E4M3, i.e. never resolved in E4M3) keep the r = 1 value.
   *       About three more tensor-core passes over every tile holding an
   *       entry resolved at p*; the workspace grows by 2 M N floats.
   *       maxprod_pnorm and maxprod_pnorm_static accept it; the grouped
   *       call, apsp_pnorm and maxprod_pnorm_backward return PN_EUNSUPPORTED,
   *       and it excludes correction 2 (PN_EINVAL). */
  int32_t estimator;
  /* Bias correction of the estimate, applied per entry in the scaled space
   * (value / (r_i c_j), where the exact result lies in (0, 1]):
   *   0 (default) = none;
   *   1 = divide by K^(1/p*), the upper end of the plain estimate's envelope
   *       (Sec. 2.1): the worst-case relative error becomes 1 - K^(-1/p*)
   *       (plain estimator only; with estimator 1 or 2 PN_EINVAL);
   *   2 = affine model fitted to a few exact sub-solutions (Discussion): at
   *       the n_fit sample entries (fit_i[s], fit_j[s]) the library computes
   *       the exact max and the estimate directly, fits exact = a_q est + b_q
   *       by least squares per p* class q (one sample, or estimates spread by
   *       less than 1e-12 of their second moment: the ratio fit, b_q = 0; no
   *       sample: unchanged) and applies it to every entry of the class.
   *       fit_i / fit_j are caller-owned device int32 arrays; an index outside
   *       [0, M) x [0, N) is skipped and sets PN_EINVAL in dev_status.
   *       fit_coef (optional, device, 2 * n_p floats) receives (a_q, b_q).
   * maxprod_pnorm and maxprod_pnorm_static accept 1 and 2, the grouped call
   * 1 (each problem's own K); apsp_pnorm and maxprod_pnorm_backward return
   * PN_EUNSUPPORTED for a nonzero correction. */
  int32_t correction;
  int32_t n_fit;
  const int32_t* fit_i;
  const int32_t* fit_j;
  float* fit_coef;
  /* Output tile height of the tensor-core kernel (no counterpart in the
   * paper): 128 = one CTA (one SM) per 128 x tile_n tile; 256 = a CTA pair
   * per 256 x tile_n tile (cta_group::2: the two SMs of a cluster each load
   * one 128-row half of A and one half of the B^T column tile, and the
   * pair's MMA reads both, so each SM moves less operand data per result:
   * a third less than one CTA per 128 x 256 tile at width 256, a quarter
   * less than one per 128 x 128 tile at width 128); 0 = automatic (pairs for
   * M and N >= 256 unless tile_n = 128, or the autotuner's choice).  A
   * pair's width with tile_n = 0 is 256 unless 128-wide tiles need no more
   * waves of clusters (small outputs): with every cluster busy a 256 x 128
   * tile takes 0.94 of the time of a 256 x 256 one, its operand traffic per
   * SM being more than L2 serves.  Pairs serve maxprod_pnorm, maxprod_pnorm_static
   * and apsp_pnorm, and the adjoint's two GEMMs (256 x 256 tiles, chosen
   * automatically when each GEMM gives every pair of SMs at least two tiles,
   * e.g. n >= 4096 on 152 SMs; tile_n = 128 or tile_m = 128 keeps one CTA per
   * tile there); the grouped call uses tiles 128 rows high. */
  int32_t tile_m;
} pn_opts;

/* Human-readable name of a status code (static string). */
PN_API const char* pn_status_string(int32_t status);

/* P = {1, 2, 4, ..., 64}, PN_BF16, default tau, per-row/column scaling,
 * diagonal reset and clamp (diag_policy 2), autotuned tiles, no status word,
 * no events. */
PN_API void pn_default_opts(pn_opts* opts);

/* Default tau for contraction length K and compute mode (reading of Sec. 2.1,
 * where tau is set by the numeric stability of H): with powered operands
 * stored as q = x^p * 2^s in a format of smallest normal mu and m mantissa
 * bits, tau = K * mu * 2^(m - s), so that flushed operands can drop at most
 * a 2^-m fraction of an accepted S.  Returns a negative value for an unknown
 * mode. */
PN_API double pn_default_tau(int64_t K, int32_t compute);

/* Number of streaming multiprocessors of the current device (0 if none). */
PN_API int32_t pn_device_sm_count(void);

/* Bytes of workspace maxprod_pnorm needs for these sizes and options
 * (0 on invalid options); with tile_n = 0 it covers every tile width the
 * autotuner may pick.  The workspace must be 256-byte aligned. */
PN_API size_t pn_workspace_size(int64_t M, int64_t N, int64_t K, const pn_opts* opts);

/* p-norm estimate of the (x, max) product C = A (x,max) B (Alg. 5 with H a
 * tensor-core GEMM; Sec. 2.1 for the scaling and the stable-p rule):
 *   r_i = scale of row i of A, c_j = scale of column j of B,
 *   S^(p)_ij = sum_k (a_ik/r_i * b_kj/c_j)^p            for p in P,
 *   p*_ij = largest p in P with S^(p)_ij >= tau,
 *   C_ij = r_i c_j (S^(p*))^(1/p*).
 * If no p is stable, p* is the smallest p of P and p_sel carries 0x80.
 * A: M x K (lda >= K), B: K x N (ldb >= N), C: M x N (ldc >= N), all FP32,
 * all entries in [0, 2^127], -0 counting as 0 (else PN_EDOMAIN on the device).
 * p_sel (nullable): M x N bytes, row stride N, log2(p*) | 0x80 if unstable.
 * S_sel (nullable): M x N FP32, row stride N, the scaled p-sum at p*.
 * ws / ws_bytes: workspace of at least pn_workspace_size() bytes. */
PN_API pn_status maxprod_pnorm(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                        const float* B, int64_t ldb, float* C, int64_t ldc, uint8_t* p_sel,
                        float* S_sel, const pn_opts* opts, void* ws, size_t ws_bytes,
                        void* stream);

/* Size of the scratch array behind maxprod_pnorm_static: 64 MiB of device
 * memory.  With CUDA's default lazy module loading it is reserved on a device
 * once maxprod_pnorm_static is first used there, until the process exits or
 * the device is reset. */
#define PN_STATIC_SCRATCH_BYTES ((size_t)64 << 20)

/* maxprod_pnorm for callers that cannot allocate device memory (no citation:
 * the paper has no counterpart; this is a library convenience).  Some callers
 * are handed only their inputs and outputs and may not call cudaMalloc -- for
 * instance a plugin whose host framework owns all device memory, or code on
 * a path where an allocation would stall.  This call takes no workspace: it
 * uses a fixed array of PN_STATIC_SCRATCH_BYTES inside the library and
 * allocates nothing.  Arguments and results are those of maxprod_pnorm.
 * Returns PN_EWORKSPACE when pn_workspace_size(M, N, K, opts) exceeds
 * PN_STATIC_SCRATCH_BYTES (with P = {1..64}, square products fit up to about
 * n = 3900 with BF16 operands and n = 2000 with PN_F32_EXACT).  A call made
 * outside a stream capture looks up the array's device address (so a device
 * reset, which moves the array, is picked up); a call made while `stream` is
 * capturing uses the address of an earlier call on that device, so make one
 * call on each device before capturing (PN_ECUDA otherwise).  Every call uses
 * the same array, so calls whose GPU work can overlap (other streams, other
 * host threads) race and must be serialised by the caller. */
PN_API pn_status maxprod_pnorm_static(int64_t M, int64_t N, int64_t K, const float* A,
                                      int64_t lda, const float* B, int64_t ldb, float* C,
                                      int64_t ldc, uint8_t* p_sel, float* S_sel,
                                      const pn_opts* opts, void* stream);

/* Exact semiring product on the CUDA cores (FP32, the plain comparison):
 * semiring 0: C_ij = max_k a_ik * b_kj  (Alg. 2; empty max = 0)
 * semiring 1: C_ij = min_k a_ik + b_kj  (Alg. 1; empty min = +inf)
 * Every product/sum is one correctly rounded FP32 operation and max/min are
 * exact, so the result is bit-identical to any sequential FP32 evaluation.
 * No workspace. */
PN_API pn_status maxprod_exact(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                        const float* B, int64_t ldb, float* C, int64_t ldc, int32_t semiring,
                        void* stream);

/* maxprod_exact with an explicit kernel variant, for comparing them:
 * variant 0 issues one FP32 multiply (add) and one max (min) per semiring
 * operation; variant 1 forms two consecutive products with one paired
 * mul.rn.f32x2 (add.rn.f32x2) and folds both with one 3-input max (min);
 * variant 2 (the default of maxprod_exact) issues variant 1's instructions in
 * a software-pipelined order.  All give identical results.  A variant outside
 * 0..2 returns PN_EINVAL. */
PN_API pn_status pn_maxprod_exact_variant(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                                   const float* B, int64_t ldb, float* C, int64_t ldc,
                                   int32_t semiring, int32_t variant, void* stream);

/* ------------------------------------------------------------------------
 * Max-convolution (Sec. 1): for each of `batch` independent problems,
 *   z_m = max_i x_i y_(m-i),  m = 0 .. nx + ny - 2,
 * over the indices where both factors exist.  Layout: x is batch x nx
 * (row stride ldx >= nx), y is batch x ny (ldy >= ny), z is batch x
 * (nx + ny - 1) (ldz >= nx + ny - 1), all row-major FP32 device arrays owned
 * by the caller; nx, ny >= 1 (else PN_EINVAL); batch 0 does nothing.
 * ------------------------------------------------------------------------ */

/* p-norm estimate with H = FFT convolution (Sec. 1; the scaled H' and the
 * threshold tau of Sec. 2.1): x' = x / max x, y' = y / max y (a zero vector
 * keeps scale 1); for each p of the family (largest first) the ring
 * convolution S^(p) = x'^p * y'^p by a double-precision FFT; index m takes
 * the largest p with S^(p)_m >= tau (none: the smallest p, flag 0x80 in
 * p_sel) and z_m = max x * max y * (S^(p*)_m)^(1/p*).  One CTA per problem
 * holds its transforms in shared memory: nx + ny - 1 <= 8192, else
 * PN_EUNSUPPORTED.  opts: n_p / p_log2, tau (<= 0: pn_maxconv_default_tau()),
 * dev_status (PN_EDOMAIN for an input outside [0, FLT_MAX]); compute,
 * scaling and tile_n are not used; a nonzero estimator or correction returns
 * PN_EUNSUPPORTED.  p_sel (optional; ldp >= nx + ny - 1) as in maxprod_pnorm.
 * No workspace.  The first call on a device also fills a table of FFT
 * twiddle factors (one kernel on `stream`): make it before capturing
 * `stream` into a graph. */
PN_API pn_status maxconv_pnorm(int64_t batch, int64_t nx, const float* x, int64_t ldx,
                               int64_t ny, const float* y, int64_t ldy, float* z, int64_t ldz,
                               uint8_t* p_sel, int64_t ldp, const pn_opts* opts, void* stream);

/* One long max-convolution (nx + ny - 1 up to 2^22), the same estimate with
 * a four-step FFT through a caller-provided workspace: three kernels per p
 * level (column FFTs with the powered inputs formed on the fly, row pairs with
 * the spectrum product, inverse columns with the selection) and a fourth that
 * ends the call when nothing is open or sums the few open terms of the
 * remaining levels directly.  x, y, z (nx + ny - 1 floats) and p_sel
 * (optional) are device arrays; ws is device memory of at least
 * pn_maxconv_long_workspace_size(nx, ny, p_sel != NULL) bytes, 256-byte
 * aligned, owned by the caller (PN_EWORKSPACE / PN_EALIGN otherwise); opts as
 * for maxconv_pnorm.  nx + ny - 1 > 2^22: PN_EUNSUPPORTED. */
PN_API pn_status maxconv_pnorm_long(int64_t nx, const float* x, int64_t ny, const float* y,
                                    float* z, uint8_t* p_sel, const pn_opts* opts, void* ws,
                                    size_t ws_bytes, void* stream);

/* Workspace bytes of maxconv_pnorm_long (0 if the sizes are out of range);
 * with_p_sel = 0 adds room for an internal p_sel. */
PN_API size_t pn_maxconv_long_workspace_size(int64_t nx, int64_t ny, int32_t with_p_sel);

/* Approximate top-k of the products x_i y_j (Alg. 9, E_(X' x Y'), with the
 * NormQueue), for `batch` independent pairs x, y of length n (row strides
 * ldx, ldy; 2n - 1 <= 8192, else PN_EUNSUPPORTED).  For every diagonal
 * m = i + j the p-sums of the max-scaled powered vectors come from FP64 FFT
 * convolutions (as in maxconv_pnorm, every p of opts' family; a family up to
 * p = 4096, p_log2 0..12, makes the pops sharp); then k times the diagonal
 * with the largest estimate is popped, psi^p is subtracted from each of its
 * p-sums and it is re-estimated, clamped to the value just popped (removing
 * a multiset's max cannot raise it); a diagonal is exhausted after as many
 * pops as it has terms.  vals[b * ldk + t] receives the t-th value (0 once
 * every diagonal is exhausted).  The same pops on y reversed give the
 * diagonals i + (n - 1 - j); pairing the two calls' pops of equal rank,
 * i = (m1 + m2 - n + 1) / 2 and j = m1 - i are written to idx_i / idx_j
 * (optional) when x_i y_j agrees with the value within 1 %, else -1.
 * ws: pn_topk_xy_workspace_size bytes, 256-byte aligned.  opts: family,
 * tau (<= 0: 1e-12), dev_status; estimator / correction must be 0. */
PN_API pn_status topk_xy(int64_t batch, int64_t n, const float* x, int64_t ldx, const float* y,
                         int64_t ldy, int64_t k, float* vals, int32_t* idx_i, int32_t* idx_j,
                         int64_t ldk, const pn_opts* opts, void* ws, size_t ws_bytes,
                         void* stream);

/* Workspace bytes of topk_xy (0 on invalid sizes or options). */
PN_API size_t pn_topk_xy_workspace_size(int64_t batch, int64_t n, int64_t k, const pn_opts* opts);

/* The paper's threshold for a double-precision FFT convolution of vectors
 * in [0, 1], 1e-12 (Sec. 2.1). */
PN_API double pn_maxconv_default_tau(void);

/* Exact max-convolution on the CUDA cores (the plain comparison): FP32
 * products, each correctly rounded, and an exact max, so the result equals
 * the FP64 max-convolution rounded to FP32.  nx + ny <= 2^30, else
 * PN_EUNSUPPORTED.  When nx > 8192 the partial maxima of several blocks of
 * terms meet in z by atomic max, after z is zeroed on `stream`. */
PN_API pn_status maxconv_exact(int64_t batch, int64_t nx, const float* x, int64_t ldx,
                               int64_t ny, const float* y, int64_t ldy, float* z, int64_t ldz,
                               void* stream);

/* Workspace bytes for apsp_pnorm (0 on invalid options). */
PN_API size_t pn_apsp_workspace_size(int64_t n, const pn_opts* opts);

/* All-pairs shortest distances estimated with p-norm squarings (Sec. 2.2):
 * X = exp(-W) with +inf -> 0, X_ii = 1 (diag_policy >= 1); then n_squarings
 * times X <- maxprod_pnorm(X, X) followed by the diag_policy rule (fused
 * into the product's epilogue); finally D = -log X (0 -> +inf).  W: n x n FP32, ldw >= n, entries >= 0 or +inf
 * (else PN_EDOMAIN); D: n x n FP32, ldd >= n.  n_squarings <= 0 selects
 * ceil(log2 n), which covers every path of up to n edges (Sec. 1, A^n by
 * powers of two). */
PN_API pn_status apsp_pnorm(int64_t n, const float* W, int64_t ldw, float* D, int64_t ldd,
                     int32_t n_squarings, const pn_opts* opts, void* ws, size_t ws_bytes,
                     void* stream);

/* Workspace bytes for maxprod_pnorm_backward (0 on invalid options). */
PN_API size_t pn_backward_workspace_size(int64_t M, int64_t N, int64_t K, const pn_opts* opts);

/* Adjoint of maxprod_pnorm with p* held fixed per entry (the p-norm rings are
 * differentiable, Sec. 4).  With C_ij = (sum_k (a_ik b_kj)^p)^(1/p):
 *   W_ij  = dC_ij * C_ij / S_sel_ij                   (0 where S_sel == 0)
 *   dA_ik = (a'_ik^(p-1) / r_i) * sum_j W_ij b'_kj^p   summed over p in P,
 *   dB_kj = (b'_kj^(p-1) / c_j) * sum_i W_ij a'_ik^p   with W masked to p*_ij == p,
 * where a' = a / r_i, b' = b / c_j are the forward's scaled operands
 * (recomputed, not stored).  A: M x K, B: K x N, C, S_sel, p_sel, dC: M x N,
 * dA: M x K, dB: K x N, all contiguous row-major (leading dimension = number
 * of columns); C, S_sel and p_sel are the outputs of maxprod_pnorm with the
 * same options.  dA and dB are overwritten.  opts->tile_m / tile_n select the
 * gradient GEMMs' tiles as described at tile_m. */
PN_API pn_status maxprod_pnorm_backward(int64_t M, int64_t N, int64_t K, const float* A,
                                 const float* B, const float* C, const float* S_sel,
                                 const uint8_t* p_sel, const float* dC, float* dA, float* dB,
                                 const pn_opts* opts, void* ws, size_t ws_bytes, void* stream);

/* Grouped launch: many independent products C_g = A_g (x,max) B_g in ONE
 * persistent launch over every problem, p level and output tile (Sec. 4: the
 * p rings and the problems parallelise coarsely).  One CTA per SM (a
 * cooperative launch) builds each operand block's maxima, scales and powered
 * images, publishes it with a ready flag, runs the tensor-core tiles of the
 * level as their blocks become ready, and meets the other CTAs at a bounded
 * barrier before the next lower p; tiles with unresolved entries carry over
 * through device work lists.  With scaling 1 (one global scale per operand)
 * the call runs one launch sequence per p level instead.  Two steps, so that
 * the run step never copies host memory and can be captured in a CUDA graph:
 *  1. pn_grouped_build_table() (host only, no CUDA calls) writes a table
 *     describing `count` problems (sizes MNK[3g..3g+2] = M_g, N_g, K_g, and
 *     DEVICE pointers A[g], B[g], C[g] of contiguous row-major FP32 matrices;
 *     K_g >= 1 unless M_g or N_g is 0) into host memory `host_table` of
 *     pn_grouped_table_bytes(count, MNK, opts) bytes (0 on invalid
 *     arguments), and returns the workspace size in *ws_bytes.  The table
 *     holds layouts for 128- and 256-wide tiles and, per layout, lookup
 *     tables from every tile / operand tile / max-pass unit to its problem.
 *  2. The caller copies the table bytes unchanged to device memory
 *     `dev_table` (16-byte aligned) and calls maxprod_pnorm_grouped() with
 *     both copies and the same options; each C_g receives the estimate
 *     maxprod_pnorm computes (no p_sel / S_sel).  opts->tile_n selects the
 *     layout; 0 uses the autotuned choice for this table, else a size rule. */
PN_API size_t pn_grouped_table_bytes(int32_t count, const int64_t* MNK, const pn_opts* opts);
PN_API pn_status pn_grouped_build_table(int32_t count, const int64_t* MNK, const float* const* A,
                                        const float* const* B, float* const* C,
                                        const pn_opts* opts, void* host_table,
                                        size_t table_bytes, size_t* ws_bytes);
PN_API pn_status maxprod_pnorm_grouped(const void* host_table, const void* dev_table,
                                       const pn_opts* opts, void* ws, size_t ws_bytes,
                                       void* stream);

/* Autotuner of the output tile shape (no counterpart in the paper).  Times
 * every candidate the options leave open -- for a product one CTA per
 * 128 x 128 or 128 x 256 tile (3xTF32: 128 x 128 only) and a CTA pair per
 * 256 x 256 or 256 x 128 tile; for a group the widths 128 and 256 -- on the caller's
 * buffers with CUDA events (three timed runs each after a warm-up) and
 * remembers the fastest for this device and shape class (ceil(log2) of M, N,
 * K for a product; the table's sizes for a group).  Later calls with
 * tile_n = 0 and tile_m = 0 use it.  Synchronises the stream; not for use
 * inside a stream capture.  The choice is returned in *chosen_tile_n
 * (nullable): the width, or 256 + the width for a CTA pair (512 or 384).
 * The buffers are overwritten
 * exactly as by the product itself. */
PN_API pn_status pn_autotune(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                             const float* B, int64_t ldb, float* C, int64_t ldc,
                             const pn_opts* opts, void* ws, size_t ws_bytes, void* stream,
                             int32_t* chosen_tile_n);
PN_API pn_status pn_grouped_autotune(const void* host_table, const void* dev_table,
                                     const pn_opts* opts, void* ws, size_t ws_bytes,
                                     void* stream, int32_t* chosen_tile_n);

#ifdef __cplusplus
}
#endif

#endif /* PNORM_H */
