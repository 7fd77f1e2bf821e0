/*
 * Oracle for the p-norm estimate of the (x,max) semiring matrix product.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, obviously-correct
 * CPU implementation (FP64 unless stated) of what the GPU library computes.
 * It shares no code, header, table or helper with the CUDA path.  Only the
 * tests, the smoke check and the CPU-baseline leg of the benchmark may load it.
 *
 * Paper: O. Serang, "Fast Computation on Semirings Isomorphic to (x, max) on
 * R+" (arXiv 1511.05690).  Each function names the passage it follows.
 *
 * Readings of the paper that this file adopts (where the paper is silent or
 * garbled) are:
 *   - scaling (Sec. 2.1, definition of H'): operands are divided by a power of
 *     two per row of A and per column of B, r_i = 2^ceil(log2 max_k a_ik),
 *     c_j = 2^ceil(log2 max_k b_kj); the scale is undone after the 1/p root.
 *     A zero row/column gets scale 1.  mode 1 = one global scale per operand
 *     (the paper's literal H'), mode 0 = no scaling.
 *   - estimator (Sec. 2.1, estimateMaxFromNormPowerSequence; Alg. 5): the
 *     plain form, (S^(p*))^(1/p*) at the largest p in P with S^(p) >= tau.
 *     If no p passes, p* is the smallest p in P and the result carries an
 *     "unstable" flag (0x80 in p_sel).
 *   - projection estimator r = 1 (Sec. 2.1, multiset projection; the
 *     printed r = 1 formula is garbled): the two evenly spaced norms are
 *     taken at p'= p* / 2 and 2p' = p*, both stable; the estimate is the root
 *     of the projection polynomial, (S^(2p') / S^(p'))^(1/p').  Entries
 *     whose p* / 2 is not in P (including p* = min P and unstable entries)
 *     keep the plain estimate.
 *   - projection estimator r = 2 (Sec. 2.1 with r = 2, the estimator of the
 *     paper's experiments): the four evenly spaced sums are taken at
 *     p' = p* / 4, 2p', 3p', 4p' = p* (the 3p' sums form the extra family
 *     1.5 * 2^k); the 2 x 3 Hankel matrix's null vector is the cross product
 *     of its rows and the estimate the larger root of its quadratic, to the
 *     power 1/p'.  Entries whose p* / 2 and p* / 4 are not the two p below
 *     p* in P keep the plain estimate; sums that do not resolve a second
 *     value (s1 s3 - s2^2 <= 1e-6 s2^2: the oracle's sums are exact up to
 *     FP64 rounding, so the margin only guards the rounding of that
 *     difference, nothing of any operand format) keep the r = 1 value, and
 *     the root is clamped between the r = 1 value and the plain norm (the
 *     interval that holds the larger Gauss node).
 *   - corrections (Sec. 2.1 bound remark; Discussion), in the scaled space
 *     where the exact value lies in (0, 1]: correction 1 divides the estimate
 *     by K^(1/p*), the upper end of its envelope; correction 2 fits
 *     exact = a_q * est + b_q by least squares on sample entries whose exact
 *     value is known, one (a_q, b_q) per p* class q, and applies it to every
 *     entry of that class.  Degenerate classes: one sample, or a spread of the
 *     estimates below 1e-12 of their second moment, fit the ratio
 *     (b_q = 0); no sample leaves the class unchanged.
 *   - APSP (Sec. 2.2, Eq. for A^n): the diagonal is reset to 1 (distance 0)
 *     after each squaring when diag_policy >= 1; with diag_policy == 2 every
 *     entry is also clamped to <= 1 (distance >= 0).
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC oracle.c
 * (-ffp-contract=off keeps every product and sum separately rounded.)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* ---------------------------------------------------------------------- */
/* Alg. 2 (F'_APSP): naive matrix multiplication on the semiring (x, max). */
/* C[i][j] = max_k A[i][k] * B[k][j].  FP64.  Empty max (K == 0) = 0, the  */
/* zero of the semiring on R+.                                             */
void orc_maxprod_f64(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda,
                     const double* B, int64_t ldb, double* C, int64_t ldc) {
  int64_t i;
#pragma omp parallel for schedule(dynamic, 1)
  for (i = 0; i < M; ++i) {
    for (int64_t j = 0; j < N; ++j) {
      double r = 0.0;
      for (int64_t k = 0; k < K; ++k) {
        double t = A[i * lda + k] * B[k * ldb + j];
        if (t > r) r = t;
      }
      C[i * ldc + j] = r;
    }
  }
}

/* Same as above with FP32 inputs: every product is rounded to float (one */
/* correctly rounded multiply), the max is exact.  This is the bit-exact   */
/* reference for the GPU's exact CUDA-core kernel.                         */
void orc_maxprod_f32(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                     const float* B, int64_t ldb, float* C, int64_t ldc) {
  int64_t i;
#pragma omp parallel for schedule(dynamic, 1)
  for (i = 0; i < M; ++i) {
    for (int64_t j = 0; j < N; ++j) {
      float r = 0.0f;
      for (int64_t k = 0; k < K; ++k) {
        volatile float t = A[i * lda + k] * B[k * ldb + j];
        if (t > r) r = t;
      }
      C[i * ldc + j] = r;
    }
  }
}

/* Alg. 1 (F_APSP): naive matrix multiplication on the semiring (+, min).  */
/* Empty min (K == 0) = +inf.                                              */
void orc_minplus_f64(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda,
                     const double* B, int64_t ldb, double* C, int64_t ldc) {
  int64_t i;
#pragma omp parallel for schedule(dynamic, 1)
  for (i = 0; i < M; ++i) {
    for (int64_t j = 0; j < N; ++j) {
      double r = INFINITY;
      for (int64_t k = 0; k < K; ++k) {
        double t = A[i * lda + k] + B[k * ldb + j];
        if (t < r) r = t;
      }
      C[i * ldc + j] = r;
    }
  }
}

void orc_minplus_f32(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                     const float* B, int64_t ldb, float* C, int64_t ldc) {
  int64_t i;
#pragma omp parallel for schedule(dynamic, 1)
  for (i = 0; i < M; ++i) {
    for (int64_t j = 0; j < N; ++j) {
      float r = INFINITY;
      for (int64_t k = 0; k < K; ++k) {
        volatile float t = A[i * lda + k] + B[k * ldb + j];
        if (t < r) r = t;
      }
      C[i * ldc + j] = r;
    }
  }
}

/* Alg. 3 (G_APSP): naive matrix multiplication on the ring (x, +).  FP64. */
void orc_ringprod_f64(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda,
                      const double* B, int64_t ldb, double* C, int64_t ldc) {
  int64_t i;
#pragma omp parallel for schedule(dynamic, 1)
  for (i = 0; i < M; ++i) {
    for (int64_t j = 0; j < N; ++j) {
      double s = 0.0;
      for (int64_t k = 0; k < K; ++k) s += A[i * lda + k] * B[k * ldb + j];
      C[i * ldc + j] = s;
    }
  }
}

/* ---------------------------------------------------------------------- */
/* Default stability threshold tau (Sec. 2.1: tau depends on the numeric    */
/* stability of H; the paper gives 1e-12 only for FFT convolution).  For a  */
/* GEMM of nonnegative terms the only loss is operand underflow.  With the  */
/* powered operands stored as q = x^p * 2^s in a format whose smallest      */
/* normal is mu and which keeps m mantissa bits, operands below mu may be   */
/* flushed, dropping at most K * mu * 2^-s from S.  Requiring that loss to  */
/* stay below 2^-m * S gives tau = K * mu * 2^(m - s).                      */
/*   compute 0 (FP32 via 3xTF32 split): mu 2^-126, m 21, s 0               */
/*   compute 1 (TF32):                  mu 2^-126, m 10, s 0               */
/*   compute 2 (BF16):                  mu 2^-126, m 7,  s 0               */
/*   compute 3 (FP16):                  mu 2^-14,  m 10, s 15              */
/*   compute 4 (FP8 E4M3):              mu 2^-6,   m 3,  s 8               */
double orc_default_tau(int64_t K, int compute) {
  int e_mu, m, s;
  switch (compute) {
    case 0: e_mu = -126; m = 21; s = 0; break;
    case 1: e_mu = -126; m = 10; s = 0; break;
    case 2: e_mu = -126; m = 7; s = 0; break;
    case 3: e_mu = -14; m = 10; s = 15; break;
    case 4: e_mu = -6; m = 3; s = 8; break;
    default: return -1.0;
  }
  return (double)(K > 0 ? K : 1) * ldexp(1.0, e_mu + m - s);
}

/* Scaling (Sec. 2.1, H'): the smallest power of two >= m, for m > 0.      */
/* m = f * 2^e with f in [0.5, 1): if f == 0.5, m = 2^(e-1) exactly.        */
static double pow2_ceil(double m) {
  if (!(m > 0.0)) return 1.0;
  int e = 0;
  double f = frexp(m, &e);
  return ldexp(1.0, f == 0.5 ? e - 1 : e);
}

/* Row scales of A (M x K): mode 2 per row, mode 1 one global, mode 0 none. */
void orc_row_scales(int64_t M, int64_t K, const double* A, int64_t lda, int mode, double* r) {
  if (mode == 0) {
    for (int64_t i = 0; i < M; ++i) r[i] = 1.0;
    return;
  }
  double gmax = 0.0;
  for (int64_t i = 0; i < M; ++i) {
    double m = 0.0;
    for (int64_t k = 0; k < K; ++k)
      if (A[i * lda + k] > m) m = A[i * lda + k];
    r[i] = pow2_ceil(m);
    if (m > gmax) gmax = m;
  }
  if (mode == 1) {
    double g = pow2_ceil(gmax);
    for (int64_t i = 0; i < M; ++i) r[i] = g;
  }
}

/* Column scales of B (K x N). */
void orc_col_scales(int64_t K, int64_t N, const double* B, int64_t ldb, int mode, double* c) {
  if (mode == 0) {
    for (int64_t j = 0; j < N; ++j) c[j] = 1.0;
    return;
  }
  double gmax = 0.0;
  for (int64_t j = 0; j < N; ++j) {
    double m = 0.0;
    for (int64_t k = 0; k < K; ++k)
      if (B[k * ldb + j] > m) m = B[k * ldb + j];
    c[j] = pow2_ceil(m);
    if (m > gmax) gmax = m;
  }
  if (mode == 1) {
    double g = pow2_ceil(gmax);
    for (int64_t j = 0; j < N; ++j) c[j] = g;
  }
}

/* ---------------------------------------------------------------------- */
/* Alg. 5 (E_APSP), first loop: for each p in P, the ring product of the   */
/* scaled, powered operands (Alg. 3 on A'^p and B'^p), FP64, term by term: */
/*   S[q][i][j] = sum_k pow(a_ik / r_i * b_kj / c_j, p_q),  p_q = 2^p_log2[q]. */
/* pow() per term is used on purpose (no squaring chain).                   */
void orc_psums(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda, const double* B,
               int64_t ldb, const double* r, const double* c, int n_p, const int* p_log2,
               double* S) {
  int64_t i;
#pragma omp parallel for schedule(dynamic, 1)
  for (i = 0; i < M; ++i) {
    for (int64_t j = 0; j < N; ++j) {
      for (int q = 0; q < n_p; ++q) {
        double p = ldexp(1.0, p_log2[q]);
        double s = 0.0;
        for (int64_t k = 0; k < K; ++k) {
          double u = (A[i * lda + k] / r[i]) * (B[k * ldb + j] / c[j]);
          s += pow(u, p);
        }
        S[((int64_t)q * M + i) * N + j] = s;
      }
    }
  }
}

/* The same sums at arbitrary real exponents pw[q] (the 3p/4 family of the */
/* r = 2 projection): S[q][i][j] = sum_k pow(a_ik / r_i * b_kj / c_j, pw[q]). */
void orc_psums_real(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda,
                    const double* B, int64_t ldb, const double* r, const double* c, int n_p,
                    const double* pw, double* S) {
  int64_t i;
#pragma omp parallel for schedule(dynamic, 1)
  for (i = 0; i < M; ++i) {
    for (int64_t j = 0; j < N; ++j) {
      for (int q = 0; q < n_p; ++q) {
        double s = 0.0;
        for (int64_t k = 0; k < K; ++k) {
          double u = (A[i * lda + k] / r[i]) * (B[k * ldb + j] / c[j]);
          s += pow(u, pw[q]);
        }
        S[((int64_t)q * M + i) * N + j] = s;
      }
    }
  }
}

/* Sec. 2.1, multiset projection with r = 1.  Given the two evenly spaced   */
/* power sums s1 = ||u||_{p'}^{p'} and s2 = ||u||_{2p'}^{2p'}, the 1 x 2     */
/* Hankel matrix [s1 s2] has the null vector gamma = (s2, -s1); the         */
/* projection polynomial gamma_0 + gamma_1 a has the single root a = -g0/g1 */
/* and the projected value is alpha = a^(1/p').                              */
static double project_r1(double s1, double s2, double p_prime) {
  double g0 = s2, g1 = -s1;
  if (g1 == 0.0) return 0.0;
  double a = -g0 / g1;
  return a > 0.0 ? pow(a, 1.0 / p_prime) : 0.0;
}

/* Sec. 2.1, multiset projection with r = 2.  Given the four evenly spaced  */
/* power sums s_m = ||u||_{m p'}^{m p'}, m = 1..4, the 2 x 3 Hankel matrix   */
/* [s1 s2 s3; s2 s3 s4] has the null vector gamma = (s2 s4 - s3^2,          */
/* s2 s3 - s1 s4, s1 s3 - s2^2), the cross product of its two rows; the     */
/* roots a of gamma_0 + gamma_1 a + gamma_2 a^2 are the two projected        */
/* values alpha^p' and the estimate is the larger alpha = a^(1/p').          */
/* The s_m are the moments of the measure with mass w x at each value x,   */
/* so the roots are its 2-point Gauss nodes and the larger one lies between */
/* the 1-point node s2 / s1 (the r = 1 value) and max x <= s4^(1/4) (the    */
/* plain norm).  Readings: when gamma_2 <= R2_ETA s2^2 the sums do not      */
/* resolve a second value (s1 s3 >= s2^2 always; R2_ETA = 1e-6 is a margin   */
/* over the FP64 rounding of exact sums) and the r = 1 value is returned;   */
/* a negative discriminant (rounding) counts as zero; a root that is not    */
/* positive gives the r = 1 value; the root is clamped to [s2 / s1, s4^(1/4)] */
/* (never binding for exact sums; with rounded sums it keeps the estimate   */
/* between the r = 1 value and the plain norm).                              */
#define R2_ETA 1e-6
double orc_project_r2(double s1, double s2, double s3, double s4, double p_prime) {
  double g0 = s2 * s4 - s3 * s3;
  double g1 = s2 * s3 - s1 * s4;
  double g2 = s1 * s3 - s2 * s2;
  if (!(g2 > R2_ETA * s2 * s2)) return project_r1(s1, s2, p_prime);
  double disc = g1 * g1 - 4.0 * g0 * g2;
  if (disc < 0.0) disc = 0.0;
  double a = (-g1 + sqrt(disc)) / (2.0 * g2);
  if (!(a > 0.0)) return project_r1(s1, s2, p_prime);
  double lo = s2 / s1, hi = sqrt(sqrt(s4));
  if (a < lo) a = lo;
  if (a > hi) a = hi;
  return pow(a, 1.0 / p_prime);
}

/* orc_project_r2 over n quadruples (s1[e], s2[e], s3[e], s4[e]).            */
void orc_project_r2_batch(int64_t n, const double* s1, const double* s2, const double* s3,
                          const double* s4, double p_prime, double* out) {
  for (int64_t e = 0; e < n; ++e)
    out[e] = orc_project_r2(s1[e], s2[e], s3[e], s4[e], p_prime);
}

/* Alg. 5, second loop, with estimateMaxFromNormPowerSequence:              */
/* p* = largest p in P with S^(p) >= tau (the stable set is a prefix of P   */
/* because S^(p) is non-increasing in p once every term is <= 1).           */
/* estimator 0 (plain): Chat = r_i * c_j * (S^(p*))^(1/p*).                  */
/* estimator 1 (projection r = 1): Chat = r_i * c_j *                      */
/*   project_r1(S^(p* / 2), S^(p*), p* / 2)                                  */
/* when p* / 2 is in P and p* is stable, else the plain form.                */
/* estimator 2 (projection r = 2): Chat = r_i * c_j *                      */
/*   orc_project_r2(S^(p* / 4), S^(p* / 2), S^(3 p* / 4), S^(p*), p* / 4)     */
/* when p* / 2 and p* / 4 are the two p below p* in P and p* is stable,     */
/* else the plain form; S34[q] holds the sums at 3 p_q / 4.                  */
/* p_sel = log2(p*) | 0x80 if unstable; S_sel = S^(p*).                      */
void orc_estimate_ex2(int64_t M, int64_t N, int n_p, const int* p_log2, const double* S,
                      const double* S34, const double* r, const double* c, double tau,
                      int estimator, double* Chat, uint8_t* psel, double* Ssel) {
  int64_t i;
#pragma omp parallel for schedule(static)
  for (i = 0; i < M; ++i) {
    for (int64_t j = 0; j < N; ++j) {
      int q_sel = -1;
      for (int q = n_p - 1; q >= 0; --q) {
        if (S[((int64_t)q * M + i) * N + j] >= tau) {
          q_sel = q;
          break;
        }
      }
      int unstable = 0;
      if (q_sel < 0) {
        q_sel = 0;
        unstable = 1;
      }
      double s = S[((int64_t)q_sel * M + i) * N + j];
      double p = ldexp(1.0, p_log2[q_sel]);
      double est = s > 0.0 ? pow(s, 1.0 / p) : 0.0;
      if (estimator == 1 && !unstable && q_sel > 0 && p_log2[q_sel - 1] == p_log2[q_sel] - 1) {
        double s_half = S[((int64_t)(q_sel - 1) * M + i) * N + j];
        est = project_r1(s_half, s, 0.5 * p);
      }
      if (estimator == 2 && S34 && !unstable && q_sel > 1 &&
          p_log2[q_sel - 1] == p_log2[q_sel] - 1 && p_log2[q_sel - 2] == p_log2[q_sel] - 2) {
        double s2 = S[((int64_t)(q_sel - 1) * M + i) * N + j];
        double s1 = S[((int64_t)(q_sel - 2) * M + i) * N + j];
        double s3 = S34[((int64_t)q_sel * M + i) * N + j];
        est = orc_project_r2(s1, s2, s3, s, 0.25 * p);
      }
      if (Chat) Chat[i * N + j] = r[i] * c[j] * est;
      if (psel) psel[i * N + j] = (uint8_t)(p_log2[q_sel] | (unstable ? 0x80 : 0));
      if (Ssel) Ssel[i * N + j] = s;
    }
  }
}

void orc_estimate_ex(int64_t M, int64_t N, int n_p, const int* p_log2, const double* S,
                     const double* r, const double* c, double tau, int estimator, double* Chat,
                     uint8_t* psel, double* Ssel) {
  orc_estimate_ex2(M, N, n_p, p_log2, S, NULL, r, c, tau, estimator, Chat, psel, Ssel);
}

/* Discussion (affine model from a few exact sub-solutions): least squares  */
/* exact_s = a_q * est_s + b_q over the samples s of class q = cls[s], from */
/* the plain sums n, sum x, sum y, sum x^2, sum x y; coef[2q] = a_q,        */
/* coef[2q + 1] = b_q.                                                       */
void orc_affine_fit(int64_t n_s, const double* est, const double* exact, const int* cls, int n_cls,
                    double* coef) {
  for (int q = 0; q < n_cls; ++q) {
    double n = 0.0, sx = 0.0, sy = 0.0, sxx = 0.0, sxy = 0.0;
    for (int64_t s = 0; s < n_s; ++s) {
      if (cls[s] != q) continue;
      n += 1.0;
      sx += est[s];
      sy += exact[s];
      sxx += est[s] * est[s];
      sxy += est[s] * exact[s];
    }
    double a = 1.0, b = 0.0;
    if (n >= 2.0 && sxx - sx * sx / n > 1e-12 * sxx) {
      a = (sxy - sx * sy / n) / (sxx - sx * sx / n);
      b = (sy - a * sx) / n;
    } else if (n >= 1.0 && sx > 0.0) {
      a = sy / sx;
    }
    coef[2 * q] = a;
    coef[2 * q + 1] = b;
  }
}

/* Applies a correction to Chat in place, per entry, in the scaled space:   */
/* est = Chat / (r_i c_j); correction 1: est / K^(1/p*); correction 2:      */
/* a_q est + b_q with q the index of p* in P.                                */
void orc_apply_correction(int64_t M, int64_t N, int64_t K, int n_p, const int* p_log2,
                          int correction, const double* coef, const uint8_t* psel,
                          const double* r, const double* c, double* Chat) {
  int64_t i;
#pragma omp parallel for schedule(static)
  for (i = 0; i < M; ++i) {
    for (int64_t j = 0; j < N; ++j) {
      int lp = psel[i * N + j] & 0x7F, q = 0;
      for (int t = 0; t < n_p; ++t)
        if (p_log2[t] == lp) q = t;
      double rc = r[i] * c[j];
      if (rc <= 0.0) continue;
      double est = Chat[i * N + j] / rc;
      if (correction == 1) est = est / pow((double)(K > 0 ? K : 1), 1.0 / ldexp(1.0, lp));
      if (correction == 2) est = coef[2 * q] * est + coef[2 * q + 1];
      Chat[i * N + j] = rc * est;
    }
  }
}

/* The plain estimator (estimator 0 of orc_estimate_ex). */
void orc_estimate(int64_t M, int64_t N, int n_p, const int* p_log2, const double* S,
                  const double* r, const double* c, double tau, double* Chat, uint8_t* psel,
                  double* Ssel) {
  orc_estimate_ex(M, N, n_p, p_log2, S, r, c, tau, 0, Chat, psel, Ssel);
}

/* Scales + p-sums + estimate.  S (n_p*M*N doubles) may be NULL, in which   */
/* case a temporary is used.                                                 */
int orc_pnorm_ex2(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda,
                  const double* B, int64_t ldb, int n_p, const int* p_log2, double tau,
                  int scaling, int estimator, double* Chat, uint8_t* psel,
                  double* Ssel, double* S_all, double* r_out, double* c_out) {
  double* r = (double*)malloc(sizeof(double) * (M > 0 ? M : 1));
  double* c = (double*)malloc(sizeof(double) * (N > 0 ? N : 1));
  double* S = S_all ? S_all : (double*)malloc(sizeof(double) * (size_t)n_p * (M * N > 0 ? M * N : 1));
  if (!r || !c || !S) return -1;
  orc_row_scales(M, K, A, lda, scaling, r);
  orc_col_scales(K, N, B, ldb, scaling, c);
  orc_psums(M, N, K, A, lda, B, ldb, r, c, n_p, p_log2, S);
  double* S34 = NULL;
  if (estimator == 2) {
    double* pw = (double*)malloc(sizeof(double) * (n_p > 0 ? n_p : 1));
    S34 = (double*)malloc(sizeof(double) * (size_t)n_p * (M * N > 0 ? M * N : 1));
    if (!pw || !S34) return -1;
    for (int q = 0; q < n_p; ++q) pw[q] = 0.75 * ldexp(1.0, p_log2[q]);
    orc_psums_real(M, N, K, A, lda, B, ldb, r, c, n_p, pw, S34);
    free(pw);
  }
  orc_estimate_ex2(M, N, n_p, p_log2, S, S34, r, c, tau, estimator, Chat, psel, Ssel);
  free(S34);
  if (r_out) memcpy(r_out, r, sizeof(double) * M);
  if (c_out) memcpy(c_out, c, sizeof(double) * N);
  free(r);
  free(c);
  if (!S_all) free(S);
  return 0;
}

int orc_pnorm_ex(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda, const double* B,
                 int64_t ldb, int n_p, const int* p_log2, double tau, int scaling, int estimator,
                 double* Chat, uint8_t* psel, double* Ssel, double* S_all, double* r_out,
                 double* c_out) {
  return orc_pnorm_ex2(M, N, K, A, lda, B, ldb, n_p, p_log2, tau, scaling, estimator, Chat,
                       psel, Ssel, S_all, r_out, c_out);
}

int orc_pnorm(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda, const double* B,
              int64_t ldb, int n_p, const int* p_log2, double tau, int scaling, double* Chat,
              uint8_t* psel, double* Ssel, double* S_all, double* r_out, double* c_out) {
  return orc_pnorm_ex(M, N, K, A, lda, B, ldb, n_p, p_log2, tau, scaling, 0, Chat, psel, Ssel,
                      S_all, r_out, c_out);
}

/* Selected entries only: for n_e pairs (ii[e], jj[e]) of the product A*B, */
/* the exact max (Alg. 2) and every p-sum (Alg. 5 first loop), given the   */
/* scales r (length M) and c (length N).  Cost O(n_e * K * n_p).            */
void orc_entries(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda, const double* B,
                 int64_t ldb, const double* r, const double* c, int n_p, const int* p_log2,
                 int64_t n_e, const int64_t* ii, const int64_t* jj, double* exact, double* S) {
  (void)M;
  (void)N;
  int64_t e;
#pragma omp parallel for schedule(dynamic, 1)
  for (e = 0; e < n_e; ++e) {
    int64_t i = ii[e], j = jj[e];
    double mx = 0.0;
    for (int64_t k = 0; k < K; ++k) {
      double t = A[i * lda + k] * B[k * ldb + j];
      if (t > mx) mx = t;
    }
    if (exact) exact[e] = mx;
    if (S) {
      for (int q = 0; q < n_p; ++q) {
        double p = ldexp(1.0, p_log2[q]);
        double s = 0.0;
        for (int64_t k = 0; k < K; ++k) {
          double u = (A[i * lda + k] / r[i]) * (B[k * ldb + j] / c[j]);
          s += pow(u, p);
        }
        S[e * n_p + q] = s;
      }
    }
  }
}

/* The p-sums at the entries (ii[e], jj[e]) for real exponents pw[q]:      */
/* S[e * n_p + q] = sum_k pow(a_ik / r_i * b_kj / c_j, pw[q]).               */
void orc_entries_real(int64_t K, const double* A, int64_t lda, const double* B, int64_t ldb,
                      const double* r, const double* c, int n_p, const double* pw, int64_t n_e,
                      const int64_t* ii, const int64_t* jj, double* S) {
  int64_t e;
#pragma omp parallel for schedule(dynamic, 1)
  for (e = 0; e < n_e; ++e) {
    int64_t i = ii[e], j = jj[e];
    for (int q = 0; q < n_p; ++q) {
      double s = 0.0;
      for (int64_t k = 0; k < K; ++k) {
        double u = (A[i * lda + k] / r[i]) * (B[k * ldb + j] / c[j]);
        s += pow(u, pw[q]);
      }
      S[e * n_p + q] = s;
    }
  }
}

/* ---------------------------------------------------------------------- */
/* Floyd-Warshall (Sec. 3.1 comparison): exact APSP in O(n^3), in place.    */
/* D holds the weights on entry (+inf = no edge) and distances on return.  */
void orc_floyd_warshall(int64_t n, double* D, int64_t ldd) {
  for (int64_t k = 0; k < n; ++k) {
    const double* Dk = D + k * ldd;
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n; ++i) {
      double dik = D[i * ldd + k];
      if (dik == INFINITY) continue;
      double* Di = D + i * ldd;
      for (int64_t j = 0; j < n; ++j) {
        double t = dik + Dk[j];
        if (t < Di[j]) Di[j] = t;
      }
    }
  }
}

/* p-norm APSP (Sec. 2.2): X = exp(-W) (+inf -> 0), then n_sq times         */
/* X <- E(X, X) (the p-norm product above), and D = -log X.                 */
/* n_sq <= 0 means ceil(log2 n).  After the transform and after each         */
/* squaring, diag_policy >= 1 sets X_ii = 1 (distance 0); diag_policy == 2   */
/* also clamps every entry to X <= 1 (distance >= 0): with nonnegative       */
/* weights both are exact facts, and since E only overestimates X the        */
/* clamped estimate still lies between the exact X and the unclamped one.   */
int orc_apsp_pnorm(int64_t n, const double* W, int64_t ldw, int n_sq, int n_p, const int* p_log2,
                   double tau, int scaling, int diag_policy, double* D, int64_t ldd,
                   uint8_t* psel_last) {
  if (n <= 0) return 0;
  if (n_sq <= 0) {
    n_sq = 0;
    while (((int64_t)1 << n_sq) < n) ++n_sq;
  }
  double* X = (double*)malloc(sizeof(double) * n * n);
  double* Y = (double*)malloc(sizeof(double) * n * n);
  if (!X || !Y) return -1;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) {
      double w = W[i * ldw + j];
      X[i * n + j] = (w == INFINITY) ? 0.0 : exp(-w);
    }
  if (diag_policy >= 1)
    for (int64_t i = 0; i < n; ++i) X[i * n + i] = 1.0;
  for (int t = 0; t < n_sq; ++t) {
    int rc = orc_pnorm(n, n, n, X, n, X, n, n_p, p_log2, tau, scaling, Y,
                       (t == n_sq - 1) ? psel_last : NULL, NULL, NULL, NULL, NULL);
    if (rc) return rc;
    if (diag_policy == 2)
      for (int64_t e = 0; e < n * n; ++e)
        if (Y[e] > 1.0) Y[e] = 1.0;
    if (diag_policy >= 1)
      for (int64_t i = 0; i < n; ++i) Y[i * n + i] = 1.0;
    double* tmp = X;
    X = Y;
    Y = tmp;
  }
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) {
      double x = X[i * n + j];
      D[i * ldd + j] = (x > 0.0) ? -log(x) : INFINITY;
    }
  free(X);
  free(Y);
  return 0;
}

/* ---------------------------------------------------------------------- */
/* Gradient of the p-norm product with the selected p held fixed per entry */
/* (the derivative of (sum_k (a_ik b_kj)^p)^(1/p), the estimator of Alg. 5  */
/* at p = p_ij; the Discussion notes the p-norm rings are differentiable).  */
/*   dC_ij/da_ik = C_ij^(1-p) a_ik^(p-1) b_kj^p                            */
/*   dA_ik = sum_j G_ij dC_ij/da_ik,  dB_kj = sum_i G_ij dC_ij/db_kj.       */
/* Written in the scaled variables to stay in range:                       */
/*   C_ij^(1-p) a_ik^(p-1) b_kj^p = (C_ij/S_ij) (a'_ik^(p-1)/r_i) b'_kj^p,  */
/* with S_ij the scaled p-sum at p_ij.  Entries with S_ij == 0 contribute 0.*/
/* plog[i*N+j] holds log2(p_ij) (flag bits already masked off).             */
void orc_pnorm_grad(int64_t M, int64_t N, int64_t K, const double* A, const double* B,
                    const double* r, const double* c, const uint8_t* plog, const double* G,
                    double* dA, double* dB) {
  double* Wt = (double*)malloc(sizeof(double) * (M * N > 0 ? M * N : 1));
  /* W_ij = G_ij * C_ij / S_ij computed from the definition. */
  int64_t i;
#pragma omp parallel for schedule(dynamic, 1)
  for (i = 0; i < M; ++i) {
    for (int64_t j = 0; j < N; ++j) {
      double p = ldexp(1.0, plog[i * N + j]);
      double s = 0.0;
      for (int64_t k = 0; k < K; ++k) s += pow((A[i * K + k] / r[i]) * (B[k * N + j] / c[j]), p);
      double C = s > 0.0 ? r[i] * c[j] * pow(s, 1.0 / p) : 0.0;
      Wt[i * N + j] = s > 0.0 ? G[i * N + j] * C / s : 0.0;
    }
  }
#pragma omp parallel for schedule(dynamic, 1)
  for (i = 0; i < M; ++i) {
    for (int64_t k = 0; k < K; ++k) {
      double acc = 0.0;
      double ap = A[i * K + k] / r[i];
      for (int64_t j = 0; j < N; ++j) {
        double p = ldexp(1.0, plog[i * N + j]);
        double bp = B[k * N + j] / c[j];
        acc += Wt[i * N + j] * pow(ap, p - 1.0) / r[i] * pow(bp, p);
      }
      dA[i * K + k] = acc;
    }
  }
  int64_t k;
#pragma omp parallel for schedule(dynamic, 1)
  for (k = 0; k < K; ++k) {
    for (int64_t j = 0; j < N; ++j) {
      double acc = 0.0;
      double bp = B[k * N + j] / c[j];
      for (int64_t ii2 = 0; ii2 < M; ++ii2) {
        double p = ldexp(1.0, plog[ii2 * N + j]);
        double ap = A[ii2 * K + k] / r[ii2];
        acc += Wt[ii2 * N + j] * pow(ap, p) * pow(bp, p - 1.0) / c[j];
      }
      dB[k * N + j] = acc;
    }
  }
  free(Wt);
}

/* Selected entries of the same gradient: dA at (ia[e], ka[e]) for e < n_a   */
/* and dB at (kb[e], jb[e]) for e < n_b.  A dA entry needs row i of W, i.e.  */
/* S_ij for every j (O(N K) terms); a dB entry needs column j (O(M K)).     */
void orc_pnorm_grad_entries(int64_t M, int64_t N, int64_t K, const double* A, const double* B,
                            const double* r, const double* c, const uint8_t* plog,
                            const double* G, int64_t n_a, const int64_t* ia, const int64_t* ka,
                            double* dA, int64_t n_b, const int64_t* kb, const int64_t* jb,
                            double* dB) {
  int64_t e;
#pragma omp parallel for schedule(dynamic, 1)
  for (e = 0; e < n_a; ++e) {
    const int64_t i = ia[e], k = ka[e];
    double acc = 0.0;
    for (int64_t j = 0; j < N; ++j) {
      double p = ldexp(1.0, plog[i * N + j]);
      double s = 0.0;
      for (int64_t t = 0; t < K; ++t) s += pow((A[i * K + t] / r[i]) * (B[t * N + j] / c[j]), p);
      if (!(s > 0.0)) continue;
      double C = r[i] * c[j] * pow(s, 1.0 / p);
      double W = G[i * N + j] * C / s;
      acc += W * pow(A[i * K + k] / r[i], p - 1.0) / r[i] * pow(B[k * N + j] / c[j], p);
    }
    dA[e] = acc;
  }
#pragma omp parallel for schedule(dynamic, 1)
  for (e = 0; e < n_b; ++e) {
    const int64_t k = kb[e], j = jb[e];
    double acc = 0.0;
    for (int64_t i = 0; i < M; ++i) {
      double p = ldexp(1.0, plog[i * N + j]);
      double s = 0.0;
      for (int64_t t = 0; t < K; ++t) s += pow((A[i * K + t] / r[i]) * (B[t * N + j] / c[j]), p);
      if (!(s > 0.0)) continue;
      double C = r[i] * c[j] * pow(s, 1.0 / p);
      double W = G[i * N + j] * C / s;
      acc += W * pow(A[i * K + k] / r[i], p) * pow(B[k * N + j] / c[j], p - 1.0) / c[j];
    }
    dB[e] = acc;
  }
}

/* Loss L = sum_j log C_ij over one row i of the product, at fixed p per    */
/* entry; used by finite differences (a_ik only changes row i of C).       */
double orc_row_logloss(int64_t N, int64_t K, const double* arow, const double* B,
                       const uint8_t* plog_row) {
  double L = 0.0;
  for (int64_t j = 0; j < N; ++j) {
    double p = ldexp(1.0, plog_row[j]);
    double s = 0.0;
    for (int64_t k = 0; k < K; ++k) s += pow(arow[k] * B[k * N + j], p);
    L += log(pow(s, 1.0 / p));
  }
  return L;
}

/* Loss over one column j of the product (b_kj only changes column j). */
double orc_col_logloss(int64_t M, int64_t K, const double* A, const double* bcol,
                       const uint8_t* plog_col) {
  double L = 0.0;
  for (int64_t i = 0; i < M; ++i) {
    double p = ldexp(1.0, plog_col[i]);
    double s = 0.0;
    for (int64_t k = 0; k < K; ++k) s += pow(A[i * K + k] * bcol[k], p);
    L += log(pow(s, 1.0 / p));
  }
  return L;
}

/* ---------------------------------------------------------------------- */
/* Max-convolution (Sec. 1): z_m = max_i x_i y_(m-i) over the indices where */
/* both factors exist, m = 0 .. nx + ny - 2.  One problem per batch row;    */
/* x is batch x nx, y is batch x ny, z is batch x (nx + ny - 1), row-major.  */
void orc_maxconv(int64_t batch, int64_t nx, const double* x, int64_t ny, const double* y,
                 double* z) {
  int64_t b;
  int64_t nz = nx + ny - 1;
#pragma omp parallel for schedule(dynamic, 1)
  for (b = 0; b < batch; ++b) {
    const double* xb = x + b * nx;
    const double* yb = y + b * ny;
    for (int64_t m = 0; m < nz; ++m) {
      double mx = 0.0;
      for (int64_t i = 0; i < nx; ++i) {
        int64_t t = m - i;
        if (t < 0 || t >= ny) continue;
        double v = xb[i] * yb[t];
        if (v > mx) mx = v;
      }
      z[b * nz + m] = mx;
    }
  }
}

/* The ring convolution G done naively (what an FFT convolution H computes */
/* up to rounding): w_m = sum_i x_i y_(m-i).  Same layout as orc_maxconv.   */
void orc_conv(int64_t batch, int64_t nx, const double* x, int64_t ny, const double* y, double* w) {
  int64_t b;
  int64_t nz = nx + ny - 1;
#pragma omp parallel for schedule(dynamic, 1)
  for (b = 0; b < batch; ++b) {
    const double* xb = x + b * nx;
    const double* yb = y + b * ny;
    for (int64_t m = 0; m < nz; ++m) {
      double s = 0.0;
      for (int64_t i = 0; i < nx; ++i) {
        int64_t t = m - i;
        if (t < 0 || t >= ny) continue;
        s += xb[i] * yb[t];
      }
      w[b * nz + m] = s;
    }
  }
}

/* p-norm estimate of the max-convolution (Sec. 1; the scaled H' of Sec.    */
/* 2.1 with one scale per vector): x' = x / max x, y' = y / max y (a zero   */
/* vector keeps scale 1); for each p in P the p-sums                        */
/* S^(p)_m = sum_i x'_i^p y'_(m-i)^p by the naive convolution, with pow per */
/* term; p* = the largest p with S^(p)_m >= tau (none: the smallest p,      */
/* flagged 0x80 in p_sel); z_m = max x * max y * (S^(p*)_m)^(1/p*).          */
/* S_all (optional) receives S as [batch][n_p][nz].                          */
void orc_maxconv_pnorm(int64_t batch, int64_t nx, const double* x, int64_t ny, const double* y,
                       int n_p, const int* p_log2, double tau, double* z, uint8_t* psel,
                       double* S_all) {
  int64_t b;
  int64_t nz = nx + ny - 1;
#pragma omp parallel for schedule(dynamic, 1)
  for (b = 0; b < batch; ++b) {
    const double* xb = x + b * nx;
    const double* yb = y + b * ny;
    double mx = 0.0, my = 0.0;
    for (int64_t i = 0; i < nx; ++i)
      if (xb[i] > mx) mx = xb[i];
    for (int64_t i = 0; i < ny; ++i)
      if (yb[i] > my) my = yb[i];
    double sx = mx > 0.0 ? mx : 1.0, sy = my > 0.0 ? my : 1.0;
    for (int64_t m = 0; m < nz; ++m) {
      int q_sel = -1;
      double s_sel = 0.0;
      for (int q = n_p - 1; q >= 0; --q) {
        double p = ldexp(1.0, p_log2[q]);
        double s = 0.0;
        for (int64_t i = 0; i < nx; ++i) {
          int64_t t = m - i;
          if (t < 0 || t >= ny) continue;
          s += pow(xb[i] / sx, p) * pow(yb[t] / sy, p);
        }
        if (S_all) S_all[(b * n_p + q) * nz + m] = s;
        if (q_sel < 0 && s >= tau) {
          q_sel = q;
          s_sel = s;
        }
        if (q == 0 && q_sel < 0) s_sel = s;
      }
      int unstable = q_sel < 0;
      if (unstable) q_sel = 0;
      double p = ldexp(1.0, p_log2[q_sel]);
      z[b * nz + m] = sx * sy * (s_sel > 0.0 ? pow(s_sel, 1.0 / p) : 0.0);
      if (psel) psel[b * nz + m] = (uint8_t)(p_log2[q_sel] | (unstable ? 0x80 : 0));
    }
  }
}

/* Selected outputs m[e] of one max-convolution: the exact max and every    */
/* p-sum S^(p)_m of the max-scaled vectors (as in orc_maxconv_pnorm), with   */
/* pow per term; S[e * n_p + q].  Cost O(n_e * min(nx, ny) * n_p).           */
void orc_maxconv_entries(int64_t nx, const double* x, int64_t ny, const double* y, int n_p,
                         const int* p_log2, int64_t n_e, const int64_t* m, double* exact,
                         double* S) {
  double mx = 0.0, my = 0.0;
  for (int64_t i = 0; i < nx; ++i)
    if (x[i] > mx) mx = x[i];
  for (int64_t i = 0; i < ny; ++i)
    if (y[i] > my) my = y[i];
  double sx = mx > 0.0 ? mx : 1.0, sy = my > 0.0 ? my : 1.0;
  int64_t e;
#pragma omp parallel for schedule(dynamic, 1)
  for (e = 0; e < n_e; ++e) {
    int64_t mm = m[e];
    double best = 0.0;
    for (int64_t i = 0; i < nx; ++i) {
      int64_t t = mm - i;
      if (t < 0 || t >= ny) continue;
      double v = x[i] * y[t];
      if (v > best) best = v;
    }
    if (exact) exact[e] = best;
    for (int q = 0; q < n_p; ++q) {
      double p = ldexp(1.0, p_log2[q]);
      double s = 0.0;
      for (int64_t i = 0; i < nx; ++i) {
        int64_t t = mm - i;
        if (t < 0 || t >= ny) continue;
        s += pow(x[i] / sx, p) * pow(y[t] / sy, p);
      }
      S[e * n_p + q] = s;
    }
  }
}

/* ---------------------------------------------------------------------- */
/* Approximate top-k of the products x_i y_j (Alg. 9, E_(X' x Y'), with the  */
/* NormQueue).  x' = x / max x, y' = y / max y; for every diagonal          */
/* m = i + j the p-sums sigma^(p)_m = sum_i x'_i^p y'_(m-i)^p (naive ring    */
/* convolution, FP64, pow per term); psi_m = estimateMaxFromNormPowerSequence */
/* (the plain form: (sigma^(p*))^(1/p*) at the largest p with sigma >= tau,  */
/* none: 0).  k times: take the diagonal m* with the largest psi (ties: the   */
/* smallest m), emit (psi_m* max x max y, m*), subtract psi_m*^p from every  */
/* sigma^(p)_m* (the NormQueue pop) and re-estimate psi_m* once; a diagonal  */
/* is exhausted after as many pops as it has terms.  Readings of the printed */
/* listing: the subtraction touches sigma_m* (not sigma_m), the re-estimate */
/* follows the update of every p, and it is clamped to the value just       */
/* popped from that diagonal (removing a multiset's max cannot raise its    */
/* max; without the clamp, residuals of large p falling below tau hand the  */
/* estimate to small p, whose norms are near the diagonal's whole sum).     */
/* vals[k], diag[k] (-1 when every                                           */
/* diagonal is exhausted).  y_rev != 0 uses y reversed (the second call of   */
/* the index recovery).                                                     */
void orc_topk_xy(int64_t n, const double* x, const double* y, int y_rev, int n_p,
                 const int* p_log2, double tau, int64_t k, double* vals, int64_t* diag) {
  int64_t nz = 2 * n - 1;
  double mx = 0.0, my = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    if (x[i] > mx) mx = x[i];
    if (y[i] > my) my = y[i];
  }
  double sx = mx > 0.0 ? mx : 1.0, sy = my > 0.0 ? my : 1.0;
  double* sig = (double*)malloc(sizeof(double) * (size_t)nz * n_p);
  double* psi = (double*)malloc(sizeof(double) * (size_t)nz);
  int64_t* left = (int64_t*)malloc(sizeof(int64_t) * (size_t)nz);
  if (!sig || !psi || !left) {
    free(sig); free(psi); free(left);
    return;
  }
  int64_t m;
#pragma omp parallel for schedule(dynamic, 16)
  for (m = 0; m < nz; ++m) {
    int64_t lo = m - n + 1 > 0 ? m - n + 1 : 0, hi = m < n - 1 ? m : n - 1;
    left[m] = hi - lo + 1;
    for (int q = 0; q < n_p; ++q) {
      double p = ldexp(1.0, p_log2[q]), s = 0.0;
      for (int64_t i = lo; i <= hi; ++i) {
        double yv = y_rev ? y[n - 1 - (m - i)] : y[m - i];
        s += pow(x[i] / sx, p) * pow(yv / sy, p);
      }
      sig[m * n_p + q] = s;
    }
  }
  for (m = 0; m < nz; ++m) {
    psi[m] = 0.0;
    for (int q = n_p - 1; q >= 0; --q)
      if (sig[m * n_p + q] >= tau) {
        psi[m] = pow(sig[m * n_p + q], 1.0 / ldexp(1.0, p_log2[q]));
        break;
      }
  }
  for (int64_t t = 0; t < k; ++t) {
    int64_t best = -1;
    for (m = 0; m < nz; ++m)
      if (left[m] > 0 && (best < 0 || psi[m] > psi[best])) best = m;
    if (best < 0 || psi[best] <= 0.0) {
      vals[t] = 0.0;
      diag[t] = -1;
      continue;
    }
    double a = psi[best];
    vals[t] = a * sx * sy;
    diag[t] = best;
    left[best] -= 1;
    for (int q = 0; q < n_p; ++q) sig[best * n_p + q] -= pow(a, ldexp(1.0, p_log2[q]));
    psi[best] = 0.0;
    if (left[best] > 0)
      for (int q = n_p - 1; q >= 0; --q)
        if (sig[best * n_p + q] >= tau) {
          psi[best] = pow(sig[best * n_p + q], 1.0 / ldexp(1.0, p_log2[q]));
          break;
        }
    /* the next max of a multiset never exceeds the one just removed */
    if (psi[best] > a) psi[best] = a;
  }
  free(sig);
  free(psi);
  free(left);
}
