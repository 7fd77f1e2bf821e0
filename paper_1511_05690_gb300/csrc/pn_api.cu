// Host runtime and C ABI of the p-norm semiring library (include/pnorm.h):
// argument checks, workspace layout, the per-level launch sequence of the
// p-norm product (Alg. 5), the APSP driver (Sec. 2.2) and the exact product.
#include <cmath>
#include <cstring>
#include <mutex>

#include "pn_internal.h"
#include <cuda_runtime.h>

namespace pn {

namespace {

constexpr size_t WS_ALIGN = 256;
constexpr size_t IMG_ALIGN = 1024;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

struct DevInfo {
  int sms = 0;
  int ok = -1;  // -1 unknown, 0 unsupported, 1 sm_103
};
std::mutex g_dev_mu;
DevInfo g_dev[64];

// Streaming multiprocessors of the current device, or 0 if it is not an
// sm_103 (GB300-class) device.
int device_sms() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  std::lock_guard<std::mutex> lk(g_dev_mu);
  DevInfo& d = g_dev[dev];
  if (d.ok < 0) {
    int major = 0, minor = 0, sms = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    d.ok = (major == 10 && minor == 3) ? 1 : 0;
    d.sms = sms;
  }
  return d.ok == 1 ? d.sms : 0;
}

bool opts_valid(const pn_opts* o) {
  if (!o) return false;
  if (o->n_p < 1 || o->n_p > PN_MAX_P) return false;
  for (int q = 0; q < o->n_p; ++q) {
    if (o->p_log2[q] < 0 || o->p_log2[q] > 15) return false;
    if (q > 0 && o->p_log2[q] <= o->p_log2[q - 1]) return false;
  }
  if (o->compute < PN_F32_EXACT || o->compute > PN_E4M3) return false;
  if (o->scaling < 0 || o->scaling > 2) return false;
  if (o->diag_policy < 0 || o->diag_policy > 2) return false;
  if (o->tile_n != 0 && o->tile_n != 128 && o->tile_n != 256) return false;
  if (o->tile_m != 0 && o->tile_m != 128 && o->tile_m != 256) return false;
  if (o->timeout_ns < 0) return false;
  if (std::isnan(o->tau)) return false;
  if (o->estimator < 0 || o->estimator > 2) return false;
  if (o->correction < 0 || o->correction > 2) return false;
  if (o->correction == 1 && o->estimator != 0) return false;
  if (o->correction == 2 && o->estimator == 2) return false;
  if (o->correction == 2 && (o->n_fit < 1 || !o->fit_i || !o->fit_j)) return false;
  return true;
}

// A CTA pair (cta_group::2) per 256 x BN tile, or one CTA per 128 x BN tile.
// The autotune cache records a pair as 256 + BN (512 or 384).
int choose_cg(const pn_opts* o, int64_t M, int64_t N, int64_t K) {
  if (o->tile_m) return o->tile_m == 256 ? 2 : 1;
  if (o->tile_n == 128) return 1;
  const int tuned = host_tuned_bn(o->compute, M, N, K);
  if (tuned) return tuned > 256 ? 2 : 1;
  return (M >= 256 && N >= 256) ? 2 : 1;
}

// Time of a 256 x 128 pair tile relative to a 256 x 256 one with every
// cluster busy (measured, BF16, n = 8192 and 16384: 0.93 and 0.945).  The
// narrow tile does half the MMAs, but each SM then loads 24 KB of operand
// images per 256 tensor cycles instead of 32 KB per 512, more than L2 serves
// to all SMs at once.
constexpr double PAIR_NARROW_COST = 0.94;

// Width of a pair tile when the options leave it open: tiles run in waves of
// one per cluster (two SMs); the narrow tile wins only where it needs no more
// waves than the wide one (small outputs, where it spreads the work over
// twice the SMs).  A 4096 x 4096 output: 4 waves of 256 wide tiles on 76
// clusters against 7 of 128 wide ones (7 x 0.94 > 4).
int pair_width(int64_t M, int64_t N) {
  const int sms = device_sms();
  const int64_t clusters = sms > 1 ? sms / 2 : 76;
  const int64_t rows = ceil_div(M, 2 * TILE_M);
  const int64_t w256 = ceil_div(rows * ceil_div(N, 256), clusters);
  const int64_t w128 = ceil_div(rows * ceil_div(N, 128), clusters);
  return static_cast<double>(w128) * PAIR_NARROW_COST < static_cast<double>(w256) ? 128 : 256;
}

// Tile width: 3xTF32 carries two operand planes, so only 128 fits one CTA's
// ring; a CTA pair's tile is 256 or 128 wide.
int choose_bn(const pn_opts* o, int64_t M, int64_t N, int64_t K) {
  if (choose_cg(o, M, N, K) == 2) {
    if (o->tile_n) return o->tile_n;
    if (o->tile_m == 0) {
      const int tuned = host_tuned_bn(o->compute, M, N, K);
      if (tuned == 512 || tuned == 384) return tuned - 256;
    }
    return pair_width(M, N);
  }
  if (o->compute == PN_F32_EXACT) return 128;
  if (o->tile_n) return o->tile_n;
  const int tuned = host_tuned_bn(o->compute, M, N, K);  // autotune cache
  if (tuned == 128 || tuned == 256) return tuned;
  return N > 128 ? 256 : 128;
}

// Smallest float >= t (so that S >= result  <=>  S >= t for float S).
float tau_up(double t) {
  if (!(t > 0.0)) return 0.0f;
  if (t > 3.0e38) return INFINITY;
  float f = static_cast<float>(t);
  if (static_cast<double>(f) < t) f = std::nextafter(f, INFINITY);
  if (f == 0.0f) f = std::nextafter(0.0f, 1.0f);
  return f;
}

// Workspace layout of one product (single problem).
struct Layout {
  int BN = 0, KB = 0, RBA = 0, RBB = 0, tiles_m = 0, tiles_n = 0, total_tiles = 0;
  int cg = 1, pair_tiles = 0;
  int state_ld = 0, n_p = 0, n_slots = 0, planes = 1;
  size_t off_rmax = 0, off_cmax = 0, off_gmax = 0, off_counts = 0, off_rflag = 0,
         off_cflag = 0, off_pushed = 0;
  size_t ctrl_bytes = 0, off_coef = 0, off_samp = 0, off_scls = 0;
  size_t off_r = 0, off_c = 0, off_work = 0, off_state = 0, off_pend = 0, off_pend2 = 0,
         off_park = 0, off_aimg = 0, off_bimg = 0;
  size_t a_level_bytes = 0, b_level_bytes = 0, a_plane = 0, b_plane = 0;
  size_t total = 0;
};

Layout make_layout(int64_t M, int64_t N, int64_t K, const pn_opts* o) {
  Layout L;
  const int mode = o->compute;
  L.cg = choose_cg(o, M, N, K);
  L.BN = choose_bn(o, M, N, K);
  L.n_p = o->n_p;
  L.n_slots = make_schedule(o).n;
  L.planes = mode_planes(mode);
  L.KB = static_cast<int>(ceil_div(K, mode_bk(mode)));
  L.tiles_m = static_cast<int>(ceil_div(M, TILE_M));
  L.tiles_n = static_cast<int>(ceil_div(N, L.BN));
  // a pair's second CTA reads A row block 2 TM + 1: an odd last one is padded
  // with a block of zeros (rows past M)
  L.RBA = L.cg == 2 ? (L.tiles_m + 1) / 2 * 2 : L.tiles_m;
  L.RBB = L.tiles_n * (L.BN / TILE_M);
  L.pair_tiles = L.cg == 2 ? (L.tiles_m + 1) / 2 * L.tiles_n : 0;
  L.total_tiles = L.cg == 2 ? L.pair_tiles : L.tiles_m * L.tiles_n;
  L.state_ld = L.tiles_n * (L.BN / 32);
  size_t off = 0;
  // control words, cleared at the start of every call
  L.off_rmax = off; off += sizeof(uint32_t) * M;
  L.off_cmax = off; off += sizeof(uint32_t) * N;
  L.off_gmax = off; off += sizeof(uint32_t) * 2;
  L.off_counts = off; off += sizeof(int32_t) * 2 * PN_MAX_P;
  L.off_rflag = off; off += static_cast<size_t>(L.n_slots) * L.RBA;
  L.off_cflag = off; off += static_cast<size_t>(L.n_slots) * L.tiles_n;
  off = align_up(off, 4);
  L.off_pushed = off; off += sizeof(uint32_t) * static_cast<size_t>(L.n_slots) * L.pair_tiles;
  L.ctrl_bytes = align_up(off, 16);
  off = align_up(off, WS_ALIGN);
  L.off_coef = off; off = align_up(off + sizeof(float) * 2 * PN_MAX_P, WS_ALIGN);
  if (o->correction == 2) {
    // the affine correction's per-sample records (estimate, exact value, class)
    L.off_samp = off; off = align_up(off + sizeof(double) * 2 * (size_t)o->n_fit, WS_ALIGN);
    L.off_scls = off; off = align_up(off + sizeof(int32_t) * (size_t)o->n_fit, WS_ALIGN);
  }
  L.off_r = off; off = align_up(off + sizeof(float) * M, WS_ALIGN);
  L.off_c = off; off = align_up(off + sizeof(float) * N, WS_ALIGN);
  L.off_work = off;
  off = align_up(off + sizeof(int32_t) * L.n_slots * (size_t)L.total_tiles, WS_ALIGN);
  L.off_state = off; off = align_up(off + sizeof(uint32_t) * (size_t)M * L.state_ld, IMG_ALIGN);
  if (o->estimator >= 1) {
    L.off_pend = off; off = align_up(off + sizeof(uint32_t) * (size_t)M * L.state_ld, IMG_ALIGN);
  }
  if (o->estimator == 2) {
    L.off_pend2 = off; off = align_up(off + sizeof(uint32_t) * (size_t)M * L.state_ld, IMG_ALIGN);
    L.off_park = off; off = align_up(off + sizeof(float) * 2 * (size_t)M * N, IMG_ALIGN);
  }
  L.a_plane = static_cast<size_t>(L.RBA) * L.KB * IMG_BYTES;
  L.b_plane = static_cast<size_t>(L.RBB) * L.KB * IMG_BYTES;
  L.a_level_bytes = L.a_plane * L.planes;
  L.b_level_bytes = L.b_plane * L.planes;
  // One image buffer per operand serves every level: level q reads only the
  // images written for level q, after the previous level's GEMM has finished
  // (stream order).
  L.off_aimg = off; off += L.a_level_bytes;
  L.off_bimg = off; off += L.b_level_bytes;
  L.total = align_up(off, WS_ALIGN);
  return L;
}

double default_tau(int64_t K, int compute) {
  int e_mu, m, s;
  switch (compute) {
    case PN_F32_EXACT: e_mu = -126; m = 21; s = 0; break;
    case PN_TF32: e_mu = -126; m = 10; s = 0; break;
    case PN_BF16: e_mu = -126; m = 7; s = 0; break;
    case PN_F16: e_mu = -14; m = 10; s = 15; break;
    case PN_E4M3: e_mu = -6; m = 3; s = 8; break;
    default: return -1.0;
  }
  return static_cast<double>(K > 0 ? K : 1) * std::ldexp(1.0, e_mu + m - s);
}

pn_status cuda_status(int e) { return e == 0 ? PN_OK : PN_ECUDA; }

}  // namespace

// Shared with the grouped and autotune code (pn_grouped.cu).
int host_device_sms() { return device_sms(); }
bool host_opts_valid(const pn_opts* o) { return opts_valid(o); }
double host_default_tau(int64_t K, int compute) { return default_tau(K, compute); }
float host_tau_up(double t) { return tau_up(t); }

namespace {

// Fills the Common / Prob description of one product laid out by `L` in `ws`.
void fill_common(Common& cm, const Layout& L, int64_t M, int64_t N, int64_t K, const float* A,
                 int64_t lda, const float* B, int64_t ldb, float* C, int64_t ldc, uint8_t* p_sel,
                 float* S_sel, const pn_opts* o, uint8_t* ws) {
  std::memset(&cm, 0, sizeof(cm));
  Prob& P = cm.single;
  P.A = A; P.B = B; P.C = C; P.psel = p_sel; P.Ssel = S_sel;
  P.lda = lda; P.ldb = ldb; P.ldc = ldc; P.ldaux = N;
  P.M = static_cast<int32_t>(M); P.N = static_cast<int32_t>(N); P.K = static_cast<int32_t>(K);
  P.KB = L.KB; P.RBA = L.RBA; P.RBB = L.RBB;
  P.tiles_m = L.tiles_m; P.tiles_n = L.tiles_n;
  P.tile_base = 0; P.xa_base = 0; P.xb_base = 0; P.tm_base = 0; P.tn_base = 0;
  P.KMA = static_cast<int32_t>(ceil_div(K, MAXSEG_A));
  P.KMB = static_cast<int32_t>(ceil_div(K, MAXSEG_B));
  P.ma_base = 0; P.mb_base = 0;
  const bool vc = ((ldc & 3) == 0) && ((reinterpret_cast<uintptr_t>(C) & 15) == 0) &&
                  ((N & 15) == 0) &&
                  (!p_sel || (reinterpret_cast<uintptr_t>(p_sel) & 15) == 0) &&
                  (!S_sel || (reinterpret_cast<uintptr_t>(S_sel) & 15) == 0);
  P.vec_c = vc ? 1 : 0;
  P.state_ld = L.state_ld;
  P.a_img = 0; P.b_img = 0;
  P.a_plane = static_cast<int64_t>(L.a_plane);
  P.b_plane = static_cast<int64_t>(L.b_plane);
  P.rc_r = 0; P.rc_c = 0; P.state_off = 0;
  const double tau = o->tau > 0.0 ? o->tau : default_tau(K, o->compute);
  P.tau_d = tau;
  P.tau = tau_up(tau);
  cm.probs = nullptr;
  cm.nprob = 1;
  cm.cg = L.cg;
  cm.total_tiles = L.total_tiles;
  cm.total_xa = L.RBA * L.KB;
  cm.total_xb = L.RBB * L.KB;
  cm.total_tm = L.RBA;
  cm.total_tn = L.tiles_n;
  cm.total_ma = L.RBA * P.KMA;
  cm.total_mb = L.RBB * P.KMB;
  cm.mode = o->compute;
  cm.BN = L.BN;
  cm.s_op = mode_op_shift(o->compute);
  cm.scaling = o->scaling;
  cm.unscale = std::ldexp(1.0f, -2 * cm.s_op);
  cm.rmax = reinterpret_cast<uint32_t*>(ws + L.off_rmax);
  cm.cmax = reinterpret_cast<uint32_t*>(ws + L.off_cmax);
  cm.gmax = reinterpret_cast<uint32_t*>(ws + L.off_gmax);
  cm.r = reinterpret_cast<float*>(ws + L.off_r);
  cm.c = reinterpret_cast<float*>(ws + L.off_c);
  cm.state = reinterpret_cast<uint32_t*>(ws + L.off_state);
  cm.pend = o->estimator >= 1 ? reinterpret_cast<uint32_t*>(ws + L.off_pend) : nullptr;
  cm.pend2 = o->estimator == 2 ? reinterpret_cast<uint32_t*>(ws + L.off_pend2) : nullptr;
  cm.park = o->estimator == 2 ? reinterpret_cast<float*>(ws + L.off_park) : nullptr;
  // r = 2 projection: its Hankel determinant must clear the p-sums' relative
  // error (of order u, the powered operands' unit roundoff) by a margin
  cm.r2_eta = std::ldexp(1.0f, 5 - (o->compute == PN_F32_EXACT ? 21
                                    : o->compute == PN_BF16     ? 8
                                    : o->compute == PN_E4M3     ? 4
                                                                : 11));
  cm.corr = o->correction;
  cm.coef = reinterpret_cast<const float*>(ws + L.off_coef);
  cm.status = o->dev_status;
  cm.timeout_ns = o->timeout_ns > 0 ? static_cast<uint64_t>(o->timeout_ns) : 2000000000ull;
  cm.debug_flags = o->debug_flags;
  cm.n_levels = o->n_p;
  // For operand formats with the FP32 exponent range (3xTF32, TF32, BF16) the
  // threshold tau = K mu 2^(m-s) lies near FP32 underflow, and entries within
  // a decade of it are selected and rooted in FP64.  FP16 / E4M3 thresholds
  // lie far above FP32 underflow, where an FP32 S is exact to 2^-24, far
  // finer than the operands' own 2^-11 / 2^-4.
  cm.fp64_near = (o->compute == PN_F32_EXACT || o->compute == PN_TF32 || o->compute == PN_BF16);
}

// Slot t of the level schedule (slot 0 is the largest p).
Level make_level(const Layout& L, const pn_opts* o, uint8_t* ws, const Schedule& sc, int t) {
  Level lv;
  std::memset(&lv, 0, sizeof(lv));
  int32_t* counts = reinterpret_cast<int32_t*>(ws + L.off_counts);
  int32_t* work = reinterpret_cast<int32_t*>(ws + L.off_work);
  uint8_t* rflag = ws + L.off_rflag;
  uint8_t* cflag = ws + L.off_cflag;
  const int q = sc.q[t];
  const int tn = t + 1 < sc.n ? t + 1 : t;
  lv.q = q;
  lv.half = sc.half[t];
  lv.plog = o->p_log2[q] - lv.half;  // a half level's p is 1.5 * 2^(log2 p_q - 1)
  lv.is_top = t == 0;
  lv.is_bottom = t == sc.n - 1;
  lv.a_level = ws + L.off_aimg;
  lv.b_level = ws + L.off_bimg;
  lv.work = work + static_cast<size_t>(t) * L.total_tiles;
  lv.work_count = counts + t;
  lv.next_work = work + static_cast<size_t>(tn) * L.total_tiles;
  lv.next_count = counts + tn;
  lv.rflag = rflag + static_cast<size_t>(t) * L.RBA;
  lv.cflag = cflag + static_cast<size_t>(t) * L.tiles_n;
  lv.next_rflag = rflag + static_cast<size_t>(tn) * L.RBA;
  lv.next_cflag = cflag + static_cast<size_t>(tn) * L.tiles_n;
  if (L.cg == 2)
    lv.pair_pushed = reinterpret_cast<uint32_t*>(ws + L.off_pushed) +
                     static_cast<size_t>(tn) * L.pair_tiles;
  if (o->estimator == 2) {
    lv.r2_state = t > 0;
    lv.r2_new = !lv.half && t + 1 < sc.n && sc.half[t + 1];
    if (lv.r2_new && t + 2 < sc.n) {
      const int ts = t + 2;
      lv.skip_work = work + static_cast<size_t>(ts) * L.total_tiles;
      lv.skip_count = counts + ts;
      lv.skip_rflag = rflag + static_cast<size_t>(ts) * L.RBA;
      lv.skip_cflag = cflag + static_cast<size_t>(ts) * L.tiles_n;
    }
  } else {
    set_projection(lv, o, q);
  }
  return lv;
}

// The product proper, arguments already checked.
pn_status run_pnorm(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, const float* B,
                    int64_t ldb, float* C, int64_t ldc, uint8_t* p_sel, float* S_sel,
                    const pn_opts* o, uint8_t* ws, void* stream, int sms, int post = 0) {
  if (M == 0 || N == 0) return PN_OK;
  const Layout L = make_layout(M, N, K, o);
  Common cm;
  fill_common(cm, L, M, N, K, A, lda, B, ldb, C, ldc, p_sel, S_sel, o, ws);
  cm.post = post;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (K == 0) return cuda_status(launch_fill_empty(cm, o->p_log2[0], stream));
  int e = cudaMemsetAsync(ws, 0, L.ctrl_bytes, s);
  if (e) return PN_ECUDA;
  if ((e = launch_maxes(cm, stream))) return PN_ECUDA;
  OperandMaps maps;
  make_operand_maps(cm, maps);
  const Schedule sc = make_schedule(o);
  for (int t = 0; t < sc.n; ++t) {
    const Level lv = make_level(L, o, ws, sc, t);
    if ((e = launch_power_a(cm, lv, stream, &maps))) return PN_ECUDA;
    if ((e = launch_power_b(cm, lv, stream, &maps))) return PN_ECUDA;
    if (lv.is_top && o->correction == 2) {
      // the affine model's coefficients, from the scales of the top level
      FitArgs fa;
      std::memset(&fa, 0, sizeof(fa));
      fa.fi = o->fit_i;
      fa.fj = o->fit_j;
      fa.n_fit = o->n_fit;
      fa.n_p = o->n_p;
      for (int t = 0; t < o->n_p; ++t) fa.p_log2[t] = o->p_log2[t];
      fa.estimator = o->estimator;
      fa.samp = reinterpret_cast<double*>(ws + L.off_samp);
      fa.scls = reinterpret_cast<int32_t*>(ws + L.off_scls);
      fa.coef = reinterpret_cast<float*>(ws + L.off_coef);
      fa.user_coef = o->fit_coef;
      if ((e = launch_fit(cm, fa, stream))) return PN_ECUDA;
    }
    if (lv.is_top && o->ev_gemm_begin)
      if (cudaEventRecord(static_cast<cudaEvent_t>(o->ev_gemm_begin), s)) return PN_ECUDA;
    if ((e = launch_gemm_level(cm, lv, sms, stream))) return PN_ECUDA;
    if (lv.is_top && o->ev_gemm_end)
      if (cudaEventRecord(static_cast<cudaEvent_t>(o->ev_gemm_end), s)) return PN_ECUDA;
  }
  return PN_OK;
}

// Adjoint: supported operand formats (FP32 exponent range; W is not scaled).
bool bw_mode_ok(int compute) {
  return compute == PN_F32_EXACT || compute == PN_TF32 || compute == PN_BF16;
}

// Workspace of the adjoint: control words, scales and the four operand images
// of one p (reused for every p, stream order).
struct BwLayout {
  int BN = 0, cg = 1, KB1 = 0, KB2 = 0, RB1a = 0, RB1b = 0, RB2a = 0, RB2b = 0;
  size_t off_rmax = 0, off_cmax = 0, off_gmax = 0, off_mask = 0, ctrl_bytes = 0;
  size_t off_r = 0, off_c = 0, off_w1 = 0, off_b1 = 0, off_a2 = 0, off_w2 = 0;
  size_t plane_w1 = 0, plane_b1 = 0, plane_a2 = 0, plane_w2 = 0, total = 0;
};

BwLayout make_bw_layout(int64_t M, int64_t N, int64_t K, const pn_opts* o) {
  BwLayout L;
  const int mode = o->compute;
  const int bk = mode_bk(mode), planes = mode_planes(mode);
  // CTA pairs on 256 x 256 tiles for both gradient GEMMs (outputs M x K and
  // K x N) when each gives every cluster at least two pair tiles, so that a
  // pair's gradient epilogue overlaps its next tile's MMAs (measured, 3xTF32,
  // P = {16}: n = 2048 0.43 ms with pairs against 0.40 with one CTA per tile,
  // 4096 1.40 against 1.56, 8192 7.42 against 9.54); unless the options ask
  // for one CTA per tile or for 128-wide tiles
  const int sms = device_sms();
  const int64_t clusters = sms > 1 ? sms / 2 : 76;
  const int64_t t1 = ceil_div(M, 256) * ceil_div(K, 256), t2 = ceil_div(K, 256) * ceil_div(N, 256);
  const bool many = t1 >= 2 * clusters && t2 >= 2 * clusters;
  L.cg = (o->tile_m == 256 || (o->tile_m == 0 && many)) && o->tile_n != 128 ? 2 : 1;
  L.BN = L.cg == 2 ? 256 : mode == PN_F32_EXACT ? 128 : (o->tile_n ? o->tile_n : 256);
  const int per = L.BN / TILE_M;
  auto even = [&](int rb) { return L.cg == 2 ? (rb + 1) / 2 * 2 : rb; };
  L.KB1 = static_cast<int>(ceil_div(N, bk));
  L.KB2 = static_cast<int>(ceil_div(M, bk));
  // a pair's second CTA reads A row block 2 TM + 1: an odd count is padded
  // with a block of zeros (the image kernel zero-fills rows past the source)
  L.RB1a = even(static_cast<int>(ceil_div(M, TILE_M)));
  L.RB1b = static_cast<int>(ceil_div(K, L.BN)) * per;
  L.RB2a = even(static_cast<int>(ceil_div(K, TILE_M)));
  L.RB2b = static_cast<int>(ceil_div(N, L.BN)) * per;
  size_t off = 0;
  L.off_rmax = off; off += sizeof(uint32_t) * M;
  L.off_cmax = off; off += sizeof(uint32_t) * N;
  L.off_gmax = off; off += sizeof(uint32_t) * 2;
  L.off_mask = off; off += sizeof(uint32_t);
  L.ctrl_bytes = align_up(off, 16);
  off = align_up(off, WS_ALIGN);
  L.off_r = off; off = align_up(off + sizeof(float) * M, WS_ALIGN);
  L.off_c = off; off = align_up(off + sizeof(float) * N, IMG_ALIGN);
  L.plane_w1 = static_cast<size_t>(L.RB1a) * L.KB1 * IMG_BYTES;
  L.plane_b1 = static_cast<size_t>(L.RB1b) * L.KB1 * IMG_BYTES;
  L.plane_a2 = static_cast<size_t>(L.RB2a) * L.KB2 * IMG_BYTES;
  L.plane_w2 = static_cast<size_t>(L.RB2b) * L.KB2 * IMG_BYTES;
  L.off_w1 = off; off += L.plane_w1 * planes;
  L.off_b1 = off; off += L.plane_b1 * planes;
  L.off_a2 = off; off += L.plane_a2 * planes;
  L.off_w2 = off; off += L.plane_w2 * planes;
  L.total = align_up(off, WS_ALIGN);
  return L;
}

bool dims_ok(int64_t M, int64_t N, int64_t K) {
  const int64_t lim = (int64_t)1 << 30;
  return M >= 0 && N >= 0 && K >= 0 && M < lim && N < lim && K < lim;
}

}  // namespace

}  // namespace pn

using namespace pn;

extern "C" {

const char* pn_status_string(int32_t status) {
  switch (status) {
    case PN_OK: return "PN_OK";
    case PN_EINVAL: return "PN_EINVAL: invalid argument";
    case PN_EALIGN: return "PN_EALIGN: workspace not 256-byte aligned";
    case PN_EWORKSPACE: return "PN_EWORKSPACE: workspace too small";
    case PN_EDOMAIN: return "PN_EDOMAIN: input outside the semiring domain";
    case PN_ECUDA: return "PN_ECUDA: CUDA runtime error";
    case PN_ETIMEOUT: return "PN_ETIMEOUT: a bounded device wait ran out";
    case PN_EUNSUPPORTED: return "PN_EUNSUPPORTED: unsupported device or mode";
    default: return "unknown pn_status";
  }
}

void pn_default_opts(pn_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->n_p = 7;
  for (int q = 0; q < 7; ++q) o->p_log2[q] = q;
  o->tau = 0.0;
  o->compute = PN_BF16;
  o->scaling = 2;
  o->diag_policy = 2;
  o->tile_n = 0;
}

double pn_default_tau(int64_t K, int32_t compute) { return pn::default_tau(K, compute); }

int32_t pn_device_sm_count(void) { return pn::device_sms(); }

size_t pn_workspace_size(int64_t M, int64_t N, int64_t K, const pn_opts* opts) {
  if (!opts_valid(opts) || !dims_ok(M, N, K)) return 0;
  // large enough for every tile shape the options leave open (the autotuner
  // or the automatic rule may pick any of them later)
  size_t best = 0;
  for (int tile_m : {128, 256}) {
    for (int tile_n : {128, 256}) {
      if (opts->tile_m && opts->tile_m != tile_m) continue;
      if (opts->tile_n && opts->tile_n != tile_n) continue;
      pn_opts o = *opts;
      o.tile_m = tile_m;
      o.tile_n = tile_n;
      const size_t b = make_layout(M, N, K, &o).total;
      if (b > best) best = b;
    }
  }
  return best;
}

pn_status maxprod_pnorm(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                        const float* B, int64_t ldb, float* C, int64_t ldc, uint8_t* p_sel,
                        float* S_sel, const pn_opts* opts, void* ws, size_t ws_bytes,
                        void* stream) {
  if (!opts_valid(opts) || !dims_ok(M, N, K)) return PN_EINVAL;
  if (M == 0 || N == 0) return PN_OK;
  if (!C || ldc < N) return PN_EINVAL;
  if (K > 0 && (!A || !B || lda < K || ldb < N)) return PN_EINVAL;
  const size_t need = make_layout(M, N, K, opts).total;
  if (!ws || ws_bytes < need) return PN_EWORKSPACE;
  if (reinterpret_cast<uintptr_t>(ws) % WS_ALIGN) return PN_EALIGN;
  const int sms = device_sms();
  if (sms <= 0) return PN_EUNSUPPORTED;
  return run_pnorm(M, N, K, A, lda, B, ldb, C, ldc, p_sel, S_sel, opts,
                   static_cast<uint8_t*>(ws), stream, sms);
}

pn_status maxprod_exact(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                        const float* B, int64_t ldb, float* C, int64_t ldc, int32_t semiring,
                        void* stream) {
  if (!dims_ok(M, N, K) || (semiring != 0 && semiring != 1)) return PN_EINVAL;
  if (M == 0 || N == 0) return PN_OK;
  if (!C || ldc < N) return PN_EINVAL;
  if (K > 0 && (!A || !B || lda < K || ldb < N)) return PN_EINVAL;
  if (device_sms() <= 0) return PN_EUNSUPPORTED;
  return cuda_status(launch_exact(M, N, K, A, lda, B, ldb, C, ldc, semiring, 2, stream));
}

// Exact product with an explicit kernel variant (0: FMUL + FMNMX, 1: paired
// mul.f32x2 + 3-input max, 2: variant 1 software-pipelined); used to compare
// them.  Same results.
pn_status pn_maxprod_exact_variant(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                                   const float* B, int64_t ldb, float* C, int64_t ldc,
                                   int32_t semiring, int32_t variant, void* stream) {
  if (!dims_ok(M, N, K) || (semiring != 0 && semiring != 1)) return PN_EINVAL;
  if (variant < 0 || variant > 2) return PN_EINVAL;
  if (M == 0 || N == 0) return PN_OK;
  if (!C || ldc < N) return PN_EINVAL;
  if (K > 0 && (!A || !B || lda < K || ldb < N)) return PN_EINVAL;
  if (device_sms() <= 0) return PN_EUNSUPPORTED;
  return cuda_status(launch_exact(M, N, K, A, lda, B, ldb, C, ldc, semiring, variant, stream));
}

size_t pn_apsp_workspace_size(int64_t n, const pn_opts* opts) {
  if (!opts_valid(opts) || !dims_ok(n, n, n)) return 0;
  const size_t x_bytes = align_up(sizeof(float) * n * n, IMG_ALIGN);
  // like pn_workspace_size: with tile_n = 0 large enough for either width the
  // autotuner may pick later
  return x_bytes + pn_workspace_size(n, n, n, opts);
}

pn_status apsp_pnorm(int64_t n, const float* W, int64_t ldw, float* D, int64_t ldd,
                     int32_t n_squarings, const pn_opts* opts, void* ws, size_t ws_bytes,
                     void* stream) {
  if (!opts_valid(opts) || !dims_ok(n, n, n)) return PN_EINVAL;
  if (opts->estimator != 0 || opts->correction != 0) return PN_EUNSUPPORTED;
  if (n == 0) return PN_OK;
  if (!W || !D || ldw < n || ldd < n) return PN_EINVAL;
  const size_t need = pn_apsp_workspace_size(n, opts);
  if (!ws || ws_bytes < need) return PN_EWORKSPACE;
  if (reinterpret_cast<uintptr_t>(ws) % WS_ALIGN) return PN_EALIGN;
  const int sms = device_sms();
  if (sms <= 0) return PN_EUNSUPPORTED;
  int T = n_squarings;
  if (T <= 0) {
    T = 0;
    while (((int64_t)1 << T) < n) ++T;
  }
  uint8_t* wsb = static_cast<uint8_t*>(ws);
  float* X = reinterpret_cast<float*>(wsb);
  uint8_t* pws = wsb + align_up(sizeof(float) * n * n, IMG_ALIGN);
  if (launch_apsp_init(n, W, ldw, X, opts->diag_policy, opts->dev_status, stream)) return PN_ECUDA;
  // ping-pong between the workspace copy X (ld n) and the output D (ld ldd)
  float* src = X;
  int64_t lds = n;
  float* dst = D;
  int64_t ldt = ldd;
  pn_opts o = *opts;
  for (int t = 0; t < T; ++t) {
    if (t > 0) o.ev_gemm_begin = o.ev_gemm_end = nullptr;
    // the diagonal reset / clamp of diag_policy is applied by the epilogue
    const pn_status st = run_pnorm(n, n, n, src, lds, src, lds, dst, ldt, nullptr, nullptr, &o,
                                   pws, stream, sms, opts->diag_policy);
    if (st != PN_OK) return st;
    float* tp = src; src = dst; dst = tp;
    const int64_t tl = lds; lds = ldt; ldt = tl;
  }
  if (launch_apsp_final(n, src, lds, D, ldd, stream)) return PN_ECUDA;
  return PN_OK;
}

size_t pn_backward_workspace_size(int64_t M, int64_t N, int64_t K, const pn_opts* opts) {
  if (!opts_valid(opts) || !dims_ok(M, N, K) || !bw_mode_ok(opts->compute)) return 0;
  return make_bw_layout(M, N, K, opts).total;
}

pn_status maxprod_pnorm_backward(int64_t M, int64_t N, int64_t K, const float* A,
                                 const float* B, const float* C, const float* S_sel,
                                 const uint8_t* p_sel, const float* dC, float* dA, float* dB,
                                 const pn_opts* opts, void* ws, size_t ws_bytes, void* stream) {
  if (!opts_valid(opts) || !dims_ok(M, N, K)) return PN_EINVAL;
  if (!bw_mode_ok(opts->compute) || opts->estimator != 0 || opts->correction != 0)
    return PN_EUNSUPPORTED;
  if (K == 0) return PN_OK;  // dA and dB are empty
  if ((M > 0 && !dA) || (N > 0 && !dB)) return PN_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (M == 0 || N == 0) {
    // no output entry depends on the other operand: the gradient is zero
    if (M > 0 && cudaMemsetAsync(dA, 0, sizeof(float) * M * K, s)) return PN_ECUDA;
    if (N > 0 && cudaMemsetAsync(dB, 0, sizeof(float) * K * N, s)) return PN_ECUDA;
    return PN_OK;
  }
  if (!A || !B || !C || !S_sel || !p_sel || !dC) return PN_EINVAL;
  const BwLayout L = make_bw_layout(M, N, K, opts);
  if (!ws || ws_bytes < L.total) return PN_EWORKSPACE;
  if (reinterpret_cast<uintptr_t>(ws) % WS_ALIGN) return PN_EALIGN;
  const int sms = device_sms();
  if (sms <= 0) return PN_EUNSUPPORTED;
  uint8_t* w = static_cast<uint8_t*>(ws);

  // scales of the forward operands (same rule as maxprod_pnorm)
  const Layout FL = make_layout(M, N, K, opts);
  Common fw;
  fill_common(fw, FL, M, N, K, A, K, B, N, nullptr, N, nullptr, nullptr, opts, w);
  fw.rmax = reinterpret_cast<uint32_t*>(w + L.off_rmax);
  fw.cmax = reinterpret_cast<uint32_t*>(w + L.off_cmax);
  fw.gmax = reinterpret_cast<uint32_t*>(w + L.off_gmax);
  fw.r = reinterpret_cast<float*>(w + L.off_r);
  fw.c = reinterpret_cast<float*>(w + L.off_c);
  uint32_t* mask = reinterpret_cast<uint32_t*>(w + L.off_mask);
  if (cudaMemsetAsync(w, 0, L.ctrl_bytes, s)) return PN_ECUDA;
  if (launch_maxes(fw, stream)) return PN_ECUDA;
  if (launch_scales(fw, stream)) return PN_ECUDA;
  if (launch_bw_mask(p_sel, M * N, opts->p_log2, opts->n_p, mask, stream)) return PN_ECUDA;

  // G1: dA (M x K) = W^(p) (M x N) . B'^p^T, contraction over N
  Common g1;
  std::memset(&g1, 0, sizeof(g1));
  {
    Prob& P = g1.single;
    P.A = A; P.lda = K; P.C = dA; P.ldc = K;
    P.M = static_cast<int32_t>(M); P.N = static_cast<int32_t>(K); P.K = static_cast<int32_t>(N);
    P.KB = L.KB1; P.RBA = L.RB1a; P.RBB = L.RB1b;
    P.tiles_m = static_cast<int32_t>(ceil_div(M, TILE_M));
    P.tiles_n = static_cast<int32_t>(ceil_div(K, L.BN));
    P.a_plane = static_cast<int64_t>(L.plane_w1);
    P.b_plane = static_cast<int64_t>(L.plane_b1);
    P.vec_c = (K % 4 == 0) && (reinterpret_cast<uintptr_t>(dA) % 16 == 0) &&
              (reinterpret_cast<uintptr_t>(A) % 16 == 0);
    g1.total_tiles = (L.cg == 2 ? (P.tiles_m + 1) / 2 : P.tiles_m) * P.tiles_n;
  }
  // G2: dB (K x N) = A'^p^T (K x M) . W^(p), contraction over M
  Common g2;
  std::memset(&g2, 0, sizeof(g2));
  {
    Prob& P = g2.single;
    P.A = B; P.lda = N; P.C = dB; P.ldc = N;
    P.M = static_cast<int32_t>(K); P.N = static_cast<int32_t>(N); P.K = static_cast<int32_t>(M);
    P.KB = L.KB2; P.RBA = L.RB2a; P.RBB = L.RB2b;
    P.tiles_m = static_cast<int32_t>(ceil_div(K, TILE_M));
    P.tiles_n = static_cast<int32_t>(ceil_div(N, L.BN));
    P.a_plane = static_cast<int64_t>(L.plane_a2);
    P.b_plane = static_cast<int64_t>(L.plane_w2);
    P.vec_c = (N % 4 == 0) && (reinterpret_cast<uintptr_t>(dB) % 16 == 0) &&
              (reinterpret_cast<uintptr_t>(B) % 16 == 0);
    g2.total_tiles = (L.cg == 2 ? (P.tiles_m + 1) / 2 : P.tiles_m) * P.tiles_n;
  }
  for (Common* g : {&g1, &g2}) {
    g->nprob = 1;
    g->cg = L.cg;
    g->mode = opts->compute;
    g->BN = L.BN;
    g->r = fw.r;
    g->c = fw.c;
    g->status = opts->dev_status;
    g->timeout_ns = fw.timeout_ns;
    g->debug_flags = 0;
    g->unscale = 1.0f;
  }
  g1.grad_axis = 0;
  g2.grad_axis = 1;

  for (int q = opts->n_p - 1; q >= 0; --q) {
    const int plog = opts->p_log2[q];
    BwImage im;
    std::memset(&im, 0, sizeof(im));
    im.plog = plog; im.q = q; im.pmask = mask;
    im.dC = dC; im.Cv = C; im.S = S_sel; im.psel = p_sel;
    // W^(p) rows (i, contraction j) and B'^p rows (k, contraction j)
    im.kind = 1; im.trans = 0; im.srows = static_cast<int32_t>(M); im.scols = static_cast<int32_t>(N);
    im.dst = w + L.off_w1; im.plane = static_cast<int64_t>(L.plane_w1); im.RB = L.RB1a; im.KB = L.KB1;
    if (launch_bw_image(opts->compute, im, stream)) return PN_ECUDA;
    im.kind = 0; im.trans = 0; im.src = B; im.lds = N; im.scale = fw.c;
    im.srows = static_cast<int32_t>(K); im.scols = static_cast<int32_t>(N);
    im.dst = w + L.off_b1; im.plane = static_cast<int64_t>(L.plane_b1); im.RB = L.RB1b; im.KB = L.KB1;
    if (launch_bw_image(opts->compute, im, stream)) return PN_ECUDA;
    // A'^p transposed (k, contraction i) and W^(p) transposed (j, contraction i)
    im.kind = 0; im.trans = 1; im.src = A; im.lds = K; im.scale = fw.r;
    im.srows = static_cast<int32_t>(M); im.scols = static_cast<int32_t>(K);
    im.dst = w + L.off_a2; im.plane = static_cast<int64_t>(L.plane_a2); im.RB = L.RB2a; im.KB = L.KB2;
    if (launch_bw_image(opts->compute, im, stream)) return PN_ECUDA;
    im.kind = 1; im.trans = 1; im.src = nullptr; im.scale = nullptr;
    im.srows = static_cast<int32_t>(M); im.scols = static_cast<int32_t>(N);
    im.dst = w + L.off_w2; im.plane = static_cast<int64_t>(L.plane_w2); im.RB = L.RB2b; im.KB = L.KB2;
    if (launch_bw_image(opts->compute, im, stream)) return PN_ECUDA;

    Level lv;
    std::memset(&lv, 0, sizeof(lv));
    lv.q = q; lv.plog = plog; lv.is_top = 1; lv.is_bottom = 1; lv.pmask = mask;
    lv.a_level = w + L.off_w1; lv.b_level = w + L.off_b1;
    if (launch_gemm_grad(g1, lv, sms, stream)) return PN_ECUDA;
    lv.a_level = w + L.off_a2; lv.b_level = w + L.off_w2;
    if (launch_gemm_grad(g2, lv, sms, stream)) return PN_ECUDA;
  }
  return PN_OK;
}

}  // extern "C"
