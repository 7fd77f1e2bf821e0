// Grouped products and the tile-width autotuner.
//
// Grouped: many independent (x,max) products evaluated together (the problems
// and the p rings parallelise coarsely, Sec. 4): the maxima and the top
// level's operand images in two image kernels, then every level of every
// problem in one persistent tensor-core launch (pn_grouped_kernel.cuh); the
// global scale of scaling 1 keeps one launch sequence per level.  Every kernel of the
// product works on global ids (operand tile, output tile, tile row / column,
// max-pass unit); a group is a table of Prob records with running offsets
// into one shared workspace, plus id -> problem lookup tables so that a kernel
// finds the problem of an id with one load.  The table is built on the host
// and copied to the device by the caller once; the run step then only launches kernels and can
// be captured in a CUDA graph.  The table holds two layouts, for 128- and
// 256-wide output tiles, so the autotuner can time both on the same buffers.
//
// Autotuner: times the candidate tile widths of a product (or of a group) with
// CUDA events and keeps the fastest per device and shape class; calls with
// tile_n = 0 then use it.
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "pn_internal.h"
#include <cuda_runtime.h>

namespace pn {

namespace {

constexpr uint64_t GROUP_MAGIC = 0x3250524750504e50ull;  // "PNPPGRP2"
constexpr size_t WS_ALIGN = 256;
constexpr size_t IMG_ALIGN = 1024;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

struct GroupLayout {
  int32_t BN, total_tiles, total_xa, total_xb, total_tm, total_tn, total_ma, total_mb;
  uint64_t off_rmax, off_cmax, off_gmax, off_counts, off_rflag, off_cflag, off_ready, off_ldone,
      ctrl_bytes;
  uint64_t off_r, off_c, off_work, off_state, off_pend, off_aimg, off_bimg, total;
  uint64_t probs_offset;  // bytes from the table start to this layout's Prob[count]
  uint64_t lut_offset[7]; // bytes from the table start to each id -> problem table
};

// Id counts of a layout (tile width BN): tiles, A tiles, B tiles, tile rows,
// tile columns, A max units, B max units.
void id_counts(int32_t count, const int64_t* MNK, int mode, int BN, int64_t out[7]) {
  const int bk = mode_bk(mode);
  for (int w = 0; w < 7; ++w) out[w] = 0;
  for (int32_t g = 0; g < count; ++g) {
    const int64_t M = MNK[3 * g], N = MNK[3 * g + 1], K = MNK[3 * g + 2];
    if (M <= 0 || N <= 0) continue;
    const int64_t tm = ceil_div(M, TILE_M), tn = ceil_div(N, BN), KB = ceil_div(K, bk);
    const int64_t rbb = tn * (BN / TILE_M);
    out[0] += tm * tn;
    out[1] += tm * KB;
    out[2] += rbb * KB;
    out[3] += tm;
    out[4] += tn;
    out[5] += tm * ceil_div(K, MAXSEG_A);
    out[6] += rbb * ceil_div(K, MAXSEG_B);
  }
}

struct GroupHeader {
  uint64_t magic;
  int32_t count, n_p, mode, scaling;
  int32_t estimator, pad;
  uint64_t signature;  // of the sizes, for the autotune cache
  int64_t sum_cube;    // sum of M*N*K over the problems
  GroupLayout layout[2];
};

size_t table_bytes(int32_t count, const int64_t* MNK, int mode) {
  size_t b = align_up(sizeof(GroupHeader), 64) + 2 * static_cast<size_t>(count) * sizeof(Prob);
  for (int l = 0; l < 2; ++l) {
    int64_t ids[7];
    id_counts(count, MNK, mode, (mode == MODE_3XTF32 || l == 0) ? 128 : 256, ids);
    for (int w = 0; w < 7; ++w) b += align_up(sizeof(int32_t) * static_cast<size_t>(ids[w]), 16);
  }
  return b;
}

// -------------------------------------------------------------- autotune ---
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int>, int> g_tune_single;  // dev, mode, lgM, lgN, lgK
std::map<std::tuple<int, int, uint64_t>, int> g_tune_group;        // dev, mode, signature

int lg(int64_t x) {
  int b = 0;
  while ((int64_t(1) << b) < x) ++b;
  return b;
}

int current_device() {
  int d = 0;
  cudaGetDevice(&d);
  return d;
}

// Average milliseconds of `reps` runs of fn on the stream (after one warm-up).
template <class F>
float time_ms(F fn, cudaStream_t s, int reps, pn_status* st) {
  *st = fn();
  if (*st != PN_OK) return 0.0f;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaEventRecord(a, s);
  for (int i = 0; i < reps && *st == PN_OK; ++i) *st = fn();
  cudaEventRecord(b, s);
  cudaEventSynchronize(b);
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms / reps;
}

}  // namespace

int grouped_persist_f16(const Common& cm, const GroupedRun& gr, int sms, void* stream);
int grouped_persist_tf32(const Common& cm, const GroupedRun& gr, int sms, void* stream);
int grouped_persist_f8(const Common& cm, const GroupedRun& gr, int sms, void* stream);

int launch_grouped_persist(const Common& cm, const GroupedRun& gr, int num_sms, void* stream) {
  switch (cm.mode) {
    case MODE_BF16:
    case MODE_F16: return grouped_persist_f16(cm, gr, num_sms, stream);
    case MODE_TF32:
    case MODE_3XTF32: return grouped_persist_tf32(cm, gr, num_sms, stream);
    case MODE_E4M3: return grouped_persist_f8(cm, gr, num_sms, stream);
    default: return cudaErrorInvalidValue;
  }
}

int host_tuned_bn(int mode, int64_t M, int64_t N, int64_t K) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  const auto it = g_tune_single.find({current_device(), mode, lg(M), lg(N), lg(K)});
  return it == g_tune_single.end() ? 0 : it->second;
}

}  // namespace pn

using namespace pn;

extern "C" {

size_t pn_grouped_table_bytes(int32_t count, const int64_t* MNK, const pn_opts* opts) {
  if (count < 0 || !host_opts_valid(opts) || (count > 0 && !MNK)) return 0;
  for (int32_t g = 0; g < count; ++g)
    for (int t = 0; t < 3; ++t)
      if (MNK[3 * g + t] < 0 || MNK[3 * g + t] >= (int64_t(1) << 30)) return 0;
  return table_bytes(count, MNK, opts->compute);
}

pn_status pn_grouped_build_table(int32_t count, const int64_t* MNK, const float* const* A,
                                 const float* const* B, float* const* C, const pn_opts* opts,
                                 void* host_table, size_t tbytes, size_t* ws_bytes) {
  if (count < 0 || !host_opts_valid(opts) || !host_table) return PN_EINVAL;
  if (count > 0 && (!MNK || !A || !B || !C)) return PN_EINVAL;
  const int mode = opts->compute;
  const int bk = mode_bk(mode), planes = mode_planes(mode);
  uint64_t sig = 1469598103934665603ull;
  int64_t sum_cube = 0;
  for (int32_t g = 0; g < count; ++g) {
    const int64_t M = MNK[3 * g], N = MNK[3 * g + 1], K = MNK[3 * g + 2];
    if (M < 0 || N < 0 || K < 0 || M >= (1 << 30) || N >= (1 << 30) || K >= (1 << 30))
      return PN_EINVAL;
    if (M > 0 && N > 0 && (K == 0 || !A[g] || !B[g] || !C[g])) return PN_EINVAL;
    for (int t = 0; t < 3; ++t) sig = (sig ^ static_cast<uint64_t>(MNK[3 * g + t])) * 1099511628211ull;
    sum_cube += M * N * K;
  }
  if (tbytes < table_bytes(count, MNK, mode)) return PN_EINVAL;
  auto* H = static_cast<GroupHeader*>(host_table);
  std::memset(H, 0, sizeof(GroupHeader));
  H->magic = GROUP_MAGIC;
  H->count = count;
  H->n_p = opts->n_p;
  H->mode = mode;
  H->scaling = opts->scaling;
  H->estimator = opts->estimator;
  H->signature = sig;
  H->sum_cube = sum_cube;
  size_t off_probs = align_up(sizeof(GroupHeader), 64);
  size_t off_lut = off_probs + 2 * static_cast<size_t>(count) * sizeof(Prob);
  size_t need = 0;
  for (int l = 0; l < 2; ++l) {
    GroupLayout& L = H->layout[l];
    L.BN = (mode == MODE_3XTF32 || l == 0) ? 128 : 256;
    L.probs_offset = off_probs + static_cast<size_t>(l) * count * sizeof(Prob);
    Prob* probs = reinterpret_cast<Prob*>(static_cast<uint8_t*>(host_table) + L.probs_offset);
    int64_t tiles = 0, xa = 0, xb = 0, tm = 0, tn = 0, ma = 0, mb = 0, rows = 0, cols = 0,
            words = 0, abytes = 0, bbytes = 0;
    for (int32_t g = 0; g < count; ++g) {
      const int64_t M = MNK[3 * g], N = MNK[3 * g + 1], K = MNK[3 * g + 2];
      Prob& P = probs[g];
      std::memset(&P, 0, sizeof(P));
      const bool empty = M == 0 || N == 0;
      P.A = A[g]; P.B = B[g]; P.C = C[g]; P.psel = nullptr; P.Ssel = nullptr;
      P.lda = K; P.ldb = N; P.ldc = N; P.ldaux = N;
      P.M = empty ? 0 : static_cast<int32_t>(M);
      P.N = empty ? 0 : static_cast<int32_t>(N);
      P.K = static_cast<int32_t>(K);
      P.KB = empty ? 0 : static_cast<int32_t>(ceil_div(K, bk));
      P.tiles_m = static_cast<int32_t>(ceil_div(P.M, TILE_M));
      P.tiles_n = static_cast<int32_t>(ceil_div(P.N, L.BN));
      P.RBA = P.tiles_m;
      P.RBB = P.tiles_n * (L.BN / TILE_M);
      P.KMA = empty ? 0 : static_cast<int32_t>(ceil_div(K, MAXSEG_A));
      P.KMB = empty ? 0 : static_cast<int32_t>(ceil_div(K, MAXSEG_B));
      P.tile_base = static_cast<int32_t>(tiles);
      P.xa_base = static_cast<int32_t>(xa);
      P.xb_base = static_cast<int32_t>(xb);
      P.tm_base = static_cast<int32_t>(tm);
      P.tn_base = static_cast<int32_t>(tn);
      P.ma_base = static_cast<int32_t>(ma);
      P.mb_base = static_cast<int32_t>(mb);
      P.vec_c = (N % 4 == 0) && (reinterpret_cast<uintptr_t>(C[g]) % 16 == 0);
      P.state_ld = P.tiles_n * (L.BN / 32);
      P.a_plane = static_cast<int64_t>(P.RBA) * P.KB * IMG_BYTES;
      P.b_plane = static_cast<int64_t>(P.RBB) * P.KB * IMG_BYTES;
      P.a_img = abytes;
      P.b_img = bbytes;
      P.rc_r = rows;
      P.rc_c = cols;
      P.state_off = words;
      const double tau = opts->tau > 0.0 ? opts->tau : host_default_tau(K, mode);
      P.tau_d = tau;
      P.tau = host_tau_up(tau);
      tiles += static_cast<int64_t>(P.tiles_m) * P.tiles_n;
      xa += static_cast<int64_t>(P.RBA) * P.KB;
      xb += static_cast<int64_t>(P.RBB) * P.KB;
      tm += P.tiles_m;
      tn += P.tiles_n;
      ma += static_cast<int64_t>(P.RBA) * P.KMA;
      mb += static_cast<int64_t>(P.RBB) * P.KMB;
      rows += align_up(P.M, 4);
      cols += align_up(P.N, 4);
      words += static_cast<int64_t>(P.M) * P.state_ld;
      abytes += P.a_plane * planes;
      bbytes += P.b_plane * planes;
    }
    if (tiles >= (int64_t(1) << 31) || xa >= (int64_t(1) << 31) || xb >= (int64_t(1) << 31) ||
        ma >= (int64_t(1) << 31) || mb >= (int64_t(1) << 31))
      return PN_EINVAL;
    // id -> problem lookup tables of this layout
    const int64_t totals[7] = {tiles, xa, xb, tm, tn, ma, mb};
    for (int w = 0; w < 7; ++w) {
      L.lut_offset[w] = off_lut;
      int32_t* lut = reinterpret_cast<int32_t*>(static_cast<uint8_t*>(host_table) + off_lut);
      for (int32_t g = 0; g < count; ++g) {
        const Prob& P = probs[g];
        const int64_t base = w == 0 ? P.tile_base : w == 1 ? P.xa_base : w == 2 ? P.xb_base
                           : w == 3 ? P.tm_base : w == 4 ? P.tn_base : w == 5 ? P.ma_base : P.mb_base;
        const int64_t cnt = w == 0 ? int64_t(P.tiles_m) * P.tiles_n
                          : w == 1 ? int64_t(P.RBA) * P.KB
                          : w == 2 ? int64_t(P.RBB) * P.KB
                          : w == 3 ? P.tiles_m
                          : w == 4 ? P.tiles_n
                          : w == 5 ? int64_t(P.RBA) * P.KMA
                                   : int64_t(P.RBB) * P.KMB;
        for (int64_t e = 0; e < cnt; ++e) lut[base + e] = g;
      }
      off_lut += align_up(sizeof(int32_t) * static_cast<size_t>(totals[w]), 16);
    }
    L.total_tiles = static_cast<int32_t>(tiles);
    L.total_xa = static_cast<int32_t>(xa);
    L.total_xb = static_cast<int32_t>(xb);
    L.total_tm = static_cast<int32_t>(tm);
    L.total_tn = static_cast<int32_t>(tn);
    L.total_ma = static_cast<int32_t>(ma);
    L.total_mb = static_cast<int32_t>(mb);
    size_t off = 0;
    L.off_rmax = off; off += sizeof(uint32_t) * rows;
    L.off_cmax = off; off += sizeof(uint32_t) * cols;
    L.off_gmax = off; off += sizeof(uint32_t) * 2 * static_cast<size_t>(count);
    L.off_counts = off; off += sizeof(int32_t) * PN_MAX_P;
    L.off_rflag = off; off += static_cast<size_t>(opts->n_p) * tm;
    L.off_cflag = off; off += static_cast<size_t>(opts->n_p) * tn;
    // persistent launch: a ready flag per operand block, a counter per level
    off = align_up(off, 4);
    L.off_ready = off; off += sizeof(int32_t) * static_cast<size_t>(tm + tn);
    L.off_ldone = off; off += sizeof(int32_t) * PN_MAX_P;
    L.ctrl_bytes = align_up(off, 16);
    off = align_up(off, WS_ALIGN);
    L.off_r = off; off = align_up(off + sizeof(float) * rows, WS_ALIGN);
    L.off_c = off; off = align_up(off + sizeof(float) * cols, WS_ALIGN);
    L.off_work = off; off = align_up(off + sizeof(int32_t) * opts->n_p * static_cast<size_t>(tiles), WS_ALIGN);
    L.off_state = off; off = align_up(off + sizeof(uint32_t) * static_cast<size_t>(words), IMG_ALIGN);
    L.off_pend = 0;
    if (opts->estimator == 1) {
      L.off_pend = off;
      off = align_up(off + sizeof(uint32_t) * static_cast<size_t>(words), IMG_ALIGN);
    }
    L.off_aimg = off; off += static_cast<size_t>(abytes);
    L.off_bimg = off; off += static_cast<size_t>(bbytes);
    L.total = align_up(off, WS_ALIGN);
    if (L.total > need) need = L.total;
  }
  if (ws_bytes) *ws_bytes = need;
  return PN_OK;
}

// Runs the group with layout l (0: 128-wide tiles, 1: 256-wide).
static pn_status run_group(const GroupHeader* H, const void* dev_table, int l, const pn_opts* o,
                           uint8_t* ws, void* stream, int sms) {
  const GroupLayout& L = H->layout[l];
  Common cm;
  std::memset(&cm, 0, sizeof(cm));
  cm.probs = reinterpret_cast<const Prob*>(static_cast<const uint8_t*>(dev_table) + L.probs_offset);
  for (int w = 0; w < 7; ++w)
    cm.lut[w] = reinterpret_cast<const int32_t*>(static_cast<const uint8_t*>(dev_table) + L.lut_offset[w]);
  cm.nprob = H->count;
  cm.total_tiles = L.total_tiles;
  cm.total_xa = L.total_xa;
  cm.total_xb = L.total_xb;
  cm.total_tm = L.total_tm;
  cm.total_tn = L.total_tn;
  cm.total_ma = L.total_ma;
  cm.total_mb = L.total_mb;
  cm.mode = H->mode;
  cm.BN = L.BN;
  cm.s_op = mode_op_shift(H->mode);
  cm.scaling = H->scaling;
  cm.unscale = std::ldexp(1.0f, -2 * cm.s_op);
  cm.rmax = reinterpret_cast<uint32_t*>(ws + L.off_rmax);
  cm.cmax = reinterpret_cast<uint32_t*>(ws + L.off_cmax);
  cm.gmax = reinterpret_cast<uint32_t*>(ws + L.off_gmax);
  cm.r = reinterpret_cast<float*>(ws + L.off_r);
  cm.c = reinterpret_cast<float*>(ws + L.off_c);
  cm.state = reinterpret_cast<uint32_t*>(ws + L.off_state);
  cm.pend = H->estimator == 1 ? reinterpret_cast<uint32_t*>(ws + L.off_pend) : nullptr;
  cm.corr = o->correction;
  cm.status = o->dev_status;
  cm.timeout_ns = o->timeout_ns > 0 ? static_cast<uint64_t>(o->timeout_ns) : 2000000000ull;
  cm.debug_flags = o->debug_flags;
  cm.n_levels = o->n_p;
  cm.fp64_near = (H->mode == MODE_3XTF32 || H->mode == MODE_TF32 || H->mode == MODE_BF16);
  if (L.total_tiles == 0) return PN_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(ws, 0, L.ctrl_bytes, s)) return PN_ECUDA;
  int32_t* counts = reinterpret_cast<int32_t*>(ws + L.off_counts);
  int32_t* work = reinterpret_cast<int32_t*>(ws + L.off_work);
  uint8_t* rflag = ws + L.off_rflag;
  uint8_t* cflag = ws + L.off_cflag;
  // One persistent launch for every level (scaling 2 and 0: the block
  // builders find each block's maxima themselves); the global scale of
  // scaling 1 needs every block of a problem first, so it keeps one launch
  // per level.  debug_flags bit 2 forces the per-level launches (tests).
  const bool persist = H->scaling != 1 && !(o->debug_flags & 4);
  GroupedRun gr;
  std::memset(&gr, 0, sizeof(gr));
  gr.n_slots = o->n_p;
  gr.n_a = L.total_tm;
  gr.n_b = L.total_tn;
  gr.ready = reinterpret_cast<int32_t*>(ws + L.off_ready);
  gr.level_done = reinterpret_cast<int32_t*>(ws + L.off_ldone);
  // A kernel of one CTA per operand block, several per SM, keeps far more
  // loads in flight than the persistent kernel's eight builder warps per SM,
  // so it writes the maxima and the top level's images (every block) before
  // the persistent launch, which builds only the pushed blocks of the lower
  // levels.  debug_flags bit 3 builds the top level inside the persistent
  // kernel too.
  const bool top_inside = persist && (o->debug_flags & 8);
  gr.maxima = top_inside ? 1 : 0;
  gr.plain = (H->estimator == 0 && o->correction != 2) ? 1 : 0;
  gr.top_built = top_inside ? 0 : 1;
  if (!persist && launch_maxes(cm, stream)) return PN_ECUDA;
  for (int q = o->n_p - 1; q >= 0; --q) {
    const int qn = q > 0 ? q - 1 : 0;
    Level lv;
    std::memset(&lv, 0, sizeof(lv));
    lv.q = q;
    lv.plog = o->p_log2[q];
    lv.is_top = q == o->n_p - 1;
    lv.is_bottom = q == 0;
    lv.a_level = ws + L.off_aimg;
    lv.b_level = ws + L.off_bimg;
    lv.work = work + static_cast<size_t>(q) * L.total_tiles;
    lv.work_count = counts + q;
    lv.next_work = work + static_cast<size_t>(qn) * L.total_tiles;
    lv.next_count = counts + qn;
    lv.rflag = rflag + static_cast<size_t>(q) * L.total_tm;
    lv.cflag = cflag + static_cast<size_t>(q) * L.total_tn;
    lv.next_rflag = rflag + static_cast<size_t>(qn) * L.total_tm;
    lv.next_cflag = cflag + static_cast<size_t>(qn) * L.total_tn;
    set_projection(lv, o, q);
    if (persist) {
      gr.lv[o->n_p - 1 - q] = lv;
      if (lv.is_top && !top_inside && launch_strips(cm, lv, stream)) return PN_ECUDA;
      continue;
    }
    if (launch_power_a(cm, lv, stream)) return PN_ECUDA;
    if (launch_power_b(cm, lv, stream)) return PN_ECUDA;
    if (lv.is_top && o->ev_gemm_begin)
      if (cudaEventRecord(static_cast<cudaEvent_t>(o->ev_gemm_begin), s)) return PN_ECUDA;
    if (launch_gemm_level(cm, lv, sms, stream)) return PN_ECUDA;
    if (lv.is_top && o->ev_gemm_end)
      if (cudaEventRecord(static_cast<cudaEvent_t>(o->ev_gemm_end), s)) return PN_ECUDA;
  }
  if (!persist) return PN_OK;
  // the events bracket the whole persistent launch (every level)
  if (o->ev_gemm_begin && cudaEventRecord(static_cast<cudaEvent_t>(o->ev_gemm_begin), s))
    return PN_ECUDA;
  if (launch_grouped_persist(cm, gr, sms, stream)) return PN_ECUDA;
  if (o->ev_gemm_end && cudaEventRecord(static_cast<cudaEvent_t>(o->ev_gemm_end), s))
    return PN_ECUDA;
  return PN_OK;
}

static pn_status check_group(const void* host_table, const void* dev_table, const pn_opts* o,
                             void* ws, size_t ws_bytes, const GroupHeader** out) {
  if (!host_table || !host_opts_valid(o)) return PN_EINVAL;
  const auto* H = static_cast<const GroupHeader*>(host_table);
  if (H->magic != GROUP_MAGIC || H->n_p != o->n_p || H->mode != o->compute ||
      H->scaling != o->scaling || H->estimator != o->estimator)
    return PN_EINVAL;
  if (H->count > 0 && (!dev_table || reinterpret_cast<uintptr_t>(dev_table) % 16)) return PN_EINVAL;
  const size_t need = H->layout[0].total > H->layout[1].total ? H->layout[0].total : H->layout[1].total;
  if (!ws || ws_bytes < need) return PN_EWORKSPACE;
  if (reinterpret_cast<uintptr_t>(ws) % WS_ALIGN) return PN_EALIGN;
  *out = H;
  return PN_OK;
}

pn_status maxprod_pnorm_grouped(const void* host_table, const void* dev_table,
                                const pn_opts* opts, void* ws, size_t ws_bytes, void* stream) {
  const GroupHeader* H = nullptr;
  const pn_status st = check_group(host_table, dev_table, opts, ws, ws_bytes, &H);
  if (st != PN_OK) return st;
  if (opts->correction == 2) return PN_EUNSUPPORTED;  // sample entries index one product
  if (opts->estimator == 2) return PN_EUNSUPPORTED;
  const int sms = host_device_sms();
  if (sms <= 0) return PN_EUNSUPPORTED;
  int l;
  if (opts->tile_n == 128 || H->mode == MODE_3XTF32) {
    l = 0;
  } else if (opts->tile_n == 256) {
    l = 1;
  } else {
    int tuned = 0;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      const auto it = g_tune_group.find({current_device(), H->mode, H->signature});
      if (it != g_tune_group.end()) tuned = it->second;
    }
    // untuned: 256-wide tiles once the average problem is large
    l = tuned ? (tuned == 256 ? 1 : 0)
              : (H->count > 0 && H->sum_cube / H->count >= (int64_t(512) * 512 * 512) ? 1 : 0);
  }
  return run_group(H, dev_table, l, opts, static_cast<uint8_t*>(ws), stream, sms);
}

pn_status pn_grouped_autotune(const void* host_table, const void* dev_table, const pn_opts* opts,
                              void* ws, size_t ws_bytes, void* stream, int32_t* chosen_tile_n) {
  const GroupHeader* H = nullptr;
  pn_status st = check_group(host_table, dev_table, opts, ws, ws_bytes, &H);
  if (st != PN_OK) return st;
  if (opts->correction == 2 || opts->estimator == 2) return PN_EUNSUPPORTED;
  const int sms = host_device_sms();
  if (sms <= 0) return PN_EUNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int best = 0;
  float best_ms = 0.0f;
  for (int l = 0; l < (H->mode == MODE_3XTF32 ? 1 : 2); ++l) {
    const float ms = time_ms([&] { return run_group(H, dev_table, l, opts, static_cast<uint8_t*>(ws), stream, sms); },
                             s, 3, &st);
    if (st != PN_OK) return st;
    if (l == 0 || ms < best_ms) {
      best = l;
      best_ms = ms;
    }
  }
  const int bn = H->layout[best].BN;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_group[{current_device(), H->mode, H->signature}] = bn;
  }
  if (chosen_tile_n) *chosen_tile_n = bn;
  return PN_OK;
}

pn_status pn_autotune(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                      const float* B, int64_t ldb, float* C, int64_t ldc, const pn_opts* opts,
                      void* ws, size_t ws_bytes, void* stream, int32_t* chosen_tile_n) {
  if (!host_opts_valid(opts)) return PN_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  pn_opts o = *opts;
  o.ev_gemm_begin = o.ev_gemm_end = nullptr;
  // candidates: one CTA per 128 x 128 and per 128 x 256 tile, and a CTA pair
  // per 256 x 256 and per 256 x 128 tile (recorded as 512 and 384); the
  // options may fix some of these
  int best = 0;
  float best_ms = 0.0f;
  for (int c = 0; c < 4; ++c) {
    const int tile_m = c >= 2 ? 256 : 128, tile_n = (c == 0 || c == 3) ? 128 : 256;
    if (opts->tile_m && opts->tile_m != tile_m) continue;
    if (opts->tile_n && opts->tile_n != tile_n) continue;
    if (c == 1 && opts->compute == PN_F32_EXACT) continue;  // one CTA: 128 wide only
    o.tile_m = tile_m;
    o.tile_n = tile_n;
    pn_status st = PN_OK;
    const float ms = time_ms([&] {
      return maxprod_pnorm(M, N, K, A, lda, B, ldb, C, ldc, nullptr, nullptr, &o, ws, ws_bytes, stream);
    }, s, 3, &st);
    if (st != PN_OK) return st;
    if (best == 0 || ms < best_ms) {
      best = c >= 2 ? 256 + tile_n : tile_n;
      best_ms = ms;
    }
  }
  if (best == 0) return PN_EINVAL;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_single[{current_device(), opts->compute, lg(M), lg(N), lg(K)}] = best;
  }
  if (chosen_tile_n) *chosen_tile_n = best;
  return PN_OK;
}

}  // extern "C"
