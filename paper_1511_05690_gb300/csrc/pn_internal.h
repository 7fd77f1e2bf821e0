// Internal types shared by the host runtime and the kernels of the p-norm
// semiring library.  Not part of the public ABI (see include/pnorm.h).
#pragma once
#include <cstddef>
#include <cstdint>

#include "../../include/pnorm.h"

namespace pn {

constexpr int TILE_M = 128;         // output rows per tensor-core tile (MMA M)
constexpr int IMG_BYTES = 16384;    // one operand tile image: 128 rows x 128 bytes
constexpr int IMG_ROW_BYTES = 128;  // bytes of K per image row (one 128-byte swizzle row)
constexpr int RASTER_GM = 16;       // tile rows per raster group (L2 reuse of B)
constexpr int MAXSEG_A = 1024;      // columns of A per max-pass unit
constexpr int MAXSEG_B = 256;       // rows of B per max-pass unit

// Operand formats of the tensor-core path (values equal pn_compute).
enum Mode : int32_t { MODE_3XTF32 = 0, MODE_TF32 = 1, MODE_BF16 = 2, MODE_F16 = 3, MODE_E4M3 = 4 };

__host__ __device__ constexpr int mode_elem_bytes(int mode) {
  return mode == MODE_E4M3 ? 1 : (mode == MODE_BF16 || mode == MODE_F16) ? 2 : 4;
}
// K elements per 128-byte image row.
__host__ __device__ constexpr int mode_bk(int mode) { return IMG_ROW_BYTES / mode_elem_bytes(mode); }
__host__ __device__ constexpr int mode_planes(int mode) { return mode == MODE_3XTF32 ? 2 : 1; }
// Exponent s of the power-of-two factor 2^s applied to powered operands.
__host__ __device__ constexpr int mode_op_shift(int mode) {
  return mode == MODE_F16 ? 15 : mode == MODE_E4M3 ? 8 : 0;
}

// One (x,max) product problem and where its pieces live in the workspace.
struct Prob {
  const float* A;
  const float* B;
  float* C;
  uint8_t* psel;  // nullable
  float* Ssel;    // nullable
  int64_t lda, ldb, ldc, ldaux;
  int32_t M, N, K;
  int32_t KB;               // k-blocks of mode_bk(mode) elements
  int32_t RBA, RBB;         // 128-row blocks of the A image / of the B^T image
  int32_t tiles_m, tiles_n; // output tiles (128 x BN)
  int32_t tile_base;        // first global tile id of this problem
  int32_t xa_base, xb_base; // first global operand-tile id (RBA*KB / RBB*KB per problem)
  int32_t tm_base, tn_base; // offsets into per-level row / column flag arrays
  int32_t KMA, KMB;         // max-pass segments: 1024 columns of A / 256 rows of B
  int32_t ma_base, mb_base; // first global max-pass unit (RBA*KMA / RBB*KMB per problem)
  int32_t vec_c;            // C, p_sel, S_sel rows allow 16-byte vector stores
  int32_t state_ld;         // 32-bit state words per row (tiles_n * BN / 32)
  int64_t a_img, b_img;     // byte offsets inside one level's A / B image region
  int64_t a_plane, b_plane; // bytes of one image plane (the 3xTF32 lo plane follows hi)
  int64_t rc_r, rc_c;       // element offsets into the row / column scale arrays
  int64_t state_off;        // word offset into the state array
  float tau;
  float pad0;
  double tau_d;
};

// Everything a launch needs besides the per-level control.
struct Common {
  const Prob* probs;  // device table (grouped) or nullptr
  // grouped: problem index of every global id, per id space (tiles, A operand
  // tiles, B operand tiles, tile rows, tile columns, A / B max-pass units)
  const int32_t* lut[7];
  Prob single;        // the problem when nprob == 1
  int32_t nprob;
  int32_t total_tiles, total_xa, total_xb;
  int32_t total_tm, total_tn;  // tile rows / tile columns summed over problems
  int32_t total_ma, total_mb;  // max-pass units summed over problems
  int32_t mode, BN, s_op, scaling;
  float unscale;      // 2^(-2 s_op)
  int32_t cg;         // 2: a CTA pair (cta_group::2) per 256 x BN tile, total_tiles counts pairs
  uint32_t* rmax;     // per-row max of A (float bits)
  uint32_t* cmax;     // per-column max of B
  uint32_t* gmax;     // per-problem global max of A (2g) and B (2g+1)
  float* r;           // row scales
  float* c;           // column scales
  uint32_t* state;    // resolved-entry bits of tiles that go to a lower level
  uint32_t* pend;     // r = 1 projection: bits of entries resolved at the level
                      // above whose C holds S^(2p) (same layout as state), or null;
                      // r = 2 projection: bit 0 of each entry's pending stage
  uint32_t* pend2;    // r = 2 projection: bit 1 of the pending stage, or null
  float* park;        // r = 2 projection: S^(3p*/4) (M x N), then S^(p*/2) (M x N)
  float r2_eta;       // r = 2 projection: resolution margin, 32 u of the operand format
  int32_t* status;
  uint64_t timeout_ns;
  int32_t debug_flags;
  int32_t n_levels;
  int32_t fp64_near;  // FP64 selection/root for entries with S < 10 tau (FP32-range formats)
  int32_t grad_axis;  // gradient epilogue: 0 = scale per output row (r), 1 = per column (c)
  int32_t post;       // APSP squaring: 1 = C_ii = 1, 2 = also C = min(C, 1)
  int32_t corr;       // bias correction: 0 none, 1 divide by K^(1/p*), 2 affine per p* class
  const float* coef;  // correction 2: (a_q, b_q) per level q of P, device
};

// Sample entries and class sums of the affine correction (pn_correct.cu).
struct FitArgs {
  const int32_t* fi;
  const int32_t* fj;
  int32_t n_fit;
  int32_t n_p;
  int32_t p_log2[PN_MAX_P];
  int32_t estimator;
  int32_t pad;
  double* samp;       // [n_fit][2]: each sample's estimate and exact value
  int32_t* scls;      // [n_fit]: each sample's p* class (-1: entry outside the product)
  float* coef;        // [PN_MAX_P][2]
  float* user_coef;   // optional copy for the caller
};

// Control of one p level (one p of the family).
struct Level {
  int32_t q;          // index into P (0 = smallest p)
  int32_t plog;       // log2 p
  int32_t is_top;     // largest p: every tile, nothing resolved yet
  int32_t is_bottom;  // smallest p: resolve every entry that is left
  uint8_t* a_level;   // this level's A image region
  uint8_t* b_level;   // this level's B image region
  const int32_t* work;        // tiles of this level (ignored at the top)
  const int32_t* work_count;
  int32_t* next_work;         // tiles pushed to the next lower level
  int32_t* next_count;
  const uint8_t* rflag;       // this level's needed A row blocks (not at top)
  const uint8_t* cflag;       // this level's needed B column tiles (not at top)
  uint8_t* next_rflag;
  uint8_t* next_cflag;
  const uint32_t* pmask;      // gradient launches: bit q set if some entry has p* = P[q]
  uint32_t* pair_pushed;      // CTA pairs: one word per pair tile, set once the tile is
                              // pushed to the next level (either half may push it)
  int32_t proj_here;          // r = 1 projection: finish entries resolved at 2p (the level above)
  int32_t proj_next;          // r = 1 projection: the next level is p/2; park S^(p) of new entries
  // r = 2 projection.  A pending entry's 2-bit stage s (planes pend, pend2)
  // names the sum it waits for: 1 = S^(3p*/4), 2 = S^(p*/2), 3 = S^(p*/4).
  int32_t half;               // extra level p = 1.5 * 2^plog (= 3p/4 of the level above): no
                              // entry resolves here, stage-1 entries park S^(p)
  int32_t r2_new;             // entries resolving here start a chain (C keeps S^(p*), stage 1)
  int32_t r2_state;           // pending stages are read and written at this level
  // With r2_new the next slot is the half level 3p/4, which only entries
  // resolved here need: tiles that start no chain skip it and go to the
  // slot after it (the next p of P) through these lists.
  int32_t* skip_work;
  int32_t* skip_count;
  uint8_t* skip_rflag;
  uint8_t* skip_cflag;
};

// One persistent grouped launch (k_grouped_persist): the levels of the
// schedule in slot order (largest p first) and the cross-CTA control words.
// Operand blocks: A row blocks are the tile rows (global ids 0 .. n_a - 1),
// B column blocks the tile columns (ids n_a .. n_a + n_b - 1).
struct GroupedRun {
  Level lv[PN_MAX_P];
  int32_t n_slots;
  int32_t n_a, n_b;
  int32_t maxima;        // top level: maxima and domain test in the block builders
  int32_t top_built;     // the top level's images were written before the launch
  int32_t plain;         // plain estimator, no affine line: the epilogue without those paths
  int32_t* ready;        // [n_a + n_b]: slot + 1 once the block's images of that slot are written
  int32_t* level_done;   // [n_slots]: CTAs that finished the slot
};

// The level schedule: every p of P from the largest down, each followed --
// for the r = 2 projection (estimator 2) -- by an extra "half" level at
// 3p/4 when p/2 and p/4 are the two p below it in P.  Slot t runs level
// (q[t], half[t]); its work list, counts and flags are slot t's.
struct Schedule {
  int n;
  int8_t q[2 * PN_MAX_P];
  int8_t half[2 * PN_MAX_P];
};
inline Schedule make_schedule(const pn_opts* o) {
  Schedule s;
  s.n = 0;
  for (int q = o->n_p - 1; q >= 0; --q) {
    s.q[s.n] = static_cast<int8_t>(q);
    s.half[s.n++] = 0;
    if (o->estimator == 2 && q >= 2 && o->p_log2[q - 1] == o->p_log2[q] - 1 &&
        o->p_log2[q - 2] == o->p_log2[q] - 2) {
      s.q[s.n] = static_cast<int8_t>(q);
      s.half[s.n++] = 1;
    }
  }
  return s;
}

// One operand image of the adjoint (maxprod_pnorm_backward).
//   kind 0: (src / scale)^p with one scale per contraction index
//   kind 1: W^(p) = dC * C / S where p_sel == p, else 0
//   trans 0: image row r = source row r, contraction = source column
//   trans 1: image row r = source column r, contraction = source row
struct BwImage {
  const float* src;
  int64_t lds;
  int32_t srows, scols;
  const float* scale;
  const float* dC;
  const float* Cv;
  const float* S;
  const uint8_t* psel;
  uint8_t* dst;
  int64_t plane;           // bytes to the lo plane (3xTF32)
  int32_t RB, KB;          // image row blocks (128 rows), contraction blocks
  int32_t plog, q;
  const uint32_t* pmask;
  int32_t kind, trans;
};

__host__ __device__ inline const Prob& prob_at(const Common& cm, int g) {
  return cm.nprob == 1 ? cm.single : cm.probs[g];
}

// Problem index owning global id `id` in id space `which` (0 tiles, 1 A
// operand tiles, 2 B operand tiles, 3 tile rows, 4 tile columns, 5 A max
// units, 6 B max units): a table lookup for groups.
__host__ __device__ inline int find_prob(const Common& cm, int id, int which) {
  if (cm.nprob == 1) return 0;
  return cm.lut[which][id];
}

// Local tile index -> (tile row, tile column), grouped raster order: groups
// of `group_m` tile rows (RASTER_GM for 128-row tiles; a CTA pair's 256-row
// tiles use half as many, so that a group covers the same rows of A).
__host__ __device__ inline void raster(int lt, int tiles_m, int tiles_n, int& tm, int& tn,
                                       int group_m = RASTER_GM) {
  const int group = group_m * tiles_n;
  const int g = lt / group;
  const int first_m = g * group_m;
  const int gm = (tiles_m - first_m) < group_m ? (tiles_m - first_m) : group_m;
  const int local = lt - g * group;
  tm = first_m + local % gm;
  tn = local / gm;
}

// --------------------------------------------------------- host helpers ---
// r = 1 projection flags of level q (estimator 1, Sec. 2.1): level q finishes
// the entries resolved at the level above when that level's p is 2p, and
// parks S^(p) of the entries it resolves when the level below is p/2.
inline void set_projection(Level& lv, const pn_opts* o, int q) {
  const bool proj = o->estimator == 1;
  lv.proj_next = (proj && q > 0 && o->p_log2[q - 1] == o->p_log2[q] - 1) ? 1 : 0;
  lv.proj_here = (proj && q + 1 < o->n_p && o->p_log2[q + 1] == o->p_log2[q] + 1) ? 1 : 0;
}

int host_device_sms();                      // SMs of the current sm_103 device, else 0
bool host_opts_valid(const pn_opts* o);
double host_default_tau(int64_t K, int compute);
float host_tau_up(double t);                // smallest float >= t
int host_tuned_bn(int mode, int64_t M, int64_t N, int64_t K);  // autotune cache, 0 if none

// Launch with programmatic stream serialisation (the kernel must call
// pdl_wait() before it touches global memory): its CTAs may be scheduled as
// soon as every CTA of the previous kernel has called pdl_trigger().
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              void* stream, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = static_cast<cudaStream_t>(stream);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// ------------------------------------------------------------ launchers ---
// All return a cudaError_t value as int (0 = success).
// Tensor maps (CUtensorMap, 128 opaque bytes) of the FP32 operands of a
// single product, for the top-level image kernels; has_a / has_b are 0 when
// the operand's rows are not 16-byte aligned or the driver's encoder is not
// available (the per-tile kernels are used then).
struct alignas(64) TensorMapBytes {
  uint64_t w[16];
};
struct OperandMaps {
  TensorMapBytes a, b;
  int32_t has_a, has_b;
};
// Tensor maps over the A and B operand-image regions of a CTA-pair launch:
// each region as rows of 128 bytes (one image block = 128 rows), copied
// unswizzled (the blocks are stored in their shared-memory layout).
struct ImgMaps {
  TensorMapBytes a, b;
};
struct NoMaps {};
// Encodes a region of `bytes` bytes (a multiple of 128, base 16-byte aligned)
// as a 2-D tensor of 128-byte rows with boxes of box_rows x 128 bytes; false
// if the driver's encoder is unavailable or the region is out of range.
bool encode_img_rows(TensorMapBytes& out, const void* base, int64_t bytes, int box_rows = 128);
void make_operand_maps(const Common& cm, OperandMaps& maps);

int launch_maxes(const Common& cm, void* stream);
// Grouped top level (scaling 0 or 2): maxima, domain test, scales and images
// of every operand block in one launch (a CTA per 32-row / 32-column strip).
int launch_strips(const Common& cm, const Level& lv, void* stream);
int launch_power_a(const Common& cm, const Level& lv, void* stream,
                   const OperandMaps* maps = nullptr);
int launch_power_b(const Common& cm, const Level& lv, void* stream,
                   const OperandMaps* maps = nullptr);
int launch_gemm_level(const Common& cm, const Level& lv, int num_sms, void* stream);
int launch_exact(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, const float* B,
                 int64_t ldb, float* C, int64_t ldc, int semiring, int variant, void* stream);
int launch_fill_empty(const Common& cm, int plog0, void* stream);
int launch_apsp_init(int64_t n, const float* W, int64_t ldw, float* X, int diag, int32_t* status,
                     void* stream);
int launch_apsp_final(int64_t n, const float* X, int64_t ldx, float* D, int64_t ldd,
                      void* stream);
int launch_gemm_grad(const Common& cm, const Level& lv, int num_sms, void* stream);
int launch_fit(const Common& cm, const FitArgs& fa, void* stream);

// Batched max-convolution problems (pn_maxconv.cu).
struct MaxconvArgs {
  const float* x;
  const float* y;
  float* z;
  uint8_t* psel;
  int64_t ldx, ldy, ldz, ldp;
  int64_t batch;
  int32_t nx, ny, nz;
  int32_t logN;        // FFT length 2^logN >= nz
  int32_t n_p;
  int32_t p_log2[PN_MAX_P];
  double tau;
  int32_t* status;
};
constexpr int MAXCONV_LOG_NMAX = 13;  // FFT length of the shared-memory kernel, at most
int maxconv_fft_smem_bytes(int logN);
int maxconv_exact_smem_bytes();
int launch_maxconv_fft(const MaxconvArgs& ma, void* stream);
int launch_maxconv_exact(const MaxconvArgs& ma, void* stream);
int launch_bw_mask(const uint8_t* psel, int64_t count, const int32_t* plog_list, int n_p,
                   uint32_t* mask, void* stream);
int launch_scales(const Common& cm, void* stream);
int launch_bw_image(int mode, const BwImage& im, void* stream);
int gemm_smem_bytes(int mode, int BN);
// Persistent grouped launch: every level of a group in one cooperative launch
// (returns a cudaError_t value).
int launch_grouped_persist(const Common& cm, const GroupedRun& gr, int num_sms, void* stream);
int gemm_stages(int mode, int BN);

}  // namespace pn
