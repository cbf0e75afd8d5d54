// emc_abi.cu -- the C ABI of include/emc.h: context, workspace layout,
// argument checks and the stream-ordered step calls.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <utility>
#include <vector>

#include "emc_common.cuh"
#include "emc_internal.h"
#include "pixel_groups.h"

using namespace emc;

namespace {

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
  int64_t ld_pix, ld_data, rows, chunk_rows, part_tiles;
  int nrep;  // grid replicas of the fused iterations' compression
  size_t qh, ql, quat, rot, logw, Kb, status, L, bias, lse_m, lse_s, lse2, part_m, part_s, S, P,
      Num, den, gnum, gden, scalar, fbin, finv, cand, ccnt, coff, cent, Sc, Pc, lsec, gk, gauss,
      Kb2, skcnt, skoff, skent, dupsrc, duprank, pixmax, fcn, finvn, fB, kbflag, kbcnt, kblist,
      Kp, perm, perm2, iperm, nsum, nsum_p, cn_p, invn_p, best, lsem_s, lses_s, live, tlist,
      tcount, sortH, sortoff, cgs, cgp, cgqh, cgql, cgqi, cgqlo, cgqf, L2, bias2, Ub, Ub2, Lk, Mk, Mk2, best2,
      osrc, Dd, Cd, bpm, g4, Ua, Ua2, dcand, pflag, plist, flags, qi, qlo, rotfx, epart, total;
  int64_t sort_entries;
  int64_t ntp;  // row tiles rounded up to 128: rows of each half of the bound increments
};

// Gaussian scalars inside the 256-byte block at Layout::gauss
constexpr size_t kGaussMaxOff = 0;    // unsigned: bits of max(grid)
constexpr size_t kGaussNmaxOff = 8;   // unsigned long long: largest frame total
constexpr size_t kGaussScaleOff = 16; // float4: (s, 1/s^2, ps, 1/ps)

size_t score_bytes(int64_t rows, int64_t ld_data) {
  return sizeof(float) * (size_t)(rows + rows / 32) * ld_data;
}

bool is_gauss(const emc_config* c) { return c->model == EMC_MODEL_GAUSSIAN; }
bool is_flu(const emc_config* c) { return c->model == EMC_MODEL_POISSON_FLUENCE; }
// emc_iteration's bound-pruned pass 1 (EMC_FLAG_DENSE_ESTEP clears it)
bool prune_ok(const emc_config* c) {
  return !(c->flags & EMC_FLAG_DENSE_ESTEP) &&
         (c->precision == EMC_PREC_BF16_SPLIT || c->precision == EMC_PREC_FP16_SPLIT) &&
         (c->model == EMC_MODEL_POISSON || c->model == EMC_MODEL_POISSON_FLUENCE);
}
// |S - S_hi| <= n_k / bound_div + 1: the rest below the hi grid is at most 1/16
// (BF16 split, hi on the 1/8 grid) or 1/128 (FP16 split, hi on the 1/64 grid)
float bound_div(const emc_config* c) { return c->precision == EMC_PREC_FP16_SPLIT ? 128.f : 16.f; }
// Poisson-fluence model: the constant c of L = log(W / B_j) + c, log n_pix on
// the 1/8 grid (L is then the log of W over the slice's mean)
double flu_shift(const emc_config* c) { return rint(8.0 * log((double)c->n_pix)) / 8.0; }

// bytes of L (emc_expand) and P (emc_normalize) for `rows` rotations
size_t L_bytes(const emc_config* c, int64_t rows, int64_t ld_pix) {
  const int p = c->precision;
  const int planes = is_gauss(c) ? 3 : (p == EMC_PREC_BF16_SPLIT ? 3 : (p == EMC_PREC_FP16_SPLIT ? 2 : 1));
  return (size_t)planes * (p == EMC_PREC_FP32 ? 4 : 2) * (size_t)rows * ld_pix;
}
// Gaussian and Poisson-fluence: after the planes, den[rows] (float)
size_t P_plane_bytes(const emc_config* c, int64_t rows, int64_t ld_data) {
  const int p = c->precision;
  return (size_t)(p == EMC_PREC_FP32 ? 1 : 2) * (p == EMC_PREC_FP32 ? 4 : 2) * (size_t)rows * ld_data;
}
size_t P_bytes(const emc_config* c, int64_t rows, int64_t ld_data) {
  return P_plane_bytes(c, rows, ld_data) +
         (is_gauss(c) || is_flu(c) ? align256(sizeof(float) * rows) : 0);
}

int check_config(const emc_config* c) {
  if (!c) return EMC_ERR_ARG;
  if (c->N < 4 || c->N > 1024) return EMC_ERR_ARG;
  if (c->n_pix < 1 || c->n_rot < 1 || c->n_data < 1) return EMC_ERR_ARG;
  if (c->n_pix > (1LL << 24) || c->n_rot > (1LL << 31) || c->n_data > (1LL << 31))
    return EMC_ERR_ARG;
  if (c->precision < EMC_PREC_FP32 || c->precision > EMC_PREC_FP16_SPLIT) return EMC_ERR_ARG;
  if (c->compress_mode != EMC_COMPRESS_DEFERRED && c->compress_mode != EMC_COMPRESS_IDW)
    return EMC_ERR_ARG;
  if (!(c->w_floor > 0.0) || !isfinite(c->w_floor)) return EMC_ERR_ARG;
  if (c->model != EMC_MODEL_POISSON && c->model != EMC_MODEL_GAUSSIAN && !is_flu(c))
    return EMC_ERR_ARG;
  if (is_gauss(c)) {
    if (!(c->sigma > 0.0) || !isfinite(c->sigma)) return EMC_ERR_ARG;
    if (c->precision != EMC_PREC_FP16_SPLIT || !(c->flags & EMC_FLAG_STORE_SCORES) ||
        c->n_cand != 0 || (c->flags & EMC_FLAG_SPARSE_K))
      return EMC_ERR_UNSUPPORTED;
  } else if (is_flu(c)) {
    // one rounded value of log(W / B_j) per element (FP32, FP16 rest, BF16)
    // carries a per-rotation rounding bias that the contraction multiplies by
    // N_k; the three-term split carries log B_j's low part exactly
    if (c->precision != EMC_PREC_BF16_SPLIT) return EMC_ERR_UNSUPPORTED;
  } else if ((c->precision == EMC_PREC_BF16_SPLIT || c->precision == EMC_PREC_FP16_SPLIT) &&
             log(c->w_floor) < (double)kHiMin) {
    return EMC_ERR_UNSUPPORTED;
  }
  if (c->rot_chunk < 0 || (c->flags & ~(EMC_FLAG_STORE_SCORES | EMC_FLAG_SPARSE_K |
                                         EMC_FLAG_WIDE_COUNTS | EMC_FLAG_DENSE_ESTEP)) != 0)
    return EMC_ERR_ARG;
  if ((c->flags & EMC_FLAG_SPARSE_K) && c->n_pix > 65536) return EMC_ERR_UNSUPPORTED;
  if (c->n_cand < 0 || c->n_cand > c->n_rot || c->n_cand > 4096) return EMC_ERR_ARG;
  return EMC_OK;
}

Layout make_layout(const emc_config* c) {
  Layout y;
  const bool wide = (c->flags & EMC_FLAG_WIDE_COUNTS) != 0;
  // pixels, the column of ones, and (wide counts) the duplicate columns
  y.ld_pix = round_up(c->n_pix + 1 + (wide ? kDupCols : 0), 64);
  y.ld_data = round_up(c->n_data, 256);
  y.rows = round_up(c->n_rot, 128);
  y.chunk_rows = c->rot_chunk > 0 ? std::min(round_up(c->rot_chunk, 128), y.rows) : y.rows;
  y.part_tiles = y.rows / 64;
  const int64_t nvox = (int64_t)c->N * c->N * c->N;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align256(o + bytes);
    return at;
  };
  y.qh = take(sizeof(float4) * y.ld_pix);
  y.ql = take(sizeof(float4) * y.ld_pix);
  y.cgs = take(sizeof(int32_t) * (c->n_pix + 1));
  y.cgp = take(sizeof(int32_t) * (c->n_pix + 1));
  y.cgqh = take(sizeof(float4) * (c->n_pix + 1));
  y.cgql = take(sizeof(float4) * (c->n_pix + 1));
  y.cgqi = take(sizeof(int4) * (c->n_pix + 1));
  y.cgqlo = take(sizeof(float4) * (c->n_pix + 1));
  y.cgqf = take(sizeof(float4) * (c->n_pix + 1));
  y.qi = take(sizeof(int4) * y.ld_pix);
  y.qlo = take(sizeof(float4) * y.ld_pix);
  y.quat = take(sizeof(double) * 4 * c->n_rot);
  y.rot = take(sizeof(RotDF) * c->n_rot);
  y.rotfx = take(sizeof(RotFX) * c->n_rot);
  y.epart = take(sizeof(double) * (size_t)expand_tile_slices(y.ld_pix) * y.rows);
  // the model in the corner-pair layout of the expansions' gathers (16 B a voxel;
  // grids up to 256^3, 268 MB)
  y.g4 = c->N <= 256 ? take(sizeof(float4) * (size_t)nvox) : 0;
  y.logw = take(sizeof(double) * c->n_rot);
  y.Kb = take(2 * (size_t)y.ld_data * y.ld_pix);
  y.status = take(256);
  y.L = take(L_bytes(c, y.rows, y.ld_pix));
  y.bias = take(sizeof(double) * y.rows * (is_flu(c) ? 2 : 1));
  y.lse_m = take(sizeof(double) * y.ld_data);
  y.lse_s = take(sizeof(double) * y.ld_data);
  y.lse2 = take(sizeof(float2) * y.ld_data);
  y.part_m = take(sizeof(double) * (size_t)y.part_tiles * y.ld_data);
  y.part_s = take(sizeof(float) * (size_t)y.part_tiles * y.ld_data);
  y.S = (c->flags & EMC_FLAG_STORE_SCORES) ? take(score_bytes(y.rows, y.ld_data)) : 0;
  y.P = take(P_bytes(c, y.chunk_rows, y.ld_data));
  // the sparse update (n_cand > 0) writes Num and den for every rotation at once
  const int64_t num_rows = c->n_cand > 0 ? y.rows : y.chunk_rows;
  y.Num = take(sizeof(float) * (size_t)num_rows * y.ld_pix);
  y.den = take(sizeof(float) * num_rows);
  // replicas spread the reductions into the central voxels every slice crosses;
  // as many as fit 64 MB for both grids, at most 16 (16 measured best at 64^3,
  // 8 and 32 slower; one for large grids)
  y.nrep = (int)std::max<int64_t>(1, std::min<int64_t>(16, (64ll << 20) / (16 * nvox)));
  y.gnum = take(sizeof(double) * nvox * y.nrep);
  y.gden = take(sizeof(double) * nvox * y.nrep);
  y.scalar = take(256);
  y.fbin = take(sizeof(int16_t) * y.ld_pix);
  y.finv = take(sizeof(float) * kFeat);
  const int64_t M = c->n_cand;
  y.cand = M ? take(sizeof(int32_t) * (size_t)y.ld_data * M) : 0;
  y.ccnt = M ? take(sizeof(int32_t) * (size_t)y.rows) : 0;
  y.coff = M ? take(sizeof(int64_t) * (size_t)(y.rows + 1)) : 0;
  y.cent = M ? take(sizeof(int2) * (size_t)c->n_data * M) : 0;
  y.Sc = M ? take(sizeof(double) * (size_t)y.ld_data * M) : 0;
  y.Pc = M ? take(sizeof(float) * (size_t)y.ld_data * M) : 0;
  y.lsec = M ? take(sizeof(double) * (size_t)y.ld_data) : 0;
  y.gk = is_gauss(c) ? take(sizeof(float4) * (size_t)y.ld_data) : 0;
  y.gauss = take(256);
  y.Kb2 = is_gauss(c) ? take(2 * (size_t)y.ld_data * y.ld_pix) : 0;
  const bool sk = (c->flags & EMC_FLAG_SPARSE_K) != 0;
  y.skcnt = sk ? take(sizeof(int32_t) * (size_t)y.ld_data) : 0;
  y.skoff = sk ? take(sizeof(int64_t) * (size_t)(y.ld_data + 1)) : 0;
  y.skent = sk ? take(sizeof(uint32_t) * (size_t)c->n_data * c->n_pix) : 0;
  y.dupsrc = wide ? take(sizeof(int32_t) * kDupCols) : 0;
  y.duprank = wide ? take(sizeof(int32_t) * kDupCols) : 0;
  y.pixmax = wide ? take(sizeof(int32_t) * (size_t)c->n_pix) : 0;
  y.fcn = is_flu(c) ? take(sizeof(double) * (size_t)y.ld_data) : 0;
  y.finvn = is_flu(c) ? take(sizeof(float) * (size_t)y.ld_data) : 0;
  // B_j at rot0 + row for every padded row of an emc_expand block: one tile beyond rows
  y.fB = is_flu(c) ? take(sizeof(double) * (size_t)(y.rows + 128)) : 0;
  // non-zero P blocks of a pass-2 chunk (tensor-core update over those only)
  const bool tc = c->precision != EMC_PREC_FP32;
  const int64_t ctiles = y.chunk_rows / 128, kbs = y.ld_data / 64;
  y.kbflag = tc ? take((size_t)ctiles * kbs) : 0;
  y.kbcnt = tc ? take(sizeof(int32_t) * (size_t)ctiles) : 0;
  y.kblist = tc ? take(sizeof(int32_t) * (size_t)ctiles * kbs) : 0;
  // bound-pruned pass 1: frames in their internal order and the tile bookkeeping
  const bool pr = prune_ok(c);
  const int64_t nmt = y.rows / 128, nnt = y.ld_data / 256;
  // the frame sort's histogram; also the tile lists' per-CTA counts (not live at once)
  y.sort_entries = pr ? std::max(sort_scratch_entries(c->n_data, (int)nmt),
                                 tile_list_scratch_entries(nmt, y.ld_data / 256))
                      : 0;
  y.Kp = pr ? take(2 * (size_t)y.ld_data * y.ld_pix) : 0;
  y.perm = pr ? take(sizeof(int32_t) * (size_t)y.ld_data) : 0;
  y.perm2 = pr ? take(sizeof(int32_t) * (size_t)y.ld_data) : 0;
  y.iperm = pr ? take(sizeof(int32_t) * (size_t)y.ld_data) : 0;
  y.nsum = pr ? take(sizeof(float) * (size_t)y.ld_data) : 0;
  y.nsum_p = pr ? take(sizeof(float) * (size_t)y.ld_data) : 0;
  y.cn_p = pr && is_flu(c) ? take(sizeof(double) * (size_t)y.ld_data) : 0;
  y.invn_p = pr && is_flu(c) ? take(sizeof(float) * (size_t)y.ld_data) : 0;
  y.best = pr ? take(sizeof(int32_t) * (size_t)y.ld_data) : 0;
  y.lsem_s = pr ? take(sizeof(double) * (size_t)y.ld_data) : 0;
  y.lses_s = pr ? take(sizeof(double) * (size_t)y.ld_data) : 0;
  y.live = pr ? take((size_t)nmt * nnt) : 0;
  y.tlist = pr ? take(sizeof(int32_t) * (size_t)nmt * nnt) : 0;
  y.tcount = pr ? take(256) : 0;
  y.sortH = pr ? take(sizeof(int32_t) * (size_t)y.sort_entries) : 0;
  y.sortoff = pr ? take(sizeof(int64_t) * (size_t)(y.sort_entries + 1)) : 0;
  // the incremental bound between consecutive iterations: a second L and bias
  // (the last iteration's stay for the differences), per-tile bounds Ub in the
  // internal frame order (and a copy for reordering), per-frame lower bounds,
  // the last exact maxima, the BF16 increments D and their products C
  y.ntp = round_up(nmt, 128);
  const int64_t npairs = (nmt + 1) / 2;
  y.L2 = pr ? take(L_bytes(c, y.rows, y.ld_pix)) : 0;
  y.bias2 = pr ? take(sizeof(double) * y.rows * (is_flu(c) ? 2 : 1)) : 0;
  y.Ub = pr ? take(sizeof(float) * (size_t)nmt * y.ld_data) : 0;
  y.Ub2 = pr ? take(sizeof(float) * (size_t)nmt * y.ld_data) : 0;
  y.Ua = pr ? take(sizeof(float) * (size_t)nmt * y.ld_data) : 0;
  y.Ua2 = pr ? take(sizeof(float) * (size_t)nmt * y.ld_data) : 0;
  y.Lk = pr ? take(sizeof(double) * (size_t)y.ld_data) : 0;
  y.Mk = pr ? take(sizeof(double) * (size_t)y.ld_data) : 0;
  y.Mk2 = pr ? take(sizeof(double) * (size_t)y.ld_data) : 0;
  y.best2 = pr ? take(sizeof(int32_t) * (size_t)y.ld_data) : 0;
  y.osrc = pr ? take(sizeof(int32_t) * (size_t)y.ld_data) : 0;
  y.Dd = pr ? take(2 * (size_t)(3 * y.ntp) * y.ld_pix) : 0;
  y.Cd = pr ? take(sizeof(float) * (size_t)(3 * y.ntp) * y.ld_data) : 0;
  y.bpm = pr ? take(sizeof(float) * 2 * (size_t)nmt) : 0;
  y.dcand = pr ? take((size_t)nmt * nnt) : 0;
  y.pflag = pr ? take((size_t)npairs * nnt) : 0;
  y.plist = pr ? take(sizeof(int32_t) * (size_t)npairs * nnt) : 0;
  // int32 [0]: the frames changed since the last iteration; [2]: the device
  // status when the last pass 1 ended (non-zero voids the tile bounds)
  y.flags = pr ? take(256) : 0;
  y.total = o;
  return y;
}

#define CU(x)                                      \
  do {                                             \
    if ((x) != cudaSuccess) return EMC_ERR_CUDA;   \
  } while (0)

}  // namespace

struct emc_ctx {
  emc_config cfg;
  Layout lay;
  char* ws;
  size_t ws_bytes;
  Geom geom;
  double* quat;
  const RotDF* rot;
  double* logw;
  uint16_t* Kb;
  int32_t* status;
  uint16_t* Kb2;              // Gaussian: BF16 copy of the frames (the update operand)
  float4* gk;                 // Gaussian per-frame constants
  unsigned* gmax;             // Gaussian: bits of max(grid) of the last emc_expand
  unsigned long long* nmax;   // Gaussian: largest frame total
  float4* gsc;                // Gaussian scales of the last emc_expand
  double* flu_cn;             // Poisson-fluence: per-frame score shift c N_k
  float* flu_invn;            // Poisson-fluence: 1 / N_k (0 for empty frames)
  double* flu_B;              // Poisson-fluence: B_j = sum_i W_ij of the last emc_expand
  double flu_c;               // Poisson-fluence: c of L = log(W / B_j) + c
  bool prune;                 // emc_iteration prunes pass 1 (prune_ok)
  bool perm_valid;            // the internal frame order comes from an iteration
  int32_t* perm;              // internal position -> frame (swapped with perm2)
  int32_t* perm2;
  bool order_pending;         // perm2 holds the order for the next iteration
  bool scores_internal;       // the stored scores are in the internal order (iperm)
  bool last_pruned;           // ... and hold only the live tiles (live flags)
  bool frames_loaded;
  bool cand_loaded;
  bool iterated;              // an emc_iteration ran on the loaded frames
  int lcur;                   // L and bias buffer of the last emc_iteration (pruned contexts)
  bool ub_valid;              // the tile bounds, maxima and best tiles belong to that iteration
  int32_t* best;              // per-frame state in the internal order (swapped with *2)
  int32_t* best2;
  double* Mk;
  double* Mk2;
  float* Ub;
  float* Ub2;
  float* Ua;  // widening gathered since each tile bound's refresh (swapped with Ua2)
  float* Ua2;
  CollectBuf col;   // responsibilities recorded by emc_iteration (emc_set_collect)
  bool collecting;
  bool collected;   // the last emc_iteration recorded into col
  cudaEvent_t ev[8];
  int kernels;  // launches made by the last emc_iteration
  TcCtl tcctl;  // bounded waits of the tensor-core launches (emc_ctx_set_wait_limit)
};

// The internal frame order the last iteration found (perm2) becomes the
// current one. The per-frame state of the incremental bound (tile bounds, last
// exact maxima, best tiles) moves with the frames: each new position takes the
// values of its frame's old position (iperm before the frames are permuted).
// The caller then permutes the frames themselves (launch_permute_frames).
static int reorder_state(emc_ctx* c, cudaStream_t s) {
  const Layout& y = c->lay;
  std::swap(c->perm, c->perm2);
  CU(launch_reorder_state(c->perm, (const int32_t*)(c->ws + y.iperm), c->cfg.n_data, y.ld_data,
                          y.rows / 128, (int32_t*)(c->ws + y.osrc), c->Ub, c->Ub2, c->Ua, c->Ua2,
                          c->Mk, c->Mk2, c->best, c->best2, s));
  std::swap(c->Ub, c->Ub2);
  std::swap(c->Ua, c->Ua2);
  std::swap(c->Mk, c->Mk2);
  std::swap(c->best, c->best2);
  c->order_pending = false;
  return EMC_OK;
}

extern "C" {

const char* emc_status_string(int status) {
  switch (status) {
    case EMC_OK: return "ok";
    case EMC_ERR_ARG: return "invalid argument, size or alignment";
    case EMC_ERR_CUDA: return "CUDA runtime error";
    case EMC_ERR_NOMEM: return "workspace too small";
    case EMC_ERR_UNSUPPORTED: return "input outside the exactly handled range";
    case EMC_ERR_TIMEOUT: return "bounded device wait gave up";
    case EMC_ERR_NUMERIC: return "non-finite or out-of-range value on device";
    default: return "unknown status";
  }
}

int64_t emc_quat_count(int n) {
  if (n < 1) return -1;
  return 10LL * (5LL * n * n * n + n);
}

int64_t emc_quat_generate(int n, int uniform, double* quat, double* weight, int64_t cap) {
  try {  // no C++ exception crosses the C ABI
    return emc::quat_generate(n, uniform, quat, weight, cap);
  } catch (...) {
    return EMC_ERR_NOMEM;
  }
}

int emc_buffer_sizes_for(const emc_config* cfg, int64_t nrot, emc_buffer_sizes* out) {
  int st = check_config(cfg);
  if (st) return st;
  if (!out || nrot < 1 || nrot > cfg->n_rot) return EMC_ERR_ARG;
  Layout y = make_layout(cfg);
  out->ld_pix = y.ld_pix;
  out->ld_data = y.ld_data;
  out->rows = round_up(nrot, 128);
  out->logw_bytes = L_bytes(cfg, out->rows, y.ld_pix);
  out->bias_bytes = sizeof(double) * out->rows * (is_flu(cfg) ? 2 : 1);
  out->prob_bytes = P_bytes(cfg, out->rows, y.ld_data);
  out->num_bytes = sizeof(float) * (size_t)out->rows * y.ld_pix;
  out->den_bytes = sizeof(float) * out->rows;
  out->lse_bytes = sizeof(double) * y.ld_data;
  out->score_bytes = score_bytes(out->rows, y.ld_data);
  out->grid_bytes = sizeof(double) * (size_t)cfg->N * cfg->N * cfg->N;
  return EMC_OK;
}

int emc_workspace_size(const emc_config* cfg, size_t* bytes) {
  int st = check_config(cfg);
  if (st) return st;
  if (!bytes) return EMC_ERR_ARG;
  *bytes = make_layout(cfg).total;
  return EMC_OK;
}

static int ctx_create(const emc_config* cfg, const double* q, const double* quat,
                      const double* weight, void* workspace, size_t workspace_bytes,
                      emc_stream stream, emc_ctx** out);

int emc_ctx_create(const emc_config* cfg, const double* q, const double* quat, const double* weight,
                   void* workspace, size_t workspace_bytes, emc_stream stream, emc_ctx** out) {
  // the host staging vectors are all allocated before the context itself, so a
  // failed allocation leaves nothing behind; no C++ exception crosses the C ABI
  try {
    return ctx_create(cfg, q, quat, weight, workspace, workspace_bytes, stream, out);
  } catch (...) {
    return EMC_ERR_NOMEM;
  }
}

static int ctx_create(const emc_config* cfg, const double* q, const double* quat,
                      const double* weight, void* workspace, size_t workspace_bytes,
                      emc_stream stream, emc_ctx** out) {
  int st = check_config(cfg);
  if (st) return st;
  if (!q || !quat || !weight || !workspace || !out) return EMC_ERR_ARG;
  if (((uintptr_t)workspace) & 255) return EMC_ERR_ARG;
  Layout y = make_layout(cfg);
  if (workspace_bytes < y.total) return EMC_ERR_NOMEM;
  for (int64_t j = 0; j < cfg->n_rot; j++) {
    if (!(weight[j] > 0.0) || !isfinite(weight[j])) return EMC_ERR_ARG;
    double n2 = 0;
    for (int c = 0; c < 4; c++) n2 += quat[4 * j + c] * quat[4 * j + c];
    if (fabs(n2 - 1.0) > 1e-6) return EMC_ERR_ARG;
  }
  const double qlim = 0.5 * cfg->N;
  for (int64_t i = 0; i < cfg->n_pix; i++)
    for (int c = 0; c < 3; c++)
      if (!isfinite(q[3 * i + c]) || fabs(q[3 * i + c]) > qlim) return EMC_ERR_ARG;

  // host staging of the small geometry arrays
  std::vector<float4> qh(y.ld_pix), ql(y.ld_pix);
  for (int64_t i = 0; i < y.ld_pix; i++) {
    float4 a = make_float4(0, 0, 0, 0), b = make_float4(0, 0, 0, 0);
    if (i < cfg->n_pix) {
      float h[3], l[3];
      for (int c = 0; c < 3; c++) {
        h[c] = (float)q[3 * i + c];
        l[c] = (float)(q[3 * i + c] - (double)h[c]);
      }
      a = make_float4(h[0], h[1], h[2], 1.f);
      b = make_float4(l[0], l[1], l[2], 0.f);
    }
    qh[i] = a;
    ql[i] = b;
  }
  // compression groups (pixel_groups.h) and their geometry in group order
  std::vector<int32_t> gord, gstart;
  build_pixel_groups(q, cfg->n_pix, kCompressExtent, kCompressGroup, gord, gstart);
  std::vector<float4> gqh(cfg->n_pix + 1), gql(cfg->n_pix + 1);
  for (int64_t p = 0; p < cfg->n_pix; p++) {
    gqh[p] = qh[gord[p]];
    gql[p] = ql[gord[p]];
  }
  std::vector<double> lw(cfg->n_rot);
  for (int64_t j = 0; j < cfg->n_rot; j++) lw[j] = log(weight[j]);
  std::vector<RotDF> rot(cfg->n_rot);
  for (int64_t j = 0; j < cfg->n_rot; j++) quat_to_rot_df(quat + 4 * j, &rot[j]);
  // the same matrices in fixed point: hi = round(R 2^20), lo = R - hi 2^-20
  std::vector<RotFX> rotfx(cfg->n_rot);
  for (int64_t j = 0; j < cfg->n_rot; j++) {
    double R[9];
    quat_to_rot(quat + 4 * j, R);
    for (int e = 0; e < 9; e++) {
      const double h = rint(R[e] * 1048576.0);
      rotfx[j].hi[e] = (int32_t)h;
      rotfx[j].lo[e] = (float)(R[e] - h / 1048576.0);
    }
  }
  // feature bins of the learned proposal: radial floor(32 |q| / max|q|),
  // angular floor(16 (atan2(q_y, q_x) + pi) / (2 pi)); both capped at the top bin
  std::vector<int16_t> fbin(y.ld_pix, 0);
  std::vector<float> finv(kFeat, 0.f);
  {
    std::vector<double> r(cfg->n_pix);
    double rmax = 0.0;
    for (int64_t i = 0; i < cfg->n_pix; i++) {
      const double* qi = q + 3 * i;
      r[i] = sqrt(qi[0] * qi[0] + qi[1] * qi[1] + qi[2] * qi[2]);
      rmax = r[i] > rmax ? r[i] : rmax;
    }
    std::vector<int64_t> cnt(kFeat, 0);
    for (int64_t i = 0; i < cfg->n_pix; i++) {
      const double* qi = q + 3 * i;
      int64_t rb = rmax > 0 ? (int64_t)floor(32.0 * r[i] / rmax) : 0;
      rb = rb > 31 ? 31 : rb;
      int64_t ab = (int64_t)floor(16.0 * (atan2(qi[1], qi[0]) + M_PI) / (2.0 * M_PI));
      ab = ab > 15 ? 15 : (ab < 0 ? 0 : ab);
      fbin[i] = (int16_t)(rb * 16 + ab);
      cnt[rb * 16 + ab]++;
    }
    for (int b = 0; b < kFeat; b++) finv[b] = cnt[b] ? (float)(1.0 / (double)cnt[b]) : 0.f;
  }

  emc_ctx* c = (emc_ctx*)calloc(1, sizeof(emc_ctx));
  if (!c) return EMC_ERR_NOMEM;
  c->cfg = *cfg;
  c->lay = y;
  c->ws = (char*)workspace;
  c->ws_bytes = workspace_bytes;
  c->geom.qh = (const float4*)(c->ws + y.qh);
  c->geom.ql = (const float4*)(c->ws + y.ql);
  c->geom.qi = (const int4*)(c->ws + y.qi);
  c->geom.qlo = (const float4*)(c->ws + y.qlo);
  c->geom.n_pix = cfg->n_pix;
  c->geom.ld_pix = y.ld_pix;
  c->geom.N = cfg->N;
  c->geom.ngroups = (int)gstart.size() - 1;
  c->geom.gstart = (const int32_t*)(c->ws + y.cgs);
  c->geom.gpix = (const int32_t*)(c->ws + y.cgp);
  c->geom.gqh = (const float4*)(c->ws + y.cgqh);
  c->geom.gql = (const float4*)(c->ws + y.cgql);
  c->geom.gqi = (const int4*)(c->ws + y.cgqi);
  c->geom.gqlo = (const float4*)(c->ws + y.cgqlo);
  c->geom.gqf = (const float4*)(c->ws + y.cgqf);
  {
    // |R q| = |q|: with every |q_i| below N/2 - 1 (less a margin far above the
    // 1e-9-voxel error of the rotation) each p = R q + N/2 has floor in
    // [1, N - 2], so the trilinear corners need no bounds checks
    double r2max = 0.0;
    for (int64_t i = 0; i < cfg->n_pix; i++) {
      const double* qi = q + 3 * i;
      const double r2 = qi[0] * qi[0] + qi[1] * qi[1] + qi[2] * qi[2];
      r2max = r2 > r2max ? r2 : r2max;
    }
    c->geom.interior = sqrt(r2max) < 0.5 * cfg->N - 1.0 - 1e-4 ? 1 : 0;
  }
  c->quat = (double*)(c->ws + y.quat);
  c->rot = (const RotDF*)(c->ws + y.rot);
  c->logw = (double*)(c->ws + y.logw);
  c->Kb = (uint16_t*)(c->ws + y.Kb);
  c->status = (int32_t*)(c->ws + y.status);
  c->gk = y.gk ? (float4*)(c->ws + y.gk) : nullptr;
  c->Kb2 = y.Kb2 ? (uint16_t*)(c->ws + y.Kb2) : nullptr;
  c->gmax = (unsigned*)(c->ws + y.gauss + kGaussMaxOff);
  c->nmax = (unsigned long long*)(c->ws + y.gauss + kGaussNmaxOff);
  c->gsc = (float4*)(c->ws + y.gauss + kGaussScaleOff);
  c->flu_cn = y.fcn ? (double*)(c->ws + y.fcn) : nullptr;
  c->flu_invn = y.finvn ? (float*)(c->ws + y.finvn) : nullptr;
  c->flu_B = y.fB ? (double*)(c->ws + y.fB) : nullptr;
  c->flu_c = is_flu(cfg) ? flu_shift(cfg) : 0.0;
  c->prune = prune_ok(cfg);
  c->perm = y.perm ? (int32_t*)(c->ws + y.perm) : nullptr;
  c->perm2 = y.perm2 ? (int32_t*)(c->ws + y.perm2) : nullptr;
  c->best = y.best ? (int32_t*)(c->ws + y.best) : nullptr;
  c->best2 = y.best2 ? (int32_t*)(c->ws + y.best2) : nullptr;
  c->Mk = y.Mk ? (double*)(c->ws + y.Mk) : nullptr;
  c->Mk2 = y.Mk2 ? (double*)(c->ws + y.Mk2) : nullptr;
  c->Ub = y.Ub ? (float*)(c->ws + y.Ub) : nullptr;
  c->Ub2 = y.Ub2 ? (float*)(c->ws + y.Ub2) : nullptr;
  c->Ua = y.Ua ? (float*)(c->ws + y.Ua) : nullptr;
  c->Ua2 = y.Ua2 ? (float*)(c->ws + y.Ua2) : nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  bool ok = true;
  ok &= cudaMemcpyAsync(c->ws + y.qh, qh.data(), sizeof(float4) * y.ld_pix,
                        cudaMemcpyHostToDevice, s) == cudaSuccess;
  ok &= cudaMemcpyAsync(c->ws + y.ql, ql.data(), sizeof(float4) * y.ld_pix,
                        cudaMemcpyHostToDevice, s) == cudaSuccess;
  ok &= cudaMemcpyAsync(c->ws + y.cgs, gstart.data(), sizeof(int32_t) * gstart.size(),
                        cudaMemcpyHostToDevice, s) == cudaSuccess;
  ok &= cudaMemcpyAsync(c->ws + y.cgp, gord.data(), sizeof(int32_t) * cfg->n_pix,
                        cudaMemcpyHostToDevice, s) == cudaSuccess;
  ok &= cudaMemcpyAsync(c->ws + y.cgqh, gqh.data(), sizeof(float4) * cfg->n_pix,
                        cudaMemcpyHostToDevice, s) == cudaSuccess;
  ok &= cudaMemcpyAsync(c->ws + y.cgql, gql.data(), sizeof(float4) * cfg->n_pix,
                        cudaMemcpyHostToDevice, s) == cudaSuccess;
  ok &= cudaMemcpyAsync(c->quat, quat, sizeof(double) * 4 * cfg->n_rot, cudaMemcpyHostToDevice,
                        s) == cudaSuccess;
  ok &= cudaMemcpyAsync(c->logw, lw.data(), sizeof(double) * cfg->n_rot, cudaMemcpyHostToDevice,
                        s) == cudaSuccess;
  ok &= cudaMemcpyAsync(c->ws + y.rot, rot.data(), sizeof(RotDF) * cfg->n_rot,
                        cudaMemcpyHostToDevice, s) == cudaSuccess;
  ok &= cudaMemcpyAsync(c->ws + y.rotfx, rotfx.data(), sizeof(RotFX) * cfg->n_rot,
                        cudaMemcpyHostToDevice, s) == cudaSuccess;
  ok &= launch_fixed_geometry((const float4*)(c->ws + y.qh), (const float4*)(c->ws + y.ql),
                              y.ld_pix, (int4*)(c->ws + y.qi), (float4*)(c->ws + y.qlo),
                              nullptr, s) == cudaSuccess;
  ok &= launch_fixed_geometry((const float4*)(c->ws + y.cgqh), (const float4*)(c->ws + y.cgql),
                              cfg->n_pix, (int4*)(c->ws + y.cgqi), (float4*)(c->ws + y.cgqlo),
                              (float4*)(c->ws + y.cgqf), s) == cudaSuccess;
  ok &= cudaMemsetAsync(c->status, 0, 256, s) == cudaSuccess;
  ok &= cudaMemsetAsync(c->ws + y.gauss, 0, 256, s) == cudaSuccess;
  if (y.flags) ok &= cudaMemsetAsync(c->ws + y.flags, 0, 256, s) == cudaSuccess;
  ok &= cudaMemcpyAsync(c->ws + y.fbin, fbin.data(), sizeof(int16_t) * y.ld_pix,
                        cudaMemcpyHostToDevice, s) == cudaSuccess;
  ok &= cudaMemcpyAsync(c->ws + y.finv, finv.data(), sizeof(float) * kFeat, cudaMemcpyHostToDevice,
                        s) == cudaSuccess;
  ok &= cudaStreamSynchronize(s) == cudaSuccess;  // host staging buffers go out of scope
  for (int e = 0; e < 8 && ok; e++) ok &= cudaEventCreate(&c->ev[e]) == cudaSuccess;
  if (!ok) {
    for (int e = 0; e < 8; e++)
      if (c->ev[e]) cudaEventDestroy(c->ev[e]);
    free(c);
    return EMC_ERR_CUDA;
  }
  *out = c;
  return EMC_OK;
}

int emc_ctx_destroy(emc_ctx* ctx) {
  if (!ctx) return EMC_ERR_ARG;
  for (int e = 0; e < 8; e++)
    if (ctx->ev[e]) cudaEventDestroy(ctx->ev[e]);
  free(ctx);
  return EMC_OK;
}

int emc_ctx_set_wait_limit(emc_ctx* ctx, uint64_t wait_limit_ns, int stall) {
  if (!ctx) return EMC_ERR_ARG;
  ctx->tcctl.wait_ns = wait_limit_ns;
  ctx->tcctl.stall = stall ? 1 : 0;
  return EMC_OK;
}

int emc_ctx_status(emc_ctx* ctx, int* device_status) {
  if (!ctx || !device_status) return EMC_ERR_ARG;
  int32_t v = 0;
  CU(cudaMemcpy(&v, ctx->status, sizeof(int32_t), cudaMemcpyDeviceToHost));
  CU(cudaMemset(ctx->status, 0, sizeof(int32_t)));
  *device_status = v;
  return EMC_OK;
}

int emc_set_frames(emc_ctx* ctx, const int32_t* K, int64_t ld_k, emc_stream stream) {
  if (!ctx || !K || ld_k < ctx->cfg.n_pix) return EMC_ERR_ARG;
  const Layout& y = ctx->lay;
  const bool g = is_gauss(&ctx->cfg);
  cudaStream_t s = (cudaStream_t)stream;
  const int32_t* dsrc = nullptr;
  const int32_t* drank = nullptr;
  if (ctx->cfg.flags & EMC_FLAG_WIDE_COUNTS) {
    // duplicate columns for counts above 256 (geometry and bins rewritten)
    dsrc = (const int32_t*)(ctx->ws + y.dupsrc);
    drank = (const int32_t*)(ctx->ws + y.duprank);
    CU(launch_assign_duplicates(K, ld_k, ctx->cfg.n_data, ctx->cfg.n_pix, y.ld_data,
                                (int32_t*)(ctx->ws + y.pixmax), (float4*)(ctx->ws + y.qh),
                                (float4*)(ctx->ws + y.ql), (int16_t*)(ctx->ws + y.fbin),
                                (int32_t*)(ctx->ws + y.dupsrc), (int32_t*)(ctx->ws + y.duprank),
                                ctx->status, s));
    CU(launch_fixed_geometry((const float4*)(ctx->ws + y.qh), (const float4*)(ctx->ws + y.ql),
                             y.ld_pix, (int4*)(ctx->ws + y.qi), (float4*)(ctx->ws + y.qlo),
                             nullptr, s));
  }
  if (ctx->prune) {
    // the incremental bound of the next iteration holds for the frames of the
    // last one only: flag counts that differ from the held copy (frames with
    // counts above 256 are always flagged: their copy holds parts of them)
    int32_t* changed = (int32_t*)(ctx->ws + y.flags);
    if (ctx->frames_loaded && !(ctx->cfg.flags & EMC_FLAG_WIDE_COUNTS)) {
      CU(launch_frames_differ(K, ld_k, ctx->cfg.n_data, ctx->cfg.n_pix, ctx->Kb, y.ld_pix,
                              ctx->cfg.precision == EMC_PREC_FP16_SPLIT ? 1 : 0, changed, s));
    } else {
      CU(cudaMemsetAsync(changed, 1, sizeof(int32_t), s));
    }
  }
  CU(launch_prep_frames(K, ld_k, ctx->cfg.n_data, ctx->cfg.n_pix, y.ld_data, y.ld_pix, ctx->Kb,
                        g ? 3 : (ctx->cfg.precision == EMC_PREC_FP16_SPLIT ? 1 : 0), dsrc, drank,
                        ctx->status, s));
  if (ctx->cfg.flags & EMC_FLAG_SPARSE_K)
    CU(launch_sparse_k_frames(K, ld_k, ctx->cfg.n_data, ctx->cfg.n_pix, y.ld_data,
                              (int32_t*)(ctx->ws + y.skcnt), (int64_t*)(ctx->ws + y.skoff),
                              (uint32_t*)(ctx->ws + y.skent), (cudaStream_t)stream));
  if (is_flu(&ctx->cfg))
    CU(launch_flu_frames(K, ld_k, ctx->cfg.n_data, ctx->cfg.n_pix, y.ld_data, ctx->flu_c,
                         ctx->flu_cn, ctx->flu_invn, s));
  if (ctx->prune) {
    // the internal frame order starts as the given one; a context that already
    // has one keeps it for new frames (it only decides how many pass-1 tiles
    // the bound skips, and the same frames loaded again keep their grouping)
    float* nsum = (float*)(ctx->ws + y.nsum);
    CU(launch_frame_totals(K, ld_k, ctx->cfg.n_data, ctx->cfg.n_pix, y.ld_data, nsum, s));
    if (!ctx->perm_valid) {
      CU(launch_identity(ctx->perm, y.ld_data, s));
      CU(launch_identity(ctx->perm2, y.ld_data, s));
    } else if (ctx->order_pending) {
      int st = reorder_state(ctx, s);
      if (st) return st;
    }
    CU(launch_permute_frames(ctx->perm, y.ld_data, y.ld_pix, ctx->Kb, (uint16_t*)(ctx->ws + y.Kp),
                             nsum, (float*)(ctx->ws + y.nsum_p), ctx->flu_cn,
                             y.cn_p ? (double*)(ctx->ws + y.cn_p) : nullptr, ctx->flu_invn,
                             y.invn_p ? (float*)(ctx->ws + y.invn_p) : nullptr,
                             (int32_t*)(ctx->ws + y.iperm), s));
    ctx->scores_internal = false;
  }
  if (g) {
    CU(launch_prep_frames(K, ld_k, ctx->cfg.n_data, ctx->cfg.n_pix, y.ld_data, y.ld_pix, ctx->Kb2,
                          2, dsrc, drank, ctx->status, s));
    CU(launch_gauss_frames(K, ld_k, ctx->cfg.n_data, ctx->cfg.n_pix, y.ld_data, ctx->cfg.sigma,
                           ctx->gk, ctx->nmax, (cudaStream_t)stream));
  }
  ctx->frames_loaded = true;
  ctx->iterated = false;
  return EMC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Internal step implementations (used by both the step calls and the fused
// iteration).
// ---------------------------------------------------------------------------
namespace {

// Lold, bias_old (optional, Poisson model): the last iteration's L and bias;
// the expansion then also writes the incremental bound's increments.
int do_expand(emc_ctx* c, const float* grid, int64_t rot0, int64_t nrot, void* L, double* bias,
              cudaStream_t s, const void* Lold = nullptr, const double* bias_old = nullptr) {
  const int64_t rows = round_up(nrot, 128);
  Planes p{L, rows * c->lay.ld_pix, c->lay.ld_pix};
  const bool g = is_gauss(&c->cfg);
  const Layout& y = c->lay;
  float4* g4 = (y.g4 && c->geom.interior) ? (float4*)(c->ws + y.g4) : nullptr;
  if (g4) CU(launch_grid_pairs(grid, c->cfg.N, g4, s));
  if (!g && !is_flu(&c->cfg)) {
    CU(launch_expand_tile(c->geom, grid, g4, (const RotFX*)(c->ws + y.rotfx) + rot0, c->logw + rot0,
                          nrot, rows, c->cfg.precision, (float)c->cfg.w_floor, p, bias,
                          (double*)(c->ws + y.epart), Lold, bias_old,
                          Lold ? (uint16_t*)(c->ws + y.Dd) : nullptr, y.ntp,
                          Lold ? (float*)(c->ws + y.bpm) : nullptr, c->status, s));
    return EMC_OK;
  }
  if (is_flu(&c->cfg)) {
    CU(launch_expand_flu(c->geom, grid, g4, c->rot + rot0, c->logw + rot0, nrot, rows,
                         c->cfg.precision, (float)c->cfg.w_floor, c->flu_c, p, bias,
                         c->flu_B + rot0, c->status, s));
    return EMC_OK;
  }
  if (g)
    CU(launch_gauss_scales(grid, (int64_t)c->cfg.N * c->cfg.N * c->cfg.N, c->gmax, c->nmax,
                           c->gsc, c->status, s));
  CU(launch_expand(c->geom, grid, g4, c->rot + rot0, c->logw + rot0, nrot, rows,
                   c->cfg.precision, (float)c->cfg.w_floor, p, bias, g ? c->gsc : nullptr,
                   c->cfg.sigma, c->status, s));
  return EMC_OK;
}

// L is the full block [planes][rows][ld_pix] (plane stride = Lrows * ld_pix);
// the rows processed here start at row_off inside it.
// scores: NULL or a buffer of score_bytes(rows, ld_data) for this block.
int do_loglik(emc_ctx* c, const void* L, int64_t Lrows, int64_t row_off, const double* bias,
              int64_t nrot, double* lse_m, double* lse_s, int accumulate, void* scores,
              cudaStream_t s) {
  const Layout& y = c->lay;
  const int64_t rows = round_up(nrot, 128);
  double* pm = (double*)(c->ws + y.part_m);
  float* ps = (float*)(c->ws + y.part_s);
  float* S = (float*)scores;
  float* Sref = S ? S + rows * y.ld_data : nullptr;
  int64_t tiles;
  if (c->cfg.precision == EMC_PREC_FP32) {
    const float* Lf = (const float*)L + row_off * y.ld_pix;
    CU(launch_simt_pass1(Lf, y.ld_pix, bias, rows, c->Kb, y.ld_data, c->cfg.n_data, pm, ps, S,
                         Sref, s));
    tiles = simt_pass1_tiles(rows);
  } else {
    Planes p{(void*)((const uint16_t*)L + row_off * y.ld_pix), Lrows * y.ld_pix, y.ld_pix};
    const bool g = is_gauss(&c->cfg);
    CU(launch_tc_pass1(p, c->cfg.precision, bias, rows, c->Kb, y.ld_data, c->cfg.n_data, y.ld_pix, pm, ps,
                       S, Sref, g ? c->gk : nullptr, g ? c->gsc : nullptr, c->status, s, nullptr,
                       nullptr, c->tcctl));
    tiles = tc_pass1_tiles(rows);
  }
  CU(launch_lse_merge(pm, ps, tiles, y.ld_data, c->cfg.n_data, lse_m, lse_s, accumulate,
                      is_gauss(&c->cfg), c->status, s, c->flu_cn));
  return EMC_OK;
}

// Frames in emc_iteration's internal order (bound-pruned pass 1): their BF16
// matrix, the Poisson-fluence arrays, and the contracted tiles of these rows.
struct FrameView {
  const uint16_t* K;
  const double* cn;
  const float* invn;
  const uint8_t* tile_live;   // stored scores: the contracted tiles of these rows
  const int32_t* tile_list;   // recomputed scores: the live tiles of these rows
  const int32_t* tile_count;
};

// S, Sref: stored scores of these rows, S frame-major with leading dimension
// ldS (NULL: recompute from L and bias). Bsum: the rows' B_j (Poisson-fluence model).
// fv (may be NULL): frames in the internal order.
int do_normalize(emc_ctx* c, const void* L, int64_t Lrows, int64_t row_off, const double* bias,
                 int64_t nrot, const double* lse_m, const double* lse_s, const float* S,
                 int64_t ldS, const float* Sref, void* P, int64_t Prows, cudaStream_t s,
                 const double* Bsum = nullptr, uint8_t* kbf = nullptr,
                 const FrameView* fv = nullptr) {
  const Layout& y = c->lay;
  const int64_t rows = round_up(nrot, 128);
  const uint8_t* tlive = fv ? fv->tile_live : nullptr;
  const uint16_t* Kf = fv ? fv->K : c->Kb;
  const int32_t* tl = fv ? fv->tile_list : nullptr;
  const int32_t* tc = fv ? fv->tile_count : nullptr;
  if (is_flu(&c->cfg)) {
    if (!bias || !Bsum) return EMC_ERR_ARG;
    float2* lse2 = (float2*)(c->ws + y.lse2);
    float* den = (float*)((char*)P + P_plane_bytes(&c->cfg, Prows, y.ld_data));
    const double* cn = fv ? fv->cn : c->flu_cn;
    const float* invn = fv ? fv->invn : c->flu_invn;
    if (S) {
      CU(launch_lse_split(lse_m, lse_s, c->cfg.n_data, y.ld_data, lse2, s, cn));
      CU(launch_normalize_scores_flu(S, ldS, Sref, lse2, Bsum, invn, rows, nrot,
                                     y.ld_data, c->cfg.n_data, (uint16_t*)P, Prows * y.ld_data,
                                     den, s, kbf, tlive));
    } else {
      Planes lp{(void*)((const uint16_t*)L + row_off * y.ld_pix), Lrows * y.ld_pix, y.ld_pix};
      Planes pp{P, Prows * y.ld_data, y.ld_data};
      CU(launch_tc_normalize(lp, c->cfg.precision, bias, rows, nrot, Kf, y.ld_data,
                             c->cfg.n_data, y.ld_pix, lse_m, lse_s, lse2, pp, c->status, s,
                             cn, Bsum, invn, den, kbf, tl, tc, c->tcctl));
    }
    return EMC_OK;
  }
  if (is_gauss(&c->cfg)) {
    if (!S || !bias) return EMC_ERR_UNSUPPORTED;
    float2* lse2 = (float2*)(c->ws + y.lse2);
    float* den = (float*)((char*)P + P_plane_bytes(&c->cfg, Prows, y.ld_data));
    CU(launch_lse_split(lse_m, lse_s, c->cfg.n_data, y.ld_data, lse2, s));
    CU(launch_normalize_scores_gauss(S, ldS, Sref, lse2, bias, c->gk, rows, nrot,
                                     y.ld_data, c->cfg.n_data, (uint16_t*)P, Prows * y.ld_data,
                                     den, s, kbf));
    return EMC_OK;
  }
  if (S) {
    float2* lse2 = (float2*)(c->ws + y.lse2);
    CU(launch_lse_split(lse_m, lse_s, c->cfg.n_data, y.ld_data, lse2, s));
    CU(launch_normalize_scores(S, ldS, Sref, lse2, rows, nrot, y.ld_data, c->cfg.n_data,
                               c->cfg.precision, P, Prows * y.ld_data, s, kbf, tlive));
    return EMC_OK;
  }
  if (c->cfg.precision == EMC_PREC_FP32) {
    const float* Lf = (const float*)L + row_off * y.ld_pix;
    CU(launch_simt_normalize(Lf, y.ld_pix, bias, rows, nrot, c->Kb, y.ld_data, c->cfg.n_data,
                             lse_m, lse_s, (float*)P, s));
  } else {
    Planes lp{(void*)((const uint16_t*)L + row_off * y.ld_pix), Lrows * y.ld_pix, y.ld_pix};
    Planes pp{P, Prows * y.ld_data, y.ld_data};
    CU(launch_tc_normalize(lp, c->cfg.precision, bias, rows, nrot, Kf, y.ld_data, c->cfg.n_data,
                           y.ld_pix, lse_m, lse_s, (float2*)(c->ws + y.lse2), pp, c->status, s,
                           nullptr, nullptr, nullptr, nullptr, kbf, tl, tc, c->tcctl));
  }
  return EMC_OK;
}

// kbc, kbl (optional): the non-zero 64-frame blocks of each row tile of P;
// Kf (optional): frames in emc_iteration's internal order
int do_update(emc_ctx* c, const void* P, int64_t Prows, int64_t nrot, float* Num, float* den,
              cudaStream_t s, const int32_t* kbc = nullptr, const int32_t* kbl = nullptr,
              const uint16_t* Kf = nullptr) {
  const Layout& y = c->lay;
  const int64_t rows = round_up(nrot, 128);
  if (c->cfg.precision == EMC_PREC_FP32) {
    CU(launch_simt_update((const float*)P, y.ld_data, rows, c->Kb, y.ld_pix, c->cfg.n_pix, Num,
                          den, s));
  } else {
    Planes pp{(void*)P, Prows * y.ld_data, y.ld_data};
    if (is_gauss(&c->cfg) || is_flu(&c->cfg)) {
      // BF16 hi + lo planes of P / phi against the BF16 frames (the Gaussian
      // model's BF16 copy)
      // (the Gaussian model's P is not sparse: its update stays on the tensor
      // pipe's rate and keeps every pipeline stage)
      CU(launch_tc_update(pp, EMC_PREC_BF16_SPLIT, rows,
                          Kf ? Kf : (is_gauss(&c->cfg) ? c->Kb2 : c->Kb), y.ld_data, y.ld_pix,
                          c->cfg.n_pix, Num, nullptr, c->status, s, kbc, kbl, c->tcctl,
                          kbc != nullptr && !is_gauss(&c->cfg)));
      const char* tail = (const char*)P + P_plane_bytes(&c->cfg, Prows, y.ld_data);
      CU(cudaMemcpyAsync(den, tail, sizeof(float) * rows, cudaMemcpyDeviceToDevice, s));
    } else {
      // over the listed blocks of a sparse P the update is bound by its output
      CU(launch_tc_update(pp, c->cfg.precision, rows, Kf ? Kf : c->Kb, y.ld_data, y.ld_pix,
                          c->cfg.n_pix, Num, den, c->status, s, kbc, kbl, c->tcctl,
                          kbc != nullptr));
    }
  }
  return EMC_OK;
}

int check_rot_range(emc_ctx* c, int64_t rot0, int64_t nrot) {
  if (rot0 < 0 || nrot < 1 || rot0 + nrot > c->cfg.n_rot) return EMC_ERR_ARG;
  return EMC_OK;
}

}  // namespace

extern "C" {

int emc_expand(emc_ctx* ctx, const float* grid, int64_t rot0, int64_t nrot, void* L, double* bias,
               emc_stream stream) {
  if (!ctx || !grid || !L || !bias) return EMC_ERR_ARG;
  if (check_rot_range(ctx, rot0, nrot)) return EMC_ERR_ARG;
  return do_expand(ctx, grid, rot0, nrot, L, bias, (cudaStream_t)stream);
}

int emc_loglik(emc_ctx* ctx, const void* L, const double* bias, int64_t nrot, double* lse_m,
               double* lse_s, int accumulate, void* scores, emc_stream stream) {
  if (!ctx || !L || !bias || !lse_m || !lse_s) return EMC_ERR_ARG;
  if (check_rot_range(ctx, 0, nrot)) return EMC_ERR_ARG;
  if (!ctx->frames_loaded) return EMC_ERR_ARG;
  if (((uintptr_t)scores) & 15) return EMC_ERR_ARG;
  return do_loglik(ctx, L, round_up(nrot, 128), 0, bias, nrot, lse_m, lse_s, accumulate, scores,
                   (cudaStream_t)stream);
}

int emc_loglik_sparse_k(emc_ctx* ctx, const float* L, const double* bias, int64_t nrot,
                        double* lse_m, double* lse_s, int accumulate, emc_stream stream) {
  if (!ctx || !L || !bias || !lse_m || !lse_s) return EMC_ERR_ARG;
  if (check_rot_range(ctx, 0, nrot)) return EMC_ERR_ARG;
  if (!ctx->frames_loaded) return EMC_ERR_ARG;
  if (!(ctx->cfg.flags & EMC_FLAG_SPARSE_K) || ctx->cfg.precision != EMC_PREC_FP32)
    return EMC_ERR_UNSUPPORTED;
  const Layout& y = ctx->lay;
  if (sparse_k_smem(y.ld_pix) > 220u * 1024u) return EMC_ERR_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t rows = round_up(nrot, 128);
  double* pm = (double*)(ctx->ws + y.part_m);
  float* ps = (float*)(ctx->ws + y.part_s);
  CU(launch_sparse_k_pass1(L, y.ld_pix, ctx->cfg.n_pix, bias, rows, (int64_t*)(ctx->ws + y.skoff),
                           (uint32_t*)(ctx->ws + y.skent), y.ld_data, ctx->cfg.n_data, pm, ps,
                           s));
  CU(launch_lse_merge(pm, ps, rows / 128, y.ld_data, ctx->cfg.n_data, lse_m, lse_s, accumulate, 0,
                      ctx->status, s));
  return EMC_OK;
}

int emc_normalize(emc_ctx* ctx, const void* L, const double* bias, int64_t nrot,
                  const double* lse_m, const double* lse_s, const void* scores, void* P,
                  emc_stream stream) {
  if (!ctx || !lse_m || !lse_s || !P) return EMC_ERR_ARG;
  if (!scores && (!L || !bias)) return EMC_ERR_ARG;
  if (is_gauss(&ctx->cfg) && !scores) return EMC_ERR_UNSUPPORTED;
  if ((is_gauss(&ctx->cfg) || is_flu(&ctx->cfg)) && !bias) return EMC_ERR_ARG;
  if (check_rot_range(ctx, 0, nrot)) return EMC_ERR_ARG;
  if (!ctx->frames_loaded) return EMC_ERR_ARG;
  if (((uintptr_t)scores) & 15) return EMC_ERR_ARG;
  const int64_t rows = round_up(nrot, 128);
  const float* S = (const float*)scores;
  const float* Sref = S ? S + rows * ctx->lay.ld_data : nullptr;
  // Poisson-fluence model: B_j follows log w_j in the bias buffer
  return do_normalize(ctx, L, rows, 0, bias, nrot, lse_m, lse_s, S, rows, Sref, P, rows,
                      (cudaStream_t)stream, is_flu(&ctx->cfg) ? bias + rows : nullptr);
}

int emc_update(emc_ctx* ctx, const void* P, int64_t nrot, float* Num, float* den,
               emc_stream stream) {
  if (!ctx || !P || !Num || !den) return EMC_ERR_ARG;
  if (check_rot_range(ctx, 0, nrot)) return EMC_ERR_ARG;
  if (!ctx->frames_loaded) return EMC_ERR_ARG;
  return do_update(ctx, P, round_up(nrot, 128), nrot, Num, den, (cudaStream_t)stream);
}

int emc_compress(emc_ctx* ctx, int64_t rot0, int64_t nrot, const float* Num, const float* den,
                 double* g_num, double* g_den, int accumulate, emc_stream stream) {
  if (!ctx || !Num || !den || !g_num || !g_den) return EMC_ERR_ARG;
  if (check_rot_range(ctx, rot0, nrot)) return EMC_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t gb = sizeof(double) * (size_t)ctx->cfg.N * ctx->cfg.N * ctx->cfg.N;
  if (!accumulate) {
    CU(cudaMemsetAsync(g_num, 0, gb, s));
    CU(cudaMemsetAsync(g_den, 0, gb, s));
  }
  CU(launch_compress(ctx->geom, (const RotFX*)(ctx->ws + ctx->lay.rotfx) + rot0, nrot, Num, den, ctx->cfg.compress_mode, g_num,
                     g_den, 1, s));
  return EMC_OK;
}

int emc_finalize(emc_ctx* ctx, const double* g_num, const double* g_den, const float* grid_prev,
                 float* grid_out, emc_stream stream) {
  if (!ctx || !g_num || !g_den || !grid_prev || !grid_out) return EMC_ERR_ARG;
  const int64_t nvox = (int64_t)ctx->cfg.N * ctx->cfg.N * ctx->cfg.N;
  CU(launch_finalize(nvox, g_num, g_den, 1, grid_prev, grid_out, (cudaStream_t)stream));
  return EMC_OK;
}

int emc_iteration(emc_ctx* c, const float* grid_in, float* grid_out, emc_iter_stats* stats,
                  emc_stream stream) {
  if (!c || !grid_in || !grid_out || grid_in == grid_out) return EMC_ERR_ARG;
  if (!c->frames_loaded) return EMC_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const Layout& y = c->lay;
  const int64_t n_rot = c->cfg.n_rot;
  // pruned contexts alternate between two L and bias buffers: the last
  // iteration's stay for the incremental bound
  const bool pr = c->prune;
  const int lnew = pr ? 1 - c->lcur : 0;
  void* L = c->ws + (lnew ? y.L2 : y.L);
  double* bias = (double*)(c->ws + (lnew ? y.bias2 : y.bias));
  double* lse_m = (double*)(c->ws + y.lse_m);
  double* lse_s = (double*)(c->ws + y.lse_s);
  void* P = c->ws + y.P;
  float* Num = (float*)(c->ws + y.Num);
  float* den = (float*)(c->ws + y.den);
  double* gn = (double*)(c->ws + y.gnum);
  double* gd = (double*)(c->ws + y.gden);
  double* ll = (double*)(c->ws + y.scalar);
  const size_t gb = sizeof(double) * (size_t)c->cfg.N * c->cfg.N * c->cfg.N * c->lay.nrep;
  int kernels = 0;
  int st;
  bool delta = false;  // the incremental bound ran

  // the incremental bound runs when the last iteration left its tile bounds;
  // for the Poisson model the expansion computes its increments on the way
  const bool pruned = pr && c->perm_valid;
  delta = pruned && c->ub_valid;
  const void* Lold = delta ? c->ws + (lnew ? y.L : y.L2) : nullptr;
  const double* bold = delta ? (const double*)(c->ws + (lnew ? y.bias : y.bias2)) : nullptr;
  const bool fused = delta && !is_flu(&c->cfg);
  if (stats) CU(cudaEventRecord(c->ev[0], s));
  c->collected = false;
  if (c->collecting) CU(cudaMemsetAsync(c->col.count, 0, sizeof(unsigned long long), s));
  if ((st = do_expand(c, grid_in, 0, n_rot, L, bias, s, fused ? Lold : nullptr,
                      fused ? bold : nullptr)))
    return st;
  // Gaussian: grid maximum and scales first; Poisson: the row tiles and the bias
  // sums; the corner-pair layout of the model first where it is used
  kernels += (is_gauss(&c->cfg) ? 3 : (is_flu(&c->cfg) ? 1 : 2)) +
             ((y.g4 && c->geom.interior) ? 1 : 0);
  if (stats) CU(cudaEventRecord(c->ev[1], s));
  float* S = (c->cfg.flags & EMC_FLAG_STORE_SCORES) ? (float*)(c->ws + y.S) : nullptr;
  // bound-pruned pass 1 over the frames in their internal order
  const int64_t nmt = y.rows / 128, nnt = y.ld_data / 256;
  const uint16_t* Kp = pr ? (const uint16_t*)(c->ws + y.Kp) : nullptr;
  uint8_t* live = pr ? (uint8_t*)(c->ws + y.live) : nullptr;
  double* lm = pr ? (double*)(c->ws + y.lsem_s) : lse_m;  // lse in the internal order
  double* ls = pr ? (double*)(c->ws + y.lses_s) : lse_s;
  const double* cn_p = y.cn_p ? (const double*)(c->ws + y.cn_p) : nullptr;
  if (pr && c->order_pending) {
    // the order the previous iteration found: frames, their arrays and the
    // per-frame state of the incremental bound follow it
    if ((st = reorder_state(c, s))) return st;
    CU(launch_permute_frames(c->perm, y.ld_data, y.ld_pix, c->Kb, (uint16_t*)(c->ws + y.Kp),
                             (const float*)(c->ws + y.nsum), (float*)(c->ws + y.nsum_p),
                             c->flu_cn, y.cn_p ? (double*)(c->ws + y.cn_p) : nullptr,
                             c->flu_invn, y.invn_p ? (float*)(c->ws + y.invn_p) : nullptr,
                             (int32_t*)(c->ws + y.iperm), s));
    kernels += 3;
  }
  if (pr) {
    double* pm = (double*)(c->ws + y.part_m);
    float* ps = (float*)(c->ws + y.part_s);
    Planes p3{L, y.rows * y.ld_pix, y.ld_pix};
    int32_t* tlist = (int32_t*)(c->ws + y.tlist);
    int32_t* tcount = (int32_t*)(c->ws + y.tcount);
    const float* nsum_p = (const float*)(c->ws + y.nsum_p);
    if (pruned) {
      // 1. the incremental bound from the last iteration (same frames, its L
      //    and tile bounds kept): candidates for the hi-plane bound
      uint8_t* cand = (uint8_t*)(c->ws + y.dcand);
      uint8_t* pf = (uint8_t*)(c->ws + y.pflag);
      int32_t* plist = (int32_t*)(c->ws + y.plist);
      int32_t* pcount = tcount + 32;
      const float* Cd = (const float*)(c->ws + y.Cd);
      const float* bpm = (const float*)(c->ws + y.bpm);
      if (delta) {
        const int f16 = c->cfg.precision == EMC_PREC_FP16_SPLIT ? 1 : 0;
        if (!fused) {  // Poisson-fluence: the increments from both L in a pass of their own
          CU(launch_delta_planes((const uint16_t*)Lold, (const uint16_t*)L, y.rows * y.ld_pix,
                                 y.ld_pix, n_rot, bold, bias, y.ntp, (uint16_t*)(c->ws + y.Dd),
                                 (float*)bpm, f16, s));
          kernels++;
        }
        Planes pd{c->ws + y.Dd, 3 * y.ntp * y.ld_pix, y.ld_pix};
        CU(launch_tc_store(pd, 3 * y.ntp, Kp, y.ld_data, y.ld_pix, (float*)Cd, f16, c->status, s,
                           c->tcctl));
        kernels++;
      }
      CU(launch_delta_live(Cd, y.ntp, bpm, c->Ub, c->Ua, (double*)(c->ws + y.Lk), c->Mk,
                           c->best,
                           nsum_p, bound_div(&c->cfg), y.ld_pix, nmt, y.ld_data, c->cfg.n_data,
                           delta ? 1 : 0,
                           (const int32_t*)(c->ws + y.flags), cand, s));
      // 2. the hi plane alone (the first plane of L) over the candidate pairs of
      //    row tiles (none when the incremental bound is tighter everywhere):
      //    per-tile maxima of S_hi
      CU(launch_pair_flags(cand, nmt, nnt, pf, s));
      CU(launch_tile_list(pf, (int)((nmt + 1) / 2), (int)nnt, 4, plist, pcount,
                            (int32_t*)(c->ws + y.sortH), s));
      CU(launch_tc_bound(p3, c->cfg.precision, bias, y.rows, Kp, y.ld_data, y.ld_pix, pm,
                         c->status, s, c->tcctl, plist, pcount));
      // 3. both bounds together: the live tiles, listed for the exact pass
      CU(launch_final_live(pm, pf, c->Ub, c->Ua, (double*)(c->ws + y.Lk), nsum_p,
                           bound_div(&c->cfg),
                           nmt, y.ld_data, c->cfg.n_data, live, s));
      CU(launch_tile_list(live, (int)nmt, (int)nnt, 8, tlist, tcount, (int32_t*)(c->ws + y.sortH),
                            s));
      kernels += 10;  // a tile list is three launches
    }
    CU(launch_tc_pass1(p3, c->cfg.precision, bias, y.rows, Kp, y.ld_data, c->cfg.n_data, y.ld_pix,
                       pm, ps, S, S + y.rows * y.ld_data, nullptr, nullptr, c->status, s,
                       pruned ? tlist : nullptr, pruned ? tcount : nullptr, c->tcctl));
    // the merge also keeps, for the next iteration's incremental bound, every
    // contracted tile's maximum (plus 1/64) in Ub, the frames' largest maxima and best tiles
    CU(launch_lse_merge(pm, ps, nmt, y.ld_data, c->cfg.n_data, lm, ls, 0, 0, c->status, s, cn_p,
                        pruned ? live : nullptr, c->best, c->Ub, c->Mk, c->Ua));
    CU(launch_unpermute_lse(c->perm, c->cfg.n_data, lm, ls, lse_m, lse_s, s));
    // the frames are consumed; a device status recorded by now (a wait that
    // gave up, a non-finite value) voids the tile bounds for the next iteration
    CU(cudaMemsetAsync(c->ws + y.flags, 0, sizeof(int32_t), s));
    CU(cudaMemcpyAsync(c->ws + y.flags + 8, c->status, sizeof(int32_t), cudaMemcpyDeviceToDevice,
                       s));
    kernels += 3;  // pass 1, merge, lse order
  } else {
    if ((st = do_loglik(c, L, y.rows, 0, bias, n_rot, lse_m, lse_s, 0, S, s))) return st;
    kernels += 2;
  }
  CU(launch_loglik_sum(lse_m, lse_s, c->cfg.n_data, ll, s));
  kernels += 1;
  if (stats) CU(cudaEventRecord(c->ev[2], s));
  CU(cudaMemsetAsync(gn, 0, gb, s));
  CU(cudaMemsetAsync(gd, 0, gb, s));
  float t_norm = 0.f, t_upd = 0.f, t_cmp = 0.f;
  for (int64_t r0 = 0; r0 < n_rot; r0 += y.chunk_rows) {
    const int64_t nr = std::min(y.chunk_rows, n_rot - r0);
    const int64_t crows = round_up(nr, 128);
    if (stats) CU(cudaEventRecord(c->ev[3], s));
    const float* Sc = S ? S + r0 : nullptr;  // frame-major: rows r0.. of every frame
    const float* Sr = S ? S + y.rows * y.ld_data + (r0 / 32) * y.ld_data : nullptr;
    // the tensor-core update contracts only the 128 x 64 blocks of P that the
    // normalisation found non-zero (skipping blocks of exact zeros changes no sum)
    uint8_t* kbf = y.kbflag ? (uint8_t*)(c->ws + y.kbflag) : nullptr;
    const int32_t* kbc = kbf ? (const int32_t*)(c->ws + y.kbcnt) : nullptr;
    const int32_t* kbl = kbf ? (const int32_t*)(c->ws + y.kblist) : nullptr;
    // (the chunk's count sits after pass 1's in the same block, which the stats read)
    int32_t* tlist = pr ? (int32_t*)(c->ws + y.tlist) : nullptr;
    int32_t* tcount = pr ? (int32_t*)(c->ws + y.tcount) + 16 : nullptr;
    if (pruned && !S) {  // recomputed pass 2: the live tiles of this chunk's rows
      CU(launch_tile_list(live + (r0 / 128) * nnt, (int)(crows / 128), (int)nnt, 8, tlist, tcount,
                          (int32_t*)(c->ws + y.sortH), s));
      kernels += 3;
    }
    FrameView fv{Kp, cn_p, y.invn_p ? (const float*)(c->ws + y.invn_p) : nullptr,
                 pruned && S ? live + (r0 / 128) * nnt : nullptr,
                 pruned && !S ? tlist : nullptr, pruned && !S ? tcount : nullptr};
    if ((st = do_normalize(c, L, y.rows, r0, bias + r0, nr, lm, ls, Sc, y.rows, Sr, P, crows, s,
                           c->flu_B ? c->flu_B + r0 : nullptr, kbf, pr ? &fv : nullptr)))
      return st;
    if (kbf)
      CU(launch_kb_lists(kbf, crows / 128, (int)(y.ld_data / 64), (int32_t*)kbc, (int32_t*)kbl,
                         s));
    if (c->collecting && kbf) {  // the chunk's non-zero P_jk, before the update reads them
      const float* invn = is_flu(&c->cfg)
                              ? ((pr && y.invn_p) ? (const float*)(c->ws + y.invn_p) : c->flu_invn)
                              : nullptr;
      CU(launch_collect(P, crows * y.ld_data, y.ld_data, c->cfg.precision,
                        c->flu_B ? c->flu_B + r0 : nullptr, invn, r0, nr, crows / 128, kbc, kbl,
                        (int)(y.ld_data / 64), pr ? c->perm : nullptr, c->cfg.n_data, c->col,
                        s));
      kernels++;
    }
    if (stats) CU(cudaEventRecord(c->ev[4], s));
    if ((st = do_update(c, P, crows, nr, Num, den, s, kbc, kbl, Kp))) return st;
    if (stats) CU(cudaEventRecord(c->ev[5], s));
    CU(launch_compress(c->geom, (const RotFX*)(c->ws + y.rotfx) + r0, nr, Num, den, c->cfg.compress_mode, gn, gd, y.nrep,
                       s));
    if (stats) CU(cudaEventRecord(c->ev[6], s));
    // normalize: lse split + the pass (one SIMT kernel when recomputing in FP32)
    kernels += (S || c->cfg.precision != EMC_PREC_FP32 ? 2 : 1) + 2 + (kbf ? 1 : 0);
    if (stats) {
      // chunk timings need a host wait per chunk; only when stats are asked for
      float a = 0, b = 0, d = 0;
      CU(cudaEventSynchronize(c->ev[6]));
      CU(cudaEventElapsedTime(&a, c->ev[3], c->ev[4]));
      CU(cudaEventElapsedTime(&b, c->ev[4], c->ev[5]));
      CU(cudaEventElapsedTime(&d, c->ev[5], c->ev[6]));
      t_norm += a;
      t_upd += b;
      t_cmp += d;
    }
  }
  if (stats) CU(cudaEventRecord(c->ev[3], s));
  CU(launch_finalize((int64_t)c->cfg.N * c->cfg.N * c->cfg.N, gn, gd, y.nrep, grid_in, grid_out,
                     s));
  kernels++;
  if (pr) {
    // the next iteration's frame order: grouped by the row tile of the best
    // rotation (counting sort, stable); applied when that iteration starts, so
    // that until then the stored scores, iperm and the live flags agree
    // (sort_frames writes positions below n_data only; the tails stay the identity)
    CU(launch_sort_frames(c->best, c->perm, c->cfg.n_data, (int)nmt,
                          (int32_t*)(c->ws + y.sortH), (int64_t*)(c->ws + y.sortoff), c->perm2,
                          s));
    c->order_pending = true;
    c->perm_valid = true;
    c->scores_internal = true;
    c->last_pruned = pruned;
    c->lcur = lnew;
    c->ub_valid = true;
    kernels += 3;
  }
  if (stats) CU(cudaEventRecord(c->ev[7], s));
  c->kernels = kernels;
  c->iterated = true;
  c->collected = c->collecting;
  if (stats) {
    CU(cudaEventSynchronize(c->ev[7]));
    float te = 0, tl = 0, tf = 0, tt = 0;
    CU(cudaEventElapsedTime(&te, c->ev[0], c->ev[1]));
    CU(cudaEventElapsedTime(&tl, c->ev[1], c->ev[2]));
    CU(cudaEventElapsedTime(&tf, c->ev[3], c->ev[7]));
    CU(cudaEventElapsedTime(&tt, c->ev[0], c->ev[7]));
    memset(stats, 0, sizeof(*stats));
    stats->ms_expand = te;
    stats->ms_loglik = tl;
    stats->ms_normalize = t_norm;
    stats->ms_update = t_upd;
    stats->ms_compress = t_cmp + tf;
    stats->ms_total = tt;
    CU(cudaMemcpy(&stats->loglik, ll, sizeof(double), cudaMemcpyDeviceToHost));
    int32_t dst = 0;
    CU(cudaMemcpy(&dst, c->status, sizeof(int32_t), cudaMemcpyDeviceToHost));
    stats->device_status = dst;
    stats->kernels = kernels;
    stats->pass1_tiles = nmt * nnt;
    stats->pass1_exact = nmt * nnt;
    if (pruned) {
      int32_t cnt[33] = {0};
      CU(cudaMemcpy(cnt, c->ws + y.tcount, sizeof(cnt), cudaMemcpyDeviceToHost));
      stats->pass1_exact = cnt[0];
      stats->pass1_pruned = 1;
      stats->pass1_delta = delta ? 1 : 0;
      stats->pass1_bound_pairs = cnt[32];
    }
  }
  return EMC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Learned rotation proposal and the sparse Maximize
// ---------------------------------------------------------------------------
extern "C" {

int emc_features(emc_ctx* ctx, float* feat, emc_stream stream) {
  if (!ctx || !feat || !ctx->frames_loaded) return EMC_ERR_ARG;
  const Layout& y = ctx->lay;
  CU(launch_features(ctx->Kb, ctx->cfg.precision == EMC_PREC_FP16_SPLIT, y.ld_pix,
                     ctx->cfg.n_pix, ctx->cfg.n_data, y.ld_data,
                     (const int16_t*)(ctx->ws + y.fbin), (const float*)(ctx->ws + y.finv), feat,
                     (cudaStream_t)stream));
  return EMC_OK;
}

int64_t emc_mlp_param_count(int64_t n_out) {
  if (n_out < 1) return EMC_ERR_ARG;
  return mlp_layout(n_out, 1).n_params;
}

int emc_mlp_work_size(int64_t n_out, int64_t batch, size_t* bytes) {
  if (n_out < 1 || batch < 1 || !bytes) return EMC_ERR_ARG;
  *bytes = sizeof(float) * (size_t)mlp_layout(n_out, batch).work_floats;
  return EMC_OK;
}

int emc_mlp_forward(int64_t n_out, const float* params, const float* X, int64_t batch, void* work,
                    float* logits, emc_stream stream) {
  if (n_out < 1 || batch < 1 || batch > (1 << 30) || !params || !X || !work || !logits)
    return EMC_ERR_ARG;
  CU(mlp_forward(mlp_layout(n_out, batch), params, X, (int)batch, (float*)work, logits,
                 (cudaStream_t)stream));
  return EMC_OK;
}

int emc_mlp_train_step(int64_t n_out, float* params, float* grads, float* adam_m, float* adam_v,
                       int step, float lr, const float* X, const int32_t* tidx, const float* tprob,
                       int64_t batch, int R, void* work, double* loss, emc_stream stream) {
  if (n_out < 1 || batch < 1 || batch > (1 << 30) || step < 1 || !(lr > 0.f) || R < 1 ||
      !params || !grads || !adam_m || !adam_v || !X || !tidx || !tprob || !work || !loss)
    return EMC_ERR_ARG;
  CU(mlp_train_step(mlp_layout(n_out, batch), params, grads, adam_m, adam_v, step, lr, X, tidx,
                    tprob, (int)batch, R, (float*)work, loss, (cudaStream_t)stream));
  return EMC_OK;
}

int emc_topm(const float* logits, int64_t batch, int64_t n, int64_t ld, int M, int32_t* cand,
             emc_stream stream) {
  if (!logits || !cand || batch < 0 || n < 1 || n > INT32_MAX || ld < n || M < 1 || M > n)
    return EMC_ERR_ARG;
  CU(launch_topm(logits, batch, n, ld, M, cand, (cudaStream_t)stream));
  return EMC_OK;
}

int emc_targets_from_scores(emc_ctx* ctx, const void* scores, int R, int32_t* tidx, float* tprob,
                            emc_stream stream) {
  if (!ctx || !tidx || !tprob || R < 1 || R > kMaxTargets || R > ctx->cfg.n_rot) return EMC_ERR_ARG;
  const Layout& y = ctx->lay;
  if (!scores) {
    if (!(ctx->cfg.flags & EMC_FLAG_STORE_SCORES)) return EMC_ERR_ARG;
    scores = ctx->ws + y.S;
  }
  const float* S = (const float*)scores;
  // the context's own scores after emc_iteration: its internal frame order and,
  // if that pass was bound-pruned, its live tiles only
  const bool internal = scores == (const void*)(ctx->ws + y.S) && ctx->scores_internal;
  CU(launch_topr_columns(S, y.rows, S + y.rows * y.ld_data, y.ld_data, ctx->cfg.n_rot,
                         ctx->cfg.n_data, R, tidx, tprob, (cudaStream_t)stream,
                         internal ? (const int32_t*)(ctx->ws + y.iperm) : nullptr,
                         internal && ctx->last_pruned ? (const uint8_t*)(ctx->ws + y.live)
                                                      : nullptr));
  return EMC_OK;
}

int emc_merge_candidates(const int32_t* first, int R, const int32_t* rest, int M_rest, int64_t n,
                         int M, int32_t* out, emc_stream stream) {
  if (!rest || !out || n < 0 || M < 1 || R < 0 || R > kMaxTargets || M_rest < M) return EMC_ERR_ARG;
  if (R > 0 && !first) return EMC_ERR_ARG;
  CU(launch_merge_candidates(first, R, rest, M_rest, n, M, out, (cudaStream_t)stream));
  return EMC_OK;
}

int emc_set_candidates(emc_ctx* ctx, const int32_t* cand, emc_stream stream) {
  if (!ctx || !cand || ctx->cfg.n_cand < 1) return EMC_ERR_ARG;
  const Layout& y = ctx->lay;
  const int M = ctx->cfg.n_cand;
  cudaStream_t s = (cudaStream_t)stream;
  int32_t* dc = (int32_t*)(ctx->ws + y.cand);
  CU(cudaMemcpyAsync(dc, cand, sizeof(int32_t) * (size_t)ctx->cfg.n_data * M,
                     cudaMemcpyDeviceToDevice, s));
  CU(launch_csr_build(dc, ctx->cfg.n_data, M, ctx->cfg.n_rot, y.rows,
                      (int32_t*)(ctx->ws + y.ccnt), (int64_t*)(ctx->ws + y.coff),
                      (int2*)(ctx->ws + y.cent), ctx->status, s));
  ctx->cand_loaded = true;
  return EMC_OK;
}

int emc_sparse_estep(emc_ctx* ctx, const void* L, const double* bias, float* P, double* lse,
                     emc_stream stream) {
  if (!ctx || !L || !bias || !P || !lse || !ctx->frames_loaded || !ctx->cand_loaded)
    return EMC_ERR_ARG;
  const Layout& y = ctx->lay;
  cudaStream_t s = (cudaStream_t)stream;
  const int M = ctx->cfg.n_cand;
  Planes lp{(void*)L, y.rows * y.ld_pix, y.ld_pix};
  double* Sc = (double*)(ctx->ws + y.Sc);
  const bool csr = (ctx->cfg.flags & EMC_FLAG_SPARSE_K) != 0;  // frames' non-zero lists
  CU(launch_sparse_scores(lp, ctx->cfg.precision, y.rows, bias, ctx->Kb, y.ld_pix,
                          (const int64_t*)(ctx->ws + y.coff), (const int2*)(ctx->ws + y.cent), M,
                          csr ? (const int64_t*)(ctx->ws + y.skoff) : nullptr,
                          csr ? (const uint32_t*)(ctx->ws + y.skent) : nullptr, Sc, s));
  CU(launch_sparse_lse(Sc, ctx->cfg.n_data, y.ld_data, M, P, lse, ctx->status, s, ctx->flu_cn));
  return EMC_OK;
}

int emc_sparse_update(emc_ctx* ctx, const float* P, float* Num, float* den, emc_stream stream) {
  if (!ctx || !P || !Num || !den || !ctx->frames_loaded || !ctx->cand_loaded) return EMC_ERR_ARG;
  const Layout& y = ctx->lay;
  const bool csr = (ctx->cfg.flags & EMC_FLAG_SPARSE_K) != 0;  // frames' non-zero lists
  CU(launch_sparse_update(ctx->Kb, ctx->cfg.precision == EMC_PREC_FP16_SPLIT, y.ld_pix,
                          ctx->cfg.n_pix, (const int64_t*)(ctx->ws + y.coff),
                          (const int2*)(ctx->ws + y.cent), ctx->cfg.n_cand, P, y.rows,
                          csr ? (const int64_t*)(ctx->ws + y.skoff) : nullptr,
                          csr ? (const uint32_t*)(ctx->ws + y.skent) : nullptr, Num, den,
                          (cudaStream_t)stream, ctx->flu_B, ctx->flu_invn));
  return EMC_OK;
}

int emc_sparse_iteration(emc_ctx* c, const float* grid_in, float* grid_out, emc_iter_stats* stats,
                         emc_stream stream) {
  if (!c || !grid_in || !grid_out || grid_in == grid_out) return EMC_ERR_ARG;
  if (!c->frames_loaded || !c->cand_loaded) return EMC_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const Layout& y = c->lay;
  // pruned contexts: the buffer the last emc_iteration did not write, so that
  // its L stays for the next one's incremental bound
  const bool other = c->prune && c->lcur == 0;
  void* L = c->ws + (other ? y.L2 : y.L);
  double* bias = (double*)(c->ws + (other ? y.bias2 : y.bias));
  float* Pc = (float*)(c->ws + y.Pc);
  double* lsec = (double*)(c->ws + y.lsec);
  float* Num = (float*)(c->ws + y.Num);
  float* den = (float*)(c->ws + y.den);
  double* gn = (double*)(c->ws + y.gnum);
  double* gd = (double*)(c->ws + y.gden);
  double* ll = (double*)(c->ws + y.scalar);
  const size_t gb = sizeof(double) * (size_t)c->cfg.N * c->cfg.N * c->cfg.N * c->lay.nrep;
  int st;
  if (stats) CU(cudaEventRecord(c->ev[0], s));
  if ((st = do_expand(c, grid_in, 0, c->cfg.n_rot, L, bias, s))) return st;
  if (stats) CU(cudaEventRecord(c->ev[1], s));
  if ((st = emc_sparse_estep(c, L, bias, Pc, lsec, stream))) return st;
  CU(launch_loglik_sum(lsec, nullptr, c->cfg.n_data, ll, s));  // sum_k lse_k over C_k
  if (stats) CU(cudaEventRecord(c->ev[2], s));
  if ((st = emc_sparse_update(c, Pc, Num, den, stream))) return st;
  if (stats) CU(cudaEventRecord(c->ev[3], s));
  CU(cudaMemsetAsync(gn, 0, gb, s));
  CU(cudaMemsetAsync(gd, 0, gb, s));
  CU(launch_compress(c->geom, (const RotFX*)(c->ws + y.rotfx), c->cfg.n_rot, Num, den, c->cfg.compress_mode, gn, gd,
                     y.nrep, s));
  CU(launch_finalize((int64_t)c->cfg.N * c->cfg.N * c->cfg.N, gn, gd, y.nrep, grid_in, grid_out,
                     s));
  if (stats) CU(cudaEventRecord(c->ev[4], s));
  if (stats) {
    CU(cudaEventSynchronize(c->ev[4]));
    float te = 0, tl = 0, tu = 0, tc = 0, tt = 0;
    CU(cudaEventElapsedTime(&te, c->ev[0], c->ev[1]));
    CU(cudaEventElapsedTime(&tl, c->ev[1], c->ev[2]));
    CU(cudaEventElapsedTime(&tu, c->ev[2], c->ev[3]));
    CU(cudaEventElapsedTime(&tc, c->ev[3], c->ev[4]));
    CU(cudaEventElapsedTime(&tt, c->ev[0], c->ev[4]));
    memset(stats, 0, sizeof(*stats));
    stats->ms_expand = te;
    stats->ms_loglik = tl;
    stats->ms_update = tu;
    stats->ms_compress = tc;
    stats->ms_total = tt;
    CU(cudaMemcpy(&stats->loglik, ll, sizeof(double), cudaMemcpyDeviceToHost));
    int32_t dst = 0;
    CU(cudaMemcpy(&dst, c->status, sizeof(int32_t), cudaMemcpyDeviceToHost));
    stats->device_status = dst;
    stats->kernels = 9;
  }
  return EMC_OK;
}

int emc_missed_mass(emc_ctx* ctx, const void* scores, const double* lse_m, const double* lse_s,
                    float* missed, emc_stream stream) {
  if (!ctx || !missed || !ctx->cand_loaded) return EMC_ERR_ARG;
  const Layout& y = ctx->lay;
  if (!scores) {
    if (!(ctx->cfg.flags & EMC_FLAG_STORE_SCORES)) return EMC_ERR_ARG;
    scores = ctx->ws + y.S;
  }
  if (!lse_m) lse_m = (const double*)(ctx->ws + y.lse_m);
  if (!lse_s) lse_s = (const double*)(ctx->ws + y.lse_s);
  cudaStream_t s = (cudaStream_t)stream;
  float2* lse2 = (float2*)(ctx->ws + y.lse2);
  CU(launch_lse_split(lse_m, lse_s, ctx->cfg.n_data, y.ld_data, lse2, s, ctx->flu_cn));
  const float* S = (const float*)scores;
  const bool internal = scores == (const void*)(ctx->ws + y.S) && ctx->scores_internal;
  CU(launch_missed_mass(S, y.rows, S + y.rows * y.ld_data, y.ld_data, lse2,
                        (const int32_t*)(ctx->ws + y.cand), ctx->cfg.n_cand, ctx->cfg.n_data,
                        missed, s, internal ? (const int32_t*)(ctx->ws + y.iperm) : nullptr,
                        internal && ctx->last_pruned ? (const uint8_t*)(ctx->ws + y.live)
                                                     : nullptr));
  return EMC_OK;
}

size_t emc_collect_bytes(const emc_ctx* ctx, int64_t cap) {
  if (!ctx || cap < 1) return 0;
  return collect_layout(cap, ctx->cfg.n_data, nullptr, nullptr);
}

int emc_set_collect(emc_ctx* ctx, void* buf, int64_t cap) {
  if (!ctx) return EMC_ERR_ARG;
  if (!buf) {
    ctx->collecting = false;
    ctx->collected = false;
    return EMC_OK;
  }
  if (cap < 1 || cap > (1LL << 31) || ((uintptr_t)buf & 255)) return EMC_ERR_ARG;
  const int p = ctx->cfg.precision;
  if (p == EMC_PREC_FP32 || is_gauss(&ctx->cfg)) return EMC_ERR_UNSUPPORTED;
  if (is_flu(&ctx->cfg) && p != EMC_PREC_BF16 && p != EMC_PREC_BF16_SPLIT)
    return EMC_ERR_UNSUPPORTED;
  collect_layout(cap, ctx->cfg.n_data, &ctx->col, (char*)buf);
  ctx->collecting = true;
  ctx->collected = false;
  return EMC_OK;
}

int emc_collected_targets(emc_ctx* ctx, int R, int32_t* tidx, float* tprob, float* missed,
                          emc_stream stream) {
  if (!ctx || !tidx || !tprob || R < 1 || R > 64 || R > ctx->cfg.n_rot) return EMC_ERR_ARG;
  if (!ctx->collected || !ctx->collecting) return EMC_ERR_ARG;
  if (missed && !ctx->cand_loaded) return EMC_ERR_ARG;
  CU(launch_collected_targets(ctx->col, ctx->cfg.n_data, ctx->cfg.n_rot, R, tidx, tprob,
                              missed ? (const int32_t*)(ctx->ws + ctx->lay.cand) : nullptr,
                              ctx->cfg.n_cand, missed, ctx->status, (cudaStream_t)stream));
  return EMC_OK;
}

int emc_iteration_lse(emc_ctx* ctx, double* lse, emc_stream stream) {
  if (!ctx || !lse || !ctx->iterated) return EMC_ERR_ARG;
  const Layout& y = ctx->lay;
  CU(launch_lse_values((const double*)(ctx->ws + y.lse_m), (const double*)(ctx->ws + y.lse_s),
                       ctx->cfg.n_data, lse, (cudaStream_t)stream));
  return EMC_OK;
}

int emc_responsibilities(emc_ctx* ctx, const int32_t* frames, int64_t n, float* P,
                         emc_stream stream) {
  if (!ctx || !frames || !P || n < 1 || !ctx->iterated) return EMC_ERR_ARG;
  if (!(ctx->cfg.flags & EMC_FLAG_STORE_SCORES)) return EMC_ERR_ARG;
  const Layout& y = ctx->lay;
  cudaStream_t s = (cudaStream_t)stream;
  float2* lse2 = (float2*)(ctx->ws + y.lse2);
  CU(launch_lse_split((const double*)(ctx->ws + y.lse_m), (const double*)(ctx->ws + y.lse_s),
                      ctx->cfg.n_data, y.ld_data, lse2, s, ctx->flu_cn));
  const float* S = (const float*)(ctx->ws + y.S);
  CU(launch_responsibilities(S, y.rows, S + y.rows * y.ld_data, y.ld_data, lse2, frames, n,
                             ctx->cfg.n_rot, ctx->cfg.n_data, P, ctx->status, s,
                             ctx->scores_internal ? (const int32_t*)(ctx->ws + y.iperm) : nullptr,
                             ctx->scores_internal && ctx->last_pruned
                                 ? (const uint8_t*)(ctx->ws + y.live)
                                 : nullptr));
  return EMC_OK;
}

}  // extern "C"
