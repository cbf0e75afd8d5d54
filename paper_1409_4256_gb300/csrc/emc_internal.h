// emc_internal.h -- launchers shared between the ABI layer and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/emc.h"

namespace emc {

// Rotation matrix R_j (row-major 3x3) as double-float pairs (h, l) of FP32,
// computed once per context on the host in FP64.
struct RotDF;

// Rotation R_j in fixed point for the e-step: R = hi 2^-20 + lo (hi integer,
// |lo| <= 2^-21), row-major 3x3.
struct RotFX {
  int32_t hi[9];
  float lo[9];
};

// Pixel geometry as stored in the workspace: positions q_i split into FP32
// hi/lo pairs, w component 1 for a used pixel and 0 for padding; the same in
// fixed point for the e-step: q = qi 2^-12 + qlo (qi.w = the w component).
struct Geom {
  const float4* qh;
  const float4* ql;
  const int4* qi;
  const float4* qlo;
  int64_t n_pix;
  int64_t ld_pix;
  int N;
  int interior;  // every |q_i| < N/2 - 1 with margin: all 8 corners of every R_j q_i lie in the grid
  // compression groups: the used pixels split by (q_x, q_y) into groups of at
  // most kCompressGroup pixels spanning at most kCompressExtent voxels along
  // q_x and q_y (pixel_groups.h); group g holds the positions
  // gstart[g] .. gstart[g + 1] of gpix (pixel columns) and of gqh/gql (their
  // geometry in that order)
  int ngroups;
  const int32_t* gstart;
  const int32_t* gpix;
  const float4* gqh;
  const float4* gql;
  const int4* gqi;    // the same in fixed point
  const float4* gqlo;
  const float4* gqf;  // gqi 2^-12 as FP32
};
constexpr int kCompressGroup = 32;
constexpr double kCompressExtent = 8.0;

// A block of rows of a (possibly multi-plane) row-major matrix.
struct Planes {
  void* base;            // first row of plane 0
  int64_t plane_stride;  // elements between planes
  int64_t ld;            // elements between rows
};

// fp16: bit 0 FP16 frames (EMC_PREC_FP16_SPLIT), else BF16; bit 1 no limit on
// the frame total (the Gaussian model's two copies)
// dup_src/dup_rank (device int32[kDupCols], NULL without duplicates): source
// pixel of each duplicate column n_pix + 1 + d and its rank among that pixel's
// duplicates; counts are then split in parts of at most kDupCount.
cudaError_t launch_prep_frames(const int32_t* K, int64_t ld_k, int64_t n_data, int64_t n_pix,
                               int64_t ld_data, int64_t ld_pix, uint16_t* Kb, int fp16,
                               const int32_t* dup_src, const int32_t* dup_rank,
                               int32_t* status, cudaStream_t s);
// Duplicate columns for counts above kDupCount: per-pixel maxima over the
// frames, then one thread assigns columns in pixel order and writes their
// geometry (w = kDupMark) and feature bins. pixmax: int32[n_pix] scratch.
cudaError_t launch_assign_duplicates(const int32_t* K, int64_t ld_k, int64_t n_data, int64_t n_pix,
                                     int64_t ld_data, int32_t* pixmax, float4* qh, float4* ql,
                                     int16_t* fbin, int32_t* dup_src, int32_t* dup_rank,
                                     int32_t* status, cudaStream_t s);

// gsc != NULL: Gaussian model (FP16 three-plane s W, bias log w - sum W^2 / 2 sigma^2)
// g4 (may be NULL): the grid in the corner-pair layout (launch_grid_pairs)
cudaError_t launch_expand(const Geom& g, const float* grid, const float4* g4, const RotDF* rot,
                          const double* logw, int64_t nrot, int64_t rows, int precision,
                          float w_floor, Planes L, double* bias, const float4* gsc, double sigma,
                          int32_t* status, cudaStream_t s);

// Poisson model: the e-step per row tile of 128 rotations (expand_tile.cu).
// partial: scratch of expand_tile_slices(ld_pix) x rows doubles. With Lold
// (the last iteration's L, same layout) it also writes the incremental bound's
// increments D ([2 ntp][ld_pix], rounded up to the frames' type), dabs[t] and,
// from bias_old, bpm (as launch_delta_planes).
int64_t expand_tile_slices(int64_t ld_pix);
// g4 (may be NULL): the grid in the corner-pair layout (launch_grid_pairs),
// read where every corner lies inside the grid
cudaError_t launch_grid_pairs(const float* grid, int N, float4* g4, cudaStream_t s);
cudaError_t launch_expand_tile(const Geom& g, const float* grid, const float4* g4,
                               const RotFX* rot,
                               const double* logw, int64_t nrot, int64_t rows, int precision,
                               float w_floor, Planes L, double* bias, double* partial,
                               const void* Lold, const double* bias_old, uint16_t* D, int64_t ntp,
                               float* bpm, int32_t* status, cudaStream_t s);
// qi, qlo (and qf = qi 2^-12 as FP32, if non-NULL) from qh, ql for ld_pix columns
cudaError_t launch_fixed_geometry(const float4* qh, const float4* ql, int64_t ld_pix, int4* qi,
                                  float4* qlo, float4* qf, cudaStream_t s);

// Poisson-fluence model: L = log(W / B_j) + c as the BF16 three-term split
// (precision EMC_PREC_BF16_SPLIT only); bias = double[2][rows]: log w_j, then
// B_j = sum_i W_ij; Bctx[row] = B_j too.
cudaError_t launch_expand_flu(const Geom& g, const float* grid, const float4* g4, const RotDF* rot,
                              const double* logw, int64_t nrot, int64_t rows, int precision,
                              float w_floor, double c, Planes L, double* bias, double* Bctx,
                              int32_t* status, cudaStream_t s);
// Per frame: cn[k] = c N_k, invn[k] = 1 / N_k (0 for empty and padding frames).
cudaError_t launch_flu_frames(const int32_t* K, int64_t ld_k, int64_t n_data, int64_t n_pix,
                              int64_t ld_data, double c, double* cn, float* invn,
                              cudaStream_t s);
// Pass 2 from stored scores: BF16 hi + lo planes of P B_j / N_k, den[rows] = sum_k P.
cudaError_t launch_normalize_scores_flu(const float* S, int64_t ldS, const float* Sref,
                                        const float2* lse2, const double* Bsum, const float* invn,
                                        int64_t rows, int64_t nrot, int64_t ld_data,
                                        int64_t n_data, uint16_t* P, int64_t P_plane, float* den,
                                        cudaStream_t s, uint8_t* kb_flag = nullptr,
                                        const uint8_t* tile_live = nullptr);
// Non-zero P blocks (update over those only): the normalisations set
// flag[mt * kb_ld + kb] (kb_ld = ld_data / 64) for every 128-row x 64-frame
// block of P with a non-zero entry; this lists them per row tile.
cudaError_t launch_kb_lists(const uint8_t* flag, int64_t n_mtiles, int kb_ld, int32_t* cnt,
                            int32_t* list, cudaStream_t s);

// ---- Gaussian model (misc.cu) ----
// Per-frame constants gk[ld_data] = (c_k hi, c_k lo, 2 sigma^2 / A_k, 0) and the
// largest frame total (*nmax).
cudaError_t launch_gauss_frames(const int32_t* K, int64_t ld_k, int64_t n_data, int64_t n_pix,
                                int64_t ld_data, double sigma, float4* gk,
                                unsigned long long* nmax, cudaStream_t s);
// max(grid) into *gmax, then the scales (s, 1/s^2, 0, 0) into *gsc.
cudaError_t launch_gauss_scales(const float* grid, int64_t n_vox, unsigned* gmax,
                                const unsigned long long* nmax, float4* gsc, int32_t* status,
                                cudaStream_t s);
// Pass 2 from stored scores: BF16 hi + lo planes of P / phi, den[rows] = sum_k P.
cudaError_t launch_normalize_scores_gauss(const float* S, int64_t ldS, const float* Sref,
                                          const float2* lse2, const double* bias,
                                          const float4* gk, int64_t rows,
                                          int64_t nrot, int64_t ld_data, int64_t n_data,
                                          uint16_t* P, int64_t P_plane, float* den,
                                          cudaStream_t s, uint8_t* kb_flag = nullptr);

// FP32 SIMT forms (precision EMC_PREC_FP32).
// S, Sref (optional, both or neither): scores relative to 32-row group maxima,
// frame-major [ld_data][rows], and the maxima (on the 1/64 grid) [rows / 32][ld_data].
cudaError_t launch_simt_pass1(const float* L, int64_t ld_pix, const double* bias, int64_t rows,
                              const uint16_t* Kb, int64_t ld_data, int64_t n_data,
                              double* part_m, float* part_s, float* S, float* Sref,
                              cudaStream_t s);
cudaError_t launch_simt_normalize(const float* L, int64_t ld_pix, const double* bias, int64_t rows,
                                  int64_t nrot, const uint16_t* Kb, int64_t ld_data,
                                  int64_t n_data, const double* lse_m, const double* lse_s,
                                  float* P, cudaStream_t s);
cudaError_t launch_simt_update(const float* P, int64_t ld_data, int64_t rows, const uint16_t* Kb,
                               int64_t ld_pix, int64_t n_pix, float* Num, float* den,
                               cudaStream_t s);
int64_t simt_pass1_tiles(int64_t rows);

// Merge of per-tile (max, sum) pairs into the running per-frame (m, s).
// shift (may be NULL): per-frame constant carried by the tiles' scores
// (double[ld_data]), removed before the merge.
// live (may be NULL): [n_tiles][ld_data / 256] flags of the contracted tiles
// of a pruned pass 1; best (may be NULL): row tile of each frame's largest maximum.
// Ub, Mk (may be NULL): for the incremental bound, every merged tile's maximum
// + 1/64 into Ub[tile][frame] (rounded up to FP32) and each frame's largest
// maximum, as the scores carry it (shift included), into Mk.
cudaError_t launch_lse_merge(const double* part_m, const float* part_s, int64_t n_tiles,
                             int64_t ld_data, int64_t n_data, double* lse_m, double* lse_s,
                             int accumulate, int gauss, int32_t* status, cudaStream_t s,
                             const double* shift = nullptr, const uint8_t* live = nullptr,
                             int32_t* best = nullptr, float* Ub = nullptr, double* Mk = nullptr,
                             float* Ua = nullptr);
// ---- incremental bound between consecutive iterations (prune.cu) ----
// D ([3 ntp][ld_pix], BF16, or FP16 when f16) rows t and ntp + t: max over the
// tile's valid rows of L1 - L0 and of L0 - L1 (BF16 split: three planes; f16,
// the FP16 split's two; plane stride `plane`), rows 2 ntp + t: a bound of both
// magnitudes; all rounded up; bpm[t], bpm[nt + t] = the same maxima of the
// bias change (b1 - b0), rounded up.
cudaError_t launch_delta_planes(const uint16_t* L0, const uint16_t* L1, int64_t plane,
                                int64_t ld_pix, int64_t nrot, const double* b0, const double* b1,
                                int64_t ntp, uint16_t* D, float* bpm, int f16, cudaStream_t s);
// Ub += C+ + b+ + err, Lk from Mk, best and C- (C = D K^T, rows t, ntp + t and
// 2 ntp + t, the last giving err);
// cand[t][nt] where Ub >= Lk - 111 and the widening exceeds the hi-plane
// bound's 2 (N_k / div + 1); valid = 0, changed[0] or changed[2]: every tile
// a candidate, Ub = +inf, Lk = -inf.
// Ua: the widening gathered since each tile bound's last refresh (cleared by
// the refreshes: the hi-plane bound in launch_final_live, the exact maxima in
// the merge).
cudaError_t launch_delta_live(const float* C, int64_t ntp, const float* bpm,
                              float* Ub, float* Ua, double* Lk, const double* Mk,
                              const int32_t* best,
                              const float* nsum, float div, int64_t ld_pix, int64_t n_mtiles,
                              int64_t ld_data, int64_t n_data, int valid,
                              const int32_t* changed, uint8_t* cand, cudaStream_t s);
// pf[mp][nt] = cand[2 mp][nt] | cand[2 mp + 1][nt]
cudaError_t launch_pair_flags(const uint8_t* cand, int64_t n_mtiles, int64_t nnt, uint8_t* pf,
                              cudaStream_t s);
// hi-plane maxima of the flagged pairs tighten Ub and Lk; live[t][nt] where Ub >= Lk - 111
cudaError_t launch_final_live(const double* part_m, const uint8_t* pf, float* Ub, float* Ua,
                              double* Lk,
                              const float* nsum, float div, int64_t n_mtiles, int64_t ld_data,
                              int64_t n_data, uint8_t* live, cudaStream_t s);
// Ub2, Mk2, best2 = Ub, Mk, best at each frame's old position
// (src[pos] = iperm_old[perm_new[pos]])
cudaError_t launch_reorder_state(const int32_t* perm_new, const int32_t* iperm_old, int64_t n_data,
                                 int64_t ld_data, int64_t n_mtiles, int32_t* src, const float* Ub,
                                 float* Ub2, const float* Ua, float* Ua2, const double* Mk,
                                 double* Mk2, const int32_t* best, int32_t* best2,
                                 cudaStream_t s);
// *flag = 1 if any count of K (columns < n_pix) differs from the BF16 (FP16) copy Kb
cudaError_t launch_frames_differ(const int32_t* K, int64_t ld_k, int64_t n_data, int64_t n_pix,
                                 const uint16_t* Kb, int64_t ld_pix, int fp16, int32_t* flag,
                                 cudaStream_t s);
// shift (may be NULL): added back to lse before the split.
cudaError_t launch_lse_split(const double* lse_m, const double* lse_s, int64_t n_data,
                             int64_t ld_data, float2* out, cudaStream_t s,
                             const double* shift = nullptr);
// E-step pass 2 from stored scores (frame-major, ld ldS); P layout as
// emc_normalize documents.
cudaError_t launch_normalize_scores(const float* S, int64_t ldS, const float* Sref,
                                    const float2* lse2, int64_t rows, int64_t nrot,
                                    int64_t ld_data, int64_t n_data, int precision, void* P,
                                    int64_t P_plane, cudaStream_t s, uint8_t* kb_flag = nullptr,
                                    const uint8_t* tile_live = nullptr);
cudaError_t launch_loglik_sum(const double* lse_m, const double* lse_s, int64_t n_data,
                              double* out, cudaStream_t s);

// Control of the tensor-core launches' bounded waits: wait_ns = 0 is the
// default limit (2 s); stall != 0 is the test hook of emc_ctx_set_wait_limit
// (the MMA issuer's first wait is on a barrier nothing completes).
struct TcCtl {
  uint64_t wait_ns;
  int stall;
};

// tcgen05 forms (precision EMC_PREC_BF16 / BF16_SPLIT / FP16_SPLIT).
// gk, gsc != NULL: the Gaussian model's pass 1 (three FP16 planes of s W).
// tile_list, tile_count (device, optional): contract only the listed
// (row tile, frame tile) pairs, codes mt * (ld_data / 256) + nt, *tile_count of them
cudaError_t launch_tc_pass1(const Planes& L, int precision, const double* bias, int64_t rows,
                            const uint16_t* Kb, int64_t ld_data, int64_t n_data, int64_t ld_pix,
                            double* part_m, float* part_s, float* S, float* Sref,
                            const float4* gk, const float4* gsc, int32_t* status,
                            cudaStream_t s, const int32_t* tile_list = nullptr,
                            const int32_t* tile_count = nullptr, TcCtl ctl = TcCtl{});
// lse2: scratch float2[ld_data] for lse_k split into a 1/8-grid part and a rest.
// Bsum != NULL: Poisson-fluence model -- shift[ld_data] is added back to lse,
// the planes receive BF16 hi + lo of P B_j invn[k] and den[rows] = sum_k P_jk
// (zeroed here, then FP32 atomics). tile_list, tile_count (optional): only the
// listed (row tile, frame tile) pairs are recomputed and written (P elsewhere
// is left as it was: with kb_flag, readers skip those blocks).
cudaError_t launch_tc_normalize(const Planes& L, int precision, const double* bias, int64_t rows,
                                int64_t nrot, const uint16_t* Kb, int64_t ld_data, int64_t n_data,
                                int64_t ld_pix, const double* lse_m, const double* lse_s,
                                float2* lse2, Planes P, int32_t* status, cudaStream_t s,
                                const double* shift = nullptr, const double* Bsum = nullptr,
                                const float* invn = nullptr, float* den = nullptr,
                                uint8_t* kb_flag = nullptr, const int32_t* tile_list = nullptr,
                                const int32_t* tile_count = nullptr, TcCtl ctl = TcCtl{});
// P planes: hi + lo (BF16 split, FP16 split) or hi only (BF16); FP16 planes
// carry the scale 2^14. den NULL: not written.
// kb_cnt, kb_list (optional, from launch_kb_lists): contract only the listed
// 64-frame blocks of each row tile (the others of P are zero). staged: write
// Num through a shared-memory staging block, for updates bound by their output
// (few listed blocks); it costs the two-plane update a pipeline stage
cudaError_t launch_tc_update(const Planes& P, int precision, int64_t rows, const uint16_t* Kb,
                             int64_t ld_data, int64_t ld_pix, int64_t n_pix, float* Num, float* den,
                             int32_t* status, cudaStream_t s, const int32_t* kb_cnt = nullptr,
                             const int32_t* kb_list = nullptr, TcCtl ctl = TcCtl{},
                             bool staged = false);
int64_t tc_pass1_tiles(int64_t rows);
// C (float[rows][ld_data]) = A Kb^T over ld_pix columns, A one plane of rows
// (a multiple of 128) x ld_pix, Kb [ld_data][ld_pix], both BF16 (or both FP16
// when f16): a plain tensor-core product, FP32 accumulation, stored as it is.
cudaError_t launch_tc_store(const Planes& A, int64_t rows, const uint16_t* Kb, int64_t ld_data,
                            int64_t ld_pix, float* C, int f16, int32_t* status, cudaStream_t s,
                            TcCtl ctl = TcCtl{});
// Bound pass of the pruned pass 1: per 128-row tile and frame, the maximum of
// S^hi = (first plane of L) K^T + bias into part_m[rows / 128][ld_data]
// (pairs of row tiles per CTA tile sharing the frame operand).
// pair_list, pair_count (device, optional): contract only the listed pairs,
// codes mp * (ld_data / 256) + nt for row tiles 2 mp and 2 mp + 1.
cudaError_t launch_tc_bound(const Planes& L, int precision, const double* bias, int64_t rows,
                            const uint16_t* Kb, int64_t ld_data, int64_t ld_pix, double* part_m,
                            int32_t* status, cudaStream_t s, TcCtl ctl = TcCtl{},
                            const int32_t* pair_list = nullptr,
                            const int32_t* pair_count = nullptr);

// nrep grid replicas of n_vox each (row j reduces into replica j mod nrep)
cudaError_t launch_compress(const Geom& g, const RotFX* rot, int64_t nrot, const float* Num,
                            const float* den, int mode, double* g_num, double* g_den, int nrep,
                            cudaStream_t s);
// grid_out = (sum of nrep numerator replicas) / (sum of denominator replicas)
cudaError_t launch_finalize(int64_t n_vox, const double* g_num, const double* g_den, int nrep,
                            const float* grid_prev, float* grid_out, cudaStream_t s);

// ---- learned proposal (learned.cu) ----
constexpr int kFeat = 512;        // 32 radial x 16 angular bins = MLP width
constexpr int kMaxTargets = 64;   // soft targets per frame at most

struct MlpLayout {
  int64_t n_out, ld_out;          // logits per frame, padded to 64
  int64_t W[4], b[4];             // offsets (floats) in the parameter array
  int64_t n_params;
  int64_t B;                      // batch rows the work buffer holds
  int64_t work_floats;
};
MlpLayout mlp_layout(int64_t n_out, int64_t B);
// kf16 != 0: frames in FP16, else BF16 (likewise for the sparse update)
cudaError_t launch_features(const uint16_t* Kb, int kf16, int64_t ld_pix, int64_t n_pix,
                            int64_t n_data, int64_t ld_data, const int16_t* bin,
                            const float* inv_count, float* feat, cudaStream_t s);
cudaError_t mlp_forward(const MlpLayout& y, const float* params, const float* X, int B,
                        float* work, float* logits, cudaStream_t s);
cudaError_t mlp_train_step(const MlpLayout& y, float* params, float* grads, float* adam_m,
                           float* adam_v, int step, float lr, const float* X,
                           const int32_t* tidx, const float* tprob, int B, int R, float* work,
                           double* loss, cudaStream_t s);

// ---- candidates and the sparse Maximize (sparse.cu) ----
cudaError_t launch_topm(const float* logits, int64_t B, int64_t n, int64_t ld, int M,
                        int32_t* cand, cudaStream_t s);
// iperm, live (may be NULL): scores in emc_iteration's internal frame order
// (frame k in column iperm[k]) holding only the live row tiles
cudaError_t launch_topr_columns(const float* S, int64_t ldS, const float* Sref, int64_t ld, int64_t nrot,
                                int64_t n_data, int R, int32_t* tidx, float* tprob,
                                cudaStream_t s, const int32_t* iperm = nullptr,
                                const uint8_t* live = nullptr);
cudaError_t launch_merge_candidates(const int32_t* first, int R, const int32_t* rest, int M_rest,
                                    int64_t n, int M, int32_t* out, cudaStream_t s);
cudaError_t launch_csr_build(const int32_t* cand, int64_t n_data, int M, int64_t n_rot,
                             int64_t rows, int32_t* cnt, int64_t* off, int2* ent,
                             int32_t* status, cudaStream_t s);
// koff/kent (non-NULL): the frames' non-zero pixel lists (EMC_FLAG_SPARSE_K)
// replace their dense rows in both sparse contractions
cudaError_t launch_sparse_scores(const Planes& L, int precision, int64_t rows, const double* bias,
                                 const uint16_t* Kb, int64_t ld_pix, const int64_t* off,
                                 const int2* ent, int M, const int64_t* koff,
                                 const uint32_t* kent, double* Sc, cudaStream_t s);
// shift (may be NULL): per-frame constant of the scores, removed from lse_c
cudaError_t launch_sparse_lse(const double* Sc, int64_t n_data, int64_t ld_data, int M, float* Pc,
                              double* lse_c, int32_t* status, cudaStream_t s,
                              const double* shift = nullptr);
// Bsum, invn (non-NULL): Poisson-fluence model, Num_j = sum P_jk K_k B_j / N_k
// and den_j = sum P_jk
cudaError_t launch_sparse_update(const uint16_t* Kb, int kf16, int64_t ld_pix, int64_t n_pix,
                                 const int64_t* off, const int2* ent, int M, const float* Pc,
                                 int64_t rows, const int64_t* koff, const uint32_t* kent,
                                 float* Num, float* den, cudaStream_t s,
                                 const double* Bsum = nullptr, const float* invn = nullptr);
cudaError_t launch_missed_mass(const float* S, int64_t ldS, const float* Sref, int64_t ld_data,
                               const float2* lse2, const int32_t* cand, int M, int64_t n_data,
                               float* missed, cudaStream_t s, const int32_t* iperm = nullptr,
                               const uint8_t* live = nullptr);

// P[f][j] (float[n][nrot]) = exp(S_jk - lse_k) of frames k = frames[f] from
// stored scores (iperm, live as launch_missed_mass); an index outside
// [0, n_data) sets EMC_ERR_ARG and leaves that row unwritten
cudaError_t launch_responsibilities(const float* S, int64_t ldS, const float* Sref,
                                    int64_t ld_data, const float2* lse2, const int32_t* frames,
                                    int64_t n, int64_t nrot, int64_t n_data, float* P,
                                    int32_t* status, cudaStream_t s,
                                    const int32_t* iperm = nullptr,
                                    const uint8_t* live = nullptr);
// lse[k] = m[k] + log s[k] for k < n
cudaError_t launch_lse_values(const double* m, const double* sm, int64_t n, double* lse,
                              cudaStream_t s);

// ---- pruned pass 1 and the frame order (prune.cu) ----
// the live tiles (flags live[mt][nt]) as codes mt * n_ntiles + nt in raster
// order (groups of `group` row tiles) into list, their number into *count;
// scratch: tile_list_scratch_entries int32
cudaError_t launch_tile_list(const uint8_t* live, int n_mtiles, int n_ntiles, int group,
                             int32_t* list, int32_t* count, int32_t* scratch, cudaStream_t s);
int64_t tile_list_scratch_entries(int64_t n_mtiles, int64_t n_ntiles);
// entries of the histogram scratch H (int32) of launch_sort_frames; off needs one more (int64)
int64_t sort_scratch_entries(int64_t n_data, int nbins);
// new_perm[pos] = perm[s] for the frames s stably sorted by key[s] in [0, nbins)
cudaError_t launch_sort_frames(const int32_t* key, const int32_t* perm, int64_t n_data, int nbins,
                               int32_t* H, int64_t* off, int32_t* new_perm, cudaStream_t s);
// frames in the order perm: rows of Kb into Kp, nsum (and cn, invn if non-NULL); iperm
cudaError_t launch_permute_frames(const int32_t* perm, int64_t ld_data, int64_t ld_pix,
                                  const uint16_t* Kb, uint16_t* Kp, const float* nsum,
                                  float* nsum_p, const double* cn, double* cn_p, const float* invn,
                                  float* invn_p, int32_t* iperm, cudaStream_t s);
cudaError_t launch_frame_totals(const int32_t* K, int64_t ld_k, int64_t n_data, int64_t n_pix,
                                int64_t ld_data, float* nsum, cudaStream_t s);
cudaError_t launch_identity(int32_t* p, int64_t n, cudaStream_t s);
cudaError_t launch_unpermute_lse(const int32_t* perm, int64_t n_data, const double* m_s,
                                 const double* s_s, double* m, double* s, cudaStream_t st);

// exclusive scan of cnt[0, n) into off[0, n] (off[n] = total), one CTA
cudaError_t launch_scan_counts(const int32_t* cnt, int64_t n, int64_t* off, cudaStream_t s);

// ---- sparse-K pass 1 (sparse_k.cu) ----
// non-zero pixels of every frame: cnt[ld_data], off[ld_data + 1],
// ent[] = pixel | count << 16 in pixel order
cudaError_t launch_sparse_k_frames(const int32_t* K, int64_t ld_k, int64_t n_data, int64_t n_pix,
                                   int64_t ld_data, int32_t* cnt, int64_t* off, uint32_t* ent,
                                   cudaStream_t s);
// per 128-row tile (max, sum) pairs like the dense pass 1, from FP32 log W
cudaError_t launch_sparse_k_pass1(const float* L, int64_t ld_pix, int64_t n_pix, const double* bias,
                                  int64_t rows, const int64_t* off, const uint32_t* ent,
                                  int64_t ld_data, int64_t n_data, double* part_m, float* part_s,
                                  cudaStream_t s);
size_t sparse_k_smem(int64_t ld_pix);

// ---- recorded responsibilities (collect.cu) ----
// A caller-owned list of the non-zero P_jk of an iteration and the scratch of
// the targets computed from it.
struct CollectBuf {
  unsigned long long* count;  // entries appended (may exceed cap: overflow)
  int32_t* ek;                // frame (the user's order)
  int32_t* ej;                // rotation
  float* ep;                  // P_jk
  int32_t* sj;                // the entries grouped by frame
  float* sp;
  int32_t* cnt;               // [n_data + 1]
  int32_t* off;               // [n_data + 1]
  int32_t* fill;              // [n_data]
  int64_t cap;
};
// bytes of a list of cap entries for n_data frames; with b and base, the
// pointers into base
size_t collect_layout(int64_t cap, int64_t n_data, CollectBuf* b, char* base);
// the non-zero entries of the listed blocks of one chunk's P planes (rows
// row0 .. row0 + nr of the rotations; frame positions mapped by perm if given)
cudaError_t launch_collect(const void* P, int64_t plane, int64_t ld_data, int precision,
                           const double* Bsum, const float* invn, int64_t row0, int64_t nr,
                           int64_t n_mtiles, const int32_t* kbc, const int32_t* kbl, int kb_ld,
                           const int32_t* perm, int64_t n_data, const CollectBuf& b,
                           cudaStream_t s);
// top-R targets, their weights and (cand non-NULL) the candidate sets' missed mass
cudaError_t launch_collected_targets(const CollectBuf& b, int64_t n_data, int64_t n_rot, int R,
                                     int32_t* tidx, float* tprob, const int32_t* cand, int n_cand,
                                     float* missed, int32_t* status, cudaStream_t s);

// Host side of Eq. 2.7 (emc_quat.cpp).
int64_t quat_generate(int n, int uniform, double* quat, double* weight, int64_t cap);

}  // namespace emc
