/*
 * emc.h -- C ABI of libemc, the GB300 (sm_103a) EMC hot path.
 *
 * EMC (Expand-Maximize-Compress), Ekeberg, Engblom & Liu, arXiv:1409.4256,
 * Algorithm 2.1, with the Poisson noise model of Sec. 2.2:
 *   e-step  (Eq. 2.9)  W_ij  = sum_l f(p_l - R_j q_i) WW_l      (trilinear f)
 *   E-step  (Eq. 2.4)  P_jk  = w_j T_jk / sum_j' w_j' T_j'k,
 *                      log T_jk = sum_i K_ik log W_ij - W_ij    (log K! dropped)
 *   M-step  (Eq. 2.11) Num_ij = sum_k P_jk K_ik,  den_j = sum_k P_jk
 *   c-step  (Eq. 2.12) WW'_l = sum_ij f Num_ij / sum_ij f den_j
 * Indices: i pixel, j rotation, k frame (pattern), l grid voxel.
 *
 * Conventions for every call
 *  - Return value: EMC_OK (0) or a negative emc_status. Arguments, sizes and
 *    alignments are checked on the host before anything is launched; a failed
 *    check launches nothing. Calls taking a stream are asynchronous and
 *    stream-ordered; problems found on the device (counts out of range, a
 *    non-finite score, a bounded wait that gave up) are recorded in a device
 *    status word that emc_ctx_status() reads.
 *  - Ownership: every array argument is owned by the caller. Device arrays
 *    are plain device pointers; host arrays are marked "host". The library
 *    never allocates device memory: all scratch comes from the workspace the
 *    caller passes to emc_ctx_create(), sized by emc_workspace_size().
 *  - Grid layout: float [N][N][N], voxel (x, y, z) at (x*N + y)*N + z; the
 *    zero frequency sits at index N/2 along each axis, and a point q maps to
 *    grid coordinate q + N/2.
 *  - Rotations: unit quaternions (w, x, y, z), R_j applied to pixel positions.
 *  - Padding: pixels are padded to ld_pix (a multiple of 64, strictly more than
 *    n_pix), frames to ld_data (a multiple of 256), rotation blocks to a
 *    multiple of 128 rows. Sizes of every per-call buffer come from
 *    emc_buffer_sizes().
 */
#ifndef EMC_H
#define EMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* emc_stream; /* a cudaStream_t; NULL = legacy default */

typedef enum emc_status {
  EMC_OK = 0,
  EMC_ERR_ARG = -1,         /* bad argument, size or alignment */
  EMC_ERR_CUDA = -2,        /* a CUDA runtime call failed */
  EMC_ERR_NOMEM = -3,       /* workspace too small, or host memory for the staging ran out */
  EMC_ERR_UNSUPPORTED = -4, /* input outside what the kernels handle exactly */
  EMC_ERR_TIMEOUT = -5,     /* a bounded device wait gave up */
  EMC_ERR_NUMERIC = -6      /* non-finite or out-of-range value met on device */
} emc_status;

typedef enum emc_precision {
  /* log W in FP32, FP32 SIMT contractions with compensated accumulation */
  EMC_PREC_FP32 = 0,
  /* log W rounded to one BF16, tcgen05 BF16 MMA with FP32 accumulation */
  EMC_PREC_BF16 = 1,
  /* log W = hi + mid + lo in BF16 with hi on a fixed 1/8 grid (accumulated
   * exactly), tcgen05 BF16 MMA; P = hi + lo in BF16 for the update */
  EMC_PREC_BF16_SPLIT = 2,
  /* log W = hi + rest in FP16 with hi on a fixed 1/64 grid (accumulated
   * exactly), frames in FP16 (counts <= 2048 exact), tcgen05 FP16 MMA;
   * P = (hi + lo) / 2^14 in FP16 for the update. Two MMAs per K step where
   * the BF16 split needs three. Frames must keep sum_i K_ik below 8192. */
  EMC_PREC_FP16_SPLIT = 3
} emc_precision;

/* Noise model of the frames given W_ij (Sec. 2.2). */
typedef enum emc_model {
  /* Poisson: log P(K_ik | W_ij) = K_ik log W_ij - W_ij - log K_ik! */
  EMC_MODEL_POISSON = 0,
  /* Gaussian with per-(j,k) fluence (Eqs. 2.2-2.3, 2.5-2.6):
   * log P = -(K_ik / phi_jk - W_ij)^2 / (2 sigma^2) + const, with
   * phi_jk = sum_i K_ik^2 / sum_i W_ij K_ik evaluated on the model of the
   * current iteration (its least-squares optimum) and used in that
   * iteration's E- and M-step. Then
   *   S_jk = (G_jk^2 / A_k - B_j) / (2 sigma^2) + log w_j,
   *   G_jk = sum_i W_ij K_ik, A_k = sum_i K_ik^2, B_j = sum_i W_ij^2,
   * so the E-step is the same contraction over pixels with W in place of
   * log W. Needs precision EMC_PREC_FP16_SPLIT and EMC_FLAG_STORE_SCORES;
   * the sparse Maximize and emc_loglik_static are Poisson only. */
  EMC_MODEL_GAUSSIAN = 1,
  /* Poisson with a per-(j,k) fluence phi_jk (frames of unequal, unknown
   * intensity): K_ik ~ Poisson(phi_jk W_ij) with phi_jk its maximum-likelihood
   * value N_k / B_j (N_k = sum_i K_ik, B_j = sum_i W_ij) on the model of the
   * current iteration, the Poisson counterpart of Eq. 2.6. Then
   *   S_jk = sum_i K_ik log(W_ij / B_j) + log w_j
   * (the per-frame constant N_k log N_k - N_k and log K! left out), and the
   * M-step divides each frame by its fluence as Eq. 2.5 does:
   *   Num_ij = sum_k P_jk K_ik B_j / N_k, den_j = sum_k P_jk
   * (an empty frame contributes only to den). The E-step is the Poisson
   * contraction on log(W / B_j) in place of log W. Needs precision
   * EMC_PREC_BF16_SPLIT (the other forms hold one rounded value of
   * log(W / B_j) per element, whose per-rotation rounding bias the
   * contraction would multiply by N_k); emc_loglik_static and
   * emc_loglik_sparse_k are Poisson only. */
  EMC_MODEL_POISSON_FLUENCE = 2
} emc_model;

typedef enum emc_compress_mode {
  EMC_COMPRESS_DEFERRED = 0, /* Eq. 2.11-2.12: normalise after compression */
  EMC_COMPRESS_IDW = 1       /* Eq. 2.5 per slice, then Eq. 2.10 */
} emc_compress_mode;

/* emc_config.flags */
#define EMC_FLAG_STORE_SCORES 1 /* emc_iteration keeps pass-1 scores in the
                                   workspace (rows x ld_data x 4 B plus 1/32 of
                                   that) and derives P from them instead of
                                   recomputing the contraction */
#define EMC_FLAG_WIDE_COUNTS 4  /* counts above 256 (the largest integer range
                                   BF16 holds exactly): ld_pix reserves 64
                                   more columns, and emc_set_frames gives every
                                   pixel whose count exceeds 256 in some frame
                                   duplicate columns (same q_i) carrying the
                                   count in parts of at most 256; expansion
                                   leaves duplicates out of sum_i W_ij and
                                   compression out of the denominators, so every
                                   result is unchanged. More than 64 duplicate
                                   columns needed: EMC_ERR_UNSUPPORTED in the
                                   device status. Frame totals keep their
                                   limits. Not for emc_loglik_static. */
#define EMC_FLAG_DENSE_ESTEP 8  /* emc_iteration contracts every (rotation tile,
                                   frame tile) in pass 1. Without it, a context
                                   with a split precision (BF16 or FP16) and a
                                   Poisson model first bounds every tile's
                                   scores by a contraction of the hi plane alone
                                   (|S - S_hi| <= N_k/16 + 1 for the BF16
                                   split, N_k/128 + 1 for the FP16 split),
                                   then contracts exactly (in pass 1, and in a
                                   recomputing pass 2) only the tiles
                                   that can hold a score within 110 of their
                                   frames' maxima. The others have P = 0 in
                                   FP32 and no weight in lse at FP64 precision,
                                   so the results are those of the dense pass.
                                   From the second pruned iteration on the same
                                   frames, an incremental bound (the last
                                   iteration's tile maxima plus the largest
                                   change of log W over each tile, contracted
                                   per tile against the frames) first rules out
                                   tiles, and the hi-plane bound runs only over
                                   the rest. The context keeps the last
                                   iteration's L and bias for that (a second
                                   copy of each in the workspace); emc_set_frames
                                   with other counts voids it for one iteration.
                                   Frames are regrouped internally by the row
                                   tile of their best rotation after every
                                   iteration (a second copy of the frames in
                                   the workspace); the grouping is kept when
                                   emc_set_frames loads frames again. The
                                   context's stored scores are then in that
                                   internal order and hold only the contracted
                                   tiles; emc_targets_from_scores and
                                   emc_missed_mass read them that way (a
                                   target among the skipped tiles would carry
                                   a weight below e^-110). */
#define EMC_FLAG_SPARSE_K 2     /* emc_set_frames also lists every frame's
                                   non-zero pixels (n_data x n_pix x 4 B of
                                   workspace at most) for emc_loglik_sparse_k;
                                   the sparse Maximize (emc_sparse_estep,
                                   emc_sparse_update) then reads those lists
                                   instead of the frames' rows. Needs
                                   n_pix <= 65536 */

typedef struct emc_config {
  int32_t N;             /* grid side, 4 <= N <= 1024 */
  int32_t precision;     /* emc_precision */
  int64_t n_pix;         /* used (unmasked, inside-support) pixels, >= 1 */
  int64_t n_rot;         /* sampled rotations M_rot, >= 1 */
  int64_t n_data;        /* frames M_data, >= 1 */
  double w_floor;        /* expanded W_ij is floored at this value, > 0 */
  int32_t compress_mode; /* emc_compress_mode */
  int32_t flags;         /* EMC_FLAG_* bits */
  int64_t rot_chunk;     /* rotations per pass-2 chunk inside emc_iteration;
                            0 = all rotations in one chunk */
  int32_t n_cand;        /* candidate rotations per frame for the sparse
                            Maximize (0 = none; at most min(n_rot, 4096)) */
  int32_t model;         /* emc_model (0 = Poisson) */
  double sigma;          /* sigma of Eq. 2.2 (> 0) for EMC_MODEL_GAUSSIAN;
                            not read for the Poisson model */
} emc_config;

/* Per-call buffer sizes in bytes for a block of nrot rotations. */
typedef struct emc_buffer_sizes {
  int64_t ld_pix;      /* padded pixel stride (elements) */
  int64_t ld_data;     /* padded frame stride (elements) */
  int64_t rows;        /* nrot padded to a multiple of 128 */
  size_t logw_bytes;   /* emc_expand output L */
  size_t bias_bytes;   /* double[rows] */
  size_t prob_bytes;   /* emc_normalize output P */
  size_t num_bytes;    /* float[rows][ld_pix] */
  size_t den_bytes;    /* float[rows] */
  size_t lse_bytes;    /* double[ld_data] (each of lse_m, lse_s) */
  size_t score_bytes;  /* optional stored scores of emc_loglik / emc_normalize */
  size_t grid_bytes;   /* double[N^3] (each of g_num, g_den) */
} emc_buffer_sizes;

typedef struct emc_iter_stats {
  double loglik;       /* sum_k lse_k (Poisson: the log-likelihood without
                          sum log K!; Gaussian: without the per-frame
                          normal-density constants) */
  double ms_expand, ms_loglik, ms_normalize, ms_update, ms_compress, ms_total;
  int32_t device_status; /* emc_status recorded on the device (0 = OK) */
  int32_t kernels;       /* kernel launches made by the call */
  int64_t pass1_tiles;   /* (128-rotation, 256-frame) tiles of the E-step pass 1 */
  int64_t pass1_exact;   /* of those, contracted with every plane (all of them
                            unless the pass was bound-pruned) */
  int32_t pass1_pruned;  /* 1: the pass was bound-pruned (a hi-plane bound ran first) */
  int32_t pass1_delta;   /* 1: the incremental bound from the last iteration ran before
                            the hi-plane bound, which then covered only the tiles it
                            could not rule out */
  int64_t pass1_bound_pairs; /* pairs of row tiles x frame tiles the hi-plane bound
                                contracted (pruned passes) */
} emc_iter_stats;

typedef struct emc_ctx emc_ctx;

/* Text for a status code (static storage). */
const char* emc_status_string(int status);

/* Rotation sampling of Eq. 2.7 (Sec. 2.2): the 600-cell with each cell
 * divided n times gives M_rot = 10 (5 n^3 + n) rotations, q ~ -q identified.
 * emc_quat_count returns that number (or -1 for n < 1).
 * emc_quat_generate writes unit quaternions quat[cap][4] (host, w first,
 * first non-zero component positive; ordered along a space-filling curve:
 * by the 30-bit Morton code of the top 10 bits of round(q_c * 2^30) + 2^30
 * for c = x, y, z, ties by round(q * 2^30) lexicographically) and prior
 * weights weight[cap] (host, sum 1; w_j ~ 1/|x_j|^4 for the flat lattice point
 * x_j, or equal weights when uniform != 0). Returns the count written, or a
 * negative emc_status (EMC_ERR_ARG if cap is too small, EMC_ERR_NOMEM if the
 * host memory of the construction runs out). */
int64_t emc_quat_count(int n);
int64_t emc_quat_generate(int n, int uniform, double* quat, double* weight, int64_t cap);

/* Buffer sizes for a configuration and a rotation block of nrot rows. */
int emc_buffer_sizes_for(const emc_config* cfg, int64_t nrot, emc_buffer_sizes* out);

/* Bytes of device workspace emc_ctx_create needs for cfg. */
int emc_workspace_size(const emc_config* cfg, size_t* bytes);

/* Create a context. q: host double[n_pix][3] pixel positions (Sec. 2.2,
 * q_i on the Ewald sphere, grid units). quat: host double[n_rot][4].
 * weight: host double[n_rot] prior weights w_j (> 0). workspace: device
 * memory of at least emc_workspace_size() bytes, 256-byte aligned, owned by
 * the caller and used until emc_ctx_destroy. Geometry and rotations are
 * staged in host memory and copied into the workspace on `stream`; if that
 * host memory cannot be had, EMC_ERR_NOMEM and nothing is created. */
int emc_ctx_create(const emc_config* cfg, const double* q, const double* quat,
                   const double* weight, void* workspace, size_t workspace_bytes,
                   emc_stream stream, emc_ctx** out);
int emc_ctx_destroy(emc_ctx* ctx);

/* Read (synchronously) and clear the device status word. */
int emc_ctx_status(emc_ctx* ctx, int* device_status);

/* Bounded waits of the context's tensor-core launches (no counterpart in the
 * paper: a control of the failure path). Every mbarrier wait in those kernels
 * gives up after wait_limit_ns (0 restores the default, 2 s); a launch whose
 * wait gives up records EMC_ERR_TIMEOUT in the device status, lets the copies
 * and MMAs it issued complete, frees its tensor memory and returns, leaving
 * its outputs undefined. stall != 0 is a test hook for that path: in every
 * tensor-core launch made while it is set, the MMA issuer's first wait is on a
 * barrier that nothing completes, so that wait runs out after wait_limit_ns.
 * Production code leaves both at 0. Takes effect for launches made after the
 * call; returns EMC_ERR_ARG for a NULL context. */
int emc_ctx_set_wait_limit(emc_ctx* ctx, uint64_t wait_limit_ns, int stall);

/* Load frames K (Sec. 2.1, photon counts): device int32 [n_data][ld_k],
 * ld_k >= n_pix, into the context's padded frame buffer (BF16, or FP16 for
 * EMC_PREC_FP16_SPLIT). Counts must lie in [0, 256] (exact in BF16; [0, 2048]
 * in FP16) and sum to below 65536 per frame (8192 for FP16_SPLIT); otherwise
 * the device status becomes EMC_ERR_UNSUPPORTED. The Gaussian model keeps an
 * FP16 copy (the E-step operand) and a BF16 copy (the M-step operand), so its
 * counts must lie in [0, 256]; frame totals are not limited. It also records
 * A_k = sum_i K_ik^2 and the largest frame total. */
int emc_set_frames(emc_ctx* ctx, const int32_t* K, int64_t ld_k, emc_stream stream);

/* e-step, Eq. 2.9, for rotations [rot0, rot0 + nrot):
 * W_ij = max(trilinear(grid, R_j q_i), w_floor);
 * L (device): FP32 -> float[rows][ld_pix] = log W;
 *             BF16 -> bf16[rows][ld_pix];
 *             BF16_SPLIT -> bf16[3][rows][ld_pix] (hi, mid, lo planes);
 *             FP16_SPLIT -> fp16[2][rows][ld_pix] (hi, rest planes);
 *             padding columns and rows are written as 0.
 * bias (device double[rows]) = log w_j - sum_i W_ij (-inf on padding rows).
 * Gaussian model: W_ij = max(trilinear(grid, R_j q_i), 0) (w_floor is not
 * used); L = fp16[3][rows][ld_pix] holding s W = hi + mid + lo, hi integral,
 * with s = 2^e chosen from max(grid) and the largest frame total so that
 * every partial sum of hi K stays below 2^24 (exact in FP32); bias_j =
 * log w_j - sum_i W_ij^2 / (2 sigma^2). The call records s in the context;
 * emc_loglik, emc_normalize and emc_update use the scale of the last
 * emc_expand.
 * An interpolated W_ij that is NaN or infinite (a non-finite voxel of grid)
 * sets EMC_ERR_NUMERIC in the device status.
 * Poisson-fluence model: L holds log(W_ij / B_j) + c in place of log W
 * (B_j = sum_i W_ij, c = log n_pix rounded to the 1/8 grid, which keeps the
 * values and the scores in the range of the exact split); bias is
 * double[2][rows] (bias_bytes): log w_j, then B_j (0 on padding rows). The
 * context also keeps B_j of rows [rot0, rot0 + nrot) for the sparse calls
 * and emc_iteration. The scores are then shifted by c N_k per frame;
 * emc_loglik removes the shift from lse (in FP64), and the normalisation
 * adds it back. */
int emc_expand(emc_ctx* ctx, const float* grid, int64_t rot0, int64_t nrot, void* L,
               double* bias, emc_stream stream);

/* E-step pass 1 (Eq. 2.4 denominators): for every frame k, the running
 * (max m_k, sum s_k) with lse_k = m_k + log s_k over rotations in this block:
 * S_jk = sum_i K_ik log W_ij + bias_j. lse_m, lse_s: device double[ld_data];
 * accumulate = 0 starts from (m, s) = (-inf, 0), else merges into them.
 * scores (device, score_bytes, may be NULL): when given, the scores are also
 * stored, frame-major, as float d[ld_data][rows] relative to float
 * r[rows/32][ld_data] (the maximum of each 32-row group of a column, on the
 * 1/64 grid; r follows directly after d in the same buffer):
 * S_jk = d[k][j] + r[j/32][k].
 * Gaussian model: S_jk = (G_jk^2 / A_k - B_j) / (2 sigma^2) + log w_j from
 * the FP16 three-plane L (see emc_model); scores more than about 1.2e5 below
 * zero are clamped there (their exp is 0 next to any frame's best rotation),
 * and a frame whose best score lies below that makes the device status
 * EMC_ERR_NUMERIC (sigma too small for the data).
 * Poisson-fluence model: lse_k = m_k + log s_k is that of
 * S_jk = sum_i K_ik log(W_ij / B_j) + log w_j; the stored scores carry the
 * per-frame shift c N_k of emc_expand's L (P is unchanged by it). */
int emc_loglik(emc_ctx* ctx, const void* L, const double* bias, int64_t nrot, double* lse_m,
               double* lse_s, int accumulate, void* scores, emc_stream stream);

/* Sparse-K form of the E-step pass 1 (no counterpart in the paper: an
 * alternative contraction for frames with few photons). Same result as
 * emc_loglik -- (m_k, s_k) over the block's rotations of
 * S_jk = sum_i K_ik log W_ij + bias_j -- but the sum runs over each frame's
 * non-zero pixels only, gathering log W there instead of contracting densely
 * on the tensor cores. Needs EMC_FLAG_SPARSE_K and precision EMC_PREC_FP32 (L =
 * FP32 log W of emc_expand); the Poisson model only; no stored scores.
 * Returns EMC_ERR_UNSUPPORTED if one log W row (2 x 4 B x ld_pix) does not
 * fit the kernel's shared memory (ld_pix above ~27000). */
int emc_loglik_sparse_k(emc_ctx* ctx, const float* L, const double* bias, int64_t nrot,
                        double* lse_m, double* lse_s, int accumulate, emc_stream stream);

/* E-step pass 2 (Eq. 2.4): P_jk = exp(S_jk - lse_k). With scores == NULL the
 * scores are recomputed from L and bias (two-pass streamed form, nothing of
 * size rotations x frames kept); otherwise they are read from the buffer
 * emc_loglik filled (L and bias are then not read and may be NULL).
 * P (device): FP32 -> float[rows][ld_data]; BF16 / BF16_SPLIT ->
 * bf16[2][rows][ld_data] (hi, lo planes, P = hi + lo; lo is 0 for BF16);
 * FP16_SPLIT -> fp16[2][rows][ld_data], P = (hi + lo) / 2^14.
 * Padding frames and rows are written as 0.
 * Gaussian model (scores and bias required): the planes hold P_jk / phi_jk,
 * the responsibility already divided by the fluence that Eq. 2.5 applies to
 * frame k (1/phi_jk = sqrt(2 sigma^2 (S_jk - bias_j) / A_k)), as
 * bf16[2][rows][ld_data] hi + lo; after the planes the buffer holds
 * float den[rows] = sum_k P_jk (prob_bytes counts it).
 * Poisson-fluence model (either form; bias, and without scores L,
 * required): the planes hold P_jk B_j / N_k (0 for an empty frame) as
 * bf16[2][rows][ld_data] hi + lo, with B_j read from the second half of
 * bias, followed by float den[rows] = sum_k P_jk. */
int emc_normalize(emc_ctx* ctx, const void* L, const double* bias, int64_t nrot,
                  const double* lse_m, const double* lse_s, const void* scores, void* P,
                  emc_stream stream);

/* E-step pass 1 for callers that cannot allocate device memory (the paper
 * has no counterpart: this is an interface addition, not a step of the
 * method). Some callers cannot call cudaMalloc -- code inside a host
 * application or framework that owns every device allocation, or a process
 * whose memory pool is already committed -- and so cannot provide the
 * workspace emc_ctx_create needs. This call needs no context and no
 * workspace: it computes what emc_loglik computes, keeping its only scratch
 * (per-tile max/sum pairs) in a 32 MiB static device array inside the
 * library, and allocates nothing at call time.
 *  cfg: precision, n_pix, n_rot, n_data, model and flags are read (host);
 *          the Poisson model only, without EMC_FLAG_WIDE_COUNTS
 *          (EMC_ERR_UNSUPPORTED otherwise).
 *  L, bias: device, as emc_expand writes them for nrot rotations.
 *  frames: device BF16 (FP16 for EMC_PREC_FP16_SPLIT) [ld_data][ld_pix]
 *          (ld_pix = round_up(n_pix + 1, 64), ld_data = round_up(n_data, 256)):
 *          counts in columns < n_pix, 1 in column n_pix for every real frame,
 *          0 everywhere else.
 *  lse_m, lse_s, accumulate: as emc_loglik.
 *  device_status: optional device int32; a bounded wait that gives up or a
 *          non-finite merge writes a negative emc_status there (first wins).
 * Rotations are processed in blocks that fit the static array; frames with
 * ld_data above about 1.4 million make even one block too large and the call
 * returns EMC_ERR_UNSUPPORTED before launching anything. Every GPU that loads
 * the library holds the 32 MiB array until the process exits. All calls share
 * it and it keeps the last call's contents (each call overwrites what it
 * reads); calls that overlap on the GPU race on it and must be serialised by
 * the caller. The first call on a device looks the array's address up
 * (cudaGetSymbolAddress, with that device current) and keeps it for the life
 * of the process; make that first call before any stream capture, and do not
 * use the call after cudaDeviceReset (the kept address would be stale).
 * L and frames must be 16-byte aligned, bias, lse_m and lse_s 8-byte aligned
 * (EMC_ERR_ARG otherwise); n_pix is limited to 2^24 as for a context. */
int emc_loglik_static(const emc_config* cfg, const void* L, const double* bias,
                      const uint16_t* frames, int64_t nrot, double* lse_m, double* lse_s,
                      int accumulate, int32_t* device_status, emc_stream stream);

/* M-step, Eq. 2.11: Num (device float[rows][ld_pix]) = P K over frames;
 * den (device float[rows]) = sum_k P_jk.
 * Gaussian model: Num_ij = sum_k P_jk K_ik / phi_jk (Eq. 2.5 before the
 * division) from the planes emc_normalize wrote; den is copied from the end
 * of the P buffer. Poisson-fluence model: likewise, Num_ij =
 * sum_k P_jk K_ik B_j / N_k. */
int emc_update(emc_ctx* ctx, const void* P, int64_t nrot, float* Num, float* den,
               emc_stream stream);

/* c-step accumulation, Eq. 2.12 (or Eq. 2.5 + 2.10 in IDW mode), for
 * rotations [rot0, rot0 + nrot): g_num_l += sum_ij f Num_ij,
 * g_den_l += sum_ij f den_j. g_num, g_den: device double[N^3]; accumulate = 0
 * zeroes them first. */
int emc_compress(emc_ctx* ctx, int64_t rot0, int64_t nrot, const float* Num, const float* den,
                 double* g_num, double* g_den, int accumulate, emc_stream stream);

/* Final division of Eq. 2.12: grid_out_l = g_num_l / g_den_l where
 * g_den_l > 0, else grid_prev_l. grid_out may alias grid_prev. */
int emc_finalize(emc_ctx* ctx, const double* g_num, const double* g_den, const float* grid_prev,
                 float* grid_out, emc_stream stream);

/* One pass of Algorithm 2.1 on the loaded frames, using the workspace for
 * every intermediate: e-step, E-step (two passes), M-step and c-step over
 * rotation chunks of cfg.rot_chunk. grid_out may not alias grid_in. With the
 * tensor-core forms the M-step contracts only the 128-rotation x 64-frame
 * blocks of P that the normalisation found non-zero (most underflow to exact
 * zeros); the result is that of the full contraction.
 * stats (host, may be NULL) is filled after the call synchronises `stream`. */
int emc_iteration(emc_ctx* ctx, const float* grid_in, float* grid_out, emc_iter_stats* stats,
                  emc_stream stream);

/* Per-frame log-likelihood terms of the last emc_iteration (the denominators
 * of Eq. 2.4): lse (device double[n_data], frames in the order given to
 * emc_set_frames) = log sum_j exp(S_jk), S_jk the scores emc_loglik defines for
 * the context's noise model. EMC_ERR_ARG if no emc_iteration ran since the
 * last emc_set_frames. */
int emc_iteration_lse(emc_ctx* ctx, double* lse, emc_stream stream);

/* Responsibilities P_jk of Eq. 2.4 of selected frames after the last
 * emc_iteration, read from the context's stored scores (needs
 * EMC_FLAG_STORE_SCORES; EMC_ERR_ARG otherwise or if no emc_iteration ran
 * since the last emc_set_frames): P (device float[n][n_rot]) row f holds
 * P_jk for frame k = frames[f] (device int32[n]) over every rotation j, in
 * FP32. Rotations in tiles that a bound-pruned pass 1 skipped get 0 (their P
 * is 0 in FP32). An index outside [0, n_data) sets EMC_ERR_ARG in the device
 * status and leaves that row unwritten. */
int emc_responsibilities(emc_ctx* ctx, const int32_t* frames, int64_t n, float* P,
                         emc_stream stream);

/* ------------------------------------------------------------------------
 * Learned rotation proposal and the sparse Maximize. The paper has no learned
 * component; these calls implement the workload's proposal stage: a frame's
 * binned counts feed a small network whose top-M logits become the candidate
 * rotations C_k, and Eq. 2.4 / 2.11 then run over (j, k), j in C_k, only.
 * ---------------------------------------------------------------------- */

/* Features of the loaded frames: feat (device float[ld_data][512]) =
 * log(1 + mean count) over the pixels of each (radial, angular) bin, radial
 * bin floor(32 |q_i| / max|q|) (<= 31), angular bin
 * floor(16 (atan2(q_y, q_x) + pi) / (2 pi)) (<= 15), index radial * 16 +
 * angular; empty bins and padding frames give 0. */
int emc_features(emc_ctx* ctx, float* feat, emc_stream stream);

/* MLP: 512 inputs -> three hidden layers of 512 GELU units -> n_out logits.
 * Parameters (device FP32, caller-owned, emc_mlp_param_count floats):
 * W1[512][512], b1[512], W2[512][512], b2, W3[512][512], b3,
 * W4[512][ld_out], b4[ld_out], ld_out = round_up(n_out, 64); layer input x
 * (row vector) maps to x W + b. Products use BF16-rounded operands with FP32
 * accumulation. work: device scratch of emc_mlp_work_size(n_out, batch) bytes
 * (activations kept for the backward pass). */
int64_t emc_mlp_param_count(int64_t n_out);
int emc_mlp_work_size(int64_t n_out, int64_t batch, size_t* bytes);

/* Forward of `batch` rows X (device float[batch][512]) into logits (device
 * float[batch][ld_out]; columns >= n_out are not written). */
int emc_mlp_forward(int64_t n_out, const float* params, const float* X, int64_t batch, void* work,
                    float* logits, emc_stream stream);

/* One Adam step (beta 0.9 / 0.999, eps 1e-8, bias-corrected, step counts from
 * 1) on the loss -(1/batch) sum_k sum_r tprob[k][r] log softmax(z_k)[tidx[k][r]]
 * over the batch: tidx (device int32[batch][R]), tprob (device float[batch][R]);
 * grads, adam_m, adam_v: device FP32 like params (zero them before the first
 * step; grads is overwritten each step). *loss (device double) is incremented
 * by the batch loss. */
int emc_mlp_train_step(int64_t n_out, float* params, float* grads, float* adam_m, float* adam_v,
                       int step, float lr, const float* X, const int32_t* tidx,
                       const float* tprob, int64_t batch, int R, void* work, double* loss,
                       emc_stream stream);

/* Indices of the M largest of the first n values of each row of logits
 * (device float[batch][ld]) into cand (device int32[batch][M]): first the
 * values above the M-th largest in index order, then equal values in index
 * order (ties towards lower indices). */
int emc_topm(const float* logits, int64_t batch, int64_t n, int64_t ld, int M, int32_t* cand,
             emc_stream stream);

/* Soft training targets from a dense E-step: for every frame the R <= 64
 * rotations of largest S_jk and softmax weights over them (device
 * tidx int32[n_data][R], tprob float[n_data][R]). scores: a buffer filled by
 * emc_loglik, or NULL for the context's own (EMC_FLAG_STORE_SCORES, from the
 * last emc_iteration). */
int emc_targets_from_scores(emc_ctx* ctx, const void* scores, int R, int32_t* tidx, float* tprob,
                            emc_stream stream);

/* Candidate sets from two ranked lists (no counterpart in the paper: the
 * learned proposal's schedule). For each of n frames: the R rotations of
 * first (device int32[n][R], distinct, e.g. tidx of emc_targets_from_scores
 * after a dense iteration), then the entries of rest (device int32[n][M_rest],
 * e.g. emc_topm of the network's logits) that are not among them, in their
 * order, until M are written to out (device int32[n][M]). Needs
 * 0 <= R <= 64 and M_rest >= M (so that M distinct entries exist). */
int emc_merge_candidates(const int32_t* first, int R, const int32_t* rest, int M_rest, int64_t n,
                         int M, int32_t* out, emc_stream stream);

/* Load candidate sets cand (device int32[n_data][n_cand], rotation indices)
 * and build the per-rotation pair lists the sparse calls use. An index outside
 * [0, n_rot) sets EMC_ERR_ARG in the device status. */
int emc_set_candidates(emc_ctx* ctx, const int32_t* cand, emc_stream stream);

/* Eq. 2.4 over the candidate sets, from L and bias of emc_expand over all
 * rotations: P (device float[ld_data][n_cand], slot order of the candidates;
 * padding frames 0) and lse (device double[ld_data]; Poisson-fluence model:
 * without the per-frame shift of L, as emc_loglik). */
int emc_sparse_estep(emc_ctx* ctx, const void* L, const double* bias, float* P, double* lse,
                     emc_stream stream);

/* Eq. 2.11 over the candidate sets: Num (device float[rows][ld_pix]) and den
 * (device float[rows]) for every rotation (rows without candidates: 0).
 * Poisson-fluence model: Num_ij = sum_k P_jk K_ik B_j / N_k and
 * den_j = sum_k P_jk over the candidate pairs, B_j from the last emc_expand
 * over all rotations. */
int emc_sparse_update(emc_ctx* ctx, const float* P, float* Num, float* den, emc_stream stream);

/* One pass of Algorithm 2.1 with the Maximize step over the candidate sets
 * (e-step, sparse E- and M-steps, c-step). stats->loglik is sum_k of the
 * candidate-set lse_k. */
int emc_sparse_iteration(emc_ctx* ctx, const float* grid_in, float* grid_out,
                         emc_iter_stats* stats, emc_stream stream);

/* Missed responsibility mass of the candidate sets under a dense E-step:
 * missed[k] = 1 - sum_{j in C_k} P_jk (device float[n_data]). scores, lse_m,
 * lse_s: from emc_loglik, or NULL for the context's own from the last
 * emc_iteration (needs EMC_FLAG_STORE_SCORES). */
int emc_missed_mass(emc_ctx* ctx, const void* scores, const double* lse_m, const double* lse_s,
                    float* missed, emc_stream stream);

/* Responsibilities recorded during emc_iteration (no counterpart in the
 * paper: the learned schedule's targets and missed mass where the scores are
 * not stored). emc_collect_bytes: the size of the caller-owned buffer for cap
 * entries and the scratch of emc_collected_targets for the context's n_data
 * frames (0 if ctx is NULL or cap < 1). */
size_t emc_collect_bytes(const emc_ctx* ctx, int64_t cap);

/* With buf non-NULL (device, 256-byte aligned, emc_collect_bytes(ctx, cap)
 * bytes, owned by the caller and kept until emc_set_collect(ctx, NULL, 0) or
 * emc_ctx_destroy), every later emc_iteration appends each P_jk of Eq. 2.4 that
 * is non-zero in FP32 as (frame, rotation, P_jk) to it, read from the blocks of
 * P its M-step contracts (the rounding of those operands: 2^-16 relative for
 * the split forms, 2^-8 for plain BF16); each iteration starts the list
 * afresh. NULL stops recording. The tensor-core precisions with the Poisson
 * model, BF16 or BF16 split with the Poisson-fluence model; EMC_ERR_UNSUPPORTED
 * otherwise. */
int emc_set_collect(emc_ctx* ctx, void* buf, int64_t cap);

/* From the entries the last emc_iteration recorded, per frame k:
 *  tidx, tprob (device int32 / float [n_data][R], 1 <= R <= 64): the R
 *    rotations of largest P_jk (ties: the lower index first) and P_jk over
 *    their sum, the softmax of their scores. Rotations whose P_jk is 0 in FP32
 *    rank last: a frame with fewer than R non-zero entries gets distinct other
 *    rotations with weight 0 (from the 128-rotation tile of its best one on).
 *    The weights equal those of emc_targets_from_scores wherever they exceed
 *    the rounding above;
 *  missed (device float[n_data], may be NULL; needs emc_set_candidates): the
 *    sum of P_jk over the recorded j outside the frame's candidate set, i.e.
 *    1 - sum_{j in C_k} P_jk as emc_missed_mass defines it.
 * EMC_ERR_ARG if the last emc_iteration recorded nothing; a list that
 * overflowed sets EMC_ERR_UNSUPPORTED in the device status. */
int emc_collected_targets(emc_ctx* ctx, int R, int32_t* tidx, float* tprob, float* missed,
                          emc_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* EMC_H */
