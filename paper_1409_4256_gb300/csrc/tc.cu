// tc.cu -- tcgen05 (5th-generation tensor core) forms of the Maximize step.
//
// One persistent, warp-specialised kernel template serves the three dense
// contractions of the E- and M-steps (Eqs. 2.3-2.4 and 2.11):
//   PASS1     S = L K^T over pixels -> per frame (max_j, sum_j exp) per 128-row tile
//   NORMALIZE S = L K^T over pixels -> P_jk = exp(S_jk - lse_k), BF16 hi/lo planes
//   UPDATE    Num = P K over frames (K read MN-major) -> FP32 rows + den_j
//   STORE     C = A K^T over pixels -> FP32 rows [rows][ld_data] as they are
//             (the per-tile bound increments of the pruned pass 1)
// with M = 128 rotations per tile and N = 256 frames (or pixels).
//
// Roles (320 threads, one CTA per SM):
//   warp 0      one thread issues TMA loads of A (1-3 BF16 planes) and B into a
//               ring of shared-memory stages (128-byte swizzle, 64-wide K blocks)
//   warp 1      allocates TMEM; one thread issues tcgen05.mma (128x256x16) into
//               FP32 accumulators in TMEM and commits stages / tiles to mbarriers
//   warps 2-9   epilogue: tcgen05.ld from TMEM (warp w reads lanes 32*(w%4)..,
//               columns 128*((w-2)/4)..), arithmetic, global stores
// Every mbarrier wait is bounded in time; a wait that gives up records
// EMC_ERR_TIMEOUT, raises a CTA-wide abort flag and lets all roles leave.
//
// Exactness of the three-term split (precision EMC_PREC_BF16_SPLIT): the hi
// plane of log W lies on the 1/8 grid with |hi| <= 32 and counts are integers
// <= 256, so every product and every partial sum of the hi accumulator is a
// multiple of 1/8 below 2^21 and FP32 holds it exactly whatever the order or
// rounding of the accumulation. mid and lo (|mid + lo| <= 1/16) go to a second
// accumulator whose magnitude stays small. The epilogue adds the per-rotation
// bias split the same way (hi on the grid, lo small), folds the small part's
// multiples of 1/8 into the exact part and only then subtracts the reference
// (running max in pass 1, lse_k in pass 2), so the exponent is accurate to a
// few FP32 ulps of a number of order one.
//
// Gaussian model (pass 1 with three FP16 planes): the accumulators hold
// s G_jk = gh + gl, gh integral and exact (every partial sum below 2^24), and
// the epilogue forms S_jk = c'_k (gh + gl)^2 + bias_j, c'_k = 1/(2 sigma^2 A_k s^2),
// in double-float: gh^2 as an exact two-product, c' gh^2 with its FMA
// remainder, the 1/64-grid part of the product added to that of the bias
// exactly and every remainder gathered in the small part.
#include <cuda.h>
#include <cudaTypedefs.h>

// The MODE / NA / F16 instantiations compile branches that cannot run for
// them (e.g. the score epilogue under MODE_UPDATE); not a defect.
#pragma nv_diag_suppress 128

#include "emc_common.cuh"
#include "emc_internal.h"
#include "tc_ptx.cuh"

namespace emc {

using namespace tc;

namespace {

enum { MODE_PASS1 = 0, MODE_NORMALIZE = 1, MODE_UPDATE = 2, MODE_STORE = 3 };

constexpr int BM = 128, BN = 256;
constexpr int kThreads = 320;
constexpr int kEpiWarps = 8;
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s: a tile takes tens of microseconds
constexpr int kSmemBudget = 220 * 1024;
constexpr int kScratchBytes = 10 * 1024;
constexpr int kXpLd = 36;  // row stride (floats) of the update's staging block: 16-byte rows, no bank conflicts
constexpr float kSentinel = -3.0e38f;

// K-block width: 64 elements with 128-byte swizzle, or 32 with 64-byte swizzle
// for the multi-plane score contractions, whose 64-80 KB stages would
// otherwise leave room for only two or three in flight (too shallow to hide
// the load latency). F16: FP16 operands (FP16 split) instead of BF16.
template <int MODE, int NA, bool F16, bool XP = false>
struct TcCfg {
  static constexpr int BK = (MODE != MODE_UPDATE && NA >= 2) ? 32 : 64;
  static constexpr int A_BYTES = BM * BK * 2;  // one 128 x BK BF16 plane
  static constexpr int B_BYTES = BN * BK * 2;  // 256 x BK BF16
  static constexpr int STAGE = NA * A_BYTES + B_BYTES;
  static constexpr int NACC = (MODE != MODE_UPDATE && NA >= 2) ? 2 : 1;
  // XP (update over listed blocks, store): a 32 x 32 staging block per
  // epilogue warp, through which the output rows leave as whole 128-byte lines
  // (the lanes of a TMEM load hold rows). It takes a pipeline stage from the
  // two-plane update, which the output bounds there; the dense update, bound by
  // the tensor pipe, keeps its stages and stores rows directly.
  static constexpr int XPOSE =
      (XP && (MODE == MODE_UPDATE || MODE == MODE_STORE)) ? kEpiWarps * 32 * kXpLd * 4 : 0;
  static constexpr int STAGES_RAW = (kSmemBudget - kScratchBytes - XPOSE - 1024 - 256) / STAGE;
  static constexpr int STAGES = STAGES_RAW > 6 ? 6 : STAGES_RAW;
  static constexpr uint32_t TMEM_COLS = NACC * BN;
  static constexpr int SMEM = 1024 + STAGES * STAGE + 256 + kScratchBytes + XPOSE;
  static constexpr uint32_t IDESC = idesc_f16kind(BM, BN, MODE == MODE_UPDATE ? 1 : 0, F16);
  static_assert(STAGES >= 2, "shared memory too small for two stages");
};

// K-major operand descriptor for k-step kk (16 elements) inside a K block
template <int BK>
__device__ __forceinline__ uint64_t kmajor_desc(uint32_t base, int kk) {
  if (BK == 64) return sdesc_sw128(base + kk * 32, 16, 1024);
  return sdesc_sw64(base + kk * 32, 512);
}

struct TcArgs {
  int n_mtiles, n_ntiles, group, kblocks;
  int64_t rows;      // rows of A (leading dimension of the frame-major stored scores)
  int64_t nrot;      // valid rows of A
  int64_t n_data, ld_data, ld_pix, n_pix;
  const double* bias;      // scores: [rows]
  const float2* lse2;      // normalize: [ld_data] (hi on the 1/8 grid, lo)
  double* part_m;          // pass 1: [n_mtiles][ld_data]
  float* part_s;
  float* S;                // pass 1, optional: shifted scores, frame-major [ld_data][rows]
  float* Sref;             // pass 1, optional: 32-row group maxima [rows / 32][ld_data]
  const float4* gk;        // Gaussian pass 1: per frame (c_k hi, c_k lo, 2 sigma^2 / A_k, 0)
  const float4* gsc;       // Gaussian pass 1: scales (s, 1/s^2, 0, 0)
  uint16_t* P;             // normalize: planes [2][rows][ld_data]
  int64_t P_plane;
  float* Num;              // update: [rows][ld_pix]
  float* den;              // update: [rows]; Poisson-fluence normalize: sum_k P_jk (atomics)
  const double* Bsum;      // Poisson-fluence normalize: B_j [rows] (NULL otherwise)
  const float* invn;       // Poisson-fluence normalize: 1 / N_k [ld_data]
  // update over the non-zero P blocks only (NULL: every K block): per row tile
  // mt, kb_cnt[mt] K-block indices (64 frames each) in kb_list[mt * kb_ld ..]
  const int32_t* kb_cnt;
  const int32_t* kb_list;
  // normalize: kb_flag[mt * kb_ld + kb] set to 1 where the block's P is non-zero
  uint8_t* kb_flag;
  int kb_ld;
  // pass 1 over listed tiles only (NULL: every tile): tile_list[t] =
  // mt * n_ntiles + nt for t < *tile_count, in raster order
  const int32_t* tile_list;
  const int32_t* tile_count;
  int n_rowtiles;          // bound pass: 128-row tiles (n_mtiles counts pairs of them)
  int32_t* status;
  uint64_t wait_ns;        // limit of every bounded wait
  int stall;               // test hook: the MMA issuer's first wait never completes
};

// K blocks a tile contracts: every block, or (update with lists) the row
// tile's non-zero P blocks. A tile without any issues no load and no MMA; its
// epilogue writes zeros instead of reading the accumulator (P itself need not
// hold zeros there).
__device__ __forceinline__ int tile_kblocks(const TcArgs& a, int mt) {
  return a.kb_cnt ? a.kb_cnt[mt] : a.kblocks;
}
__device__ __forceinline__ int tile_kblock(const TcArgs& a, int mt, int x) {
  return a.kb_cnt ? a.kb_list[(int64_t)mt * a.kb_ld + x] : x;
}

__device__ __forceinline__ void tile_coords(int t, const TcArgs& a, int* mt, int* nt) {
  if (a.tile_list) {
    const int code = a.tile_list[t];
    *mt = code / a.n_ntiles;
    *nt = code % a.n_ntiles;
    return;
  }
  const int per_group = a.group * a.n_ntiles;
  const int g = t / per_group, rem = t % per_group;
  const int gsize = min(a.group, a.n_mtiles - g * a.group);
  *nt = rem / gsize;
  *mt = g * a.group + rem % gsize;
}

// Butterfly transpose-reduction: on entry every lane holds 32 values (one per
// column); on exit v[0] of lane l is the reduction over the 32 lanes of
// column l. 31 shuffles for 32 columns.
template <bool MAX>
__device__ __forceinline__ float warp_transpose_reduce(float (&v)[32], int lane) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const bool upper = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < off; i++) {
      const float send = upper ? v[i] : v[i + off];
      const float keep = upper ? v[i + off] : v[i];
      const float recv = __shfl_xor_sync(0xffffffffu, send, off);
      v[i] = MAX ? fmaxf(keep, recv) : keep + recv;
    }
  }
  return v[0];
}

__device__ __forceinline__ void fail(volatile int* abort, int32_t* status) {
  *abort = 1;
  set_status(status, EMC_ERR_TIMEOUT);
}

template <int MODE, int NA, bool F16, bool XP = false>
__global__ void __launch_bounds__(kThreads, 1)
    tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
              const TcArgs a) {
  using C = TcCfg<MODE, NA, F16, XP>;
  constexpr bool GAUSS = (MODE == MODE_PASS1 && NA == 3 && F16);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~(uintptr_t)1023);
  uint8_t* stages = smem;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::STAGES * C::STAGE);
  uint64_t* empty = full + C::STAGES;
  uint64_t* acc_full = empty + C::STAGES;
  uint64_t* acc_empty = acc_full + 1;
  uint64_t* drain = acc_empty + 1;
  uint64_t* never = drain + 1;  // the stall hook's barrier: nothing arrives on it
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(never + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float2* scratch = reinterpret_cast<float2*>(smem + C::STAGES * C::STAGE + 256);
  float* xpose = reinterpret_cast<float*>(smem + C::STAGES * C::STAGE + 256 + kScratchBytes);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; s++) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, kEpiWarps);
    mbar_init(drain, 1);
    mbar_init(never, 1);
    *abort = 0;
    fence_mbar_init();
  }
  if (warp == 0 && lane == 0) {
    prefetch_tmap(&mapA);
    prefetch_tmap(&mapB);
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, C::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int T = a.tile_count ? *a.tile_count : a.n_mtiles * a.n_ntiles;

  if (warp == 0) {
    // ------------------------------------------------------------ producer --
    if (lane == 0) {
      int it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < T && ok; t += gridDim.x) {
        int mt, nt;
        tile_coords(t, a, &mt, &nt);
        const int nkb = tile_kblocks(a, mt);
        for (int x = 0; x < nkb; x++, it++) {
          const int kb = tile_kblock(a, mt, x);
          const int s = it % C::STAGES;
          const uint32_t ph = (uint32_t)(it / C::STAGES) & 1u;
          if (!mbar_wait(empty + s, ph ^ 1u, abort, a.wait_ns)) {
            fail(abort, a.status);
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(full + s, C::STAGE);
          uint8_t* st = stages + s * C::STAGE;
#pragma unroll
          for (int p = 0; p < NA; p++)
            tma_load_3d(st + p * C::A_BYTES, &mapA, full + s, kb * C::BK, mt * BM, p);
          uint8_t* sb = st + NA * C::A_BYTES;
          if (MODE != MODE_UPDATE) {
            tma_load_2d(sb, &mapB, full + s, kb * C::BK, nt * BN);
          } else {
#pragma unroll
            for (int j = 0; j < BN / 64; j++)
              tma_load_2d(sb + j * (64 * C::BK * 2), &mapB, full + s, nt * BN + j * 64, kb * C::BK);
          }
        }
      }
      if (!ok) {
        // let copies already issued land before the CTA retires
        for (int back = 1; back <= C::STAGES && it - back >= 0; back++) {
          const int j = it - back;
          mbar_wait_quiet(full + (j % C::STAGES), (uint32_t)(j / C::STAGES) & 1u, kWaitLimitNs);
        }
      }
    }
  } else if (warp == 1) {
    // ----------------------------------------------------------------- MMA --
    if (lane == 0) {
      int it = 0, tcount = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < T && ok; t += gridDim.x, tcount++) {
        if (!mbar_wait(acc_empty, ((uint32_t)tcount & 1u) ^ 1u, abort, a.wait_ns)) {
          fail(abort, a.status);
          break;
        }
        tc_fence_after();
        int mt_, nt_;
        tile_coords(t, a, &mt_, &nt_);
        const int nkb = tile_kblocks(a, mt_);
        for (int kb = 0; kb < nkb; kb++, it++) {
          const int s = it % C::STAGES;
          const uint32_t ph = (uint32_t)(it / C::STAGES) & 1u;
          uint64_t* wb = (a.stall && it == 0) ? never : full + s;
          if (!mbar_wait(wb, ph, abort, a.wait_ns)) {
            fail(abort, a.status);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sA = smem_u32(stages + s * C::STAGE);
          const uint32_t sB = sA + NA * C::A_BYTES;
#pragma unroll
          for (int k = 0; k < C::BK / 16; k++) {
            if (MODE != MODE_UPDATE) {
              const uint64_t bdesc = kmajor_desc<C::BK>(sB, k);
#pragma unroll
              for (int p = 0; p < NA; p++) {
                const uint64_t adesc = kmajor_desc<C::BK>(sA + p * C::A_BYTES, k);
                const int acc = (NA >= 2 && p > 0) ? 1 : 0;
                const bool first = (kb == 0 && k == 0 && p <= 1);
                umma_bf16(tmem + acc * BN, adesc, bdesc, C::IDESC, first ? 0u : 1u);
              }
            } else {
              // B is MN-major: 64-pixel chunks 8 KB apart (LBO), 8-frame groups
              // 1 KB apart (SBO); 16 frames per instruction advance 2 KB.
              const uint64_t bdesc = sdesc_sw128(sB + k * 2048, 64 * C::BK * 2, 1024);
#pragma unroll
              for (int p = 0; p < NA; p++) {
                const uint64_t adesc = kmajor_desc<C::BK>(sA + p * C::A_BYTES, k);
                const bool first = (kb == 0 && k == 0 && p == 0);
                umma_bf16(tmem, adesc, bdesc, C::IDESC, first ? 0u : 1u);
              }
            }
          }
          umma_commit(empty + s);
        }
        if (ok) umma_commit(acc_full);
      }
      // every issued MMA must finish before TMEM is released
      umma_commit(drain);
      mbar_wait_quiet(drain, 0, kWaitLimitNs);
    }
  } else {
    // ------------------------------------------------------------ epilogue --
    const int e = warp - 2;
    const int q = warp & 3;         // TMEM lane quarter this warp may read
    const int half = e >> 2;        // column half: 0 -> [0,128), 1 -> [128,256)
    const int r_in = 32 * q + lane;
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * q) << 16);
    const int et = e * 32 + lane;   // 0..255 among epilogue threads
    int tcount = 0;
    for (int t = blockIdx.x; t < T; t += gridDim.x, tcount++) {
      int mt, nt;
      tile_coords(t, a, &mt, &nt);
      const int64_t row = (int64_t)mt * BM + r_in;
      float bh = 0.f, bl = 0.f;
      bool valid = row < a.nrot;
      if (MODE == MODE_PASS1 || MODE == MODE_NORMALIZE) {
        const double b = a.bias[row];
        valid = valid && b > -INFINITY;
        if (valid) {
          bh = (float)(rint(b * kGridD) / kGridD);  // on the 1/64 grid (coarser beyond 2^18)
          bl = (float)(b - (double)bh);
        }
      }
      float2* cs = scratch + 4 * BN;  // Gaussian: c'_k of the tile's frames
      if (GAUSS) {
        const float4 g = a.gk[(int64_t)nt * BN + et];
        const float is2 = a.gsc->y;
        cs[et] = make_float2(g.x * is2, g.y * is2);
        named_bar(1, kEpiThreads);
      }
      // Poisson-fluence normalize: P_jk B_j / N_k into the planes, den_j = sum_k P_jk
      const bool flu = MODE == MODE_NORMALIZE && a.Bsum != nullptr;
      float* sinv = reinterpret_cast<float*>(scratch + BN);
      float Bj = 0.f, dsum = 0.f;
      if (MODE == MODE_NORMALIZE) {
        scratch[et] = a.lse2[(int64_t)nt * BN + et];
        if (flu) {
          sinv[et] = a.invn[(int64_t)nt * BN + et];
          if (valid) Bj = (float)a.Bsum[row];
        }
        named_bar(1, kEpiThreads);
      }
      const bool got = mbar_wait(acc_full, (uint32_t)tcount & 1u, abort, a.wait_ns);
      if (!got) fail(abort, a.status);
      // every epilogue warp leaves together if any gave up (they share named barriers)
      if (named_bar_any(2, kEpiThreads, !got)) break;
      tc_fence_after();
      bool big = false;
#pragma unroll 1
      for (int c = 0; c < 4; c++) {
        const int col0 = half * 128 + c * 32;
        uint32_t v0[32], v1[32];
        tmem_ld32(lane_addr + col0, v0);
        if (C::NACC == 2) tmem_ld32(lane_addr + BN + col0, v1);
        tmem_ld_wait();
        if (c == 3) {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(acc_empty);
        }
        if (MODE == MODE_STORE) {  // C[row][k] for the tile's 32 columns of this step
          if (XP) {
            float* xp = xpose + e * (32 * kXpLd);  // staged as in the update below
#pragma unroll
            for (int i = 0; i < 32; i += 4)
              *reinterpret_cast<uint4*>(xp + lane * kXpLd + i) =
                  make_uint4(v0[i], v0[i + 1], v0[i + 2], v0[i + 3]);
            __syncwarp();
            const int64_t row0 = (int64_t)mt * BM + 32 * q;
            const int64_t k0 = (int64_t)nt * BN + col0;
#pragma unroll
            for (int st = 0; st < 8; st++) {
              const int r = 4 * st + (lane >> 3), c4 = 4 * (lane & 7);
              const uint4 w = *reinterpret_cast<const uint4*>(xp + r * kXpLd + c4);
              *reinterpret_cast<uint4*>(a.Num + (row0 + r) * a.ld_data + k0 + c4) = w;
            }
            __syncwarp();
          } else {
            float* dst = a.Num + row * a.ld_data + (int64_t)nt * BN + col0;
#pragma unroll
            for (int i = 0; i < 32; i += 4)
              *reinterpret_cast<uint4*>(dst + i) =
                  make_uint4(v0[i], v0[i + 1], v0[i + 2], v0[i + 3]);
          }
          continue;
        }
        if (MODE == MODE_UPDATE) {
          const int64_t n0 = (int64_t)nt * BN + col0;
          if (a.kb_cnt && a.kb_cnt[mt] == 0) {  // no non-zero block: Num = 0, den = 0
#pragma unroll
            for (int i = 0; i < 32; i++) v0[i] = 0u;
          }
          if (n0 < a.ld_pix) {
            if (F16) {  // FP16 responsibilities carry a 2^14 scale
#pragma unroll
              for (int i = 0; i < 32; i++)
                v0[i] = __float_as_uint(__uint_as_float(v0[i]) * (1.0f / kP16Scale));
            }
            if (a.den && a.n_pix >= n0 && a.n_pix < n0 + 32) {
#pragma unroll
              for (int i = 0; i < 32; i++)
                if (n0 + i == a.n_pix) a.den[row] = __uint_as_float(v0[i]);
            }
            if (XP) {
              // the lane's row into the warp's staging block, then out by rows:
              // in each step 8 lanes write one row's 32 columns (128 bytes), four
              // rows a step (16-byte rows at a stride of 36 floats: each quarter
              // warp's accesses fall on distinct banks)
              float* xp = xpose + e * (32 * kXpLd);
#pragma unroll
              for (int i = 0; i < 32; i += 4)
                *reinterpret_cast<uint4*>(xp + lane * kXpLd + i) =
                    make_uint4(v0[i], v0[i + 1], v0[i + 2], v0[i + 3]);
              __syncwarp();
              const int64_t row0 = (int64_t)mt * BM + 32 * q;
#pragma unroll
              for (int st = 0; st < 8; st++) {
                const int r = 4 * st + (lane >> 3), c4 = 4 * (lane & 7);
                const uint4 w = *reinterpret_cast<const uint4*>(xp + r * kXpLd + c4);
                *reinterpret_cast<uint4*>(a.Num + (row0 + r) * a.ld_pix + n0 + c4) = w;
              }
              __syncwarp();  // the block is rewritten by the next step
            } else {
              float* dst = a.Num + row * a.ld_pix + n0;
#pragma unroll
              for (int i = 0; i < 32; i += 4)
                *reinterpret_cast<uint4*>(dst + i) =
                    make_uint4(v0[i], v0[i + 1], v0[i + 2], v0[i + 3]);
            }
          }
          continue;
        }
        // scores: exact part xh (multiples of 1/64), small part xl
        float xh[32], xl[32];
#pragma unroll
        for (int i = 0; i < 32; i++) {
          float h, l;
          if (GAUSS) {
            const float gh = __uint_as_float(v0[i]), gl = __uint_as_float(v1[i]);
            const float2 c = cs[col0 + i];
            const float t = gh * gh;
            const float r = fmaf(gh, gh, -t) + gl * (2.f * gh + gl);  // (gh + gl)^2 - t
            const float x = c.x * t;
            const float rest = fmaf(c.x, t, -x) + fmaf(c.x, r, c.y * t);
            const float xg = rintf(x * kGrid) * (1.0f / kGrid);
            h = xg + bh;  // exact wherever |h| < 2^18
            l = ((x - xg) + rest) + bl;
          } else {
            h = __uint_as_float(v0[i]) + bh;
            l = (C::NACC == 2 ? __uint_as_float(v1[i]) : 0.f) + bl;
          }
          const float rr = rintf(l * kGrid) * (1.0f / kGrid);
          h += rr;
          l -= rr;
          if (GAUSS) {
            if (h < -kGaussClamp) {
              h = -kGaussClamp;
              l = 0.f;
            }
            big |= !(h <= 131072.f);  // also NaN
          } else {
            big |= fabsf(h) > 131072.f;
          }
          xh[i] = valid ? h : kSentinel;
          xl[i] = valid ? l : 0.f;
        }
        if (MODE == MODE_PASS1) {
          float v[32];
#pragma unroll
          for (int i = 0; i < 32; i++) v[i] = xh[i];
          const float mcol = warp_transpose_reduce<true>(v, lane);
          const int64_t k0 = (int64_t)nt * BN + col0;
#pragma unroll
          for (int i = 0; i < 32; i++) {
            const float mi = __shfl_sync(0xffffffffu, mcol, i);
            const float d = (xh[i] - mi) + xl[i];
            v[i] = valid ? __expf(d) : 0.f;
            xl[i] = d;
          }
          if (a.S) {
            // S_jk relative to the 32-row group maximum of column k, frame-major:
            // the warp's 32 lanes (consecutive rows) write one 128-byte segment per column
            float* Scol = a.S + k0 * a.rows + row;
#pragma unroll
            for (int i = 0; i < 32; i++) Scol[(int64_t)i * a.rows] = xl[i];
            a.Sref[((int64_t)mt * 4 + q) * a.ld_data + k0 + lane] = mcol;
          }
          const float scol = warp_transpose_reduce<false>(v, lane);
          scratch[q * BN + col0 + lane] = make_float2(mcol, scol);
        } else {
          const int64_t k0 = (int64_t)nt * BN + col0;
          uint32_t ph[16], pl[16];
#pragma unroll
          for (int i = 0; i < 32; i += 2) {
            float pr[2];
#pragma unroll
            for (int u = 0; u < 2; u++) {
              const float2 L = scratch[col0 + i + u];
              const float d = (xh[i + u] - L.x) + (xl[i + u] - L.y);
              pr[u] = (valid && k0 + i + u < a.n_data) ? __expf(d) : 0.f;
              if (flu) {
                dsum += pr[u];
                pr[u] *= Bj * sinv[col0 + i + u];
              }
            }
            if (F16) {  // FP16 hi + lo of 2^14 P
              const float s0 = pr[0] * kP16Scale, s1 = pr[1] * kP16Scale;
              const uint16_t h0 = fp16_bits(s0), h1 = fp16_bits(s1);
              ph[i / 2] = (uint32_t)h0 | ((uint32_t)h1 << 16);
              const uint16_t l0 = fp16_bits(s0 - fp16_val(h0)), l1 = fp16_bits(s1 - fp16_val(h1));
              pl[i / 2] = (uint32_t)l0 | ((uint32_t)l1 << 16);
            } else {
              const uint16_t h0 = bf16_bits(pr[0]), h1 = bf16_bits(pr[1]);
              ph[i / 2] = (uint32_t)h0 | ((uint32_t)h1 << 16);
              if (NA == 3 || flu) {
                const uint16_t l0 = bf16_bits(pr[0] - bf16_val(h0));
                const uint16_t l1 = bf16_bits(pr[1] - bf16_val(h1));
                pl[i / 2] = (uint32_t)l0 | ((uint32_t)l1 << 16);
              } else {
                pl[i / 2] = 0u;
              }
            }
          }
          if (a.kb_flag) {  // this warp's 32 rows x 32 frames: any non-zero P?
            uint32_t any = 0u;
#pragma unroll
            for (int i = 0; i < 16; i++) any |= ph[i] | pl[i];
            if (__any_sync(0xffffffffu, any != 0u) && lane == 0)
              a.kb_flag[(int64_t)mt * a.kb_ld + (k0 >> 6)] = 1;
          }
          uint16_t* dh = a.P + row * a.ld_data + k0;
          uint16_t* dl = dh + a.P_plane;
#pragma unroll
          for (int i = 0; i < 16; i += 4) {
            *reinterpret_cast<uint4*>(dh + 2 * i) = make_uint4(ph[i], ph[i + 1], ph[i + 2], ph[i + 3]);
            *reinterpret_cast<uint4*>(dl + 2 * i) = make_uint4(pl[i], pl[i + 1], pl[i + 2], pl[i + 3]);
          }
        }
      }
      if (NA >= 2 && big && valid) set_status(a.status, EMC_ERR_NUMERIC);
      if (flu && valid && dsum > 0.f) atomicAdd(a.den + row, dsum);
      if (MODE == MODE_PASS1) {
        named_bar(1, kEpiThreads);
        const int col = et;  // one frame column per epilogue thread
        float M = scratch[col].x;
#pragma unroll
        for (int qq = 1; qq < 4; qq++) M = fmaxf(M, scratch[qq * BN + col].x);
        float S = 0.f;
#pragma unroll
        for (int qq = 0; qq < 4; qq++) {
          const float2 ms = scratch[qq * BN + col];
          if (ms.y > 0.f) S += ms.y * __expf(ms.x - M);
        }
        const int64_t o = (int64_t)mt * a.ld_data + (int64_t)nt * BN + col;
        a.part_m[o] = (double)M;
        a.part_s[o] = S;
        named_bar(1, kEpiThreads);
      } else if (MODE == MODE_NORMALIZE) {
        named_bar(1, kEpiThreads);  // scratch is rewritten by the next tile
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, C::TMEM_COLS);
  }
}

// ------------------------------------------------------- pass-1 bound --
// The bound pass of the pruned pass 1: the hi plane of L alone, S^hi = hi K^T
// + bias, and only the maximum over each 128-row tile for every frame into
// part_m[tile][frame]. One CTA tile is a pair of row tiles sharing the
// 256-frame operand (two 128 x 256 accumulators, 512 TMEM columns): per
// 64-wide K block, 64 KB of operands feed eight 128 x 256 x 16 MMAs, where a
// single row tile would fetch its 32 KB frame block for four. A pair whose
// second row tile lies past the last one loads and contracts the first only.
// Roles, rings and bounded waits as in tc_kernel.
template <bool F16>
__global__ void __launch_bounds__(kThreads, 1)
    tc_bound_kernel(const __grid_constant__ CUtensorMap mapA,
                    const __grid_constant__ CUtensorMap mapB, const TcArgs a) {
  constexpr int BK = 64;
  constexpr int A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2;
  constexpr int STAGE = 2 * A_BYTES + B_BYTES;
  constexpr int STAGES = (kSmemBudget - kScratchBytes - 1024 - 256) / STAGE;
  constexpr uint32_t TMEM_COLS = 2 * BN;
  constexpr uint32_t IDESC = idesc_f16kind(BM, BN, 0, F16);
  static_assert(STAGES >= 2, "shared memory too small for two stages");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~(uintptr_t)1023);
  uint8_t* stages = smem;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;
  uint64_t* acc_empty = acc_full + 1;
  uint64_t* drain = acc_empty + 1;
  uint64_t* never = drain + 1;  // the stall hook's barrier: nothing arrives on it
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(never + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* scratch = reinterpret_cast<float*>(smem + STAGES * STAGE + 256);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; s++) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, kEpiWarps);
    mbar_init(drain, 1);
    mbar_init(never, 1);
    *abort = 0;
    fence_mbar_init();
  }
  if (warp == 0 && lane == 0) {
    prefetch_tmap(&mapA);
    prefetch_tmap(&mapB);
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int T = a.tile_count ? *a.tile_count : a.n_mtiles * a.n_ntiles;

  if (warp == 0) {
    // ------------------------------------------------------------ producer --
    if (lane == 0) {
      int it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < T && ok; t += gridDim.x) {
        int mp, nt;
        tile_coords(t, a, &mp, &nt);
        const bool two = 2 * mp + 1 < a.n_rowtiles;
        for (int kb = 0; kb < a.kblocks; kb++, it++) {
          const int s = it % STAGES;
          const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
          if (!mbar_wait(empty + s, ph ^ 1u, abort, a.wait_ns)) {
            fail(abort, a.status);
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(full + s, two ? STAGE : STAGE - A_BYTES);
          uint8_t* st = stages + s * STAGE;
          tma_load_3d(st, &mapA, full + s, kb * BK, 2 * mp * BM, 0);
          if (two) tma_load_3d(st + A_BYTES, &mapA, full + s, kb * BK, (2 * mp + 1) * BM, 0);
          tma_load_2d(st + 2 * A_BYTES, &mapB, full + s, kb * BK, nt * BN);
        }
      }
      if (!ok) {
        for (int back = 1; back <= STAGES && it - back >= 0; back++) {
          const int j = it - back;
          mbar_wait_quiet(full + (j % STAGES), (uint32_t)(j / STAGES) & 1u, kWaitLimitNs);
        }
      }
    }
  } else if (warp == 1) {
    // ----------------------------------------------------------------- MMA --
    if (lane == 0) {
      int it = 0, tcount = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < T && ok; t += gridDim.x, tcount++) {
        if (!mbar_wait(acc_empty, ((uint32_t)tcount & 1u) ^ 1u, abort, a.wait_ns)) {
          fail(abort, a.status);
          break;
        }
        tc_fence_after();
        int mp, nt;
        tile_coords(t, a, &mp, &nt);
        const int nr = 2 * mp + 1 < a.n_rowtiles ? 2 : 1;
        for (int kb = 0; kb < a.kblocks; kb++, it++) {
          const int s = it % STAGES;
          const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
          uint64_t* wb = (a.stall && it == 0) ? never : full + s;
          if (!mbar_wait(wb, ph, abort, a.wait_ns)) {
            fail(abort, a.status);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sA = smem_u32(stages + s * STAGE);
          const uint32_t sB = sA + 2 * A_BYTES;
#pragma unroll
          for (int k = 0; k < BK / 16; k++) {
            const uint64_t bdesc = kmajor_desc<BK>(sB, k);
            for (int r = 0; r < nr; r++)
              umma_bf16(tmem + r * BN, kmajor_desc<BK>(sA + r * A_BYTES, k), bdesc, IDESC,
                        (kb == 0 && k == 0) ? 0u : 1u);
          }
          umma_commit(empty + s);
        }
        if (ok) umma_commit(acc_full);
      }
      umma_commit(drain);
      mbar_wait_quiet(drain, 0, kWaitLimitNs);
    }
  } else {
    // ------------------------------------------------------------ epilogue --
    const int e = warp - 2;
    const int q = warp & 3;
    const int half = e >> 2;
    const int r_in = 32 * q + lane;
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * q) << 16);
    const int et = e * 32 + lane;
    int tcount = 0;
    for (int t = blockIdx.x; t < T; t += gridDim.x, tcount++) {
      int mp, nt;
      tile_coords(t, a, &mp, &nt);
      const int nr = 2 * mp + 1 < a.n_rowtiles ? 2 : 1;
      const bool got = mbar_wait(acc_full, (uint32_t)tcount & 1u, abort, a.wait_ns);
      if (!got) fail(abort, a.status);
      if (named_bar_any(2, kEpiThreads, !got)) break;
      tc_fence_after();
      for (int r = 0; r < nr; r++) {
        const int mt = 2 * mp + r;
        const int64_t row = (int64_t)mt * BM + r_in;
        const double b = a.bias[row];
        const bool valid = row < a.nrot && b > -INFINITY;
        const float bf = valid ? (float)b : 0.f;
#pragma unroll 1
        for (int c = 0; c < 4; c++) {
          const int col0 = half * 128 + c * 32;
          uint32_t v0[32];
          tmem_ld32(lane_addr + r * BN + col0, v0);
          tmem_ld_wait();
          if (r == nr - 1 && c == 3) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acc_empty);
          }
          float v[32];
#pragma unroll
          for (int i = 0; i < 32; i++) v[i] = valid ? __uint_as_float(v0[i]) + bf : kSentinel;
          scratch[q * BN + col0 + lane] = warp_transpose_reduce<true>(v, lane);
        }
        named_bar(1, kEpiThreads);
        float M = scratch[et];
#pragma unroll
        for (int qq = 1; qq < 4; qq++) M = fmaxf(M, scratch[qq * BN + et]);
        a.part_m[(int64_t)mt * a.ld_data + (int64_t)nt * BN + et] = (double)M;
        named_bar(1, kEpiThreads);
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

// ------------------------------------------------------------- host side --
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// BF16 tensor map (128- or 64-byte swizzle); dims innermost first, strides in bytes.
bool make_map(CUtensorMap* m, const void* base, int rank, const uint64_t* dims,
              const uint64_t* strides, const uint32_t* box, int swizzle_bytes = 128,
              bool fp16 = false) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t d[3], st[2];
  cuuint32_t b[3], es[3] = {1, 1, 1};
  for (int i = 0; i < rank; i++) {
    d[i] = dims[i];
    b[i] = box[i];
  }
  for (int i = 0; i < rank - 1; i++) st[i] = strides[i];
  return fn(m, fp16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
            (cuuint32_t)rank, const_cast<void*>(base), d, st,
            b, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            swizzle_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int num_sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 148;
}

template <int MODE, int NA, bool F16, bool XP = false>
cudaError_t launch(const CUtensorMap& mA, const CUtensorMap& mB, TcArgs a, cudaStream_t s) {
  using C = TcCfg<MODE, NA, F16, XP>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(tc_kernel<MODE, NA, F16, XP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int T = a.n_mtiles * a.n_ntiles;
  if (T <= 0) return cudaSuccess;
  // a device-side tile list: one persistent CTA per SM (the count is read on the device)
  const int grid = (!a.tile_list && T < num_sms()) ? T : num_sms();
  tc_kernel<MODE, NA, F16, XP><<<grid, kThreads, C::SMEM, s>>>(mA, mB, a);
  return cudaGetLastError();
}

// planes of log W and operand type of each tensor-core precision
int score_planes(int precision) {
  return precision == EMC_PREC_BF16_SPLIT ? 3 : (precision == EMC_PREC_FP16_SPLIT ? 2 : 1);
}

bool maps_scores(const Planes& L, int nterms, bool f16, int64_t rows, const uint16_t* Kb,
                 int64_t ld_data, int64_t ld_pix, CUtensorMap* mA, CUtensorMap* mB) {
  const uint32_t bk = nterms >= 2 ? 32 : 64;  // TcCfg<scores, NA, F16>::BK
  const int sw = nterms >= 2 ? 64 : 128;
  const uint64_t dA[3] = {(uint64_t)ld_pix, (uint64_t)rows, (uint64_t)nterms};
  const uint64_t sA[2] = {(uint64_t)L.ld * 2, (uint64_t)L.plane_stride * 2};
  const uint32_t bA[3] = {bk, BM, 1};
  const uint64_t dB[2] = {(uint64_t)ld_pix, (uint64_t)ld_data};
  const uint64_t sB[1] = {(uint64_t)ld_pix * 2};
  const uint32_t bB[2] = {bk, BN};
  return make_map(mA, L.base, 3, dA, sA, bA, sw, f16) && make_map(mB, Kb, 2, dB, sB, bB, sw, f16);
}

TcArgs base_args(int64_t rows, int n_ntiles, int kblocks) {
  TcArgs a{};
  a.n_mtiles = (int)(rows / BM);
  a.rows = rows;
  a.n_ntiles = n_ntiles;
  a.group = 8;
  a.kblocks = kblocks;
  a.wait_ns = kWaitLimitNs;
  return a;
}

}  // namespace

int64_t tc_pass1_tiles(int64_t rows) { return rows / BM; }

cudaError_t launch_tc_bound(const Planes& L, int precision, const double* bias, int64_t rows,
                            const uint16_t* Kb, int64_t ld_data, int64_t ld_pix, double* part_m,
                            int32_t* status, cudaStream_t s, TcCtl ctl, const int32_t* pair_list,
                            const int32_t* pair_count) {
  const bool f16 = precision == EMC_PREC_FP16_SPLIT;
  CUtensorMap mA, mB;
  if (!maps_scores(L, 1, f16, rows, Kb, ld_data, ld_pix, &mA, &mB)) return cudaErrorInvalidValue;
  const int nrt = (int)(rows / BM);
  TcArgs a = base_args(rows, (int)(ld_data / BN), (int)(ld_pix / 64));
  a.n_mtiles = (nrt + 1) / 2;  // pairs of row tiles
  a.group = 4;                 // raster groups of 8 row tiles, as the other passes
  a.n_rowtiles = nrt;
  a.nrot = rows;  // validity comes from the bias (-inf on padding rows)
  a.ld_data = ld_data;
  a.bias = bias;
  a.part_m = part_m;
  a.status = status;
  if (ctl.wait_ns) a.wait_ns = ctl.wait_ns;
  a.stall = ctl.stall;
  a.tile_list = pair_list;
  a.tile_count = pair_list ? pair_count : nullptr;
  constexpr int kStage = 2 * BM * 64 * 2 + BN * 64 * 2;
  constexpr int kStages = (kSmemBudget - kScratchBytes - 1024 - 256) / kStage;
  constexpr int kSmem = 1024 + kStages * kStage + 256 + kScratchBytes;
  static bool attr[2] = {false, false};
  cudaError_t e = cudaSuccess;
  if (!attr[f16]) {
    e = f16 ? cudaFuncSetAttribute(tc_bound_kernel<true>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem)
            : cudaFuncSetAttribute(tc_bound_kernel<false>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (e != cudaSuccess) return e;
    attr[f16] = true;
  }
  const int T = a.n_mtiles * a.n_ntiles;
  if (T <= 0) return cudaSuccess;
  // a device-side pair list: one persistent CTA per SM (the count is read on the device)
  const int grid = (!pair_list && T < num_sms()) ? T : num_sms();
  if (f16)
    tc_bound_kernel<true><<<grid, kThreads, kSmem, s>>>(mA, mB, a);
  else
    tc_bound_kernel<false><<<grid, kThreads, kSmem, s>>>(mA, mB, a);
  return cudaGetLastError();
}

cudaError_t launch_tc_store(const Planes& A, int64_t rows, const uint16_t* Kb, int64_t ld_data,
                            int64_t ld_pix, float* C, int f16, int32_t* status, cudaStream_t s,
                            TcCtl ctl) {
  CUtensorMap mA, mB;
  if (!maps_scores(A, 1, f16 != 0, rows, Kb, ld_data, ld_pix, &mA, &mB))
    return cudaErrorInvalidValue;
  TcArgs a = base_args(rows, (int)(ld_data / BN), (int)(ld_pix / 64));
  a.nrot = rows;
  a.ld_data = ld_data;
  a.ld_pix = ld_pix;
  a.Num = C;
  a.status = status;
  if (ctl.wait_ns) a.wait_ns = ctl.wait_ns;
  a.stall = ctl.stall;
  // A and B of one MMA always share their type: FP16 frames take FP16 increments
  if (f16) return launch<MODE_STORE, 1, true, true>(mA, mB, a, s);
  return launch<MODE_STORE, 1, false, true>(mA, mB, a, s);
}

cudaError_t launch_tc_pass1(const Planes& L, int precision, const double* bias, int64_t rows,
                            const uint16_t* Kb, int64_t ld_data, int64_t n_data, int64_t ld_pix,
                            double* part_m, float* part_s, float* S, float* Sref,
                            const float4* gk, const float4* gsc, int32_t* status,
                            cudaStream_t s, const int32_t* tile_list,
                            const int32_t* tile_count, TcCtl ctl) {
  const bool gauss = gk != nullptr;
  const int nterms = gauss ? 3 : score_planes(precision);
  const bool f16 = gauss || precision == EMC_PREC_FP16_SPLIT;
  CUtensorMap mA, mB;
  if (!maps_scores(L, nterms, f16, rows, Kb, ld_data, ld_pix, &mA, &mB))
    return cudaErrorInvalidValue;
  TcArgs a = base_args(rows, (int)(ld_data / BN), (int)(ld_pix / (nterms >= 2 ? 32 : 64)));
  a.nrot = rows;  // validity comes from the bias (-inf on padding rows)
  a.n_data = n_data;
  a.ld_data = ld_data;
  a.ld_pix = ld_pix;
  a.bias = bias;
  a.part_m = part_m;
  a.part_s = part_s;
  a.S = S;
  a.Sref = Sref;
  a.gk = gk;
  a.gsc = gsc;
  a.tile_list = tile_list;
  a.tile_count = tile_list ? tile_count : nullptr;
  a.status = status;
  if (ctl.wait_ns) a.wait_ns = ctl.wait_ns;
  a.stall = ctl.stall;
  if (gauss) return launch<MODE_PASS1, 3, true>(mA, mB, a, s);
  if (precision == EMC_PREC_FP16_SPLIT) return launch<MODE_PASS1, 2, true>(mA, mB, a, s);
  return nterms == 3 ? launch<MODE_PASS1, 3, false>(mA, mB, a, s)
                     : launch<MODE_PASS1, 1, false>(mA, mB, a, s);
}

cudaError_t launch_tc_normalize(const Planes& L, int precision, const double* bias, int64_t rows,
                                int64_t nrot, const uint16_t* Kb, int64_t ld_data, int64_t n_data,
                                int64_t ld_pix, const double* lse_m, const double* lse_s,
                                float2* lse2, Planes P, int32_t* status, cudaStream_t s,
                                const double* shift, const double* Bsum, const float* invn,
                                float* den, uint8_t* kb_flag, const int32_t* tile_list,
                                const int32_t* tile_count, TcCtl ctl) {
  cudaError_t e = launch_lse_split(lse_m, lse_s, n_data, ld_data, lse2, s, shift);
  if (e != cudaSuccess) return e;
  if (kb_flag) {
    e = cudaMemsetAsync(kb_flag, 0, (size_t)(rows / BM) * (ld_data / 64), s);
    if (e != cudaSuccess) return e;
  }
  if (Bsum) {
    if (!invn || !den || precision == EMC_PREC_FP16_SPLIT) return cudaErrorInvalidValue;
    e = cudaMemsetAsync(den, 0, sizeof(float) * rows, s);
    if (e != cudaSuccess) return e;
  }
  const int nterms = score_planes(precision);
  CUtensorMap mA, mB;
  if (!maps_scores(L, nterms, precision == EMC_PREC_FP16_SPLIT, rows, Kb, ld_data, ld_pix, &mA,
                   &mB))
    return cudaErrorInvalidValue;
  TcArgs a = base_args(rows, (int)(ld_data / BN), (int)(ld_pix / (nterms >= 2 ? 32 : 64)));
  a.nrot = nrot;
  a.n_data = n_data;
  a.ld_data = ld_data;
  a.ld_pix = ld_pix;
  a.bias = bias;
  a.lse2 = lse2;
  a.P = reinterpret_cast<uint16_t*>(P.base);
  a.P_plane = P.plane_stride;
  a.Bsum = Bsum;
  a.invn = invn;
  a.den = den;
  a.kb_flag = kb_flag;
  a.kb_ld = (int)(ld_data / 64);
  a.tile_list = tile_list;
  a.tile_count = tile_list ? tile_count : nullptr;
  a.status = status;
  if (ctl.wait_ns) a.wait_ns = ctl.wait_ns;
  a.stall = ctl.stall;
  if (precision == EMC_PREC_FP16_SPLIT) return launch<MODE_NORMALIZE, 2, true>(mA, mB, a, s);
  return nterms == 3 ? launch<MODE_NORMALIZE, 3, false>(mA, mB, a, s)
                     : launch<MODE_NORMALIZE, 1, false>(mA, mB, a, s);
}

cudaError_t launch_tc_update(const Planes& P, int precision, int64_t rows, const uint16_t* Kb,
                             int64_t ld_data, int64_t ld_pix, int64_t n_pix, float* Num, float* den,
                             int32_t* status, cudaStream_t s, const int32_t* kb_cnt,
                             const int32_t* kb_list, TcCtl ctl, bool staged) {
  const int nterms = precision == EMC_PREC_BF16 ? 1 : 2;
  const bool f16 = precision == EMC_PREC_FP16_SPLIT;
  CUtensorMap mA, mB;
  const uint64_t dA[3] = {(uint64_t)ld_data, (uint64_t)rows, (uint64_t)nterms};
  const uint64_t sA[2] = {(uint64_t)P.ld * 2, (uint64_t)P.plane_stride * 2};
  const uint32_t bA[3] = {64, BM, 1};
  const uint64_t dB[2] = {(uint64_t)ld_pix, (uint64_t)ld_data};
  const uint64_t sB[1] = {(uint64_t)ld_pix * 2};
  const uint32_t bB[2] = {64, 64};
  if (!make_map(&mA, P.base, 3, dA, sA, bA, 128, f16) || !make_map(&mB, Kb, 2, dB, sB, bB, 128, f16))
    return cudaErrorInvalidValue;
  TcArgs a = base_args(rows, (int)((ld_pix + BN - 1) / BN), (int)(ld_data / 64));
  a.nrot = rows;
  a.ld_pix = ld_pix;
  a.n_pix = n_pix;
  a.ld_data = ld_data;
  a.Num = Num;
  a.den = den;
  a.kb_cnt = kb_cnt;
  a.kb_list = kb_list;
  a.kb_ld = (int)(ld_data / 64);
  a.status = status;
  if (ctl.wait_ns) a.wait_ns = ctl.wait_ns;
  a.stall = ctl.stall;
  if (staged) {  // bound by its output: row stores through the staging block
    if (f16) return launch<MODE_UPDATE, 2, true, true>(mA, mB, a, s);
    return nterms == 2 ? launch<MODE_UPDATE, 2, false, true>(mA, mB, a, s)
                       : launch<MODE_UPDATE, 1, false, true>(mA, mB, a, s);
  }
  if (f16) return launch<MODE_UPDATE, 2, true>(mA, mB, a, s);
  return nterms == 2 ? launch<MODE_UPDATE, 2, false>(mA, mB, a, s)
                     : launch<MODE_UPDATE, 1, false>(mA, mB, a, s);
}

}  // namespace emc
