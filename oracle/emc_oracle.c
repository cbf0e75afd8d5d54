/*
 * emc_oracle.c -- plain, slow, FP64 CPU oracle of the EMC hot path.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library. It shares no code,
 * header, table or helper with the GPU library; both only consume the same
 * seeded inputs.
 *
 * Every function follows one passage of Ekeberg, Engblom & Liu,
 * "Machine learning for ultrafast X-ray diffraction patterns on large-scale
 * GPU clusters" (arXiv:1409.4256), in the paper's notation:
 *   i = pixel, j = rotation, k = frame (pattern), l = grid voxel.
 * Loops are written straight from the definitions: no blocking, no fusion.
 * OpenMP only distributes independent outer iterations.
 *
 * Readings taken where the paper is silent (each listed in the design notes):
 *  - Poisson noise model (Sec. 2.2, the original EMC's Poisson signal):
 *      log P(K_ik | W_ij) = K_ik log W_ij - W_ij - log K_ik!,
 *    the last term dropped (constant per frame, cancels in Eq. 2.4).
 *  - interpolation kernel f of Eq. 2.8 = trilinear (tent) weights;
 *    grid index of a point q is q + N/2; corners outside [0, N) carry no value.
 *  - expanded intensities are floored: W_ij <- max(W_ij, w_floor).
 *  - prior weights w_j of the quaternion sampling (Sec. 2.2 gives no formula):
 *    w_j proportional to 1/|x_j|^4, x_j the flat lattice point before
 *    projection to the unit sphere (Jacobian of radial projection of a flat
 *    tetrahedral cell onto S^3), normalised to sum 1.
 *  - Eq. 2.12 voxels with zero denominator keep their previous value.
 *  - Gaussian model: see the block before oracle_fluence.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Eq. 2.7: rotations from the 600-cell with each tetrahedral cell divided n */
/* times; M_rot(n) = 10 (5 n^3 + n).                                          */
/*                                                                           */
/* Coordinates of the 600-cell vertices lie in Z[sqrt 5] / 4, so all lattice */
/* points are handled exactly as integer pairs (A, B) meaning                */
/* (A + B sqrt 5) / (4 n); duplicates across shared faces are then removed   */
/* exactly.                                                                  */
/* ------------------------------------------------------------------------ */

#define NVERT 120

static int vtx[NVERT][4][2]; /* vertex v, coordinate c: (a + b sqrt5) / 4 */

static int perm_parity(const int p[4]) {
  int inv = 0;
  for (int a = 0; a < 4; a++)
    for (int b = a + 1; b < 4; b++)
      if (p[a] > p[b]) inv++;
  return inv & 1;
}

static void make_600cell_vertices(void) {
  int n = 0;
  memset(vtx, 0, sizeof(vtx));
  /* 8 vertices: +-1 along one axis */
  for (int ax = 0; ax < 4; ax++)
    for (int s = -1; s <= 1; s += 2) {
      vtx[n][ax][0] = 4 * s;
      n++;
    }
  /* 16 vertices: (+-1/2, +-1/2, +-1/2, +-1/2) */
  for (int m = 0; m < 16; m++) {
    for (int c = 0; c < 4; c++) vtx[n][c][0] = ((m >> c) & 1) ? -2 : 2;
    n++;
  }
  /* 96 vertices: even permutations of (+-phi, +-1, +-1/phi, 0) / 2, where
   * phi/2 = (1 + sqrt5)/4, 1/2 = 2/4, 1/(2 phi) = (-1 + sqrt5)/4.        */
  const int base[4][2] = {{1, 1}, {2, 0}, {-1, 1}, {0, 0}};
  int p[4];
  for (p[0] = 0; p[0] < 4; p[0]++)
    for (p[1] = 0; p[1] < 4; p[1]++)
      for (p[2] = 0; p[2] < 4; p[2]++)
        for (p[3] = 0; p[3] < 4; p[3]++) {
          if (p[0] == p[1] || p[0] == p[2] || p[0] == p[3] || p[1] == p[2] ||
              p[1] == p[3] || p[2] == p[3])
            continue;
          if (perm_parity(p)) continue;
          for (int sg = 0; sg < 8; sg++) {
            for (int t = 0; t < 4; t++) {
              int s = (t < 3 && ((sg >> t) & 1)) ? -1 : 1;
              vtx[n][p[t]][0] = s * base[t][0];
              vtx[n][p[t]][1] = s * base[t][1];
            }
            n++;
          }
        }
}

/* Two vertices share an edge iff |v - w|^2 = 1/phi^2 = (24 - 8 sqrt5)/16. */
static int is_edge(int v, int w) {
  long r = 0, s = 0;
  for (int c = 0; c < 4; c++) {
    long da = vtx[v][c][0] - vtx[w][c][0];
    long db = vtx[v][c][1] - vtx[w][c][1];
    r += da * da + 5 * db * db;
    s += da * db;
  }
  return r == 24 && s == -4;
}

/* sign of (a + b sqrt5) */
static int zr5_sign(long a, long b) {
  if (a >= 0 && b >= 0) return (a > 0 || b > 0) ? 1 : 0;
  if (a <= 0 && b <= 0) return -1;
  /* opposite signs: compare a^2 with 5 b^2 */
  if (a > 0) return (a * a > 5 * b * b) ? 1 : -1;
  return (a * a > 5 * b * b) ? -1 : 1;
}

static int cmp_key8(const void* x, const void* y) {
  const int32_t* a = (const int32_t*)x;
  const int32_t* b = (const int32_t*)y;
  for (int t = 0; t < 8; t++) {
    if (a[t] < b[t]) return -1;
    if (a[t] > b[t]) return 1;
  }
  return 0;
}

typedef struct {
  int64_t key[4];
  uint64_t z;  /* Morton code of the (x, y, z) keys, the primary order */
  double q[4];
  double w;
} qrec;

/* interleave the top 10 bits of key + 2^30 of x, y, z (bit b of axis d goes to
 * bit 3 b + d) */
static uint64_t morton_xyz(const int64_t* key) {
  uint64_t z = 0;
  for (int d = 0; d < 3; d++) {
    int64_t u = (key[1 + d] + ((int64_t)1 << 30)) / ((int64_t)1 << 21);
    if (u < 0) u = 0;
    if (u > 1023) u = 1023;
    for (int b = 0; b < 10; b++)
      if ((u >> b) & 1) z |= (uint64_t)1 << (3 * b + d);
  }
  return z;
}

static int cmp_qrec(const void* x, const void* y) {
  const qrec* a = (const qrec*)x;
  const qrec* b = (const qrec*)y;
  if (a->z != b->z) return a->z < b->z ? -1 : 1;
  for (int t = 0; t < 4; t++) {
    if (a->key[t] < b->key[t]) return -1;
    if (a->key[t] > b->key[t]) return 1;
  }
  return 0;
}

/* Number of cells of the 600-cell found as 4-cliques of the edge graph. */
long oracle_600cell_counts(long* n_vertices, long* n_edges) {
  make_600cell_vertices();
  long ne = 0, nc = 0;
  for (int a = 0; a < NVERT; a++)
    for (int b = a + 1; b < NVERT; b++)
      if (is_edge(a, b)) ne++;
  for (int a = 0; a < NVERT; a++)
    for (int b = a + 1; b < NVERT; b++) {
      if (!is_edge(a, b)) continue;
      for (int c = b + 1; c < NVERT; c++) {
        if (!is_edge(a, c) || !is_edge(b, c)) continue;
        for (int d = c + 1; d < NVERT; d++)
          if (is_edge(a, d) && is_edge(b, d) && is_edge(c, d)) nc++;
      }
    }
  if (n_vertices) *n_vertices = NVERT;
  if (n_edges) *n_edges = ne;
  return nc;
}

/*
 * Rotation sampling of Eq. 2.7. Writes up to cap unit quaternions (w,x,y,z)
 * into quat[cap][4] and prior weights (sum 1) into weight[cap]; either may be
 * NULL to count only. uniform != 0 gives equal weights. Returns the number of
 * rotations, or -1 on allocation failure, -2 if cap is too small.
 * Order (a convention shared with the library, not the paper's): q
 * canonicalised so that its first non-zero component is positive;
 * k_c = round(q_c * 2^30); sorted by the Morton code of the top 10 bits of
 * k_x + 2^30, k_y + 2^30, k_z + 2^30, ties by (k_w, k_x, k_y, k_z).
 */
long oracle_quat_generate(int n, int uniform, double* quat, double* weight, long cap) {
  if (n < 1) return -1;
  make_600cell_vertices();
  /* cells */
  int(*cells)[4] = malloc(sizeof(int[4]) * 600);
  if (!cells) return -1;
  long nc = 0;
  for (int a = 0; a < NVERT; a++)
    for (int b = a + 1; b < NVERT; b++) {
      if (!is_edge(a, b)) continue;
      for (int c = b + 1; c < NVERT; c++) {
        if (!is_edge(a, c) || !is_edge(b, c)) continue;
        for (int d = c + 1; d < NVERT; d++)
          if (is_edge(a, d) && is_edge(b, d) && is_edge(c, d)) {
            if (nc < 600) {
              cells[nc][0] = a; cells[nc][1] = b; cells[nc][2] = c; cells[nc][3] = d;
            }
            nc++;
          }
      }
    }
  if (nc != 600) { free(cells); return -1; }
  /* lattice points: sum_a (m_a / n) v_a, sum_a m_a = n, m_a >= 0 */
  long per_cell = (long)(n + 3) * (n + 2) * (n + 1) / 6;
  long total = per_cell * 600;
  int32_t* keys = malloc(sizeof(int32_t) * 8 * (size_t)total);
  if (!keys) { free(cells); return -1; }
  long np = 0;
  for (long c = 0; c < 600; c++)
    for (int m0 = 0; m0 <= n; m0++)
      for (int m1 = 0; m0 + m1 <= n; m1++)
        for (int m2 = 0; m0 + m1 + m2 <= n; m2++) {
          int m3 = n - m0 - m1 - m2;
          int m[4] = {m0, m1, m2, m3};
          int32_t* k = keys + 8 * np;
          for (int t = 0; t < 4; t++) {
            long A = 0, B = 0;
            for (int a = 0; a < 4; a++) {
              A += (long)m[a] * vtx[cells[c][a]][t][0];
              B += (long)m[a] * vtx[cells[c][a]][t][1];
            }
            k[2 * t] = (int32_t)A;
            k[2 * t + 1] = (int32_t)B;
          }
          np++;
        }
  free(cells);
  qsort(keys, (size_t)np, sizeof(int32_t) * 8, cmp_key8);
  /* unique, and keep the representative of q ~ -q whose first non-zero
   * component is positive (the set is centrally symmetric) */
  qrec* recs = malloc(sizeof(qrec) * (size_t)np);
  if (!recs) { free(keys); return -1; }
  long nr = 0;
  const double s5 = sqrt(5.0);
  for (long p = 0; p < np; p++) {
    if (p > 0 && cmp_key8(keys + 8 * p, keys + 8 * (p - 1)) == 0) continue;
    const int32_t* k = keys + 8 * p;
    int sign = 0;
    for (int t = 0; t < 4 && sign == 0; t++) sign = zr5_sign(k[2 * t], k[2 * t + 1]);
    if (sign <= 0) continue;
    double x[4], r2 = 0.0;
    for (int t = 0; t < 4; t++) {
      x[t] = ((double)k[2 * t] + (double)k[2 * t + 1] * s5) / (4.0 * n);
      r2 += x[t] * x[t];
    }
    double r = sqrt(r2);
    qrec* R = recs + nr;
    for (int t = 0; t < 4; t++) {
      R->q[t] = x[t] / r;
      R->key[t] = llround(R->q[t] * 1073741824.0);
    }
    R->z = morton_xyz(R->key);
    R->w = uniform ? 1.0 : 1.0 / (r2 * r2);
    nr++;
  }
  free(keys);
  qsort(recs, (size_t)nr, sizeof(qrec), cmp_qrec);
  if ((quat || weight) && nr > cap) { free(recs); return -2; }
  double wsum = 0.0;
  for (long p = 0; p < nr; p++) wsum += recs[p].w;
  for (long p = 0; p < nr; p++) {
    if (quat)
      for (int t = 0; t < 4; t++) quat[4 * p + t] = recs[p].q[t];
    if (weight) weight[p] = recs[p].w / wsum;
  }
  free(recs);
  return nr;
}

/* Rotation matrix of a unit quaternion (w, x, y, z), row-major R[3][3]. */
void oracle_quat_to_matrix(const double* q, double* R) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* ------------------------------------------------------------------------ */
/* Interpolation weights f(p_l - R_j q_i) of Eq. 2.8 (trilinear reading).     */
/* Fills up to 8 (voxel index, weight) pairs; returns how many.              */
/* Grid layout: voxel (x, y, z) at l = (x N + y) N + z.                       */
/* ------------------------------------------------------------------------ */
static int interp_weights(int N, const double* R, const double* qi, long* idx, double* wt) {
  double p[3];
  for (int a = 0; a < 3; a++)
    p[a] = R[3 * a] * qi[0] + R[3 * a + 1] * qi[1] + R[3 * a + 2] * qi[2] + 0.5 * N;
  long f[3];
  double t[3];
  for (int a = 0; a < 3; a++) {
    f[a] = (long)floor(p[a]);
    t[a] = p[a] - (double)f[a];
  }
  int n = 0;
  for (int c = 0; c < 8; c++) {
    long x = f[0] + (c >> 2 & 1), y = f[1] + (c >> 1 & 1), z = f[2] + (c & 1);
    if (x < 0 || y < 0 || z < 0 || x >= N || y >= N || z >= N) continue;
    double w = ((c >> 2 & 1) ? t[0] : 1 - t[0]) * ((c >> 1 & 1) ? t[1] : 1 - t[1]) *
               ((c & 1) ? t[2] : 1 - t[2]);
    idx[n] = (x * N + y) * N + z;
    wt[n] = w;
    n++;
  }
  return n;
}

/*
 * Expansion (e-step), Eq. 2.9: W_ij = sum_l f(p_l - R_j q_i) WW_l,
 * then W_ij <- max(W_ij, w_floor).
 * grid[N^3], quat[n_rot][4], q[n_pix][3] -> W[n_rot][n_pix].
 */
void oracle_expand(int N, const double* grid, long n_rot, const double* quat, long n_pix,
                   const double* q, double w_floor, double* W) {
#pragma omp parallel for schedule(dynamic, 4)
  for (long j = 0; j < n_rot; j++) {
    double R[9];
    oracle_quat_to_matrix(quat + 4 * j, R);
    for (long i = 0; i < n_pix; i++) {
      long idx[8];
      double wt[8];
      int nw = interp_weights(N, R, q + 3 * i, idx, wt);
      double v = 0.0;
      for (int c = 0; c < nw; c++) v += wt[c] * grid[idx[c]];
      W[j * n_pix + i] = v > w_floor ? v : w_floor;
    }
  }
}

/*
 * Joint log-likelihood of Eq. 2.3 under the Poisson model, plus the log prior
 * weight that Eq. 2.4 multiplies in:
 *   S_jk = sum_i (K_ik log W_ij - W_ij) + log w_j.
 * W[n_rot][n_pix], weight[n_rot], K[n_data][n_pix] -> S[n_rot][n_data].
 */
void oracle_scores(long n_rot, long n_pix, long n_data, const double* W, const double* weight,
                   const double* K, double* S) {
#pragma omp parallel
  {
    double* logWj = malloc(sizeof(double) * (size_t)n_pix);
#pragma omp for schedule(dynamic, 4)
    for (long j = 0; j < n_rot; j++) {
      const double* Wj = W + j * n_pix;
      double sumW = 0.0;
      for (long i = 0; i < n_pix; i++) {
        sumW += Wj[i];
        logWj[i] = log(Wj[i]);
      }
      double logw = log(weight[j]);
      for (long k = 0; k < n_data; k++) {
        const double* Kk = K + k * n_pix;
        double s = 0.0;
        for (long i = 0; i < n_pix; i++) s += Kk[i] * logWj[i];
        S[j * n_data + k] = s - sumW + logw;
      }
    }
    free(logWj);
  }
}

/*
 * E-step, Eq. 2.4 with T_jk = exp(Q_jk): P_jk = w_j T_jk / sum_j' w_j' T_j'k.
 * Evaluated as exp(S_jk - lse_k) with lse_k = m_k + log sum_j exp(S_jk - m_k),
 * m_k = max_j S_jk (the care against finite precision the paper asks for;
 * only maxima and sums are needed, Sec. 3.3).
 * S[n_rot][n_data] -> P[n_rot][n_data], lse[n_data]. Returns sum_k lse_k.
 */
double oracle_estep(long n_rot, long n_data, const double* S, double* P, double* lse) {
  double total = 0.0;
#pragma omp parallel for reduction(+ : total)
  for (long k = 0; k < n_data; k++) {
    double m = -INFINITY;
    for (long j = 0; j < n_rot; j++)
      if (S[j * n_data + k] > m) m = S[j * n_data + k];
    double s = 0.0;
    for (long j = 0; j < n_rot; j++) s += exp(S[j * n_data + k] - m);
    double l = m + log(s);
    if (lse) lse[k] = l;
    if (P)
      for (long j = 0; j < n_rot; j++) P[j * n_data + k] = exp(S[j * n_data + k] - l);
    total += l;
  }
  return total;
}

/*
 * M-step numerator of Eq. 2.11 (phi = 1 in the Poisson model) and the
 * responsibility sums that Eq. 2.12 places in the denominator:
 *   Num_ij = sum_k P_jk K_ik,   den_j = sum_k P_jk.
 * P[n_rot][n_data], K[n_data][n_pix] -> Num[n_rot][n_pix], den[n_rot].
 */
void oracle_mstep(long n_rot, long n_pix, long n_data, const double* P, const double* K,
                  double* Num, double* den) {
#pragma omp parallel for schedule(dynamic, 4)
  for (long j = 0; j < n_rot; j++) {
    double d = 0.0;
    for (long k = 0; k < n_data; k++) d += P[j * n_data + k];
    den[j] = d;
    for (long i = 0; i < n_pix; i++) {
      double s = 0.0;
      for (long k = 0; k < n_data; k++) s += P[j * n_data + k] * K[k * n_pix + i];
      Num[j * n_pix + i] = s;
    }
  }
}

/*
 * Compression (c-step).
 *  mode 0, Eq. 2.12 (deferred normalisation, the paper's implementation):
 *    g_num_l = sum_ij f(p_l - R_j q_i) Num_ij,
 *    g_den_l = sum_ij f(p_l - R_j q_i) den_j.
 *  mode 1, Eq. 2.5 then Eq. 2.10 (normalise each slice, then inverse distance
 *  weighting): W'_ij = Num_ij / den_j for den_j > 0 (other rotations skipped),
 *    g_num_l = sum_ij f W'_ij,  g_den_l = sum_ij f.
 *  grid_out_l = g_num_l / g_den_l where g_den_l > 0, else grid_prev_l.
 * g_num and g_den (N^3) are overwritten; grid_out may be NULL.
 */
void oracle_compress(int N, long n_rot, const double* quat, long n_pix, const double* q,
                     const double* Num, const double* den, int mode, const double* grid_prev,
                     double* g_num, double* g_den, double* grid_out) {
  long M = (long)N * N * N;
  memset(g_num, 0, sizeof(double) * (size_t)M);
  memset(g_den, 0, sizeof(double) * (size_t)M);
#pragma omp parallel
  {
    double* ln = calloc((size_t)M, sizeof(double));
    double* ld = calloc((size_t)M, sizeof(double));
#pragma omp for schedule(dynamic, 4)
    for (long j = 0; j < n_rot; j++) {
      if (mode == 1 && !(den[j] > 0)) continue;
      double R[9];
      oracle_quat_to_matrix(quat + 4 * j, R);
      for (long i = 0; i < n_pix; i++) {
        long idx[8];
        double wt[8];
        int nw = interp_weights(N, R, q + 3 * i, idx, wt);
        double v = (mode == 1) ? Num[j * n_pix + i] / den[j] : Num[j * n_pix + i];
        double dv = (mode == 1) ? 1.0 : den[j];
        for (int c = 0; c < nw; c++) {
          ln[idx[c]] += wt[c] * v;
          ld[idx[c]] += wt[c] * dv;
        }
      }
    }
#pragma omp critical
    {
      for (long l = 0; l < M; l++) {
        g_num[l] += ln[l];
        g_den[l] += ld[l];
      }
    }
    free(ln);
    free(ld);
  }
  if (grid_out)
    for (long l = 0; l < M; l++) grid_out[l] = g_den[l] > 0 ? g_num[l] / g_den[l] : grid_prev[l];
}

/*
 * Algorithm 2.1, one pass: W = e(WW) (Eq. 2.9), P = E(W) (Eq. 2.4),
 * [W, WW'] = cM(P) (Eqs. 2.11-2.12, or Eq. 2.5 + 2.10 for mode 1).
 * Optional outputs (NULL to skip): P[n_rot][n_data], lse[n_data].
 * Returns the log-likelihood sum_k lse_k (up to the dropped log K! terms),
 * or NAN on allocation failure.
 */
double oracle_iteration(int N, const double* grid, long n_rot, const double* quat,
                        const double* weight, long n_pix, const double* q, long n_data,
                        const double* K, double w_floor, int mode, double* grid_out,
                        double* P_out, double* lse_out) {
  long M = (long)N * N * N;
  double* W = malloc(sizeof(double) * (size_t)(n_rot * n_pix));
  double* S = malloc(sizeof(double) * (size_t)(n_rot * n_data));
  double* Num = malloc(sizeof(double) * (size_t)(n_rot * n_pix));
  double* den = malloc(sizeof(double) * (size_t)n_rot);
  double* gn = malloc(sizeof(double) * (size_t)M);
  double* gd = malloc(sizeof(double) * (size_t)M);
  double L = NAN;
  if (W && S && Num && den && gn && gd) {
    oracle_expand(N, grid, n_rot, quat, n_pix, q, w_floor, W);
    oracle_scores(n_rot, n_pix, n_data, W, weight, K, S);
    L = oracle_estep(n_rot, n_data, S, S, lse_out); /* S now holds P */
    if (P_out) memcpy(P_out, S, sizeof(double) * (size_t)(n_rot * n_data));
    oracle_mstep(n_rot, n_pix, n_data, S, K, Num, den);
    oracle_compress(N, n_rot, quat, n_pix, q, Num, den, mode, grid, gn, gd, grid_out);
  }
  free(W); free(S); free(Num); free(den); free(gn); free(gd);
  return L;
}

/* ------------------------------------------------------------------------ */
/* Gaussian noise model (Sec. 2.2, Eqs. 2.2-2.3, 2.5-2.6).                    */
/*                                                                           */
/* Reading (the paper's superscripts put phi^(n+1) = f(W^(n)) in the M-step   */
/* and phi^(n) in the E-step): the fluence of Eq. 2.6 is evaluated on the     */
/* model W^(n) of the current iteration and used in that iteration's E-step   */
/* and M-step. Eq. 2.6 is the least-squares optimum of Eq. 2.2 over phi for   */
/* fixed W, so each rotation is scored at its best-fitting fluence.           */
/* K/phi with phi infinite (sum_i W_ij K_ik = 0) or undefined (a frame with   */
/* no photons) is read as 0.                                                 */
/* ------------------------------------------------------------------------ */

/*
 * 1/phi_jk of Eq. 2.6: (sum_i W_ij K_ik) / (sum_i K_ik^2), 0 for an empty frame.
 * W[n_rot][n_pix], K[n_data][n_pix] -> inv_phi[n_rot][n_data].
 */
void oracle_fluence(long n_rot, long n_pix, long n_data, const double* W, const double* K,
                    double* inv_phi) {
#pragma omp parallel for schedule(dynamic, 4)
  for (long j = 0; j < n_rot; j++) {
    for (long k = 0; k < n_data; k++) {
      double kk = 0.0, wk = 0.0;
      for (long i = 0; i < n_pix; i++) {
        kk += K[k * n_pix + i] * K[k * n_pix + i];
        wk += W[j * n_pix + i] * K[k * n_pix + i];
      }
      inv_phi[j * n_data + k] = kk > 0.0 ? wk / kk : 0.0;
    }
  }
}

/*
 * Eqs. 2.2-2.3 with the log prior weight of Eq. 2.4:
 *   S_jk = -sum_i (K_ik / phi_jk - W_ij)^2 / (2 sigma^2) + log w_j.
 */
void oracle_scores_gauss(long n_rot, long n_pix, long n_data, const double* W,
                         const double* weight, const double* K, double sigma,
                         const double* inv_phi, double* S) {
  const double s2 = 2.0 * sigma * sigma;
#pragma omp parallel for schedule(dynamic, 4)
  for (long j = 0; j < n_rot; j++) {
    for (long k = 0; k < n_data; k++) {
      const double f = inv_phi[j * n_data + k];
      double q = 0.0;
      for (long i = 0; i < n_pix; i++) {
        const double r = K[k * n_pix + i] * f - W[j * n_pix + i];
        q += r * r;
      }
      S[j * n_data + k] = -q / s2 + log(weight[j]);
    }
  }
}

/*
 * M-step of the Gaussian model, Eq. 2.5 with the frames scaled by their
 * fluence, split into the numerator and denominator Eq. 2.12 consumes:
 *   Num_ij = sum_k P_jk K_ik / phi_jk,   den_j = sum_k P_jk.
 */
void oracle_mstep_gauss(long n_rot, long n_pix, long n_data, const double* P, const double* K,
                        const double* inv_phi, double* Num, double* den) {
#pragma omp parallel for schedule(dynamic, 4)
  for (long j = 0; j < n_rot; j++) {
    double d = 0.0;
    for (long k = 0; k < n_data; k++) d += P[j * n_data + k];
    den[j] = d;
    for (long i = 0; i < n_pix; i++) {
      double s = 0.0;
      for (long k = 0; k < n_data; k++)
        s += P[j * n_data + k] * K[k * n_pix + i] * inv_phi[j * n_data + k];
      Num[j * n_pix + i] = s;
    }
  }
}

/*
 * One pass of Algorithm 2.1 under the Gaussian model: expand (no floor: the
 * model has no logarithm), fluence, scores, E-step, M-step, compress.
 * Returns sum_k lse_k.
 */
double oracle_iteration_gauss(int N, const double* grid, long n_rot, const double* quat,
                              const double* weight, long n_pix, const double* q, long n_data,
                              const double* K, double sigma, int mode, double* grid_out,
                              double* P_out, double* lse_out) {
  long M = (long)N * N * N;
  double* W = malloc(sizeof(double) * (size_t)(n_rot * n_pix));
  double* F = malloc(sizeof(double) * (size_t)(n_rot * n_data));
  double* S = malloc(sizeof(double) * (size_t)(n_rot * n_data));
  double* Num = malloc(sizeof(double) * (size_t)(n_rot * n_pix));
  double* den = malloc(sizeof(double) * (size_t)n_rot);
  double* gn = malloc(sizeof(double) * (size_t)M);
  double* gd = malloc(sizeof(double) * (size_t)M);
  double L = NAN;
  if (W && F && S && Num && den && gn && gd) {
    oracle_expand(N, grid, n_rot, quat, n_pix, q, 0.0, W);
    oracle_fluence(n_rot, n_pix, n_data, W, K, F);
    oracle_scores_gauss(n_rot, n_pix, n_data, W, weight, K, sigma, F, S);
    L = oracle_estep(n_rot, n_data, S, S, lse_out); /* S now holds P */
    if (P_out) memcpy(P_out, S, sizeof(double) * (size_t)(n_rot * n_data));
    oracle_mstep_gauss(n_rot, n_pix, n_data, S, K, F, Num, den);
    oracle_compress(N, n_rot, quat, n_pix, q, Num, den, mode, grid, gn, gd, grid_out);
  }
  free(W); free(F); free(S); free(Num); free(den); free(gn); free(gd);
  return L;
}

/* ------------------------------------------------------------------------ */
/* Poisson model with a per-(j,k) fluence (the 160^3 workload's frames carry a  */
/* random intensity scale). Reading: the fluence is the Poisson maximum        */
/* likelihood phi_jk = N_k / sum_i W_ij (N_k = sum_i K_ik), evaluated on the    */
/* current model, so each rotation is scored at its best scale; the M-step     */
/* divides the frames by it as Eq. 2.11 does. The per-frame constant           */
/* N_k log N_k - N_k that appears with it is left out of the scores, like      */
/* log K!, since it cancels in Eq. 2.4. An empty frame has phi = 0.           */
/* ------------------------------------------------------------------------ */

/* 1/phi_jk = sum_i W_ij / N_k (0 for an empty frame) */
void oracle_fluence_poisson(long n_rot, long n_pix, long n_data, const double* W, const double* K,
                            double* inv_phi) {
#pragma omp parallel for schedule(dynamic, 4)
  for (long j = 0; j < n_rot; j++) {
    double sw = 0.0;
    for (long i = 0; i < n_pix; i++) sw += W[j * n_pix + i];
    for (long k = 0; k < n_data; k++) {
      double nk = 0.0;
      for (long i = 0; i < n_pix; i++) nk += K[k * n_pix + i];
      inv_phi[j * n_data + k] = nk > 0.0 ? sw / nk : 0.0;
    }
  }
}

/*
 * S_jk = sum_i (K_ik log(phi_jk W_ij) - phi_jk W_ij) + log w_j
 *        - (N_k log N_k - N_k)
 */
void oracle_scores_poisson_fluence(long n_rot, long n_pix, long n_data, const double* W,
                                   const double* weight, const double* K,
                                   const double* inv_phi, double* S) {
#pragma omp parallel for schedule(dynamic, 4)
  for (long j = 0; j < n_rot; j++) {
    for (long k = 0; k < n_data; k++) {
      const double f = inv_phi[j * n_data + k];
      double nk = 0.0;
      for (long i = 0; i < n_pix; i++) nk += K[k * n_pix + i];
      double s = 0.0;
      if (f > 0.0) {
        const double phi = 1.0 / f;
        for (long i = 0; i < n_pix; i++) {
          const double kk = K[k * n_pix + i];
          const double lam = phi * W[j * n_pix + i];
          s += (kk > 0.0 ? kk * log(lam) : 0.0) - lam;
        }
        s -= nk * log(nk) - nk;
      }
      S[j * n_data + k] = s + log(weight[j]);
    }
  }
}

/* One pass of Algorithm 2.1 under the Poisson-fluence model (M-step as in the
 * Gaussian one: Num_ij = sum_k P_jk K_ik / phi_jk, den_j = sum_k P_jk). */
double oracle_iteration_poisson_fluence(int N, const double* grid, long n_rot, const double* quat,
                                        const double* weight, long n_pix, const double* q,
                                        long n_data, const double* K, double w_floor, int mode,
                                        double* grid_out, double* P_out, double* lse_out) {
  long M = (long)N * N * N;
  double* W = malloc(sizeof(double) * (size_t)(n_rot * n_pix));
  double* F = malloc(sizeof(double) * (size_t)(n_rot * n_data));
  double* S = malloc(sizeof(double) * (size_t)(n_rot * n_data));
  double* Num = malloc(sizeof(double) * (size_t)(n_rot * n_pix));
  double* den = malloc(sizeof(double) * (size_t)n_rot);
  double* gn = malloc(sizeof(double) * (size_t)M);
  double* gd = malloc(sizeof(double) * (size_t)M);
  double L = NAN;
  if (W && F && S && Num && den && gn && gd) {
    oracle_expand(N, grid, n_rot, quat, n_pix, q, w_floor, W);
    oracle_fluence_poisson(n_rot, n_pix, n_data, W, K, F);
    oracle_scores_poisson_fluence(n_rot, n_pix, n_data, W, weight, K, F, S);
    L = oracle_estep(n_rot, n_data, S, S, lse_out); /* S now holds P */
    if (P_out) memcpy(P_out, S, sizeof(double) * (size_t)(n_rot * n_data));
    oracle_mstep_gauss(n_rot, n_pix, n_data, S, K, F, Num, den);
    oracle_compress(N, n_rot, quat, n_pix, q, Num, den, mode, grid, gn, gd, grid_out);
  }
  free(W); free(F); free(S); free(Num); free(den); free(gn); free(gd);
  return L;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
