/*
 * dash_oracle.c -- plain, slow, FP64 CPU oracle for the DASH 4D-hash
 * deformation path (arXiv 2507.19141, Sec. 4.2-4.3, Eqs. 7-11).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg load it (through oracle/__init__.py).  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * Every function evaluates the paper's definitions directly, one Gaussian
 * and one corner at a time, in double precision.  Inputs are the exact
 * values the GPU sees (FP32 coordinates, FP16/BF16-representable parameters
 * upcast exactly to double), so a difference between the two sides is the
 * GPU's arithmetic error only.
 *
 * Readings of the paper taken here (the paper is silent or garbled):
 *   - Eq. 7 prints N_l = floor(N_min * b); the level exponent is lost in the
 *     source.  Read as N_l = floor(N_min * b^l + 1e-9) (the multiresolution
 *     form the section cites), the 1e-9 guard making N_{L-1} = N_max exact.
 *   - Separate spatial (shared by x, y, z) and temporal progressions.
 *   - Hypervoxel corners are i0 and i0 + 1 per axis with
 *     i0 = min(floor(x * N_l), N_l - 1); x * N_l is the FP32 round-to-nearest
 *     product of the FP32 coordinate and N_l (exact in double, rounded once).
 *   - "mod T_l" with T a power of two is a mask; products wrap at 2^32.
 *   - A level whose (N_s+1)^3 (N_t+1) vertices fit in T is stored densely,
 *     row-major with x fastest; T_l is then that vertex count.  Each level
 *     starts at an entry offset rounded up to a multiple of 8.
 *   - The decoder is Linear-ReLU-Linear-ReLU-Linear; the three heads
 *     (dx: 3, dr: 4, ds: 3) are the row blocks of the last layer.
 *   - Smoothness term (Eq. 11): mean over the n dynamic Gaussians of the
 *     squared feature distance to a spatially and to a temporally perturbed
 *     copy, perturbed coordinates = clamp(fl32(clamp(x) + eps)).
 *   - Coordinates outside [0,1] are clamped; NaN maps to 0.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_LEVELS 32

/* Grid description shared by all oracle entry points (filled by orc_layout). */
typedef struct {
  int32_t L, F, log2_T, reserved;
  uint32_t primes[4];
  int32_t res_s[ORC_MAX_LEVELS];
  int32_t res_t[ORC_MAX_LEVELS];
  int32_t dense[ORC_MAX_LEVELS];
  int64_t size[ORC_MAX_LEVELS];       /* T_l: entries used by level l */
  int64_t offset[ORC_MAX_LEVELS + 1]; /* first entry of level l; offset[L] = total */
} orc_grid;

/* ---------------------------------------------------------------- Eq. 7 -- */
/* Level resolutions in a geometric progression between N_min and N_max. */
static int32_t orc_level_res(double nmin, double nmax, int L, int l) {
  if (L == 1) return (int32_t)floor(nmin + 1e-9);
  double b = exp((log(nmax) - log(nmin)) / (double)(L - 1));
  return (int32_t)floor(nmin * pow(b, (double)l) + 1e-9);
}

int orc_layout(orc_grid* g, int L, int F, int log2_T, double nmin_s, double nmax_s,
               double nmin_t, double nmax_t, const uint32_t* primes) {
  if (L < 1 || L > ORC_MAX_LEVELS || F < 1 || log2_T < 1 || log2_T > 30) return -1;
  if (!(nmin_s >= 1.0) || !(nmax_s >= nmin_s) || !(nmin_t >= 1.0) || !(nmax_t >= nmin_t)) return -1;
  memset(g, 0, sizeof(*g));
  g->L = L;
  g->F = F;
  g->log2_T = log2_T;
  for (int i = 0; i < 4; ++i) g->primes[i] = primes[i];
  const int64_t T = (int64_t)1 << log2_T;
  int64_t off = 0;
  for (int l = 0; l < L; ++l) {
    int32_t ns = orc_level_res(nmin_s, nmax_s, L, l);
    int32_t nt = orc_level_res(nmin_t, nmax_t, L, l);
    g->res_s[l] = ns;
    g->res_t[l] = nt;
    /* vertices per axis: N + 1 (coordinates 0..N) */
    int64_t verts = (int64_t)(ns + 1) * (ns + 1) * (ns + 1) * (nt + 1);
    g->dense[l] = verts <= T;
    g->size[l] = g->dense[l] ? verts : T;
    g->offset[l] = off;
    off += g->size[l];
    off = (off + 7) / 8 * 8; /* next level starts on a multiple of 8 entries */
  }
  g->offset[L] = off;
  return 0;
}

/* -------------------------------------------------- mask compaction ------ */
/* The dynamic set G_d is the list of Gaussians whose mask is set, in
 * ascending order (Sec. 4.1: Gaussians above the threshold are dynamic). */
int64_t orc_compact(const uint8_t* mask, int64_t n, int32_t* idx_out) {
  int64_t count = 0;
  for (int64_t i = 0; i < n; ++i)
    if (mask[i] != 0) idx_out[count++] = (int32_t)i;
  return count;
}

/* ------------------------------------------------------ coordinates ------ */
static float orc_clamp01(float v) {
  if (!(v >= 0.0f)) return 0.0f; /* negatives and NaN */
  if (v > 1.0f) return 1.0f;
  return v;
}

/* Loads the (x, y, z, t) of compact point i, clamped to [0,1]. */
static void orc_point(const float* x, const float* y, const float* z, const float* t,
                      int64_t t_stride, const int32_t* pidx, int64_t i, float p[4]) {
  int64_t j = pidx ? (int64_t)pidx[i] : i;
  p[0] = orc_clamp01(x[j]);
  p[1] = orc_clamp01(y[j]);
  p[2] = orc_clamp01(z[j]);
  p[3] = orc_clamp01(t_stride ? t[j * t_stride] : t[0]);
}

/* ------------------------------------------------- Eq. 8 and Eq. 9 ------- */
/* For level l: the 16 corner entries of the hypervoxel enclosing p and their
 * quadrilinear weights.  Corner b (bit d of b = upper corner along axis d,
 * axis order x, y, z, t) has index idx[b] (level-local) and weight w[b]. */
void orc_cell(const orc_grid* g, int l, const float p[4], uint32_t idx[16], double w[16]) {
  int64_t res[4] = {g->res_s[l], g->res_s[l], g->res_s[l], g->res_t[l]};
  int64_t i0[4];
  double frac[4];
  for (int d = 0; d < 4; ++d) {
    /* FP32 round-to-nearest product x * N_l, computed exactly then rounded once */
    double pos = (double)(float)((double)p[d] * (double)res[d]);
    int64_t c = (int64_t)floor(pos);
    if (c > res[d] - 1) c = res[d] - 1;
    i0[d] = c;
    frac[d] = pos - (double)c;
  }
  const uint32_t mask = (uint32_t)((((uint64_t)1) << g->log2_T) - 1);
  for (int b = 0; b < 16; ++b) {
    int64_t c[4];
    double wb = 1.0;
    for (int d = 0; d < 4; ++d) {
      int up = (b >> d) & 1;
      c[d] = i0[d] + up;
      wb *= up ? frac[d] : (1.0 - frac[d]);
    }
    w[b] = wb;
    if (g->dense[l]) {
      /* collision-free direct index, x fastest */
      int64_t R = res[0] + 1;
      idx[b] = (uint32_t)(c[0] + R * (c[1] + R * (c[2] + R * c[3])));
    } else {
      /* Eq. 8: XOR of coordinate * prime (mod 2^32), then mod T_l */
      uint64_t h = 0;
      for (int d = 0; d < 4; ++d) h ^= ((uint64_t)c[d] * (uint64_t)g->primes[d]) & 0xFFFFFFFFull;
      idx[b] = (uint32_t)h & mask;
    }
  }
}

/* Debug view of the encoder: all corner indices and weights.
 * idx_out: [n][L][16] level-local indices, w_out: [n][L][16]. */
void orc_corners(const orc_grid* g, const float* x, const float* y, const float* z,
                 const float* t, int64_t t_stride, const int32_t* pidx, int64_t n,
                 uint32_t* idx_out, double* w_out) {
  for (int64_t i = 0; i < n; ++i) {
    float p[4];
    orc_point(x, y, z, t, t_stride, pidx, i, p);
    for (int l = 0; l < g->L; ++l)
      orc_cell(g, l, p, idx_out + (i * g->L + l) * 16, w_out + (i * g->L + l) * 16);
  }
}

/* f_h = G_4D(p) for one point: per level the weighted sum of its 16 corner
 * feature vectors, levels concatenated (feature l*F + f). */
static void orc_encode_point(const orc_grid* g, const float p[4], const double* table,
                             double* f_h) {
  const int F = g->F;
  for (int l = 0; l < g->L; ++l) {
    uint32_t idx[16];
    double w[16];
    orc_cell(g, l, p, idx, w);
    for (int f = 0; f < F; ++f) {
      double acc = 0.0;
      for (int b = 0; b < 16; ++b) acc += w[b] * table[(g->offset[l] + idx[b]) * F + f];
      f_h[l * F + f] = acc;
    }
  }
}

/* Transpose of orc_encode_point: table_grad[entry][f] += w_b * df_h[l*F+f]. */
static void orc_encode_point_bwd(const orc_grid* g, const float p[4], const double* df_h,
                                 double* table_grad) {
  const int F = g->F;
  for (int l = 0; l < g->L; ++l) {
    uint32_t idx[16];
    double w[16];
    orc_cell(g, l, p, idx, w);
    for (int b = 0; b < 16; ++b)
      for (int f = 0; f < F; ++f)
        table_grad[(g->offset[l] + idx[b]) * F + f] += w[b] * df_h[l * F + f];
  }
}

/* Eq. 9 encoder: feat [n][L*F]. table: [offset[L]][F] entry-major. */
void orc_encode(const orc_grid* g, const float* x, const float* y, const float* z,
                const float* t, int64_t t_stride, const int32_t* pidx, int64_t n,
                const double* table, double* feat) {
  const int LF = g->L * g->F;
  for (int64_t i = 0; i < n; ++i) {
    float p[4];
    orc_point(x, y, z, t, t_stride, pidx, i, p);
    orc_encode_point(g, p, table, feat + i * LF);
  }
}

/* Gradient of the encoder w.r.t. its tables; accumulates into table_grad. */
void orc_encode_bwd(const orc_grid* g, const float* x, const float* y, const float* z,
                    const float* t, int64_t t_stride, const int32_t* pidx, int64_t n,
                    const double* dfeat, double* table_grad) {
  const int LF = g->L * g->F;
  for (int64_t i = 0; i < n; ++i) {
    float p[4];
    orc_point(x, y, z, t, t_stride, pidx, i, p);
    orc_encode_point_bwd(g, p, dfeat + i * LF, table_grad);
  }
}

/* Gradient of sum_i dfeat_i . G_4D(p_i) w.r.t. the coordinates (x, y, z, t)
 * of each compact point, through the quadrilinear weights of Eq. 9.  Within
 * a hypervoxel the encoding is multilinear in the continuous position
 * x * N_l, whose derivative is N_l (N_s for x, y, z; N_t for t); the
 * hypervoxel is the one orc_cell selects (lower corner min(floor, N - 1)), so
 * at a vertex the derivative is taken from the cell above it, at x = 1 from
 * the last cell.  The clamp to [0,1] passes the derivative for coordinates
 * in [0,1] and blocks it outside (and for NaN).  dcoord: SoA [4][n]; with a
 * broadcast t (t_stride 0) row 3 holds each point's share. */
void orc_encode_coord_grad(const orc_grid* g, const float* x, const float* y, const float* z,
                           const float* t, int64_t t_stride, const int32_t* pidx, int64_t n,
                           const double* table, const double* dfeat, double* dcoord) {
  const int F = g->F, LF = g->L * g->F;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t j = pidx ? (int64_t)pidx[i] : i;
    const float raw[4] = {x[j], y[j], z[j], t_stride ? t[j * t_stride] : t[0]};
    float p[4];
    orc_point(x, y, z, t, t_stride, pidx, i, p);
    double grad[4] = {0.0, 0.0, 0.0, 0.0};
    for (int l = 0; l < g->L; ++l) {
      const int64_t res[4] = {g->res_s[l], g->res_s[l], g->res_s[l], g->res_t[l]};
      double frac[4];
      for (int d = 0; d < 4; ++d) {
        double pos = (double)(float)((double)p[d] * (double)res[d]);
        int64_t c = (int64_t)floor(pos);
        if (c > res[d] - 1) c = res[d] - 1;
        frac[d] = pos - (double)c;
      }
      uint32_t idx[16];
      double w[16];
      orc_cell(g, l, p, idx, w);
      for (int b = 0; b < 16; ++b) {
        /* s_b = dfeat . (corner b's feature vector) */
        double s_b = 0.0;
        for (int f = 0; f < F; ++f) s_b += dfeat[i * LF + l * F + f] * table[(g->offset[l] + idx[b]) * F + f];
        for (int d = 0; d < 4; ++d) {
          /* d w_b / d pos_d: the factor of axis d becomes +1 (upper) or -1 */
          double dw = ((b >> d) & 1) ? 1.0 : -1.0;
          for (int e = 0; e < 4; ++e) {
            if (e == d) continue;
            dw *= ((b >> e) & 1) ? frac[e] : (1.0 - frac[e]);
          }
          grad[d] += s_b * dw * (double)res[d];
        }
      }
    }
    for (int d = 0; d < 4; ++d) {
      const int inside = raw[d] >= 0.0f && raw[d] <= 1.0f;
      dcoord[d * n + i] = inside ? grad[d] : 0.0;
    }
  }
}

/* ------------------------------------------------ hash collisions ------- */
typedef struct {
  int64_t vertex;  /* cx + R (cy + R (cz + R ct)), R = N_s + 1: one id per grid vertex */
  uint32_t entry;  /* the level-local table entry the vertex maps to */
} orc_touch;

static int orc_cmp_touch(const void* a, const void* b) {
  const orc_touch* u = (const orc_touch*)a;
  const orc_touch* v = (const orc_touch*)b;
  return u->vertex < v->vertex ? -1 : (u->vertex > v->vertex ? 1 : 0);
}

static int orc_cmp_u32(const void* a, const void* b) {
  const uint32_t u = *(const uint32_t*)a, v = *(const uint32_t*)b;
  return u < v ? -1 : (u > v ? 1 : 0);
}

/* Occupancy of each level by the n points (Sec. 4.2's collision argument):
 * stats[l*3 + 0] = V, the distinct grid vertices touched by the points'
 * hypervoxel corners; [1] = E, the distinct table entries those vertices map
 * to; [2] = C, the touched vertices whose entry is shared with at least one
 * other touched vertex (a collision).  Dense levels have E = V, C = 0.
 * Returns 0, or -1 if the memory for the sort cannot be had. */
int orc_collision_stats(const orc_grid* g, const float* x, const float* y, const float* z,
                        const float* t, int64_t t_stride, const int32_t* pidx, int64_t n,
                        int64_t* stats) {
  orc_touch* tv = (orc_touch*)malloc(sizeof(orc_touch) * (size_t)(n > 0 ? n * 16 : 1));
  uint32_t* ent = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n * 16 : 1));
  if (tv == NULL || ent == NULL) {
    free(tv);
    free(ent);
    return -1;
  }
  for (int l = 0; l < g->L; ++l) {
    const int64_t res[4] = {g->res_s[l], g->res_s[l], g->res_s[l], g->res_t[l]};
    const int64_t R = res[0] + 1;
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) {
      float p[4];
      orc_point(x, y, z, t, t_stride, pidx, i, p);
      uint32_t idx[16];
      double w[16];
      orc_cell(g, l, p, idx, w);
      int64_t i0[4];
      for (int d = 0; d < 4; ++d) {
        const double pos = (double)(float)((double)p[d] * (double)res[d]);
        int64_t c = (int64_t)floor(pos);
        i0[d] = c > res[d] - 1 ? res[d] - 1 : c;
      }
      for (int b = 0; b < 16; ++b) {
        int64_t c[4];
        for (int d = 0; d < 4; ++d) c[d] = i0[d] + ((b >> d) & 1);
        tv[m].vertex = c[0] + R * (c[1] + R * (c[2] + R * c[3]));
        tv[m].entry = idx[b];
        ++m;
      }
    }
    qsort(tv, (size_t)m, sizeof(orc_touch), orc_cmp_touch);
    int64_t V = 0;
    for (int64_t k = 0; k < m; ++k)
      if (k == 0 || tv[k].vertex != tv[k - 1].vertex) ent[V++] = tv[k].entry;
    qsort(ent, (size_t)V, sizeof(uint32_t), orc_cmp_u32);
    int64_t E = 0, C = 0;
    for (int64_t k = 0; k < V;) {
      int64_t r = k;
      while (r < V && ent[r] == ent[k]) ++r;
      ++E;
      if (r - k >= 2) C += r - k;
      k = r;
    }
    stats[l * 3 + 0] = V;
    stats[l * 3 + 1] = E;
    stats[l * 3 + 2] = C;
  }
  free(tv);
  free(ent);
  return 0;
}

/* ------------------------------------------------------ decoder MLP ------ */
/* phi_d followed by the heads phi_x, phi_r, phi_s (Eq. 9, Sec. 4.2):
 *   z1 = W1 f + b1, h1 = relu(z1); z2 = W2 h1 + b2, h2 = relu(z2);
 *   o = W3 h2 + b3.
 * params packs W1 [H][D], b1 [H], W2 [H][H], b2 [H], W3 [O][H], b3 [O]. */
typedef struct {
  const double *W1, *b1, *W2, *b2, *W3, *b3;
} orc_mlp_view;

static orc_mlp_view orc_mlp_split(const double* params, int D, int H, int O) {
  orc_mlp_view v;
  v.W1 = params;
  v.b1 = v.W1 + (size_t)H * D;
  v.W2 = v.b1 + H;
  v.b2 = v.W2 + (size_t)H * H;
  v.W3 = v.b2 + H;
  v.b3 = v.W3 + (size_t)O * H;
  return v;
}

int64_t orc_mlp_param_count(int D, int H, int O) {
  return (int64_t)H * D + H + (int64_t)H * H + H + (int64_t)O * H + O;
}

/* One point: z1, h1, z2, h2 (each H) and o (O). */
static void orc_mlp_point(const orc_mlp_view* m, int D, int H, int O, const double* f,
                          double* z1, double* h1, double* z2, double* h2, double* o) {
  for (int j = 0; j < H; ++j) {
    double a = m->b1[j];
    for (int k = 0; k < D; ++k) a += m->W1[(size_t)j * D + k] * f[k];
    z1[j] = a;
    h1[j] = a > 0.0 ? a : 0.0;
  }
  for (int j = 0; j < H; ++j) {
    double a = m->b2[j];
    for (int k = 0; k < H; ++k) a += m->W2[(size_t)j * H + k] * h1[k];
    z2[j] = a;
    h2[j] = a > 0.0 ? a : 0.0;
  }
  for (int j = 0; j < O; ++j) {
    double a = m->b3[j];
    for (int k = 0; k < H; ++k) a += m->W3[(size_t)j * H + k] * h2[k];
    o[j] = a;
  }
}

/* Back-propagation through one point.  dout: O values; accumulates into
 * param_grad (same packing as params) and writes df (D values). */
static void orc_mlp_point_bwd(const orc_mlp_view* m, int D, int H, int O, const double* f,
                              const double* z1, const double* h1, const double* z2,
                              const double* h2, const double* dout, double* df,
                              double* param_grad) {
  double dh2[256], dz2[256], dh1[256], dz1[256];
  orc_mlp_view gv = orc_mlp_split(param_grad, D, H, O);
  double *gW1 = (double*)gv.W1, *gb1 = (double*)gv.b1, *gW2 = (double*)gv.W2;
  double *gb2 = (double*)gv.b2, *gW3 = (double*)gv.W3, *gb3 = (double*)gv.b3;
  for (int j = 0; j < O; ++j) {
    gb3[j] += dout[j];
    for (int k = 0; k < H; ++k) gW3[(size_t)j * H + k] += dout[j] * h2[k];
  }
  for (int k = 0; k < H; ++k) {
    double a = 0.0;
    for (int j = 0; j < O; ++j) a += m->W3[(size_t)j * H + k] * dout[j];
    dh2[k] = a;
    dz2[k] = z2[k] > 0.0 ? a : 0.0;
  }
  for (int j = 0; j < H; ++j) {
    gb2[j] += dz2[j];
    for (int k = 0; k < H; ++k) gW2[(size_t)j * H + k] += dz2[j] * h1[k];
  }
  for (int k = 0; k < H; ++k) {
    double a = 0.0;
    for (int j = 0; j < H; ++j) a += m->W2[(size_t)j * H + k] * dz2[j];
    dh1[k] = a;
    dz1[k] = z1[k] > 0.0 ? a : 0.0;
  }
  for (int j = 0; j < H; ++j) {
    gb1[j] += dz1[j];
    for (int k = 0; k < D; ++k) gW1[(size_t)j * D + k] += dz1[j] * f[k];
  }
  for (int k = 0; k < D; ++k) {
    double a = 0.0;
    for (int j = 0; j < H; ++j) a += m->W1[(size_t)j * D + k] * dz1[j];
    df[k] = a;
  }
}

/* MLP forward on stored features: feat [n][D] -> out SoA [O][n]. */
int orc_mlp_fwd(int D, int H, int O, const double* params, const double* feat, int64_t n,
                double* out) {
  if (D > 256 || H > 256 || O > 256) return -1;
  orc_mlp_view m = orc_mlp_split(params, D, H, O);
  double z1[256], h1[256], z2[256], h2[256], o[256];
  for (int64_t i = 0; i < n; ++i) {
    orc_mlp_point(&m, D, H, O, feat + i * D, z1, h1, z2, h2, o);
    for (int j = 0; j < O; ++j) out[j * n + i] = o[j];
  }
  return 0;
}

/* MLP backward on stored features: dout SoA [O][n] -> dfeat [n][D] (written),
 * param_grad (accumulated). */
int orc_mlp_bwd(int D, int H, int O, const double* params, const double* feat, int64_t n,
                const double* dout, double* dfeat, double* param_grad) {
  if (D > 256 || H > 256 || O > 256) return -1;
  orc_mlp_view m = orc_mlp_split(params, D, H, O);
  double z1[256], h1[256], z2[256], h2[256], o[256], d[256];
  for (int64_t i = 0; i < n; ++i) {
    orc_mlp_point(&m, D, H, O, feat + i * D, z1, h1, z2, h2, o);
    for (int j = 0; j < O; ++j) d[j] = dout[j * n + i];
    orc_mlp_point_bwd(&m, D, H, O, feat + i * D, z1, h1, z2, h2, d, dfeat + i * D, param_grad);
  }
  return 0;
}

/* ------------------------------------------------ full deformation ------- */
/* Forward of the deformation field for the dynamic Gaussians:
 * delta SoA [O][n] (rows 0-2 dx, 3-6 dr, 7-9 ds for O = 10).
 * If attrs_in is given (SoA [O][n_all], float: x, r, s of all Gaussians),
 * Eq. 10 writes attrs_out[k][j] = attrs_in[k][j] + delta[k][i] at j = pidx[i]
 * (or i); rows of attrs_out for static Gaussians are left untouched. */
int orc_deform_fwd(const orc_grid* g, const float* x, const float* y, const float* z,
                   const float* t, int64_t t_stride, const int32_t* pidx, int64_t n,
                   const double* table, int H, int O, const double* params, double* delta,
                   const float* attrs_in, double* attrs_out, int64_t n_all) {
  const int D = g->L * g->F;
  if (D > 256 || H > 256 || O > 256) return -1;
  orc_mlp_view m = orc_mlp_split(params, D, H, O);
  double f[256], z1[256], h1[256], z2[256], h2[256], o[256];
  for (int64_t i = 0; i < n; ++i) {
    float p[4];
    orc_point(x, y, z, t, t_stride, pidx, i, p);
    orc_encode_point(g, p, table, f);
    orc_mlp_point(&m, D, H, O, f, z1, h1, z2, h2, o);
    for (int j = 0; j < O; ++j) delta[j * n + i] = o[j];
    if (attrs_in) {
      int64_t gi = pidx ? (int64_t)pidx[i] : i;
      for (int j = 0; j < O; ++j) attrs_out[j * n_all + gi] = (double)attrs_in[j * n_all + gi] + o[j];
    }
  }
  return 0;
}

/* Perturbed copy of a clamped point for the smoothness term. */
static void orc_perturb(const float p[4], const float e[4], float q[4]) {
  for (int d = 0; d < 4; ++d) q[d] = orc_clamp01((float)((double)p[d] + (double)e[d]));
}

/* Backward of the deformation field plus the smoothness term (Eq. 11).
 * ddelta SoA [O][n] is dLoss/d(delta).  Accumulates table_grad [offset[L]][F]
 * and param_grad.  If lambda_r != 0, adds lambda_r * L_r with
 *   L_r = (1/n) sum_i ( |f(p_i) - f(p_i + e_s)|^2 + |f(p_i) - f(p_i + e_t)|^2 ),
 *   e_s = (eps_s[0], eps_s[1], eps_s[2], 0), e_t = (0, 0, 0, eps_t),
 * and returns lambda_r * L_r (0 when lambda_r == 0). */
double orc_deform_bwd(const orc_grid* g, const float* x, const float* y, const float* z,
                      const float* t, int64_t t_stride, const int32_t* pidx, int64_t n,
                      const double* table, int H, int O, const double* params,
                      const double* ddelta, double* table_grad, double* param_grad,
                      float lambda_r, const float* eps_s, float eps_t) {
  const int D = g->L * g->F;
  if (D > 256 || H > 256 || O > 256) return NAN;
  orc_mlp_view m = orc_mlp_split(params, D, H, O);
  double f[256], z1[256], h1[256], z2[256], h2[256], o[256], d[256], df[256];
  double fq[256], dq[256];
  double loss = 0.0;
  const float e_s[4] = {eps_s ? eps_s[0] : 0.f, eps_s ? eps_s[1] : 0.f, eps_s ? eps_s[2] : 0.f, 0.f};
  const float e_t[4] = {0.f, 0.f, 0.f, eps_t};
  const double scale = 2.0 * (double)lambda_r / (double)(n > 0 ? n : 1);
  for (int64_t i = 0; i < n; ++i) {
    float p[4];
    orc_point(x, y, z, t, t_stride, pidx, i, p);
    orc_encode_point(g, p, table, f);
    orc_mlp_point(&m, D, H, O, f, z1, h1, z2, h2, o);
    for (int j = 0; j < O; ++j) d[j] = ddelta[j * n + i];
    orc_mlp_point_bwd(&m, D, H, O, f, z1, h1, z2, h2, d, df, param_grad);
    if (lambda_r != 0.0f) {
      const float* es[2] = {e_s, e_t};
      for (int e = 0; e < 2; ++e) {
        float q[4];
        orc_perturb(p, es[e], q);
        orc_encode_point(g, q, table, fq);
        double sq = 0.0;
        for (int k = 0; k < D; ++k) {
          double diff = f[k] - fq[k];
          sq += diff * diff;
          df[k] += scale * diff;  /* d/d f(p)   of lambda * |f(p) - f(q)|^2 / n */
          dq[k] = -scale * diff;  /* d/d f(q) */
        }
        loss += sq;
        orc_encode_point_bwd(g, q, dq, table_grad);
      }
    }
    orc_encode_point_bwd(g, p, df, table_grad);
  }
  return (double)lambda_r * loss / (double)(n > 0 ? n : 1);
}

/* Value of the smoothness term alone, lambda_r * L_r (Eq. 11), no gradients. */
double orc_smooth_loss(const orc_grid* g, const float* x, const float* y, const float* z,
                       const float* t, int64_t t_stride, const int32_t* pidx, int64_t n,
                       const double* table, float lambda_r, const float* eps_s, float eps_t) {
  const int D = g->L * g->F;
  if (D > 256) return NAN;
  double f[256], fq[256];
  double loss = 0.0;
  const float e_s[4] = {eps_s[0], eps_s[1], eps_s[2], 0.f};
  const float e_t[4] = {0.f, 0.f, 0.f, eps_t};
  const float* es[2] = {e_s, e_t};
  for (int64_t i = 0; i < n; ++i) {
    float p[4];
    orc_point(x, y, z, t, t_stride, pidx, i, p);
    orc_encode_point(g, p, table, f);
    for (int e = 0; e < 2; ++e) {
      float q[4];
      orc_perturb(p, es[e], q);
      orc_encode_point(g, q, table, fq);
      for (int k = 0; k < D; ++k) loss += (f[k] - fq[k]) * (f[k] - fq[k]);
    }
  }
  return (double)lambda_r * loss / (double)(n > 0 ? n : 1);
}

/* =========================================================================
 * Self-supervised decomposition (Sec. 4.1, Eqs. 3-4): the 3-D hash encoder
 * G_3D of the Gaussian positions, the MLPs phi_p and phi_l giving the
 * positional deformation dp, its norm, and the top-k % threshold tau.
 * Readings: G_3D uses the Eq. 7 progression of the spatial resolutions and
 * the Eq. 8 hash with the first three primes, (N+1)^3 vertices per dense
 * level; phi_p is one ReLU layer D -> H (f_3D), phi_l one linear layer
 * H -> 3 (dp).  tau is the (m+1)-th largest norm with m = floor(k N / 100);
 * Gaussians with norm > tau are dynamic, so ties at tau are static.
 * ========================================================================= */

/* 3-D level layout; the grid's res_t entries are 0 and `reserved` holds 3. */
int orc_layout3(orc_grid* g, int L, int F, int log2_T, double nmin, double nmax, const uint32_t* primes) {
  if (L < 1 || L > ORC_MAX_LEVELS || F < 1 || log2_T < 1 || log2_T > 30) return -1;
  if (!(nmin >= 1.0) || !(nmax >= nmin)) return -1;
  memset(g, 0, sizeof(*g));
  g->L = L;
  g->F = F;
  g->log2_T = log2_T;
  g->reserved = 3;
  for (int i = 0; i < 3; ++i) g->primes[i] = primes[i];
  const int64_t T = (int64_t)1 << log2_T;
  int64_t off = 0;
  for (int l = 0; l < L; ++l) {
    int32_t ns = orc_level_res(nmin, nmax, L, l);
    g->res_s[l] = ns;
    int64_t verts = (int64_t)(ns + 1) * (ns + 1) * (ns + 1);
    g->dense[l] = verts <= T;
    g->size[l] = g->dense[l] ? verts : T;
    g->offset[l] = off;
    off += g->size[l];
    off = (off + 7) / 8 * 8;
  }
  g->offset[L] = off;
  return 0;
}

/* The 8 corners of the level-l voxel around p (x, y, z) and their trilinear
 * weights; corner b: bit d set = upper corner along axis d. */
void orc_cell3(const orc_grid* g, int l, const float p[3], uint32_t idx[8], double w[8]) {
  const int64_t N = g->res_s[l];
  int64_t i0[3];
  double frac[3];
  for (int d = 0; d < 3; ++d) {
    double pos = (double)(float)((double)p[d] * (double)N);
    int64_t c = (int64_t)floor(pos);
    if (c > N - 1) c = N - 1;
    i0[d] = c;
    frac[d] = pos - (double)c;
  }
  const uint32_t mask = (uint32_t)((((uint64_t)1) << g->log2_T) - 1);
  for (int b = 0; b < 8; ++b) {
    int64_t c[3];
    double wb = 1.0;
    for (int d = 0; d < 3; ++d) {
      int up = (b >> d) & 1;
      c[d] = i0[d] + up;
      wb *= up ? frac[d] : (1.0 - frac[d]);
    }
    w[b] = wb;
    if (g->dense[l]) {
      int64_t R = N + 1;
      idx[b] = (uint32_t)(c[0] + R * (c[1] + R * c[2]));
    } else {
      uint64_t h = 0;
      for (int d = 0; d < 3; ++d) h ^= ((uint64_t)c[d] * (uint64_t)g->primes[d]) & 0xFFFFFFFFull;
      idx[b] = (uint32_t)h & mask;
    }
  }
}

/* G_3D(p) for points (x, y, z)[n] (clamped to [0,1]): feat [n][L*F]. */
void orc_encode3(const orc_grid* g, const float* x, const float* y, const float* z, int64_t n,
                 const double* table, double* feat) {
  const int F = g->F, LF = g->L * g->F;
  for (int64_t i = 0; i < n; ++i) {
    const float p[3] = {orc_clamp01(x[i]), orc_clamp01(y[i]), orc_clamp01(z[i])};
    for (int l = 0; l < g->L; ++l) {
      uint32_t idx[8];
      double w[8];
      orc_cell3(g, l, p, idx, w);
      for (int f = 0; f < F; ++f) {
        double acc = 0.0;
        for (int b = 0; b < 8; ++b) acc += w[b] * table[(g->offset[l] + idx[b]) * F + f];
        feat[i * LF + l * F + f] = acc;
      }
    }
  }
}

/* dp = phi_l(phi_p(G_3D(p))) and its Euclidean norm.  params packs
 * W1 [H][D], b1 [H], W2 [3][H], b2 [3]; dp SoA [3][n] (may be NULL). */
int orc_decomp_fwd(const orc_grid* g, const float* x, const float* y, const float* z, int64_t n,
                   const double* table, int H, const double* params, double* dp, double* norm) {
  const int D = g->L * g->F;
  if (D > 256 || H > 256) return -1;
  const double* W1 = params;
  const double* b1 = W1 + (size_t)H * D;
  const double* W2 = b1 + H;
  const double* b2 = W2 + (size_t)3 * H;
  double f[256], h[256];
  for (int64_t i = 0; i < n; ++i) {
    orc_encode3(g, x + i, y + i, z + i, 1, table, f);
    for (int j = 0; j < H; ++j) {
      double a = b1[j];
      for (int k = 0; k < D; ++k) a += W1[(size_t)j * D + k] * f[k];
      h[j] = a > 0.0 ? a : 0.0;
    }
    double s = 0.0;
    for (int j = 0; j < 3; ++j) {
      double a = b2[j];
      for (int k = 0; k < H; ++k) a += W2[(size_t)j * H + k] * h[k];
      if (dp) dp[j * n + i] = a;
      s += a * a;
    }
    norm[i] = sqrt(s);
  }
  return 0;
}

/* Backward of the decomposition (Eqs. 3-5): for the loss
 *   sum_i d_dp_i . dp_i + lambda_s * L_s,  L_s = (1/N_s) sum_{mask_i = 0} |dp_i|
 * accumulates the gradients of the G_3D tables (table_grad [offset[L]][F])
 * and of the packed W1, b1, W2, b2 (param_grad).  d_dp SoA [3][n] may be
 * NULL (no upstream term); mask may be NULL (no L_s term).  The L_s term is
 * lambda_s dp_i / (N_s |dp_i|) for static i with |dp_i| > 0.  Returns 0, or
 * -1 for unsupported widths. */
int orc_decomp_bwd(const orc_grid* g, const float* x, const float* y, const float* z, int64_t n,
                   const double* table, int H, const double* params, const double* d_dp, const uint8_t* mask,
                   double lambda_s, double* table_grad, double* param_grad) {
  const int D = g->L * g->F, F = g->F;
  if (D > 256 || H > 256) return -1;
  const double* W1 = params;
  const double* b1 = W1 + (size_t)H * D;
  const double* W2 = b1 + H;
  const double* b2 = W2 + (size_t)3 * H;
  double* gW1 = param_grad;
  double* gb1 = gW1 + (size_t)H * D;
  double* gW2 = gb1 + H;
  double* gb2 = gW2 + (size_t)3 * H;
  int64_t n_s = 0;
  if (mask != NULL)
    for (int64_t i = 0; i < n; ++i) n_s += mask[i] == 0;
  double f[256], z1[256], h[256], dz1[256], df[256];
  for (int64_t i = 0; i < n; ++i) {
    orc_encode3(g, x + i, y + i, z + i, 1, table, f);
    for (int j = 0; j < H; ++j) {
      double a = b1[j];
      for (int k = 0; k < D; ++k) a += W1[(size_t)j * D + k] * f[k];
      z1[j] = a;
      h[j] = a > 0.0 ? a : 0.0;
    }
    double dp[3], s = 0.0;
    for (int c = 0; c < 3; ++c) {
      double a = b2[c];
      for (int k = 0; k < H; ++k) a += W2[(size_t)c * H + k] * h[k];
      dp[c] = a;
      s += a * a;
    }
    const double norm = sqrt(s);
    double g_dp[3];
    for (int c = 0; c < 3; ++c) {
      g_dp[c] = d_dp != NULL ? d_dp[c * n + i] : 0.0;
      if (mask != NULL && mask[i] == 0 && norm > 0.0) g_dp[c] += lambda_s * dp[c] / ((double)n_s * norm);
    }
    for (int c = 0; c < 3; ++c) {
      gb2[c] += g_dp[c];
      for (int k = 0; k < H; ++k) gW2[(size_t)c * H + k] += g_dp[c] * h[k];
    }
    for (int j = 0; j < H; ++j) {
      double a = 0.0;
      for (int c = 0; c < 3; ++c) a += W2[(size_t)c * H + j] * g_dp[c];
      dz1[j] = z1[j] > 0.0 ? a : 0.0;
      gb1[j] += dz1[j];
      for (int k = 0; k < D; ++k) gW1[(size_t)j * D + k] += dz1[j] * f[k];
    }
    for (int k = 0; k < D; ++k) {
      double a = 0.0;
      for (int j = 0; j < H; ++j) a += W1[(size_t)j * D + k] * dz1[j];
      df[k] = a;
    }
    const float p[3] = {orc_clamp01(x[i]), orc_clamp01(y[i]), orc_clamp01(z[i])};
    for (int l = 0; l < g->L; ++l) {
      uint32_t idx[8];
      double w[8];
      orc_cell3(g, l, p, idx, w);
      for (int b = 0; b < 8; ++b)
        for (int ff = 0; ff < F; ++ff) table_grad[(g->offset[l] + idx[b]) * F + ff] += w[b] * df[l * F + ff];
    }
  }
  return 0;
}

/* Eq. 4: linear motion p(t) = p + t * dp of each Gaussian; p the coordinates
 * as given, t per Gaussian (t_stride 1) or one value for all (t_stride 0);
 * out SoA [3][n]. */
void orc_linear_motion(const float* x, const float* y, const float* z, const float* t, int64_t t_stride,
                       const double* dp, int64_t n, double* out) {
  for (int64_t i = 0; i < n; ++i) {
    const double p[3] = {x[i], y[i], z[i]};
    const double ti = t[i * t_stride];
    for (int d = 0; d < 3; ++d) out[d * n + i] = p[d] + ti * dp[d * n + i];
  }
}

/* Eq. 5: L_s = (1 / N_s) * sum of |dp| over the static Gaussians (mask 0),
 * N_s their number; 0 when every Gaussian is dynamic. */
double orc_static_loss(const double* norm, const uint8_t* mask, int64_t n) {
  double sum = 0.0;
  int64_t n_s = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (mask[i] == 0) {
      sum += norm[i];
      ++n_s;
    }
  }
  return n_s > 0 ? sum / (double)n_s : 0.0;
}

static int orc_cmp_desc(const void* a, const void* b) {
  const double x = *(const double*)a, y = *(const double*)b;
  return x < y ? 1 : (x > y ? -1 : 0);
}

/* Top-k % split: tau is the (m+1)-th largest of the n values (m = floor(k n /
 * 100)); mask[i] = values[i] > tau.  m = 0 marks nothing, m >= n marks
 * everything (tau = -1; the values are norms, never negative).  Returns tau. */
double orc_topk_mask(const double* values, int64_t n, double k_percent, uint8_t* mask) {
  int64_t m = (int64_t)floor(k_percent * (double)n / 100.0);
  if (m < 0) m = 0;
  double tau = -1.0;
  if (m < n && n > 0) {
    double* s = (double*)malloc(sizeof(double) * (size_t)n);
    memcpy(s, values, sizeof(double) * (size_t)n);
    qsort(s, (size_t)n, sizeof(double), orc_cmp_desc);
    tau = s[m];
    free(s);
  }
  for (int64_t i = 0; i < n; ++i) mask[i] = values[i] > tau;
  return tau;
}
