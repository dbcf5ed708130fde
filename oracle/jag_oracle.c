/*
 * jag_oracle.c -- plain, slow CPU oracle for JAG filtered nearest-neighbour
 * search (Joint Attribute Graphs, arXiv 2602.10258).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA path: the two meet only through the
 * seeded input arrays and the 16-byte filter record layout.
 *
 * What it computes (each function cites the passage it restates):
 *   - g(a,f) and dist_F(a,f) for label / range / subset / boolean filters
 *     (Sec. 2 "Filter Constraints"; Sec. 3.1 "Examples");
 *   - dist_A and the capped attribute distance dist_A(.,.;t) (Sec. 3.1,
 *     Sec. 3.2 "Capped attribute distance");
 *   - the lexicographic comparators D_F and D_A^t (Sec. 3.2 "Unified
 *     comparison rule"), with the point id as a final tie-break;
 *   - exact filtered k-NN by brute force (Sec. 2, "Filtered Nearest
 *     Neighbors Search"), i.e. the paper's Pre-Filtering baseline;
 *   - GreedySearch (Algorithm 1) in two forms: a literal one (L as a set with
 *     the "u not in L" test, V as a set, full re-ranking every iteration) and
 *     a direct one (seen set, rejection of keys beyond a full list's tail,
 *     sorted insertion) that also counts hops, first-seen neighbours and
 *     distance computations;
 *   - Query (Algorithm 2) = GreedySearch with D_F, plus the pre-filter route
 *     for the most selective queries;
 *   - Insert (Algorithm 3) and JointRobustPrune (Algorithm 4) with the two
 *     modifications of the implementation-details appendix (carried members,
 *     0.9 early exit), threshold quantiles from a 500-point sample per point,
 *     and a deterministic batch schedule (prefix doubling, graph frozen while
 *     a batch searches, back-edges grouped by target).
 *
 * Distances: the search uses squared L2 in fp32 in one fixed ("canonical")
 * rounding order, defined in orc_dist_canon(); an fp64 distance is also given.
 * Built with -ffp-contract=off so that no multiply-add is fused except the
 * explicit fmaf() calls, which are correctly rounded by the C standard.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* records shared by layout with the caller                                   */
/* ------------------------------------------------------------------------- */

enum { K_NONE = 0, K_LABEL = 1, K_RANGE_I32 = 2, K_RANGE_F32 = 3, K_SUBSET = 4, K_BOOL = 5 };

typedef struct {
  int32_t kind;
  int32_t aux_off;
  uint64_t payload; /* label | (lo,hi) int32 | (lo,hi) float32 | 64-bit mask */
} orc_filter;

/* Element formats of the stored base vectors. */
enum { FMT_F32 = 0, FMT_BF16 = 1, FMT_FP8 = 2 };

typedef struct {
  int64_t n, d;
  const float *x;          /* [n][d] fp32 base vectors                          */
  const int32_t *a_i32;    /* [n] label or integer attribute, or NULL           */
  const float *a_f32;      /* [n] float attribute, or NULL                      */
  const uint64_t *a_mask;  /* [n] bit-set attribute, or NULL                    */
  int32_t dist_a;          /* attribute the build compares: K_LABEL .. K_SUBSET */
  int32_t R;               /* out-degree bound                                  */
  int32_t *graph;          /* [n][R], -1 padded                                 */
  int64_t entry;           /* entry vertex s                                    */
  int32_t fmt;             /* storage format of the searched rows (FMT_*)       */
  int32_t qbytes;          /* bytes per stored row (multiple of 16)             */
  const uint8_t *xq;       /* [n][qbytes] stored rows (BF16 / FP8), or NULL     */
  const float *qscale;     /* [n] per-row scale of FP8 rows, or NULL            */
} orc_index;

/* ------------------------------------------------------------------------- */
/* small helpers                                                             */
/* ------------------------------------------------------------------------- */

static inline uint32_t f2u(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }
static inline float u2f(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }
static inline int popc64(uint64_t v) { int c = 0; while (v) { v &= v - 1; ++c; } return c; }
static inline int32_t lo32(uint64_t p) { return (int32_t)(uint32_t)(p & 0xFFFFFFFFu); }
static inline int32_t hi32(uint64_t p) { return (int32_t)(uint32_t)(p >> 32); }

/* ------------------------------------------------------------------------- */
/* vector distance                                                            */
/* ------------------------------------------------------------------------- */

/* Canonical fp32 squared L2 distance.  The row is cut into 16-byte chunks
 * (4 fp32 elements); chunk g feeds accumulator g mod 32; inside a chunk the
 * elements are taken in increasing order as acc = fmaf(t, t, acc) with
 * t = q_i - x_i rounded to fp32; the 32 accumulators are then combined by a
 * butterfly over offsets 16, 8, 4, 2, 1 (acc[l] + acc[l ^ o]) and the value
 * of accumulator 0 is the distance.  Missing tail elements count as zero,
 * which changes no partial sum. */
float orc_dist_canon(const float *q, const float *x, int64_t d) {
  float acc[32];
  for (int l = 0; l < 32; ++l) acc[l] = 0.0f;
  int64_t nch = (d + 3) / 4;
  for (int64_t g = 0; g < nch; ++g) {
    int lane = (int)(g % 32);
    for (int e = 0; e < 4; ++e) {
      int64_t i = g * 4 + e;
      if (i >= d) break;
      float t = q[i] - x[i];
      acc[lane] = fmaf(t, t, acc[lane]);
    }
  }
  for (int o = 16; o >= 1; o >>= 1) {
    float nxt[32];
    for (int l = 0; l < 32; ++l) nxt[l] = acc[l] + acc[l ^ o];
    memcpy(acc, nxt, sizeof(acc));
  }
  return acc[0];
}

/* Squared L2 distance in fp64, summed in index order. */
double orc_dist_f64(const float *q, const float *x, int64_t d) {
  double s = 0.0;
  for (int64_t i = 0; i < d; ++i) {
    double t = (double)q[i] - (double)x[i];
    s += t * t;
  }
  return s;
}

/* ------------------------------------------------------------------------- */
/* low-precision storage                                                      */
/* ------------------------------------------------------------------------- */

/* BF16 from fp32 by round to nearest, ties to even, on the upper 16 bits of
 * the fp32 encoding (finite inputs). */
uint16_t orc_bf16_encode(float x) {
  uint32_t b = f2u(x);
  uint32_t lsb = (b >> 16) & 1u;
  b += 0x7FFFu + lsb;
  return (uint16_t)(b >> 16);
}
float orc_bf16_decode(uint16_t h) { return u2f((uint32_t)h << 16); }

/* FP8 E4M3 (OCP 8-bit floating point, E4M3): sign, 4 exponent bits with bias
 * 7, 3 mantissa bits; exponent field 0 holds subnormals m/8 * 2^-6; the code
 * S.1111.111 is NaN and there is no infinity, so the largest finite magnitude
 * is 1.75 * 2^8 = 448. */
float orc_fp8_decode(uint8_t c) {
  int s = c >> 7, e = (c >> 3) & 15, m = c & 7;
  float v = e == 0 ? ldexpf((float)m / 8.0f, -6) : ldexpf(1.0f + (float)m / 8.0f, e - 7);
  return s ? -v : v;
}

/* Nearest finite E4M3 value to x, ties to the even code, magnitudes beyond the
 * largest finite value saturating to +-448: a binary search over the 127
 * non-negative finite codes, whose values increase with the code. */
uint8_t orc_fp8_encode(float x) {
  uint8_t sign = (f2u(x) >> 31) ? 0x80 : 0x00;
  double a = fabs((double)x);
  int lo = 0, hi = 126;                  /* codes 0..126 are finite, increasing */
  if (a >= (double)orc_fp8_decode(126)) return sign | 126;
  while (hi - lo > 1) {                  /* invariant: value(lo) <= a < value(hi) */
    int mid = (lo + hi) / 2;
    if ((double)orc_fp8_decode((uint8_t)mid) <= a) lo = mid; else hi = mid;
  }
  double dl = a - (double)orc_fp8_decode((uint8_t)lo), dh = (double)orc_fp8_decode((uint8_t)hi) - a;
  int c = dl < dh ? lo : (dh < dl ? hi : ((lo & 1) ? hi : lo));
  return sign | (uint8_t)c;
}

/* Bytes of one stored row: d elements rounded up to 16-byte chunks. */
int orc_row_bytes(int fmt, int64_t d) {
  int64_t eb = fmt == FMT_F32 ? 4 : (fmt == FMT_BF16 ? 2 : 1);
  return (int)((d * eb + 15) / 16 * 16);
}

/* Quantize n fp32 rows.  BF16: each element rounded, scale 1.  FP8: scale
 * s = max|x_i| / 448 (1 if the row is zero), codes of x_i / s (fp32
 * divisions).  out: [n][row_bytes], zero padded. */
void orc_quantize(const float *x, int64_t n, int64_t d, int fmt, uint8_t *out, float *scale) {
  int rb = orc_row_bytes(fmt, d);
  memset(out, 0, (size_t)(n * rb));
  for (int64_t i = 0; i < n; ++i) {
    const float *r = x + i * d;
    uint8_t *o = out + i * rb;
    if (fmt == FMT_BF16) {
      for (int64_t j = 0; j < d; ++j) { uint16_t h = orc_bf16_encode(r[j]); memcpy(o + 2 * j, &h, 2); }
      if (scale) scale[i] = 1.0f;
    } else {
      float mx = 0.0f;
      for (int64_t j = 0; j < d; ++j) if (fabsf(r[j]) > mx) mx = fabsf(r[j]);
      float s = mx > 0.0f ? mx / 448.0f : 1.0f;
      for (int64_t j = 0; j < d; ++j) o[j] = orc_fp8_encode(r[j] / s);
      scale[i] = s;
    }
  }
}

/* Element j of a stored row, as the distance uses it: s * value (fp32). */
static inline float stored_elem(const uint8_t *row, int fmt, float s, int64_t j) {
  if (fmt == FMT_BF16) { uint16_t h; memcpy(&h, row + 2 * j, 2); return orc_bf16_decode(h); }
  return s * orc_fp8_decode(row[j]);
}

/* Canonical squared distance to a stored BF16 / FP8 row: the order of
 * orc_dist_canon with 16-byte chunks of stored elements (8 BF16 or 16 FP8
 * elements), each element decoded and scaled before t = q_i - x_i. */
float orc_dist_canon_q(const float *q, const uint8_t *row, int fmt, float s, int64_t d) {
  float acc[32];
  for (int l = 0; l < 32; ++l) acc[l] = 0.0f;
  int64_t per = fmt == FMT_BF16 ? 8 : 16;
  int64_t nch = (d + per - 1) / per;
  for (int64_t g = 0; g < nch; ++g) {
    int lane = (int)(g % 32);
    for (int64_t e = 0; e < per; ++e) {
      int64_t i = g * per + e;
      if (i >= d) break;
      float t = q[i] - stored_elem(row, fmt, s, i);
      acc[lane] = fmaf(t, t, acc[lane]);
    }
  }
  for (int o = 16; o >= 1; o >>= 1) {
    float nxt[32];
    for (int l = 0; l < 32; ++l) nxt[l] = acc[l] + acc[l ^ o];
    memcpy(acc, nxt, sizeof(acc));
  }
  return acc[0];
}

/* Distance from a query to point u in the index's storage format. */
static inline float search_dist(const orc_index *ix, const float *q, int64_t u) {
  if (ix->fmt == FMT_F32 || !ix->xq) return orc_dist_canon(q, ix->x + u * ix->d, ix->d);
  return orc_dist_canon_q(q, ix->xq + u * ix->qbytes, ix->fmt, ix->qscale ? ix->qscale[u] : 1.0f, ix->d);
}

void orc_bf16_encode_batch(const float *x, int64_t n, uint16_t *out) {
  for (int64_t i = 0; i < n; ++i) out[i] = orc_bf16_encode(x[i]);
}
void orc_fp8_encode_batch(const float *x, int64_t n, uint8_t *out) {
  for (int64_t i = 0; i < n; ++i) out[i] = orc_fp8_encode(x[i]);
}
void orc_fp8_decode_batch(const uint8_t *c, int64_t n, float *out) {
  for (int64_t i = 0; i < n; ++i) out[i] = orc_fp8_decode(c[i]);
}

void orc_dist_canon_q_batch(const float *q, const uint8_t *rows, const float *scale, int fmt, int64_t n,
                            int64_t d, int64_t qbytes, float *out) {
  for (int64_t i = 0; i < n; ++i)
    out[i] = orc_dist_canon_q(q + i * d, rows + i * qbytes, fmt, scale ? scale[i] : 1.0f, d);
}

/* ------------------------------------------------------------------------- */
/* filters: g and dist_F (Sec. 2 "Filter Constraints", Sec. 3.1 "Examples")   */
/* ------------------------------------------------------------------------- */

/* Compress the bits of a selected by mask into the low bits, lowest first. */
static inline uint32_t gather_bits(uint64_t a, uint64_t mask) {
  uint32_t s = 0; int j = 0;
  for (int pos = 0; pos < 64; ++pos) {
    if ((mask >> pos) & 1u) {
      s |= (uint32_t)((a >> pos) & 1u) << j;
      ++j;
    }
  }
  return s;
}

static inline int tt_bit(const uint8_t *tt, uint32_t s) { return (tt[s >> 3] >> (s & 7)) & 1; }

/* Boolean filter distance table (Sec. 3.1, boolean example): for every
 * assignment s of the m involved variables, the least number of bit flips
 * that reaches an assignment where the predicate is true, i.e. a multi-source
 * breadth-first search on the m-cube from all satisfying assignments.  Only
 * involved variables can change the predicate, so flipping any other bit
 * never helps, and dist_F(a, f) = lut[gather_bits(a, vars)].  255 marks
 * "no satisfying assignment".  Returns 1 if the predicate is satisfiable. */
int orc_bool_lut(uint64_t vars, const uint8_t *tt, uint8_t *lut) {
  int m = popc64(vars);
  uint32_t S = 1u << m;
  uint32_t *queue = (uint32_t *)malloc(sizeof(uint32_t) * S);
  uint32_t head = 0, tail = 0;
  for (uint32_t s = 0; s < S; ++s) {
    if (tt_bit(tt, s)) { lut[s] = 0; queue[tail++] = s; }
    else lut[s] = 255;
  }
  int sat = tail > 0;
  while (head < tail) {
    uint32_t s = queue[head++];
    for (int j = 0; j < m; ++j) {
      uint32_t t = s ^ (1u << j);
      if (lut[t] == 255) { lut[t] = (uint8_t)(lut[s] + 1); queue[tail++] = t; }
    }
  }
  free(queue);
  return sat;
}

/* g(a, f): the matching predicate as written in Sec. 2. */
int orc_g(const orc_index *ix, int64_t i, const orc_filter *f, const uint8_t *aux) {
  switch (f->kind) {
    case K_NONE: return 1;
    case K_LABEL: return ix->a_i32[i] == lo32(f->payload);
    case K_RANGE_I32: {
      int32_t a = ix->a_i32[i];
      return lo32(f->payload) <= a && a <= hi32(f->payload);
    }
    case K_RANGE_F32: {
      float a = ix->a_f32[i];
      return u2f((uint32_t)lo32(f->payload)) <= a && a <= u2f((uint32_t)hi32(f->payload));
    }
    case K_SUBSET: return (f->payload & ix->a_mask[i]) == f->payload;
    case K_BOOL: return tt_bit(aux + f->aux_off, gather_bits(ix->a_mask[i], f->payload));
    default: return 0;
  }
}

/* dist_F(a, f) as an ordered 32-bit key (Sec. 3.1): label 1[a != f]; range
 * f_min - a below, a - f_max above, 0 inside (fp32 subtraction for float
 * attributes; the key is then the float's bit pattern, which orders like the
 * value for non-negative floats); subset |f \ a| = popcount(f & ~a); boolean
 * the table value above.  For the boolean kind lut is the per-query table. */
uint32_t orc_dist_F(const orc_index *ix, int64_t i, const orc_filter *f, const uint8_t *lut) {
  switch (f->kind) {
    case K_NONE: return 0;
    case K_LABEL: return ix->a_i32[i] != lo32(f->payload) ? 1u : 0u;
    case K_RANGE_I32: {
      int64_t a = ix->a_i32[i], lo = lo32(f->payload), hi = hi32(f->payload);
      if (a < lo) return (uint32_t)(lo - a);
      if (a > hi) return (uint32_t)(a - hi);
      return 0;
    }
    case K_RANGE_F32: {
      float a = ix->a_f32[i];
      float lo = u2f((uint32_t)lo32(f->payload)), hi = u2f((uint32_t)hi32(f->payload));
      if (a < lo) return f2u(lo - a);
      if (a > hi) return f2u(a - hi);
      if (lo <= a && a <= hi) return 0;
      return f2u(INFINITY); /* NaN bound: never satisfied */
    }
    case K_SUBSET: return (uint32_t)popc64(f->payload & ~ix->a_mask[i]);
    case K_BOOL: return lut[gather_bits(ix->a_mask[i], f->payload)];
    default: return f2u(INFINITY);
  }
}

/* ------------------------------------------------------------------------- */
/* attribute distance and its capped form (Sec. 3.1, Sec. 3.2)                */
/* ------------------------------------------------------------------------- */

uint32_t orc_dist_A(const orc_index *ix, int64_t i, int64_t j) {
  switch (ix->dist_a) {
    case K_LABEL: return ix->a_i32[i] != ix->a_i32[j] ? 1u : 0u;
    case K_RANGE_I32: {
      int64_t t = (int64_t)ix->a_i32[i] - (int64_t)ix->a_i32[j];
      return (uint32_t)(t < 0 ? -t : t);
    }
    case K_RANGE_F32: return f2u(fabsf(ix->a_f32[i] - ix->a_f32[j]));
    case K_SUBSET:
    case K_BOOL: return (uint32_t)popc64(ix->a_mask[i] ^ ix->a_mask[j]);
    default: return 0;
  }
}

/* dist_A(a1, a2; t) = max(dist_A - t, 0). */
uint32_t orc_capped(int32_t dist_a, uint32_t da, uint32_t t) {
  if (dist_a == K_RANGE_F32) {
    float fa = u2f(da), ft = u2f(t);
    return fa > ft ? f2u(fa - ft) : 0u;
  }
  return da > t ? da - t : 0u;
}

/* ------------------------------------------------------------------------- */
/* ordered keys: (first component, vector distance, id), lexicographic        */
/* ------------------------------------------------------------------------- */

typedef struct { uint32_t k1; float dist; int32_t id; int32_t expanded; } entry_t;

static inline int key_less(uint32_t ak, float ad, int32_t aid, uint32_t bk, float bd, int32_t bid) {
  if (ak != bk) return ak < bk;
  if (ad != bd) return ad < bd;
  return aid < bid;
}
static inline int entry_less(const entry_t *a, const entry_t *b) {
  return key_less(a->k1, a->dist, a->id, b->k1, b->dist, b->id);
}
static int entry_cmp(const void *pa, const void *pb) {
  const entry_t *a = (const entry_t *)pa, *b = (const entry_t *)pb;
  if (entry_less(a, b)) return -1;
  if (entry_less(b, a)) return 1;
  return 0;
}

/* A comparator D(x, .) for GreedySearch: first key of a point plus the
 * distance from the search point. */
typedef struct {
  const orc_index *ix;
  const float *xq;          /* search point's vector                           */
  /* query comparator D_F */
  const orc_filter *f;
  const uint8_t *lut;
  /* build comparator D_A^t */
  int64_t p;                /* base point being inserted, or -1 for a query    */
  uint32_t t;
  /* Weight-JAG build comparator D_A^w = w dist_A + dist (a scalar key) */
  int weighted;
  float w;
} comparator_t;

/* Vector distance of the comparator: the build compares fp32 rows; a query
 * compares the index's stored rows (fp32, or BF16 / FP8 before re-ranking). */
/* dist_A(a_i, a_j) as a real number: the float range distance is the fp32
 * value; the integer distances are converted to fp32 (round to nearest). */
float orc_dist_A_value(const orc_index *ix, int64_t i, int64_t j) {
  const uint32_t da = orc_dist_A(ix, i, j);
  return ix->dist_a == K_RANGE_F32 ? u2f(da) : (float)da;
}

static inline float cmp_dist(const comparator_t *c, int64_t u) {
  if (c->p >= 0) {
    const float d = orc_dist_canon(c->xq, c->ix->x + u * c->ix->d, c->ix->d);
    /* Weight-JAG: D_A^w(p, u) = w * dist_A(a_p, a_u) + dist(x_p, x_u), one fp32 fma */
    return c->weighted ? fmaf(c->w, orc_dist_A_value(c->ix, c->p, u), d) : d;
  }
  return search_dist(c->ix, c->xq, u);
}

static inline uint32_t first_key(const comparator_t *c, int64_t u) {
  if (c->p >= 0) return c->weighted ? 0u : orc_capped(c->ix->dist_a, orc_dist_A(c->ix, c->p, u), c->t);
  return orc_dist_F(c->ix, u, c->f, c->lut);
}

/* ------------------------------------------------------------------------- */
/* GreedySearch (Algorithm 1)                                                 */
/* ------------------------------------------------------------------------- */

typedef struct {
  int64_t hops;   /* expansions (iterations of the while loop)           */
  int64_t seen;   /* neighbours met for the first time                   */
  int64_t dc;     /* vector distance computations                        */
} counters_t;

/* Direct form.  L is kept sorted by (first key, distance, id) and holds at
 * most ls entries.  A neighbour met before is skipped: if it is still in L it
 * must not be added twice, and if it was dropped it cannot re-enter, since a
 * full list's last key only decreases.  For the same reason a new neighbour
 * whose first key already exceeds a full list's last entry is rejected
 * without its vector distance.  On return L[0..*len) holds the final list;
 * visited[] receives the expanded vertices in expansion order (if non-NULL,
 * up to vcap of them) with *nvis their number. */
static void greedy_direct(const comparator_t *c, int ls, entry_t *L, int *len,
                          uint8_t *seen, int64_t *touched, int64_t *ntouched,
                          entry_t *visited, int64_t vcap, int64_t *nvis, counters_t *cnt) {
  const orc_index *ix = c->ix;
  int n = 0;
  int64_t nt = 0, nv = 0;
  int64_t s = ix->entry;
  L[0].k1 = first_key(c, s);
  L[0].dist = cmp_dist(c, s);
  L[0].id = (int32_t)s;
  L[0].expanded = 0;
  n = 1;
  seen[s] = 1; touched[nt++] = s;
  cnt->dc += 1;
  for (;;) {
    int sel = -1;
    for (int i = 0; i < n; ++i) if (!L[i].expanded) { sel = i; break; }
    if (sel < 0) break;
    L[sel].expanded = 1;
    cnt->hops += 1;
    int64_t p = L[sel].id;
    if (visited && nv < vcap) visited[nv] = L[sel];
    nv++;
    const int32_t *row = ix->graph + p * ix->R;
    for (int r = 0; r < ix->R; ++r) {
      int64_t u = row[r];
      if (u < 0) continue;
      if (seen[u]) continue;
      seen[u] = 1; touched[nt++] = u;
      cnt->seen += 1;
      uint32_t k1 = first_key(c, u);
      if (n == ls && k1 > L[n - 1].k1) continue;
      float du = cmp_dist(c, u);
      cnt->dc += 1;
      if (n == ls && !key_less(k1, du, (int32_t)u, L[n - 1].k1, L[n - 1].dist, L[n - 1].id)) continue;
      int pos = n < ls ? n : ls - 1;
      while (pos > 0 && key_less(k1, du, (int32_t)u, L[pos - 1].k1, L[pos - 1].dist, L[pos - 1].id)) {
        L[pos] = L[pos - 1];
        --pos;
      }
      L[pos].k1 = k1; L[pos].dist = du; L[pos].id = (int32_t)u; L[pos].expanded = 0;
      if (n < ls) ++n;
    }
  }
  *len = n;
  if (nvis) *nvis = nv;
  *ntouched = nt;
}

/* ------------------------------------------------------------------------- */
/* learned beam width and stop hop (a search policy on top of Algorithm 1)   */
/* ------------------------------------------------------------------------- */

enum { POL_PLAIN = 0, POL_LEARNED = 1, POL_FORCED = 2 };
#define NFEAT 12
#define HID 64

typedef struct {
  int32_t mode;             /* POL_*                                            */
  int32_t h0;               /* hops at the fixed beam before the decision       */
  const uint16_t *w_bf16;   /* W1 [64][12], W2 [64][64], W3 [nl+1][64], BF16    */
  const float *b_f32;       /* b1 [64], b2 [64], b3 [nl+1]                       */
  float tau;                /* least margin between the two largest beam logits */
  float stop_scale;         /* stop hop = rint(output * stop_scale); <= 0: none */
  int32_t n_ladder;         /* beam classes (nl <= 16)                          */
  int32_t ladder[16];       /* beam of each class                               */
  const int32_t *forced;    /* [nq][2] (beam, stop) for POL_FORCED; beams are
                               taken into [k, ls]                              */
  float *features;          /* [nq][12] out, or NULL                            */
  int32_t *decisions;       /* [nq][4] out: beam, stop, last top-k change, learned */
} orc_policy;

/* Network output for feature vector x: two hidden layers of 64 ReLU units and
 * nl + 1 outputs; weights in BF16, fp32 accumulation acc = fma(w, x_i, acc)
 * over the inputs in order, starting from the bias. */
void orc_mlp_infer(const orc_policy *pol, const float *x, float *out) {
  const uint16_t *w1 = pol->w_bf16, *w2 = w1 + HID * NFEAT, *w3 = w2 + HID * HID;
  const float *b1 = pol->b_f32, *b2 = b1 + HID, *b3 = b2 + HID;
  float h1[HID], h2[HID];
  for (int j = 0; j < HID; ++j) {
    float acc = b1[j];
    for (int i = 0; i < NFEAT; ++i) acc = fmaf(orc_bf16_decode(w1[j * NFEAT + i]), x[i], acc);
    h1[j] = acc > 0.0f ? acc : 0.0f;
  }
  for (int j = 0; j < HID; ++j) {
    float acc = b2[j];
    for (int i = 0; i < HID; ++i) acc = fmaf(orc_bf16_decode(w2[j * HID + i]), h1[i], acc);
    h2[j] = acc > 0.0f ? acc : 0.0f;
  }
  for (int o = 0; o <= pol->n_ladder; ++o) {
    float acc = b3[o];
    for (int i = 0; i < HID; ++i) acc = fmaf(orc_bf16_decode(w3[o * HID + i]), h2[i], acc);
    out[o] = acc;
  }
}

/* Monotone stand-in for log2 of a non-negative float from its encoding:
 * (bits >> 16) / 128 - 127, exact in fp32. */
static inline float flog(float x) { return (float)(f2u(x) >> 16) * 0.0078125f - 127.0f; }

/* Features of the search state after the decision hop: selectivity bucket,
 * filter kind, fraction of L passing, distances of the best, k-th passing
 * (or last) and last entries, answers found, expanded prefix of L. */
static void policy_features(const entry_t *L, int n, int k, int64_t est, int kind, float *f) {
  int np = 0;
  while (np < n && L[np].k1 == 0) ++np;
  int fu = n;
  for (int i = 0; i < n; ++i) if (!L[i].expanded) { fu = i; break; }
  uint32_t e = est > 0x7FFFFFFE ? 0x7FFFFFFFu : (uint32_t)est + 1u;
  f[0] = (float)(32 - __builtin_clz(e)) * 0.05f;
  for (int i = 0; i < 5; ++i) f[1 + i] = (kind == i + 1) ? 1.0f : 0.0f;
  f[6] = (float)np / (float)n;
  f[7] = flog(L[0].dist) * 0.125f;
  f[8] = flog(np > 0 ? L[(np < k ? np : k) - 1].dist : L[n - 1].dist) * 0.125f;
  f[9] = (float)(np < k ? np : k) / (float)k;
  f[10] = (float)fu / (float)n;
  f[11] = flog(L[n - 1].dist) * 0.125f;
}

/* The same features of a list state given entry by entry (first keys,
 * distances, expanded flags of L[0..n), in the search's order), so that the
 * tests can pin them on hand-worked lists. */
void orc_policy_features(const uint32_t *k1, const float *dist, const uint8_t *expanded, int n, int k,
                         int64_t est, int kind, float *f) {
  entry_t *L = (entry_t *)malloc(sizeof(entry_t) * (size_t)(n > 0 ? n : 1));
  for (int i = 0; i < n; ++i) {
    L[i].k1 = k1[i];
    L[i].dist = dist[i];
    L[i].id = i;
    L[i].expanded = expanded[i] ? 1 : 0;
  }
  policy_features(L, n, k, est, kind, f);
  free(L);
}

/* Beam and stop hop from the network: the largest beam logit wins (lowest
 * class on a tie); if it leads the runner-up by less than tau the fixed beam
 * is kept and no stop hop is set. */
static void policy_decide(const orc_policy *pol, const float *f, int fixed, int h0, int *beam, int *stop,
                          int *learned) {
  float out[17];
  orc_mlp_infer(pol, f, out);
  int nl = pol->n_ladder, c = 0;
  for (int i = 1; i < nl; ++i) if (out[i] > out[c]) c = i;
  float second = -INFINITY;
  for (int i = 0; i < nl; ++i) if (i != c && out[i] > second) second = out[i];
  float margin = out[c] - second;
  if (!(margin >= pol->tau)) { *beam = fixed; *stop = 0; *learned = 0; return; }
  float r = rintf(out[nl] * pol->stop_scale);
  int st;
  if (!(pol->stop_scale > 0.0f)) st = 0;          /* no stop hop */
  else if (!(r == r) || r >= 65535.0f) st = 65535;
  else if (r <= (float)h0) st = h0;
  else st = (int)r;
  *beam = pol->ladder[c] < fixed ? pol->ladder[c] : fixed;
  *stop = st; *learned = 1;
}

/* The direct search (as greedy_direct) run in two phases: h0 hops at the
 * fixed beam ls0, then the beam and stop hop of the policy (L is cut to the
 * new beam if longer; the search also ends once stop hops are done).  The new
 * beam never exceeds ls0: the search only ever shrinks L, so a point it has
 * set aside can never qualify again.  Tracks the last hop that inserted an
 * entry among the first k. */
static void greedy_policy(const comparator_t *c, int ls0, int k, const orc_policy *pol, const int32_t *forced_q,
                          int64_t est, int kind, entry_t *L, int *len, uint8_t *seen, int64_t *touched,
                          int64_t *ntouched, counters_t *cnt, float *feat, int32_t *dec) {
  const orc_index *ix = c->ix;
  int n = 0, ls = ls0;
  int64_t nt = 0;
  int stop = 0, learned = 0, decided = 0;
  int64_t last_change = 0;
  int64_t s = ix->entry;
  L[0].k1 = first_key(c, s);
  L[0].dist = cmp_dist(c, s);
  L[0].id = (int32_t)s;
  L[0].expanded = 0;
  n = 1;
  seen[s] = 1; touched[nt++] = s;
  cnt->dc += 1;
  if (feat) for (int i = 0; i < NFEAT; ++i) feat[i] = 0.0f;
  for (;;) {
    if (stop > 0 && cnt->hops >= stop) break;
    int sel = -1;
    for (int i = 0; i < n; ++i) if (!L[i].expanded) { sel = i; break; }
    if (sel < 0) break;
    L[sel].expanded = 1;
    cnt->hops += 1;
    int64_t p = L[sel].id;
    const int32_t *row = ix->graph + p * ix->R;
    for (int r = 0; r < ix->R; ++r) {
      int64_t u = row[r];
      if (u < 0) continue;
      if (seen[u]) continue;
      seen[u] = 1; touched[nt++] = u;
      cnt->seen += 1;
      uint32_t k1 = first_key(c, u);
      if (n == ls && k1 > L[n - 1].k1) continue;
      float du = cmp_dist(c, u);
      cnt->dc += 1;
      if (n == ls && !key_less(k1, du, (int32_t)u, L[n - 1].k1, L[n - 1].dist, L[n - 1].id)) continue;
      int pos = n < ls ? n : ls - 1;
      while (pos > 0 && key_less(k1, du, (int32_t)u, L[pos - 1].k1, L[pos - 1].dist, L[pos - 1].id)) {
        L[pos] = L[pos - 1];
        --pos;
      }
      L[pos].k1 = k1; L[pos].dist = du; L[pos].id = (int32_t)u; L[pos].expanded = 0;
      if (n < ls) ++n;
      if (pos < k) last_change = cnt->hops;
    }
    if (!decided && pol->mode != POL_PLAIN && cnt->hops == pol->h0) {
      float f[NFEAT];
      policy_features(L, n, k, est, kind, f);
      if (feat) memcpy(feat, f, sizeof(f));
      int beam = ls;
      if (pol->mode == POL_LEARNED) {
        policy_decide(pol, f, ls0, pol->h0, &beam, &stop, &learned);
      } else {
        beam = forced_q[0] > 0 ? (forced_q[0] < k ? k : forced_q[0] > ls0 ? ls0 : forced_q[0]) : ls0;
        stop = forced_q[1] > 0 ? (forced_q[1] < pol->h0 ? pol->h0 : forced_q[1]) : 0;
        learned = forced_q[0] > 0;
      }
      ls = beam;
      if (n > ls) n = ls;
      decided = 1;
    }
  }
  *len = n;
  *ntouched = nt;
  if (dec) { dec[0] = ls; dec[1] = stop; dec[2] = (int32_t)last_change; dec[3] = learned; }
}

/* Literal form, for checking the direct one: L and V are plain sets; each
 * iteration takes the best unexpanded member of L, adds every out-neighbour
 * not already in L, and if L grew beyond ls re-ranks it and keeps the best
 * ls.  Returns the top k of V ranked by the comparator in out[0..*nout). */
static void greedy_literal(const comparator_t *c, int ls, int k, entry_t *out, int *nout,
                           int64_t *hops) {
  const orc_index *ix = c->ix;
  int64_t cap = (int64_t)ls + ix->R + 1;
  entry_t *L = (entry_t *)malloc(sizeof(entry_t) * cap);
  int64_t vcap = 1024, nv = 0;
  entry_t *V = (entry_t *)malloc(sizeof(entry_t) * vcap);
  int64_t n = 0;
  int64_t s = ix->entry;
  L[n].k1 = first_key(c, s);
  L[n].dist = cmp_dist(c, s);
  L[n].id = (int32_t)s; L[n].expanded = 0; n++;
  *hops = 0;
  for (;;) {
    /* p <- argmin over L \ V */
    int64_t best = -1;
    for (int64_t i = 0; i < n; ++i) {
      int inV = 0;
      for (int64_t j = 0; j < nv; ++j) if (V[j].id == L[i].id) { inV = 1; break; }
      if (inV) continue;
      if (best < 0 || entry_less(&L[i], &L[best])) best = i;
    }
    if (best < 0) break;
    if (nv == vcap) { vcap *= 2; V = (entry_t *)realloc(V, sizeof(entry_t) * vcap); }
    V[nv++] = L[best];
    *hops += 1;
    int64_t p = L[best].id;
    for (int r = 0; r < ix->R; ++r) {
      int64_t u = ix->graph[p * ix->R + r];
      if (u < 0) continue;
      int inL = 0;
      for (int64_t i = 0; i < n; ++i) if (L[i].id == u) { inL = 1; break; }
      if (inL) continue;
      L[n].k1 = first_key(c, u);
      L[n].dist = cmp_dist(c, u);
      L[n].id = (int32_t)u; L[n].expanded = 0; n++;
    }
    if (n > ls) {
      qsort(L, (size_t)n, sizeof(entry_t), entry_cmp);
      n = ls;
    }
  }
  qsort(V, (size_t)nv, sizeof(entry_t), entry_cmp);
  int m = (int)(nv < k ? nv : k);
  for (int i = 0; i < m; ++i) out[i] = V[i];
  *nout = m;
  free(L); free(V);
}

/* ------------------------------------------------------------------------- */
/* threads                                                                    */
/* ------------------------------------------------------------------------- */

typedef void (*range_fn)(void *ctx, int64_t lo, int64_t hi, int tid);
typedef struct { range_fn fn; void *ctx; int64_t lo, hi; int tid; } thr_arg;
static void *thr_main(void *a) {
  thr_arg *t = (thr_arg *)a;
  t->fn(t->ctx, t->lo, t->hi, t->tid);
  return NULL;
}
/* Run fn over [0, n) split into nthreads contiguous ranges. */
static void parallel_for(int64_t n, int nthreads, range_fn fn, void *ctx) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if (n < nthreads) nthreads = (int)(n > 0 ? n : 1);
  if (nthreads == 1) { fn(ctx, 0, n, 0); return; }
  pthread_t th[256];
  thr_arg args[256];
  for (int i = 0; i < nthreads; ++i) {
    args[i].fn = fn; args[i].ctx = ctx; args[i].tid = i;
    args[i].lo = n * i / nthreads; args[i].hi = n * (i + 1) / nthreads;
    pthread_create(&th[i], NULL, thr_main, &args[i]);
  }
  for (int i = 0; i < nthreads; ++i) pthread_join(th[i], NULL);
}

/* ------------------------------------------------------------------------- */
/* per-query boolean tables                                                  */
/* ------------------------------------------------------------------------- */

static uint8_t *query_lut(const orc_filter *f, const uint8_t *aux) {
  if (f->kind != K_BOOL) return NULL;
  int m = popc64(f->payload);
  uint8_t *lut = (uint8_t *)malloc((size_t)1 << m);
  orc_bool_lut(f->payload, aux + f->aux_off, lut);
  return lut;
}

/* ------------------------------------------------------------------------- */
/* exact filtered k-NN (Sec. 2; the Pre-Filtering baseline)                   */
/* ------------------------------------------------------------------------- */

typedef struct {
  const orc_index *ix;
  const float *q; const orc_filter *f; const uint8_t *aux;
  int k;
  int32_t *ids; float *d32; double *d64; int64_t *npass;
} bf_ctx;

/* Top k of {p : g(a_p, f_q) = 1} by (canonical fp32 distance, id). */
static void bf_one(const bf_ctx *c, int64_t qi) {
  const orc_index *ix = c->ix;
  const float *xq = c->q + qi * ix->d;
  const orc_filter *f = &c->f[qi];
  int k = c->k;
  float *bd = c->d32 + qi * k;
  int32_t *bi = c->ids + qi * k;
  int m = 0;
  int64_t np = 0;
  for (int64_t p = 0; p < ix->n; ++p) {
    if (!orc_g(ix, p, f, c->aux)) continue;
    np++;
    float dp = orc_dist_canon(xq, ix->x + p * ix->d, ix->d);
    if (m == k && !key_less(0, dp, (int32_t)p, 0, bd[m - 1], bi[m - 1])) continue;
    int pos = m < k ? m : k - 1;
    while (pos > 0 && key_less(0, dp, (int32_t)p, 0, bd[pos - 1], bi[pos - 1])) {
      bd[pos] = bd[pos - 1]; bi[pos] = bi[pos - 1]; --pos;
    }
    bd[pos] = dp; bi[pos] = (int32_t)p;
    if (m < k) ++m;
  }
  for (int i = 0; i < k; ++i) {
    if (i < m) {
      if (c->d64) c->d64[qi * k + i] = orc_dist_f64(xq, ix->x + (int64_t)bi[i] * ix->d, ix->d);
    } else {
      bi[i] = -1; bd[i] = INFINITY;
      if (c->d64) c->d64[qi * k + i] = INFINITY;
    }
  }
  if (c->npass) c->npass[qi] = np;
}

static void bf_range(void *ctx, int64_t lo, int64_t hi, int tid) {
  (void)tid;
  for (int64_t q = lo; q < hi; ++q) bf_one((const bf_ctx *)ctx, q);
}

void orc_brute_force(const orc_index *ix, const float *q, const orc_filter *f, const uint8_t *aux,
                     int64_t nq, int k, int32_t *ids, float *d32, double *d64, int64_t *npass,
                     int nthreads) {
  bf_ctx c = {ix, q, f, aux, k, ids, d32, d64, npass};
  parallel_for(nq, nthreads, bf_range, &c);
}

/* ------------------------------------------------------------------------- */
/* routing of the most selective queries to the exact scan                    */
/* ------------------------------------------------------------------------- */

/* Number of points passing the filter, exactly. */
int64_t orc_count_passing(const orc_index *ix, const orc_filter *f, const uint8_t *aux) {
  int64_t c = 0;
  for (int64_t p = 0; p < ix->n; ++p) c += orc_g(ix, p, f, aux);
  return c;
}

/* Route rule: a query goes to the exact scan when its estimated number of
 * passing points is below s0.  Label and range filters are counted exactly;
 * subset and boolean filters are estimated on the fixed sample of
 * S = min(4096, N) points with ids floor(j N / S), j = 0..S-1, and routed
 * when (sample hits) * N < s0 * S.  A routed query whose exact count
 * exceeds the scan capacity scan_cap goes back to the graph search.
 * Returns 1 for the scan. */
int orc_route(const orc_index *ix, const orc_filter *f, const uint8_t *aux, int64_t s0,
              int64_t scan_cap, int64_t *exact_count) {
  int64_t exact = orc_count_passing(ix, f, aux);
  if (exact_count) *exact_count = exact;
  if (s0 <= 0) return 0;
  int route;
  switch (f->kind) {
    case K_LABEL: case K_RANGE_I32: case K_RANGE_F32:
      route = exact < s0;
      break;
    case K_SUBSET: case K_BOOL: {
      int64_t S = ix->n < 4096 ? ix->n : 4096;
      int64_t hits = 0;
      for (int64_t j = 0; j < S; ++j) hits += orc_g(ix, j * ix->n / S, f, aux);
      route = hits * ix->n < s0 * S;
      break;
    }
    default: route = 0;
  }
  if (route && exact > scan_cap) route = 0;
  return route;
}

/* ------------------------------------------------------------------------- */
/* Query (Algorithm 2) over a batch                                           */
/* ------------------------------------------------------------------------- */

typedef struct {
  const orc_index *ix;
  const float *q; const orc_filter *f; const uint8_t *aux;
  int k, ls, literal;
  int64_t s0, scan_cap;
  int32_t *ids; float *dist; int64_t *counters; /* [nq][4]: hops, seen, dc, routed */
  const orc_policy *pol;                        /* NULL: plain search          */
} q_ctx;

/* Passing-count estimate the policy sees: exact for label / range filters,
 * sample hits * N / S for subset / boolean ones (the routing estimator). */
static int64_t policy_estimate(const orc_index *ix, const orc_filter *f, const uint8_t *aux) {
  if (f->kind == K_SUBSET || f->kind == K_BOOL) {
    int64_t S = ix->n < 4096 ? ix->n : 4096, hits = 0;
    for (int64_t j = 0; j < S; ++j) hits += orc_g(ix, j * ix->n / S, f, aux);
    return hits * ix->n / S;
  }
  if (f->kind == K_NONE) return ix->n;
  return orc_count_passing(ix, f, aux);
}

static void query_range(void *ctx, int64_t lo, int64_t hi, int tid) {
  (void)tid;
  const q_ctx *c = (const q_ctx *)ctx;
  const orc_index *ix = c->ix;
  int ls = c->ls, k = c->k;
  const int quant = ix->fmt != FMT_F32 && ix->xq;
  /* with BF16 / FP8 storage the leading min(4k, ls) passing entries of the
   * final list are ranked again by fp32 distance */
  const int want = quant ? (4 * k < ls ? 4 * k : ls) : k;
  entry_t *L = (entry_t *)malloc(sizeof(entry_t) * (size_t)((ls > 256 ? ls : 256) + 1));
  entry_t *top = (entry_t *)malloc(sizeof(entry_t) * (size_t)(want + 1));
  uint8_t *seen = (uint8_t *)calloc((size_t)ix->n, 1);
  int64_t *touched = (int64_t *)malloc(sizeof(int64_t) * (size_t)ix->n);
  for (int64_t qi = lo; qi < hi; ++qi) {
    const orc_filter *f = &c->f[qi];
    uint8_t *lut = query_lut(f, c->aux);
    int32_t *oid = c->ids + qi * k;
    float *od = c->dist + qi * k;
    int64_t *cn = c->counters ? c->counters + qi * 4 : NULL;
    int routed = c->s0 > 0 ? orc_route(ix, f, c->aux, c->s0, c->scan_cap, NULL) : 0;
    if (routed) {
      bf_ctx b = {ix, c->q, c->f, c->aux, k, c->ids, c->dist, NULL, NULL};
      bf_one(&b, qi);
      if (cn) { cn[0] = 0; cn[1] = 0; cn[2] = 0; cn[3] = 1; }
    } else {
      comparator_t cmp = {ix, c->q + qi * ix->d, f, lut, -1, 0, 0, 0.0f};
      int m = 0;
      counters_t cnt = {0, 0, 0};
      if (c->pol) {
        int len = 0; int64_t nt = 0;
        const int32_t *fq = c->pol->forced ? c->pol->forced + qi * 2 : NULL;
        greedy_policy(&cmp, ls, k, c->pol, fq, policy_estimate(ix, f, c->aux), f->kind, L, &len, seen, touched,
                      &nt, &cnt, c->pol->features ? c->pol->features + qi * NFEAT : NULL,
                      c->pol->decisions ? c->pol->decisions + qi * 4 : NULL);
        for (int64_t i = 0; i < nt; ++i) seen[touched[i]] = 0;
        m = len < want ? len : want;
        for (int i = 0; i < m; ++i) top[i] = L[i];
      } else if (c->literal) {
        int64_t hops = 0;
        greedy_literal(&cmp, ls, want, top, &m, &hops);
        cnt.hops = hops;
      } else {
        int len = 0; int64_t nt = 0;
        greedy_direct(&cmp, ls, L, &len, seen, touched, &nt, NULL, 0, NULL, &cnt);
        for (int64_t i = 0; i < nt; ++i) seen[touched[i]] = 0;
        m = len < want ? len : want;
        for (int i = 0; i < m; ++i) top[i] = L[i];
      }
      /* only points that pass the filter are answers (a prefix of the list) */
      int np = 0;
      while (np < m && top[np].k1 == 0) ++np;
      if (quant) {
        for (int i = 0; i < np; ++i)
          top[i].dist = orc_dist_canon(c->q + qi * ix->d, ix->x + (int64_t)top[i].id * ix->d, ix->d);
        qsort(top, (size_t)np, sizeof(entry_t), entry_cmp);
      }
      int w = 0;
      for (int i = 0; i < np && w < k; ++i) { oid[w] = top[i].id; od[w] = top[i].dist; ++w; }
      for (; w < k; ++w) { oid[w] = -1; od[w] = INFINITY; }
      if (cn) { cn[0] = cnt.hops; cn[1] = cnt.seen; cn[2] = cnt.dc; cn[3] = 0; }
    }
    free(lut);
  }
  free(L); free(top); free(seen); free(touched);
}

/* Query(G, q, ls, k) for a batch.  literal != 0 selects the literal form of
 * GreedySearch.  s0 <= 0 disables the scan route. */
int orc_query(const orc_index *ix, const float *q, const orc_filter *f, const uint8_t *aux,
              int64_t nq, int k, int ls, int literal, int64_t s0, int64_t scan_cap,
              int32_t *ids, float *dist, int64_t *counters, int nthreads) {
  if (k < 1 || ls < k) return 1;
  q_ctx c = {ix, q, f, aux, k, ls, literal, s0, scan_cap, ids, dist, counters, NULL};
  parallel_for(nq, nthreads, query_range, &c);
  return 0;
}

/* Query with a search policy (learned or forced beam and stop hop). */
int orc_query_policy(const orc_index *ix, const float *q, const orc_filter *f, const uint8_t *aux,
                     int64_t nq, int k, int ls, int64_t s0, int64_t scan_cap, const orc_policy *pol,
                     int32_t *ids, float *dist, int64_t *counters, int nthreads) {
  if (k < 1 || ls < k || ls > 256 || !pol) return 1;
  q_ctx c = {ix, q, f, aux, k, ls, 0, s0, scan_cap, ids, dist, counters, pol};
  parallel_for(nq, nthreads, query_range, &c);
  return 0;
}

void orc_mlp_infer_batch(const orc_policy *pol, const float *x, int64_t n, float *out) {
  for (int64_t i = 0; i < n; ++i) orc_mlp_infer(pol, x + i * NFEAT, out + i * (pol->n_ladder + 1));
}

/* Full final list L (ids, first keys, distances) of the direct search for
 * each query: used to check the search's termination state. */
typedef struct {
  const orc_index *ix; const float *q; const orc_filter *f; const uint8_t *aux; int ls;
  int32_t *ids; uint32_t *k1; float *dist; int32_t *len;
} list_ctx;

static void list_range(void *ctx, int64_t lo, int64_t hi, int tid) {
  (void)tid;
  const list_ctx *c = (const list_ctx *)ctx;
  const orc_index *ix = c->ix;
  entry_t *L = (entry_t *)malloc(sizeof(entry_t) * (size_t)(c->ls + 1));
  uint8_t *seen = (uint8_t *)calloc((size_t)ix->n, 1);
  int64_t *touched = (int64_t *)malloc(sizeof(int64_t) * (size_t)ix->n);
  for (int64_t qi = lo; qi < hi; ++qi) {
    uint8_t *lut = query_lut(&c->f[qi], c->aux);
    comparator_t cmp = {ix, c->q + qi * ix->d, &c->f[qi], lut, -1, 0};
    counters_t cnt = {0, 0, 0};
    int len = 0; int64_t nt = 0;
    greedy_direct(&cmp, c->ls, L, &len, seen, touched, &nt, NULL, 0, NULL, &cnt);
    for (int64_t i = 0; i < nt; ++i) seen[touched[i]] = 0;
    for (int i = 0; i < c->ls; ++i) {
      c->ids[qi * c->ls + i] = i < len ? L[i].id : -1;
      c->k1[qi * c->ls + i] = i < len ? L[i].k1 : 0xFFFFFFFFu;
      c->dist[qi * c->ls + i] = i < len ? L[i].dist : INFINITY;
    }
    c->len[qi] = len;
    free(lut);
  }
  free(L); free(seen); free(touched);
}

void orc_query_lists(const orc_index *ix, const float *q, const orc_filter *f, const uint8_t *aux,
                     int64_t nq, int ls, int32_t *ids, uint32_t *k1, float *dist, int32_t *len,
                     int nthreads) {
  list_ctx c = {ix, q, f, aux, ls, ids, k1, dist, len};
  parallel_for(nq, nthreads, list_range, &c);
}

/* ------------------------------------------------------------------------- */
/* index construction                                                         */
/* ------------------------------------------------------------------------- */

/* Entry vertex: the point nearest (fp64) to the fp64 centroid, lowest id on
 * a tie. */
int64_t orc_medoid(const float *x, int64_t n, int64_t d) {
  double *c = (double *)calloc((size_t)d, sizeof(double));
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < d; ++j) c[j] += (double)x[i * d + j];
  for (int64_t j = 0; j < d; ++j) c[j] /= (double)n;
  int64_t best = 0; double bd = INFINITY;
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t j = 0; j < d; ++j) { double t = (double)x[i * d + j] - c[j]; s += t * t; }
    if (s < bd) { bd = s; best = i; }
  }
  free(c);
  return best;
}

/* SplitMix64 (Steele, Lea, Flood, OOPSLA 2014), used as a counter-based
 * generator: the value for counter c under seed s is the generator's output
 * after c+1 steps from state s. */
static inline uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
uint64_t orc_sm64(uint64_t seed, uint64_t ctr) {
  return sm64_mix(seed + (ctr + 1) * 0x9E3779B97F4A7C15ULL);
}

/* Sample id i of point p: uniform over the other n-1 points (with
 * replacement), from counter (p << 20) | i. */
static inline int64_t sample_id(uint64_t seed, int64_t n, int64_t p, int64_t i) {
  uint64_t r = orc_sm64(seed, ((uint64_t)p << 20) | (uint64_t)i) % (uint64_t)(n - 1);
  return (int64_t)r < p ? (int64_t)r : (int64_t)r + 1;
}

static int u32_cmp(const void *a, const void *b) {
  uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
  return x < y ? -1 : x > y;
}

typedef struct {
  const orc_index *ix; const int32_t *pct; int nT; int S; uint64_t seed; uint32_t *out;
} thr_ctx;

/* Per-point thresholds (implementation-details appendix): the distribution
 * of dist_A(a_p, a_v) over a sample of S points v; the threshold for
 * percentile q is the sorted sample's element floor(q (S-1) / 100). */
static void thr_range(void *ctx, int64_t lo, int64_t hi, int tid) {
  (void)tid;
  const thr_ctx *c = (const thr_ctx *)ctx;
  const orc_index *ix = c->ix;
  int64_t S = ix->n - 1 < c->S ? ix->n - 1 : c->S;
  uint32_t *buf = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(S > 0 ? S : 1));
  for (int64_t p = lo; p < hi; ++p) {
    for (int64_t i = 0; i < S; ++i) buf[i] = orc_dist_A(ix, p, sample_id(c->seed, ix->n, p, i));
    qsort(buf, (size_t)S, sizeof(uint32_t), u32_cmp);
    for (int t = 0; t < c->nT; ++t)
      c->out[p * c->nT + t] = S > 0 ? buf[(int64_t)c->pct[t] * (S - 1) / 100] : 0u;
  }
  free(buf);
}

void orc_thresholds(const orc_index *ix, const int32_t *pct, int nT, int S, uint64_t seed,
                    uint32_t *out, int nthreads) {
  thr_ctx c = {ix, pct, nT, S, seed, out};
  parallel_for(ix->n, nthreads, thr_range, &c);
}

/* One candidate of a prune ranking: (k1, key, id) lexicographic; idx is the
 * candidate's position in the caller's arrays. */
typedef struct { uint32_t k1; float key; int32_t id; int32_t idx; } pentry_t;

static int pentry_cmp(const void *pa, const void *pb) {
  const pentry_t *a = (const pentry_t *)pa, *b = (const pentry_t *)pb;
  if (a->k1 != b->k1) return a->k1 < b->k1 ? -1 : 1;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  return a->id < b->id ? -1 : a->id > b->id;
}

/* JointRobustPrune (Algorithm 4).  cand[0..nc) are distinct candidate ids
 * (p excluded) with dpc[i] = dist(p, cand[i]).  For each parameter of p in
 * order -- a threshold t (rank by D_A^t(p, .) = (capped dist_A, dist, id)) or,
 * with weighted != 0, a weight w given as fp32 bits (rank by D_A^w(p, .) =
 * (w dist_A + dist, id), the Weight-JAG comparator) -- walk the candidates,
 * keeping v if it was already chosen for an earlier parameter, else if
 * alpha * dist(u, v) > dist(p, v) for every u kept for this parameter so far
 * (squared distances: alpha^2 d2(u,v) > d2(p,v), alpha^2 rounded to fp32 and
 * the product rounded to fp32); stop once the bucket holds 0.9 R / |T|
 * members.  The union of the buckets, in the order first chosen, is the new
 * out-list (at most R).  Returns its length. */
static int joint_prune(const orc_index *ix, int64_t p, const int32_t *cand, const float *dpc, int nc,
                       const uint32_t *T, int nT, float alpha2, int weighted, int32_t *out) {
  int R = ix->R;
  pentry_t *ord = (pentry_t *)malloc(sizeof(pentry_t) * (size_t)(nc > 0 ? nc : 1));
  int32_t *chosen = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nc + 1));
  int32_t *bucket = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nc + 1));
  int nchosen = 0;
  for (int ti = 0; ti < nT; ++ti) {
    for (int i = 0; i < nc; ++i) {
      if (weighted) {
        ord[i].k1 = 0;
        ord[i].key = fmaf(u2f(T[ti]), orc_dist_A_value(ix, p, cand[i]), dpc[i]);
      } else {
        ord[i].k1 = orc_capped(ix->dist_a, orc_dist_A(ix, p, cand[i]), T[ti]);
        ord[i].key = dpc[i];
      }
      ord[i].id = cand[i];
      ord[i].idx = i;
    }
    qsort(ord, (size_t)nc, sizeof(pentry_t), pentry_cmp);
    int nb = 0;
    for (int i = 0; i < nc; ++i) {
      int32_t v = ord[i].id;
      const float dpv = dpc[ord[i].idx];
      int carried = 0;
      for (int j = 0; j < nchosen; ++j) if (chosen[j] == v) { carried = 1; break; }
      int keep = 1;
      if (!carried) {
        for (int j = 0; j < nb; ++j) {
          float duv = orc_dist_canon(ix->x + (int64_t)bucket[j] * ix->d, ix->x + (int64_t)v * ix->d, ix->d);
          if (!(alpha2 * duv > dpv)) { keep = 0; break; }
        }
      }
      if (keep) bucket[nb++] = v;
      if ((int64_t)nb * nT * 10 >= (int64_t)9 * R) break;
    }
    for (int j = 0; j < nb; ++j) {
      int present = 0;
      for (int i = 0; i < nchosen; ++i) if (chosen[i] == bucket[j]) { present = 1; break; }
      if (!present) chosen[nchosen++] = bucket[j];
    }
  }
  int m = nchosen < R ? nchosen : R;
  for (int i = 0; i < R; ++i) out[i] = i < m ? chosen[i] : -1;
  free(ord); free(chosen); free(bucket);
  return m;
}

typedef struct {
  const orc_index *ix;
  const int64_t *batch; int64_t nb;
  const uint32_t *thr; int nT; int lb; float alpha2; int weighted;
  int32_t *newrows;       /* [nb][R] */
  int64_t *visited_total; /* statistics */
} ins_ctx;

/* Insert (Algorithm 3), first half, for the points of one batch: one
 * GreedySearch with D_A(t) per threshold, the union of the visited sets, and
 * JointRobustPrune of that union.  The graph is read only. */
static void insert_range(void *ctx, int64_t lo, int64_t hi, int tid) {
  (void)tid;
  const ins_ctx *c = (const ins_ctx *)ctx;
  const orc_index *ix = c->ix;
  int lb = c->lb;
  int64_t vcap = 1 << 16;
  entry_t *L = (entry_t *)malloc(sizeof(entry_t) * (size_t)(lb + 1));
  entry_t *vis = (entry_t *)malloc(sizeof(entry_t) * (size_t)vcap);
  int32_t *cand = (int32_t *)malloc(sizeof(int32_t) * (size_t)vcap * 4);
  float *dpc = (float *)malloc(sizeof(float) * (size_t)vcap * 4);
  uint8_t *seen = (uint8_t *)calloc((size_t)ix->n, 1);
  uint8_t *inV = (uint8_t *)calloc((size_t)ix->n, 1);
  int64_t *touched = (int64_t *)malloc(sizeof(int64_t) * (size_t)ix->n);
  for (int64_t bi = lo; bi < hi; ++bi) {
    int64_t p = c->batch[bi];
    int nc = 0;
    for (int ti = 0; ti < c->nT; ++ti) {
      const uint32_t par = c->thr[p * c->nT + ti];
      comparator_t cmp = {ix, ix->x + p * ix->d, NULL, NULL, p, par, c->weighted, u2f(par)};
      counters_t cnt = {0, 0, 0};
      int len = 0; int64_t nt = 0, nv = 0;
      greedy_direct(&cmp, lb, L, &len, seen, touched, &nt, vis, vcap, &nv, &cnt);
      for (int64_t i = 0; i < nt; ++i) seen[touched[i]] = 0;
      if (nv > vcap) nv = vcap;
      for (int64_t i = 0; i < nv; ++i) {
        int32_t v = vis[i].id;
        if (inV[v]) continue;
        inV[v] = 1;
        /* the list holds D_A^w for Weight-JAG: the prune needs dist(p, v) */
        cand[nc] = v;
        dpc[nc] = c->weighted ? orc_dist_canon(ix->x + p * ix->d, ix->x + (int64_t)v * ix->d, ix->d) : vis[i].dist;
        ++nc;
      }
    }
    for (int i = 0; i < nc; ++i) inV[cand[i]] = 0;
    joint_prune(ix, p, cand, dpc, nc, c->thr + p * c->nT, c->nT, c->alpha2, c->weighted, c->newrows + bi * ix->R);
  }
  free(L); free(vis); free(cand); free(dpc); free(seen); free(inV); free(touched);
}

typedef struct { int32_t target, source; } edge_t;
static int edge_cmp(const void *a, const void *b) {
  const edge_t *x = (const edge_t *)a, *y = (const edge_t *)b;
  if (x->target != y->target) return x->target < y->target ? -1 : 1;
  return x->source < y->source ? -1 : x->source > y->source;
}

typedef struct {
  const orc_index *ix; const edge_t *edges; const int64_t *gstart; int64_t ngroups;
  const uint32_t *thr; int nT; float alpha2; int weighted;
} back_ctx;

/* Insert, second half: add p to N_out(v) for every chosen v; a list that
 * grows beyond R is pruned again with v's own thresholds.  The edges of a
 * batch are grouped by target and taken in source-id order; each target is
 * pruned at most once per batch. */
static void back_range(void *ctx, int64_t lo, int64_t hi, int tid) {
  (void)tid;
  const back_ctx *c = (const back_ctx *)ctx;
  const orc_index *ix = c->ix;
  int R = ix->R;
  for (int64_t gi = lo; gi < hi; ++gi) {
    int64_t s = c->gstart[gi], e = c->gstart[gi + 1];
    int64_t v = c->edges[s].target;
    int32_t *row = ix->graph + v * R;
    int32_t *cand = (int32_t *)malloc(sizeof(int32_t) * (size_t)(R + (e - s)));
    int nc = 0;
    for (int r = 0; r < R; ++r) if (row[r] >= 0) cand[nc++] = row[r];
    for (int64_t i = s; i < e; ++i) {
      int32_t src = c->edges[i].source;
      int present = 0;
      for (int j = 0; j < nc; ++j) if (cand[j] == src) { present = 1; break; }
      if (!present) cand[nc++] = src;
    }
    if (nc <= R) {
      for (int r = 0; r < R; ++r) row[r] = r < nc ? cand[r] : -1;
    } else {
      float *dvc = (float *)malloc(sizeof(float) * (size_t)nc);
      for (int i = 0; i < nc; ++i)
        dvc[i] = orc_dist_canon(ix->x + v * ix->d, ix->x + (int64_t)cand[i] * ix->d, ix->d);
      joint_prune(ix, v, cand, dvc, nc, c->thr + v * c->nT, c->nT, c->alpha2, c->weighted, row);
      free(dvc);
    }
    free(cand);
  }
}

/* Build the JAG graph.  Insertion order: the entry vertex (medoid), then the
 * other points by increasing id.  Batches: after the entry, each batch takes
 * the next min(#inserted, max(1, n/50)) points; within a batch every point
 * searches the graph as it stood when the batch began, then all out-lists of
 * the batch are set, then the back-edges are applied.  thr: [n][nT] per-point
 * thresholds from orc_thresholds().  The result does not depend on
 * nthreads.  Returns 0 on success. */
static int build_graph(orc_index *ix, const uint32_t *thr, int nT, int lb, float alpha2, int weighted,
                       int nthreads) {
  int64_t n = ix->n;
  int R = ix->R;
  for (int64_t i = 0; i < n * R; ++i) ix->graph[i] = -1;
  int64_t s = ix->entry;
  int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  int64_t w = 0;
  order[w++] = s;
  for (int64_t i = 0; i < n; ++i) if (i != s) order[w++] = i;
  int64_t cap = n / 50 > 1 ? n / 50 : 1;
  int64_t pos = 1, inserted = 1;
  int32_t *newrows = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap * R);
  edge_t *edges = (edge_t *)malloc(sizeof(edge_t) * (size_t)cap * R);
  int64_t *gstart = (int64_t *)malloc(sizeof(int64_t) * (size_t)(cap * R + 1));
  while (pos < n) {
    int64_t nb = inserted < cap ? inserted : cap;
    if (nb > n - pos) nb = n - pos;
    const int64_t *batch = order + pos;
    ins_ctx ic = {ix, batch, nb, thr, nT, lb, alpha2, weighted, newrows, NULL};
    parallel_for(nb, nthreads, insert_range, &ic);
    int64_t ne = 0;
    for (int64_t bi = 0; bi < nb; ++bi) {
      int64_t p = batch[bi];
      memcpy(ix->graph + p * R, newrows + bi * R, sizeof(int32_t) * (size_t)R);
      for (int r = 0; r < R; ++r) {
        int32_t v = newrows[bi * R + r];
        if (v < 0) continue;
        edges[ne].target = v; edges[ne].source = (int32_t)p; ++ne;
      }
    }
    qsort(edges, (size_t)ne, sizeof(edge_t), edge_cmp);
    int64_t ng = 0;
    for (int64_t i = 0; i < ne; ++i)
      if (i == 0 || edges[i].target != edges[i - 1].target) gstart[ng++] = i;
    gstart[ng] = ne;
    back_ctx bc = {ix, edges, gstart, ng, thr, nT, alpha2, weighted};
    parallel_for(ng, nthreads, back_range, &bc);
    pos += nb;
    inserted += nb;
  }
  free(order); free(newrows); free(edges); free(gstart);
  return 0;
}

int orc_build(orc_index *ix, const uint32_t *thr, int nT, int lb, float alpha2, int nthreads) {
  return build_graph(ix, thr, nT, lb, alpha2, 0, nthreads);
}

/* Weight-JAG build (the weighted variant of Sec. 3): Insert and
 * JointRobustPrune iterate over each point's weights w (fp32 values, [n][nW])
 * with the comparator D_A^w; the query path is unchanged. */
int orc_build_weighted(orc_index *ix, const float *w, int nW, int lb, float alpha2, int nthreads) {
  return build_graph(ix, (const uint32_t *)w, nW, lb, alpha2, 1, nthreads);
}

/* JointRobustPrune exposed for tests: cand/dpc as in joint_prune. */
int orc_joint_prune(const orc_index *ix, int64_t p, const int32_t *cand, const float *dpc, int nc,
                    const uint32_t *T, int nT, float alpha2, int32_t *out) {
  return joint_prune(ix, p, cand, dpc, nc, T, nT, alpha2, 0, out);
}

/* Weighted JointRobustPrune exposed for tests: W holds fp32 weights. */
int orc_joint_prune_weighted(const orc_index *ix, int64_t p, const int32_t *cand, const float *dpc, int nc,
                             const float *W, int nW, float alpha2, int32_t *out) {
  return joint_prune(ix, p, cand, dpc, nc, (const uint32_t *)W, nW, alpha2, 1, out);
}

/* Per-point weight scale of Weight-JAG (implementation-details appendix):
 * over the same sample of S points v as the thresholds, h = sigma / sigma_A
 * with sigma the standard deviation of dist(x_p, x_v) and sigma_A that of
 * dist_A(a_p, a_v) (population deviations, fp64, sums taken in sample
 * order; h = 0 if sigma_A = 0).  The weights of p are w_i = fp32(c_i h). */
typedef struct {
  const orc_index *ix; const double *mult; int nW; int S; uint64_t seed; float *out; double *h;
} wgt_ctx;

static void wgt_range(void *ctx, int64_t lo, int64_t hi, int tid) {
  (void)tid;
  const wgt_ctx *c = (const wgt_ctx *)ctx;
  const orc_index *ix = c->ix;
  int64_t S = ix->n - 1 < c->S ? ix->n - 1 : c->S;
  double *a = (double *)malloc(sizeof(double) * (size_t)(S > 0 ? S : 1));
  double *d = (double *)malloc(sizeof(double) * (size_t)(S > 0 ? S : 1));
  for (int64_t p = lo; p < hi; ++p) {
    for (int64_t i = 0; i < S; ++i) {
      const int64_t v = sample_id(c->seed, ix->n, p, i);
      a[i] = (double)orc_dist_A_value(ix, p, v);
      d[i] = (double)orc_dist_canon(ix->x + p * ix->d, ix->x + v * ix->d, ix->d);
    }
    double ma = 0.0, md = 0.0, va = 0.0, vd = 0.0;
    for (int64_t i = 0; i < S; ++i) { ma += a[i]; md += d[i]; }
    if (S > 0) { ma /= (double)S; md /= (double)S; }
    for (int64_t i = 0; i < S; ++i) {
      const double ta = a[i] - ma, td = d[i] - md;
      va += ta * ta;
      vd += td * td;
    }
    if (S > 0) { va /= (double)S; vd /= (double)S; }
    const double sa = sqrt(va), sd = sqrt(vd);
    const double h = sa > 0.0 ? sd / sa : 0.0;
    if (c->h) c->h[p] = h;
    for (int i = 0; i < c->nW; ++i) c->out[p * c->nW + i] = (float)(c->mult[i] * h);
  }
  free(a); free(d);
}

void orc_weights(const orc_index *ix, const double *mult, int nW, int S, uint64_t seed, float *out, double *h,
                 int nthreads) {
  wgt_ctx c = {ix, mult, nW, S, seed, out, h};
  parallel_for(ix->n, nthreads, wgt_range, &c);
}

/* Single GreedySearch with D_A^t from base point p (as in Insert); writes the
 * visited set's ids and distances (up to vcap) and returns its size. */
int64_t orc_build_search(const orc_index *ix, int64_t p, uint32_t t, int lb, int32_t *vis_ids,
                         float *vis_d, int64_t vcap) {
  entry_t *L = (entry_t *)malloc(sizeof(entry_t) * (size_t)(lb + 1));
  entry_t *vis = (entry_t *)malloc(sizeof(entry_t) * (size_t)(vcap > 0 ? vcap : 1));
  uint8_t *seen = (uint8_t *)calloc((size_t)ix->n, 1);
  int64_t *touched = (int64_t *)malloc(sizeof(int64_t) * (size_t)ix->n);
  comparator_t cmp = {ix, ix->x + p * ix->d, NULL, NULL, p, t};
  counters_t cnt = {0, 0, 0};
  int len = 0; int64_t nt = 0, nv = 0;
  greedy_direct(&cmp, lb, L, &len, seen, touched, &nt, vis, vcap, &nv, &cnt);
  int64_t m = nv < vcap ? nv : vcap;
  for (int64_t i = 0; i < m; ++i) { vis_ids[i] = vis[i].id; vis_d[i] = vis[i].dist; }
  free(L); free(vis); free(seen); free(touched);
  return nv;
}

/* Batch helpers for tests. */
void orc_dist_F_batch(const orc_index *ix, const orc_filter *f, const uint8_t *aux, const int64_t *pts,
                      int64_t np, uint32_t *out) {
  uint8_t *lut = query_lut(f, aux);
  for (int64_t i = 0; i < np; ++i) out[i] = orc_dist_F(ix, pts[i], f, lut);
  free(lut);
}

void orc_g_batch(const orc_index *ix, const orc_filter *f, const uint8_t *aux, const int64_t *pts,
                 int64_t np, uint8_t *out) {
  for (int64_t i = 0; i < np; ++i) out[i] = (uint8_t)orc_g(ix, pts[i], f, aux);
}

void orc_dist_canon_batch(const float *q, const float *x, int64_t n, int64_t d, float *out) {
  for (int64_t i = 0; i < n; ++i) out[i] = orc_dist_canon(q + i * d, x + i * d, d);
}
