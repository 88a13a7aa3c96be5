/*
 * c2: strategy loop-nest evaluator -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain C loops that evaluate exactly the trees the pattern evaluator
 * (oracle/patterns.py) defines, fast enough for the full-size workloads.
 * Built with -O2 -ffp-contract=off and without -ffast-math, so each float +
 * and * is a separate IEEE binary32 operation rounded to nearest even
 * (FLT_EVAL_METHOD 0 on x86-64 SSE and on AArch64). Only tests/, the smoke
 * check and the bench's CPU baseline load it; the CUDA library does not.
 *
 * Threads: the independent units of a strategy -- the chunks of the first
 * level, the rows of a GEMV, the columns of its dx, the entries of a GEMM
 * sample, the elements of a map -- may be evaluated by OpenMP threads
 * (oracle_set_threads; 1 by default). Each unit writes only its own slot and
 * is computed by the same loops as with one thread; every fold across units
 * (the second level, the chunk fold of dx) runs afterwards on one thread in
 * the strategy's order. No OpenMP reduction clause is used, so the thread
 * count never changes a bit of any result.
 *
 * Paper passages followed:
 *   - reduce as a left fold from the initial value (Section 4.2, reduceI as
 *     new + for);
 *   - split n: out[i][j] = in[i*n+j]; join: out[i] = in[i/m][i%m]
 *     (Section 4.3, index rules of Stage III);
 *   - the two-level dot strategy (Section 2.1): split the zipped input into
 *     chunks, a parallel map over chunks whose threads each fold a part of the
 *     chunk sequentially, join, and a final reduce over the chunk results
 *     (the loop after the parfor nest in Section 2.2);
 *   - asVector/asScalar (Section 6): V consecutive elements form one vector.
 * Tree, lane fold and second-level rules are the build's reading of the
 * strategy (the paper has no in-block tree); they match patterns.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OK 0
#define BAD_ARGS -1
#define BAD_SHAPE -2
#define NO_MEMORY -3

/* Threads for the per-unit loops (see the header comment). */
static int g_threads = 1;

int oracle_set_threads(int t) {
  if (t < 1) return BAD_ARGS;
#ifdef _OPENMP
  g_threads = t;
#else
  g_threads = 1;
#endif
  return OK;
}

int oracle_threads(void) { return g_threads; }

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_num_procs();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* element producers                                                         */
/* ------------------------------------------------------------------------ */

/* Which item of the (padded) input a thread's r-th fold step reads, lane v. */
static int64_t item_index(int64_t c, int64_t s, int T, int V, int interleaved, int64_t t,
                          int64_t r, int v) {
  int64_t R = s / ((int64_t)T * V);
  int64_t vec = interleaved ? (r * T + t) : (t * R + r);
  return c * s + vec * V + v;
}

static int is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

static int check_strategy(int64_t s, int T, int V, int second_tree, int T2) {
  if (s <= 0 || T <= 0 || V <= 0) return BAD_ARGS;
  if (!is_pow2(T) || !is_pow2(V)) return BAD_ARGS;
  if (s % ((int64_t)T * V) != 0) return BAD_ARGS;
  if (second_tree && !is_pow2(T2)) return BAD_ARGS;
  return OK;
}

/* plain binary32 halving tree over a power-of-two array, in place */
static float tree_f32(float *q, int64_t len) {
  while (len > 1) {
    int64_t h = len / 2;
    for (int64_t l = 0; l < h; ++l) q[l] = q[l] + q[l + h];
    len = h;
  }
  return q[0];
}

/* treeLanes over groups of min(32, T), then treeWarps over the group sums */
static float block_tree_f32(float *th, int T) {
  int L = T < 32 ? T : 32;
  int W = T / L;
  for (int w = 0; w < W; ++w) th[w] = tree_f32(th + (int64_t)w * L, L);
  return tree_f32(th, W);
}

/* ---- compensated (Kahan) state ------------------------------------------ */
typedef struct {
  float s, c;
} kstate;

static kstate kahan_step(kstate a, float e) {
  float y = e - a.c;
  float t = a.s + y;
  float c = (t - a.s) - y;
  kstate r = {t, c};
  return r;
}

static kstate kahan_combine(kstate a, kstate b) { return kahan_step(a, b.s - b.c); }

static kstate tree_k(kstate *q, int64_t len) {
  while (len > 1) {
    int64_t h = len / 2;
    for (int64_t l = 0; l < h; ++l) q[l] = kahan_combine(q[l], q[l + h]);
    len = h;
  }
  return q[0];
}

static kstate block_tree_k(kstate *th, int T) {
  int L = T < 32 ? T : 32;
  int W = T / L;
  for (int w = 0; w < W; ++w) th[w] = tree_k(th + (int64_t)w * L, L);
  return tree_k(th, W);
}

/* ------------------------------------------------------------------------ */
/* generic f32 strategy reduce: kind 0 = dot (x*y), kind 1 = asum (|x|)      */
/* ------------------------------------------------------------------------ */

static float item_f32(int kind, const float *x, const float *y, int64_t n, int64_t e) {
  if (e >= n) {
    /* padding item: (+0, +0) for dot, +0 for asum */
    return kind == 0 ? (0.0f * 0.0f) : fabsf(0.0f);
  }
  return kind == 0 ? (x[e] * y[e]) : fabsf(x[e]);
}

/* First level of chunk c: thread t lane v folds its items over r from +0, the
 * lanes are folded in lane order from +0, the T thread results go through the
 * block tree. th (T floats) and lane (V floats) are scratch. */
static float chunk_f32(int kind, const float *x, const float *y, int64_t n, int64_t s, int T,
                       int V, int interleaved, int64_t c, float *th, float *lane) {
  int64_t R = s / ((int64_t)T * V);
  for (int64_t t = 0; t < T; ++t) {
    for (int v = 0; v < V; ++v) lane[v] = 0.0f;
    for (int64_t r = 0; r < R; ++r)
      for (int v = 0; v < V; ++v) {
        int64_t e = item_index(c, s, T, V, interleaved, t, r, v);
        lane[v] = lane[v] + item_f32(kind, x, y, n, e);
      }
    float acc = 0.0f;
    for (int v = 0; v < V; ++v) acc = acc + lane[v];
    th[t] = acc;
  }
  return block_tree_f32(th, T);
}

/* The same first level with Kahan states in place of floats. */
static kstate chunk_k(int kind, const float *x, const float *y, int64_t n, int64_t s, int T,
                      int V, int interleaved, int64_t c, kstate *th, kstate *lane) {
  const kstate zero = {0.0f, 0.0f};
  int64_t R = s / ((int64_t)T * V);
  for (int64_t t = 0; t < T; ++t) {
    for (int v = 0; v < V; ++v) lane[v] = zero;
    for (int64_t r = 0; r < R; ++r)
      for (int v = 0; v < V; ++v) {
        int64_t e = item_index(c, s, T, V, interleaved, t, r, v);
        lane[v] = kahan_step(lane[v], item_f32(kind, x, y, n, e));
      }
    kstate acc = zero;
    for (int v = 0; v < V; ++v) acc = kahan_combine(acc, lane[v]);
    th[t] = acc;
  }
  return block_tree_k(th, T);
}

/* part[c] = chunk_f32(c) (or chunk_k, into kpart) for c = 0..C-1; the chunks
 * are independent units, shared among nt threads. */
static int first_level(int kind, const float *x, const float *y, int64_t n, int64_t s, int T,
                       int V, int interleaved, int64_t C, int nt, float *part, kstate *kpart) {
  int err = 0;
#pragma omp parallel num_threads(nt) if (nt > 1)
  {
    float *th = NULL, *lane = NULL;
    kstate *kth = NULL, *klane = NULL;
    int ok;
    if (kpart) {
      kth = (kstate *)malloc(sizeof(kstate) * (size_t)T);
      klane = (kstate *)malloc(sizeof(kstate) * (size_t)V);
      ok = kth && klane;
    } else {
      th = (float *)malloc(sizeof(float) * (size_t)T);
      lane = (float *)malloc(sizeof(float) * (size_t)V);
      ok = th && lane;
    }
    if (!ok) {
#pragma omp atomic write
      err = 1;
    }
#pragma omp for schedule(static)
    for (int64_t c = 0; c < C; ++c) {
      if (!ok) continue;
      if (kpart)
        kpart[c] = chunk_k(kind, x, y, n, s, T, V, interleaved, c, kth, klane);
      else
        part[c] = chunk_f32(kind, x, y, n, s, T, V, interleaved, c, th, lane);
    }
    free(th); free(lane); free(kth); free(klane);
  }
  return err ? NO_MEMORY : OK;
}

/* reduce of the zipped (or single) input with strategy (s, T, V, map, second,
 * T2); the first level on nt threads, the second level on one. */
static int reduce_f32(int kind, const float *x, const float *y, int64_t n, int64_t s, int T,
                      int V, int interleaved, int second_tree, int T2, int compensated, int pad,
                      int nt, float *out) {
  if (!out || n < 0) return BAD_ARGS;
  int rc = check_strategy(s, T, V, second_tree, T2);
  if (rc) return rc;
  if (n == 0) {
    *out = 0.0f;
    return OK;
  }
  if (n % s != 0 && !pad) return BAD_SHAPE;
  int64_t C = (n + s - 1) / s;
  int64_t Cpad = second_tree ? ((C + T2 - 1) / T2) * T2 : C;
  if (!compensated) {
    float *part = (float *)calloc((size_t)Cpad, sizeof(float));
    float *th = (float *)malloc(sizeof(float) * (size_t)T2);
    if (!part || !th) {
      free(part); free(th);
      return NO_MEMORY;
    }
    rc = first_level(kind, x, y, n, s, T, V, interleaved, C, nt, part, NULL);
    float res = 0.0f;
    if (rc == OK && !second_tree) {
      for (int64_t c = 0; c < C; ++c) res = res + part[c];
    } else if (rc == OK) {
      /* pad with +0 to a multiple of T2; thread t2 folds part[r*T2 + t2] */
      int64_t R2 = Cpad / T2;
      for (int64_t t = 0; t < T2; ++t) {
        float acc = 0.0f;
        for (int64_t r = 0; r < R2; ++r) acc = acc + part[r * T2 + t];
        th[t] = acc;
      }
      res = block_tree_f32(th, T2);
    }
    *out = res;
    free(part); free(th);
    return rc;
  }
  /* compensated */
  kstate *part = (kstate *)calloc((size_t)Cpad, sizeof(kstate));
  kstate *th = (kstate *)malloc(sizeof(kstate) * (size_t)T2);
  if (!part || !th) {
    free(part); free(th);
    return NO_MEMORY;
  }
  rc = first_level(kind, x, y, n, s, T, V, interleaved, C, nt, NULL, part);
  const kstate zero = {0.0f, 0.0f};
  kstate res = zero;
  if (rc == OK && !second_tree) {
    for (int64_t c = 0; c < C; ++c) res = kahan_combine(res, part[c]);
  } else if (rc == OK) {
    int64_t R2 = Cpad / T2;
    for (int64_t t = 0; t < T2; ++t) {
      kstate acc = zero;
      for (int64_t r = 0; r < R2; ++r) acc = kahan_combine(acc, part[r * T2 + t]);
      th[t] = acc;
    }
    res = block_tree_k(th, T2);
  }
  *out = res.s;
  free(part); free(th);
  return rc;
}

int oracle_dot_f32(const float *x, const float *y, int64_t n, int64_t s, int T, int V,
                   int interleaved, int second_tree, int T2, int compensated, int pad,
                   float *out) {
  if (n > 0 && (!x || !y)) return BAD_ARGS;
  return reduce_f32(0, x, y, n, s, T, V, interleaved, second_tree, T2, compensated, pad,
                    g_threads, out);
}

int oracle_asum_f32(const float *x, int64_t n, int64_t s, int T, int V, int interleaved,
                    int second_tree, int T2, int compensated, int pad, float *out) {
  if (n > 0 && !x) return BAD_ARGS;
  return reduce_f32(1, x, NULL, n, s, T, V, interleaved, second_tree, T2, compensated, pad,
                    g_threads, out);
}

/* Partials of the first level only (chunk results in chunk order), for checks
 * of the workspace contents. */
int oracle_dot_f32_partials(const float *x, const float *y, int64_t n, int64_t s, int T, int V,
                            int interleaved, int pad, float *partials) {
  int rc = check_strategy(s, T, V, 0, 1);
  if (rc) return rc;
  if (n % s != 0 && !pad) return BAD_SHAPE;
  int64_t C = (n + s - 1) / s;
  return first_level(0, x, y, n, s, T, V, interleaved, C, g_threads, partials, NULL);
}

/* ------------------------------------------------------------------------ */
/* int32 dot: int64 products and sums (exact, so any tree gives the same)    */
/* ------------------------------------------------------------------------ */

static int64_t tree_i64(int64_t *q, int64_t len) {
  while (len > 1) {
    int64_t h = len / 2;
    for (int64_t l = 0; l < h; ++l) q[l] = q[l] + q[l + h];
    len = h;
  }
  return q[0];
}

static int64_t block_tree_i64(int64_t *th, int T) {
  int L = T < 32 ? T : 32;
  for (int w = 0; w < T / L; ++w) th[w] = tree_i64(th + (int64_t)w * L, L);
  return tree_i64(th, T / L);
}

static int64_t chunk_i32(const int32_t *x, const int32_t *y, int64_t n, int64_t s, int T, int V,
                         int interleaved, int64_t c, int64_t *th, int64_t *lane) {
  int64_t R = s / ((int64_t)T * V);
  for (int64_t t = 0; t < T; ++t) {
    for (int v = 0; v < V; ++v) lane[v] = 0;
    for (int64_t r = 0; r < R; ++r)
      for (int v = 0; v < V; ++v) {
        int64_t e = item_index(c, s, T, V, interleaved, t, r, v);
        if (e < n) lane[v] += (int64_t)x[e] * (int64_t)y[e];
      }
    int64_t acc = 0;
    for (int v = 0; v < V; ++v) acc += lane[v];
    th[t] = acc;
  }
  return block_tree_i64(th, T);
}

int oracle_dot_i32(const int32_t *x, const int32_t *y, int64_t n, int64_t s, int T, int V,
                   int interleaved, int second_tree, int T2, int pad, int64_t *out) {
  if (!out || n < 0 || (n > 0 && (!x || !y))) return BAD_ARGS;
  int rc = check_strategy(s, T, V, second_tree, T2);
  if (rc) return rc;
  if (n == 0) {
    *out = 0;
    return OK;
  }
  if (n % s != 0 && !pad) return BAD_SHAPE;
  int64_t C = (n + s - 1) / s;
  int64_t Cpad = second_tree ? ((C + T2 - 1) / T2) * T2 : C;
  int64_t *part = (int64_t *)calloc((size_t)Cpad, sizeof(int64_t));
  int64_t *th2 = (int64_t *)malloc(sizeof(int64_t) * (size_t)T2);
  if (!part || !th2) {
    free(part); free(th2);
    return NO_MEMORY;
  }
  int err = 0;
#pragma omp parallel num_threads(g_threads) if (g_threads > 1)
  {
    int64_t *th = (int64_t *)malloc(sizeof(int64_t) * (size_t)T);
    int64_t *lane = (int64_t *)malloc(sizeof(int64_t) * (size_t)V);
    int ok = th && lane;
    if (!ok) {
#pragma omp atomic write
      err = 1;
    }
#pragma omp for schedule(static)
    for (int64_t c = 0; c < C; ++c)
      if (ok) part[c] = chunk_i32(x, y, n, s, T, V, interleaved, c, th, lane);
    free(th); free(lane);
  }
  int64_t res = 0;
  if (!second_tree) {
    for (int64_t c = 0; c < C; ++c) res += part[c];
  } else {
    int64_t R2 = Cpad / T2;
    for (int64_t t = 0; t < T2; ++t) {
      int64_t acc = 0;
      for (int64_t r = 0; r < R2; ++r) acc += part[r * T2 + t];
      th2[t] = acc;
    }
    res = block_tree_i64(th2, T2);
  }
  *out = res;
  free(part); free(th2);
  return err ? NO_MEMORY : OK;
}

/* ------------------------------------------------------------------------ */
/* scal, dot backward: plain maps                                             */
/* ------------------------------------------------------------------------ */

void oracle_scal_f32(float a, const float *x, float *y, int64_t n) {
#pragma omp parallel for schedule(static) num_threads(g_threads) if (g_threads > 1)
  for (int64_t i = 0; i < n; ++i) y[i] = a * x[i];
}

/* dx = g*y, dy = g*x (adjoint of reduce(+) broadcasts g; of map(*) multiplies) */
void oracle_dot_bwd_f32(const float *x, const float *y, float g, int64_t n, float *dx,
                        float *dy) {
#pragma omp parallel for schedule(static) num_threads(g_threads) if (g_threads > 1)
  for (int64_t i = 0; i < n; ++i) {
    if (dx) dx[i] = g * y[i];
    if (dy) dy[i] = g * x[i];
  }
}

/* ------------------------------------------------------------------------ */
/* GEMV: y_i = strategy-reduce of (A_i*, x), rows independent                 */
/* ------------------------------------------------------------------------ */

int oracle_gemv_f32(const float *A, int64_t M, int64_t N, int64_t lda, const float *x, float *y,
                    int64_t s, int T, int V, int interleaved, int compensated, int pad) {
  if (!A || !x || !y || M < 0 || N < 0 || lda < N) return BAD_ARGS;
  int err = OK;
  /* rows are the units; each row's reduce runs on its thread alone */
#pragma omp parallel for schedule(dynamic, 16) num_threads(g_threads) if (g_threads > 1)
  for (int64_t i = 0; i < M; ++i) {
    int rc = reduce_f32(0, A + i * lda, x, N, s, T, V, interleaved, 0, 1, compensated, pad, 1,
                        y + i);
    if (rc) {
#pragma omp atomic write
      err = rc;
    }
  }
  return err;
}

/* dx_j = fold over row chunks of size Rs (each chunk folded in row order from
 * +0), the chunk results folded in chunk order from +0; rows past M pad with 0.
 * Columns are the units. */
int oracle_gemv_bwd_dx_f32(const float *A, int64_t M, int64_t N, int64_t lda, const float *dy,
                           int64_t Rs, float *dx) {
  if (!A || !dy || !dx || M < 0 || N < 0 || lda < N || Rs <= 0) return BAD_ARGS;
  int64_t C = (M + Rs - 1) / Rs;
#pragma omp parallel for schedule(static) num_threads(g_threads) if (g_threads > 1)
  for (int64_t j = 0; j < N; ++j) {
    float res = 0.0f;
    for (int64_t c = 0; c < C; ++c) {
      float acc = 0.0f;
      for (int64_t r = 0; r < Rs; ++r) {
        int64_t i = c * Rs + r;
        float e = (i < M) ? (A[i * lda + j] * dy[i]) : (0.0f * 0.0f);
        acc = acc + e;
      }
      res = res + acc;
    }
    dx[j] = res;
  }
  return OK;
}

void oracle_gemv_bwd_dA_f32(const float *x, const float *dy, int64_t M, int64_t N, float *dA,
                            int64_t ldda) {
#pragma omp parallel for schedule(static) num_threads(g_threads) if (g_threads > 1)
  for (int64_t i = 0; i < M; ++i)
    for (int64_t j = 0; j < N; ++j) dA[i * ldda + j] = dy[i] * x[j];
}

/* ------------------------------------------------------------------------ */
/* FP32 GEMM fold: C_ij = fold over k = 0..K-1 from +0 of op(A)_ik * op(B)_kj */
/* with separate roundings, or fmaf when the contraction is declared.        */
/* op(A) = A (M x K, row-major, lda) or A^T (A stored K x M); same for B.    */
/* Rows rows[0..nr) and columns cols[0..nc) of C are computed (a sample);    */
/* out is nr x nc row-major. Each entry is a unit.                            */
/* ------------------------------------------------------------------------ */

int oracle_gemm_f32_sample(const float *A, const float *B, int64_t M, int64_t N, int64_t K,
                           int64_t lda, int64_t ldb, int transA, int transB, int contract_fma,
                           const int64_t *rows, int64_t nr, const int64_t *cols, int64_t nc,
                           float *out) {
  if (!A || !B || !out || M < 0 || N < 0 || K < 0) return BAD_ARGS;
  for (int64_t a = 0; a < nr; ++a)
    if (rows[a] < 0 || rows[a] >= M) return BAD_ARGS;
  for (int64_t b = 0; b < nc; ++b)
    if (cols[b] < 0 || cols[b] >= N) return BAD_ARGS;
#pragma omp parallel for collapse(2) schedule(static) num_threads(g_threads) if (g_threads > 1)
  for (int64_t a = 0; a < nr; ++a) {
    for (int64_t b = 0; b < nc; ++b) {
      int64_t i = rows[a], j = cols[b];
      float acc = 0.0f;
      for (int64_t k = 0; k < K; ++k) {
        float av = transA ? A[k * lda + i] : A[i * lda + k];
        float bv = transB ? B[j * ldb + k] : B[k * ldb + j];
        if (contract_fma)
          acc = fmaf(av, bv, acc);
        else
          acc = acc + av * bv;
      }
      out[a * nc + b] = acc;
    }
  }
  return OK;
}

/* ------------------------------------------------------------------------ */
/* Lane partials: the first level of the paper's Section 6 kernel, which     */
/* stores every work-item's un-reduced vector of V lane folds. out has       */
/* C*T*V entries, out[(c*T + t)*V + v] = the fold of thread t's lane v over  */
/* its items in chunk c (kind 0 = dot, 1 = asum). Chunks are the units.      */
/* ------------------------------------------------------------------------ */

int oracle_lane_partials_f32(int kind, const float *x, const float *y, int64_t n, int64_t s, int T,
                             int V, int interleaved, int pad, float *out) {
  if (!out || n < 0 || !x || (kind == 0 && !y)) return BAD_ARGS;
  int rc = check_strategy(s, T, V, 0, 1);
  if (rc) return rc;
  if (n % s != 0 && !pad) return BAD_SHAPE;
  int64_t C = (n + s - 1) / s, R = s / ((int64_t)T * V);
#pragma omp parallel for schedule(static) num_threads(g_threads) if (g_threads > 1)
  for (int64_t c = 0; c < C; ++c)
    for (int64_t t = 0; t < T; ++t)
      for (int v = 0; v < V; ++v) {
        float acc = 0.0f;
        for (int64_t r = 0; r < R; ++r)
          acc = acc + item_f32(kind, x, y, n, item_index(c, s, T, V, interleaved, t, r, v));
        out[(c * T + t) * V + v] = acc;
      }
  return OK;
}
