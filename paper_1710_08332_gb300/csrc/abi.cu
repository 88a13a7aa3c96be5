// C ABI (include/dpia.h): argument validation, strategy planning and dispatch.
//
// Everything is checked on the host before anything is enqueued: pointers,
// sizes, alignment for the requested vector width, the legality of the level
// nesting (a map nested in another runs at a strictly finer level), the
// workspace size, and that no output overlaps an input (a parallel map writes
// only through its own acceptor -- the interference control that makes the
// paper's parfor race free).
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "../../include/dpia.h"
#include "device_common.cuh"
#include "kernels.h"

using namespace dpia;

namespace {

thread_local std::string g_err;

dpia_status fail(dpia_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

dpia_status cuda_status(cudaError_t e, const char *fn) {
  if (e == cudaSuccess) return DPIA_OK;
  return fail(DPIA_ERR_CUDA, "%s: CUDA error %d (%s)", fn, (int)e, cudaGetErrorString(e));
}

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

bool aligned(const void *p, int64_t a) { return (reinterpret_cast<uintptr_t>(p) % (uintptr_t)a) == 0; }

int64_t vec_align(int V) { return V * 4 < 16 ? V * 4 : 16; }

// [a, a+na) and [b, b+nb) overlap (bytes)
bool overlap(const void *a, int64_t na, const void *b, int64_t nb) {
  if (!a || !b || na <= 0 || nb <= 0) return false;
  auto x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + (uintptr_t)nb && y < x + (uintptr_t)na;
}

constexpr int64_t kCounterBytes = 128;

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// Granularity of a level: a nested map must be strictly finer. A GRID map runs
// its iterations on single threads, like THREAD.
int granularity(int lvl) {
  switch (lvl) {
    case DPIA_LVL_BLOCK: return 1;
    case DPIA_LVL_WARP: return 2;
    case DPIA_LVL_THREAD: return 3;
    case DPIA_LVL_GRID: return 3;
    case DPIA_LVL_SEQ: return 4;
  }
  return -1;
}

struct ReducePlan {
  ChunkLevel level;
  int threads, V, Tc, T2, second_tree, compensated, grid, staged;
  int64_t s, C, Rc, step, tstride;
};

// Validate a reduction strategy for a length n and derive the launch plan.
dpia_status plan_reduce(const char *fn, int64_t n, const dpia_reduce_strategy *st, bool allow_comp,
                        bool allow_tree, bool allow_stage, ReducePlan *pl) {
  if (!st) return fail(DPIA_ERR_NULL, "%s: strategy is NULL", fn);
  if (n < 0) return fail(DPIA_ERR_SHAPE, "%s: negative length %lld", fn, (long long)n);
  const int T = st->threads, V = st->vec;
  if (!is_pow2(T) || T < 32 || T > 1024)
    return fail(DPIA_ERR_STRATEGY, "%s: threads=%d must be a power of two in [32, 1024]", fn, T);
  if (!(V == 1 || V == 2 || V == 4 || V == 8 || V == 16))
    return fail(DPIA_ERR_STRATEGY, "%s: vec=%d must be 1, 2, 4, 8 or 16", fn, V);
  if (T > max_threads_for_vec(V))
    return fail(DPIA_ERR_STRATEGY, "%s: threads=%d exceeds %d for vec=%d", fn, T, max_threads_for_vec(V), V);
  const int gm = granularity(st->map_level), gi = granularity(st->inner_level);
  if (gm < 0 || gi < 0)
    return fail(DPIA_ERR_STRATEGY, "%s: unknown level (map_level=%d, inner_level=%d)", fn,
                st->map_level, st->inner_level);
  if (st->map_level == DPIA_LVL_THREAD)
    return fail(DPIA_ERR_STRATEGY, "%s: a thread-level map must be nested in a block or warp map", fn);
  if (gi <= gm)
    return fail(DPIA_ERR_STRATEGY,
                "%s: illegal nesting: inner_level=%d is not finer than map_level=%d", fn,
                st->inner_level, st->map_level);
  ChunkLevel level;
  int Tc;
  if (st->map_level == DPIA_LVL_BLOCK && st->inner_level == DPIA_LVL_THREAD) {
    level = ChunkLevel::Block;
    Tc = T;
  } else if (st->map_level == DPIA_LVL_WARP && st->inner_level == DPIA_LVL_THREAD) {
    level = ChunkLevel::Warp;
    Tc = 32;
  } else if (st->map_level == DPIA_LVL_GRID && st->inner_level == DPIA_LVL_SEQ) {
    level = ChunkLevel::Grid;
    Tc = 1;
  } else {
    return fail(DPIA_ERR_UNSUPPORTED, "%s: level pair (map=%d, inner=%d) is legal but not implemented",
                fn, st->map_level, st->inner_level);
  }
  if (st->thread_map != DPIA_MAP_INTERLEAVED && st->thread_map != DPIA_MAP_CONTIG)
    return fail(DPIA_ERR_STRATEGY, "%s: thread_map=%d", fn, st->thread_map);
  if (st->second != DPIA_SECOND_SEQ && st->second != DPIA_SECOND_TREE)
    return fail(DPIA_ERR_STRATEGY, "%s: second=%d", fn, st->second);
  if (st->second == DPIA_SECOND_TREE) {
    if (!allow_tree) return fail(DPIA_ERR_UNSUPPORTED, "%s: second=TREE is not implemented here", fn);
    if (!is_pow2(st->threads2) || st->threads2 > T)
      return fail(DPIA_ERR_STRATEGY, "%s: threads2=%d must be a power of two <= threads=%d", fn,
                  st->threads2, T);
  }
  if (st->compensated != 0 && st->compensated != 1)
    return fail(DPIA_ERR_STRATEGY, "%s: compensated=%d", fn, st->compensated);
  if (st->compensated && !allow_comp)
    return fail(DPIA_ERR_STRATEGY, "%s: compensated summation applies to f32 only", fn);
  if (st->pad != 0 && st->pad != 1) return fail(DPIA_ERR_STRATEGY, "%s: pad=%d", fn, st->pad);
  if (st->grid < 0) return fail(DPIA_ERR_STRATEGY, "%s: grid=%d", fn, st->grid);
  if (st->stage != DPIA_STAGE_PRIVATE && st->stage != DPIA_STAGE_LOCAL)
    return fail(DPIA_ERR_STRATEGY, "%s: stage=%d", fn, st->stage);
  if (st->stage == DPIA_STAGE_LOCAL) {
    if (!allow_stage) return fail(DPIA_ERR_UNSUPPORTED, "%s: stage=LOCAL is not implemented here", fn);
    if (level != ChunkLevel::Block || V != 4 || st->thread_map != DPIA_MAP_INTERLEAVED)
      return fail(DPIA_ERR_UNSUPPORTED,
                  "%s: stage=LOCAL is implemented for map_level BLOCK, vec 4, interleaved thread map", fn);
  }
  const int64_t s = st->split;
  if (s <= 0 || s % ((int64_t)Tc * V) != 0)
    return fail(DPIA_ERR_STRATEGY, "%s: split=%lld must be a positive multiple of %d threads x vec %d",
                fn, (long long)s, Tc, V);
  if (n % s != 0 && !st->pad)
    return fail(DPIA_ERR_SHAPE, "%s: split=%lld does not divide n=%lld (set pad=1)", fn, (long long)s,
                (long long)n);
  pl->level = level;
  pl->threads = T;
  pl->V = V;
  pl->Tc = Tc;
  pl->T2 = st->second == DPIA_SECOND_TREE ? st->threads2 : 1;
  pl->second_tree = st->second == DPIA_SECOND_TREE;
  pl->compensated = st->compensated;
  pl->grid = st->grid;
  pl->staged = st->stage == DPIA_STAGE_LOCAL;
  pl->s = s;
  pl->C = (n + s - 1) / s;
  pl->Rc = s / ((int64_t)Tc * V);
  if (st->thread_map == DPIA_MAP_INTERLEAVED) {
    pl->step = (int64_t)Tc * V;
    pl->tstride = V;
  } else {
    pl->step = V;
    pl->tstride = pl->Rc * V;
  }
  return DPIA_OK;
}

int64_t reduce_ws_bytes(const ReducePlan &pl) { return kCounterBytes + round_up(pl.C * 8, 128); }

dpia_status run_reduce(const char *fn, ReduceOp op, const void *x, const void *y, int64_t n,
                       int64_t in_size, const dpia_reduce_strategy *st, void *out, int64_t out_size,
                       void *ws, size_t ws_bytes, dpia_stream_t stream) {
  g_err.clear();
  ReducePlan pl;
  dpia_status rc = plan_reduce(fn, n, st, op != ReduceOp::DotI32, true, true, &pl);
  if (rc) return rc;
  if (!out) return fail(DPIA_ERR_NULL, "%s: out is NULL", fn);
  if (n > 0 && (!x || (op != ReduceOp::AsumF32 && !y))) return fail(DPIA_ERR_NULL, "%s: input is NULL", fn);
  if (!aligned(out, out_size)) return fail(DPIA_ERR_ALIGN, "%s: out not %lld-byte aligned", fn, (long long)out_size);
  const int64_t in_bytes = n * in_size;
  if (overlap(out, out_size, x, in_bytes) || overlap(out, out_size, y, in_bytes))
    return fail(DPIA_ERR_ALIAS, "%s: out overlaps an input", fn);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (n == 0) return cuda_status(cudaMemsetAsync(out, 0, (size_t)out_size, s), fn);
  const int64_t va = vec_align(pl.V) * in_size / 4;
  if (!aligned(x, va) || (y && !aligned(y, va)))
    return fail(DPIA_ERR_ALIGN, "%s: inputs must be %lld-byte aligned for vec=%d", fn, (long long)va, pl.V);
  const int64_t need = reduce_ws_bytes(pl);
  if (!ws) return fail(DPIA_ERR_WORKSPACE, "%s: workspace is NULL (%lld bytes needed)", fn, (long long)need);
  if ((int64_t)ws_bytes < need)
    return fail(DPIA_ERR_WORKSPACE, "%s: workspace of %zu bytes, %lld needed", fn, ws_bytes, (long long)need);
  if (!aligned(ws, 128)) return fail(DPIA_ERR_ALIGN, "%s: workspace must be 128-byte aligned", fn);
  if (overlap(ws, need, x, in_bytes) || overlap(ws, need, y, in_bytes) || overlap(ws, need, out, out_size))
    return fail(DPIA_ERR_ALIAS, "%s: workspace overlaps an input or the output", fn);
  ReduceLaunch p;
  p.x = x;
  p.y = y;
  p.n = n;
  p.s = pl.s;
  p.C = pl.C;
  p.Rc = pl.Rc;
  p.step = pl.step;
  p.tstride = pl.tstride;
  p.Tc = pl.Tc;
  p.second_tree = pl.second_tree;
  p.T2 = pl.T2;
  p.counter = static_cast<unsigned *>(ws);
  p.partials = static_cast<char *>(ws) + kCounterBytes;
  p.out = out;
  if (pl.staged) return cuda_status(launch_reduce_staged(op, pl.compensated, pl.threads, pl.grid, p, s), fn);
  return cuda_status(launch_reduce(op, pl.compensated, pl.V, pl.level, pl.threads, pl.grid, p, s), fn);
}

}  // namespace

namespace dpia {
void set_last_error(const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
}
}  // namespace dpia

extern "C" {

int32_t dpia_version(void) { return 10000; }

const char *dpia_last_error_message(void) { return g_err.c_str(); }

size_t dpia_dot_workspace_size(int64_t n, const dpia_reduce_strategy *st) {
  ReducePlan pl;
  std::string saved = g_err;
  dpia_status rc = plan_reduce("dpia_dot_workspace_size", n, st, true, true, true, &pl);
  if (rc) return 0;
  g_err = saved;
  return (size_t)reduce_ws_bytes(pl);
}

dpia_status dpia_dot_f32(const float *x, const float *y, int64_t n, const dpia_reduce_strategy *st,
                         float *out, void *ws, size_t ws_bytes, dpia_stream_t stream) {
  return run_reduce("dpia_dot_f32", ReduceOp::DotF32, x, y, n, 4, st, out, 4, ws, ws_bytes, stream);
}

dpia_status dpia_dot_i32(const int32_t *x, const int32_t *y, int64_t n, const dpia_reduce_strategy *st,
                         int64_t *out, void *ws, size_t ws_bytes, dpia_stream_t stream) {
  return run_reduce("dpia_dot_i32", ReduceOp::DotI32, x, y, n, 4, st, out, 8, ws, ws_bytes, stream);
}

dpia_status dpia_asum_f32(const float *x, int64_t n, const dpia_reduce_strategy *st, float *out,
                          void *ws, size_t ws_bytes, dpia_stream_t stream) {
  return run_reduce("dpia_asum_f32", ReduceOp::AsumF32, x, nullptr, n, 4, st, out, 4, ws, ws_bytes, stream);
}

dpia_status dpia_scal_f32(float a, const float *x, float *y, int64_t n, int32_t vec, dpia_stream_t stream) {
  const char *fn = "dpia_scal_f32";
  g_err.clear();
  if (n < 0) return fail(DPIA_ERR_SHAPE, "%s: negative length", fn);
  if (!(vec == 1 || vec == 2 || vec == 4 || vec == 8 || vec == 16))
    return fail(DPIA_ERR_STRATEGY, "%s: vec=%d must be 1, 2, 4, 8 or 16", fn, vec);
  if (n == 0) return DPIA_OK;
  if (!x || !y) return fail(DPIA_ERR_NULL, "%s: x or y is NULL", fn);
  if (!aligned(x, vec_align(vec)) || !aligned(y, vec_align(vec)))
    return fail(DPIA_ERR_ALIGN, "%s: x and y must be %lld-byte aligned for vec=%d", fn,
                (long long)vec_align(vec), vec);
  if (x != y && overlap(x, n * 4, y, n * 4))
    return fail(DPIA_ERR_ALIAS, "%s: y partially overlaps x (only y == x is allowed)", fn);
  return cuda_status(launch_scal(a, x, y, n, vec, reinterpret_cast<cudaStream_t>(stream)), fn);
}

dpia_status dpia_dot_bwd_f32(const float *x, const float *y, const float *g, int64_t n, float *dx,
                             float *dy, dpia_stream_t stream) {
  const char *fn = "dpia_dot_bwd_f32";
  g_err.clear();
  if (n < 0) return fail(DPIA_ERR_SHAPE, "%s: negative length", fn);
  if (!g) return fail(DPIA_ERR_NULL, "%s: g is NULL", fn);
  if (n == 0 || (!dx && !dy)) return DPIA_OK;
  if (!x || !y) return fail(DPIA_ERR_NULL, "%s: x or y is NULL", fn);
  if (!aligned(x, 16) || !aligned(y, 16) || (dx && !aligned(dx, 16)) || (dy && !aligned(dy, 16)))
    return fail(DPIA_ERR_ALIGN, "%s: x, y, dx, dy must be 16-byte aligned", fn);
  if (!aligned(g, 4)) return fail(DPIA_ERR_ALIGN, "%s: g must be 4-byte aligned", fn);
  const int64_t b = n * 4;
  const void *ins[3] = {x, y, g};
  const int64_t insz[3] = {b, b, 4};
  float *outs[2] = {dx, dy};
  for (float *o : outs)
    for (int i = 0; i < 3; ++i)
      if (overlap(o, b, ins[i], insz[i])) return fail(DPIA_ERR_ALIAS, "%s: an output overlaps an input", fn);
  if (overlap(dx, b, dy, b)) return fail(DPIA_ERR_ALIAS, "%s: dx overlaps dy", fn);
  return cuda_status(launch_dot_bwd(x, y, g, n, dx, dy, reinterpret_cast<cudaStream_t>(stream)), fn);
}

dpia_status dpia_gemv_f32(const float *A, int64_t M, int64_t N, int64_t lda, const float *x, float *y,
                          const dpia_reduce_strategy *st, dpia_stream_t stream) {
  const char *fn = "dpia_gemv_f32";
  g_err.clear();
  if (M < 0 || N < 0) return fail(DPIA_ERR_SHAPE, "%s: negative shape", fn);
  if (lda < (N > 1 ? N : 1)) return fail(DPIA_ERR_SHAPE, "%s: lda=%lld < N=%lld", fn, (long long)lda, (long long)N);
  ReducePlan pl;
  dpia_status rc = plan_reduce(fn, N, st, true, false, false, &pl);
  if (rc) return rc;
  if (pl.level == ChunkLevel::Grid)
    return fail(DPIA_ERR_UNSUPPORTED, "%s: rows at GRID level (a thread per row) are not implemented", fn);
  if (M == 0) return DPIA_OK;
  if (!y) return fail(DPIA_ERR_NULL, "%s: y is NULL", fn);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (N > 0 && (!A || !x)) return fail(DPIA_ERR_NULL, "%s: A or x is NULL", fn);
  const int64_t abytes = ((M - 1) * lda + N) * 4;
  if (overlap(y, M * 4, A, N > 0 ? abytes : 0) || overlap(y, M * 4, x, N * 4))
    return fail(DPIA_ERR_ALIAS, "%s: y overlaps A or x", fn);
  if (N == 0) return cuda_status(cudaMemsetAsync(y, 0, (size_t)M * 4, s), fn);
  const int64_t va = vec_align(pl.V);
  if (!aligned(A, va) || !aligned(x, va) || (lda * 4) % va != 0)
    return fail(DPIA_ERR_ALIGN, "%s: A, x and lda*4 must be %lld-byte aligned for vec=%d", fn, (long long)va, pl.V);
  if (!aligned(y, 4)) return fail(DPIA_ERR_ALIGN, "%s: y must be 4-byte aligned", fn);
  GemvLaunch p;
  p.A = A;
  p.M = M;
  p.N = N;
  p.lda = lda;
  p.x = x;
  p.y = y;
  p.s = pl.s;
  p.Crow = pl.C;
  p.Rc = pl.Rc;
  p.step = pl.step;
  p.tstride = pl.tstride;
  p.Tc = pl.Tc;
  return cuda_status(launch_gemv(pl.compensated, pl.V, pl.level, pl.threads, pl.grid, p, s), fn);
}

size_t dpia_gemv_bwd_workspace_size(int64_t M, int64_t N, int64_t row_split) {
  if (M < 0 || N < 0 || row_split <= 0) return 0;
  const int64_t Cr = (M + row_split - 1) / row_split;
  const int64_t counters = round_up(((N + 31) / 32) * 4, 128);
  return (size_t)(kCounterBytes + counters + round_up(Cr * round_up(N, 4) * 4, 128));
}

dpia_status dpia_gemv_bwd_f32(const float *A, int64_t M, int64_t N, int64_t lda, const float *x,
                              const float *dy, float *dx, float *dA, int64_t ldda, int64_t row_split,
                              void *ws, size_t ws_bytes, dpia_stream_t stream) {
  const char *fn = "dpia_gemv_bwd_f32";
  g_err.clear();
  if (M < 0 || N < 0) return fail(DPIA_ERR_SHAPE, "%s: negative shape", fn);
  if (lda < (N > 1 ? N : 1)) return fail(DPIA_ERR_SHAPE, "%s: lda < N", fn);
  if (dA && ldda < (N > 1 ? N : 1)) return fail(DPIA_ERR_SHAPE, "%s: ldda < N", fn);
  if (row_split <= 0) return fail(DPIA_ERR_STRATEGY, "%s: row_split=%lld must be positive", fn, (long long)row_split);
  const int64_t Cr = (M + row_split - 1) / row_split;
  if (Cr > 65535) return fail(DPIA_ERR_STRATEGY, "%s: %lld row chunks exceed 65535 (raise row_split)", fn, (long long)Cr);
  if (N == 0 || (!dx && !dA)) return DPIA_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!dy) return fail(DPIA_ERR_NULL, "%s: dy is NULL", fn);
  const int64_t abytes = M > 0 ? ((M - 1) * lda + N) * 4 : 0;
  if (M > 0 && !A && dx) return fail(DPIA_ERR_NULL, "%s: A is NULL", fn);
  if (dA && !x) return fail(DPIA_ERR_NULL, "%s: x is NULL", fn);
  const int64_t dabytes = M > 0 ? ((M - 1) * ldda + N) * 4 : 0;
  if (dx) {
    if (overlap(dx, N * 4, A, abytes) || overlap(dx, N * 4, dy, M * 4) || overlap(dx, N * 4, x, N * 4) ||
        overlap(dx, N * 4, dA, dabytes))
      return fail(DPIA_ERR_ALIAS, "%s: dx overlaps an input or dA", fn);
    if (!aligned(dx, 4)) return fail(DPIA_ERR_ALIGN, "%s: dx must be 4-byte aligned", fn);
  }
  if (dA && (overlap(dA, dabytes, A, abytes) || overlap(dA, dabytes, dy, M * 4) || overlap(dA, dabytes, x, N * 4)))
    return fail(DPIA_ERR_ALIAS, "%s: dA overlaps an input", fn);
  if (dA && M > 0) {
    if (!aligned(dA, 4) || !aligned(x, 4)) return fail(DPIA_ERR_ALIGN, "%s: dA and x must be 4-byte aligned", fn);
    const int vec = aligned(dA, 16) && (ldda * 4) % 16 == 0 && aligned(x, 16);
    cudaError_t e = launch_outer(x, dy, M, N, dA, ldda, vec, s);
    if (e != cudaSuccess) return cuda_status(e, fn);
  }
  if (dx) {
    if (M == 0) return cuda_status(cudaMemsetAsync(dx, 0, (size_t)N * 4, s), fn);
    if (!aligned(A, 4)) return fail(DPIA_ERR_ALIGN, "%s: A must be 4-byte aligned", fn);
    const int64_t need = (int64_t)dpia_gemv_bwd_workspace_size(M, N, row_split);
    if (!ws || (int64_t)ws_bytes < need)
      return fail(DPIA_ERR_WORKSPACE, "%s: workspace of %zu bytes, %lld needed", fn, ws_bytes, (long long)need);
    if (!aligned(ws, 128)) return fail(DPIA_ERR_ALIGN, "%s: workspace must be 128-byte aligned", fn);
    if (overlap(ws, need, A, abytes) || overlap(ws, need, dy, M * 4) || overlap(ws, need, dx, N * 4) ||
        overlap(ws, need, dA, dabytes) || overlap(ws, need, x, N * 4))
      return fail(DPIA_ERR_ALIAS, "%s: workspace overlaps an argument", fn);
    GemvBwdLaunch p;
    p.A = A;
    p.M = M;
    p.N = N;
    p.lda = lda;
    p.dy = dy;
    p.dx = dx;
    p.Rs = row_split;
    p.Cr = Cr;
    p.Npad = round_up(N, 4);
    const int64_t counters = round_up(((N + 31) / 32) * 4, 128);
    p.counters = reinterpret_cast<unsigned *>(static_cast<char *>(ws) + kCounterBytes);
    p.partials = reinterpret_cast<float *>(static_cast<char *>(ws) + kCounterBytes + counters);
    p.vec = aligned(A, 16) && (lda * 4) % 16 == 0;
    return cuda_status(launch_gemv_bwd_dx(p, s), fn);
  }
  return DPIA_OK;
}

}  // extern "C"
