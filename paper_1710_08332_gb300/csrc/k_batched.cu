// Batches of uneven dot and GEMV instances: host planner and the two
// persistent kernels (forward, backward).
//
// The planner (plain host C++) validates every instance, turns its strategy
// into launch constants (the same ones the single-instance kernels use) and
// lists the work items -- dot chunks and groups of GEMV rows for the forward
// (taken by blocks); ranges of dot gradients, groups of dA rows and (column
// tile, row chunk) pieces of dx for the backward (taken by single warps) -- in
// instance order, with the running sum of their byte costs. Items are either
// dealt round robin, longest first (schedule 0), or each block (forward) or
// warp (backward) takes the contiguous run of items whose costs fall in its
// equal share of the total (schedule 1, a binary search over the running sums),
// so the work is balanced to within one item, or (schedule 2) sorted longest
// first, the forward's dealt round robin and the backward's taken one at a
// time from a counter in the workspace by whichever warp is free (the last
// warp to finish puts the counter back to zero; nothing waits for anything).
//
// Every value is computed exactly as the single-instance kernels compute it
// (same fold order per element, same trees, same second levels), so each
// instance's result is bit-identical to the oracle's evaluation of its own
// strategy.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/dpia.h"
#include "device_common.cuh"
#include "kernels.h"

namespace dpia {

int resident_blocks(const void *kernel, int threads);
void set_last_error(const char *fmt, ...);

namespace {

constexpr uint32_t kPlanMagic = 0x44504942u;  // "DPIB"
constexpr int V = 4;

enum ItemType : int32_t { DOT_CHUNK = 0, GEMV_ROWS = 1, DOT_BWD = 2, GEMV_DA = 3, GEMV_DX = 4 };

struct PlanHeader {
  uint32_t magic;
  int32_t threads;
  int32_t n_dots, n_gemvs;
  int64_t n_fwd, n_bwd;
  int64_t dots_off, gemvs_off, fwd_off, bwd_off;  // byte offsets inside the plan
  int64_t fwd_cost_off, bwd_cost_off;             // running sums of item costs (int64 per item)
  int64_t fwd_total, bwd_total;
  int32_t schedule, pad_;
  int64_t dot_partials, dx_partials;              // floats of workspace
  int64_t dx_tiles;                               // dx tile counters
  int64_t xs_extent, as_extent, gx_extent, gy_extent;  // elements the packed arrays must hold
  int64_t bwd_elems_per_item, rows_per_item, da_rows_per_item;
  int64_t total_bytes;
};

struct DotDesc {
  int64_t off, n, s, C, Rc, step, tstride, part_base;
  int32_t second_tree, T2, pad0, pad1;
};

struct GemvDesc {
  int64_t a_off, x_off, y_off, M, N, lda;
  int64_t s, Crow, Rc, step, tstride;  // forward row strategy (a warp per row)
  int64_t Rs, Cr, Npad, part_base;     // backward dx: rows per chunk, chunks, padded width, partial offset
  int32_t tiles, tile_cnt;             // dx column tiles (kDxTile columns each), index of the first tile's counter
  int32_t da_rows, pad0;               // rows of a dA item
};

struct Item {
  int32_t type, inst;
  int64_t a;
};

struct WsLayout {
  unsigned *sched;  // schedule 2: [2] the next backward item, [3] backward warps done ([0], [1] unused)
  unsigned *dot_cnt;
  unsigned *dx_cnt;
  float *dot_part;
  float *dx_part;
};

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }
bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

int64_t ws_bytes_of(const PlanHeader &h) {
  return 128 + round_up((int64_t)h.n_dots * 4, 128) + round_up(h.dx_tiles * 4, 128) +
         round_up(h.dot_partials * 4, 128) + round_up(h.dx_partials * 4, 128);
}

WsLayout ws_layout(const PlanHeader &h, void *ws) {
  char *p = static_cast<char *>(ws) + 128;
  WsLayout L;
  L.sched = static_cast<unsigned *>(ws);  // the first 128 bytes: the dynamic schedule's counters
  L.dot_cnt = reinterpret_cast<unsigned *>(p);
  p += round_up((int64_t)h.n_dots * 4, 128);
  L.dx_cnt = reinterpret_cast<unsigned *>(p);
  p += round_up(h.dx_tiles * 4, 128);
  L.dot_part = reinterpret_cast<float *>(p);
  p += round_up(h.dot_partials * 4, 128);
  L.dx_part = reinterpret_cast<float *>(p);
  return L;
}

struct Built {
  PlanHeader h;
  std::vector<DotDesc> dots;
  std::vector<GemvDesc> gemvs;
  std::vector<Item> fwd, bwd;
  std::vector<int64_t> fwd_cost, bwd_cost;  // running sums
};

// Backward items are warp-sized: a warp takes one at a time, with no block
// barrier anywhere in the backward kernel (its warps never wait for each other).
//   dot gradient: kDotBwdElems elements (64 KiB of traffic);
//   dA: rows of one GEMV, enough that the item writes about kDaItemBytes
//       (a power of two, 1..kDaMaxRows rows), a lane per column group of 4;
//   dx: one chunk of row_split rows times a tile of kDxTile columns, a lane per
//       column group of 4; the last warp to finish a tile's chunks (ticket)
//       folds that tile's chunk partials in chunk order.
constexpr int64_t kDotBwdElems = 4096;

constexpr int kDaMaxRows = 64;
constexpr int64_t kDaItemBytes = 64 * 1024;
constexpr int64_t kDxTile = 128;

int64_t da_rows_for(int64_t N) {
  int64_t r = 1;
  while (r < kDaMaxRows && r * N * 4 < kDaItemBytes) r *= 2;
  return r;
}

// Validate and plan; returns DPIA_OK and fills b.
dpia_status build_plan(int32_t nd, const dpia_dot_instance *dots, int32_t ng, const dpia_gemv_instance *gemvs,
                       const dpia_batch_options *opt, Built &b) {
  if (!opt) {
    set_last_error("dpia_batch_plan: options are NULL");
    return DPIA_ERR_NULL;
  }
  const int32_t T = opt->threads;
  if (opt->schedule < 0 || opt->schedule > 2) {
    set_last_error("dpia_batch_plan: schedule must be 0, 1 or 2");
    return DPIA_ERR_STRATEGY;
  }
  if (nd < 0 || ng < 0) {
    set_last_error("dpia_batch_plan: negative instance count");
    return DPIA_ERR_SHAPE;
  }
  if ((nd > 0 && !dots) || (ng > 0 && !gemvs)) {
    set_last_error("dpia_batch_plan: instance array is NULL");
    return DPIA_ERR_NULL;
  }
  if (!is_pow2(T) || T < 32 || T > 256) {
    set_last_error("dpia_batch_plan: threads=%d must be a power of two in [32, 256]", T);
    return DPIA_ERR_STRATEGY;
  }
  PlanHeader &h = b.h;
  std::memset(&h, 0, sizeof h);
  h.magic = kPlanMagic;
  h.threads = T;
  h.n_dots = nd;
  h.n_gemvs = ng;
  h.schedule = opt->schedule;
  h.rows_per_item = T / 32 * 4;  // a warp per row, four rows per warp
  h.da_rows_per_item = kDaMaxRows;
  h.bwd_elems_per_item = kDotBwdElems;
  std::vector<std::pair<int64_t, Item>> fwd, bwd;  // (cost, item)
  for (int32_t i = 0; i < nd; ++i) {
    const dpia_dot_instance &in = dots[i];
    const dpia_reduce_strategy &st = in.st;
    if (in.n < 0 || in.off < 0 || in.off % 4) {
      set_last_error("dpia_batch_plan: dot %d: bad offset %lld or length %lld (offsets must be multiples of 4)", i,
                     (long long)in.off, (long long)in.n);
      return DPIA_ERR_SHAPE;
    }
    if (st.map_level != DPIA_LVL_BLOCK || st.inner_level != DPIA_LVL_THREAD || st.threads != T || st.vec != V ||
        st.compensated || st.stage != DPIA_STAGE_PRIVATE || st.split <= 0 || st.split % ((int64_t)T * V) ||
        (st.thread_map != DPIA_MAP_INTERLEAVED && st.thread_map != DPIA_MAP_CONTIG) ||
        (st.second == DPIA_SECOND_TREE && (!is_pow2(st.threads2) || st.threads2 > T)) ||
        (st.second != DPIA_SECOND_SEQ && st.second != DPIA_SECOND_TREE)) {
      set_last_error("dpia_batch_plan: dot %d: strategy must be BLOCK/THREAD, threads %d, vec 4, split a multiple "
                     "of %d, plain (not compensated), stage PRIVATE, threads2 a power of two <= threads", i, T, T * V);
      return DPIA_ERR_STRATEGY;
    }
    DotDesc d{};
    d.off = in.off;
    d.n = in.n;
    d.s = st.split;
    d.C = in.n > 0 ? (in.n + d.s - 1) / d.s : 1;  // an empty dot is one all-identity chunk: +0
    d.Rc = d.s / ((int64_t)T * V);
    if (st.thread_map == DPIA_MAP_INTERLEAVED) {
      d.step = (int64_t)T * V;
      d.tstride = V;
    } else {
      d.step = V;
      d.tstride = d.Rc * V;
    }
    d.part_base = h.dot_partials;
    d.second_tree = st.second == DPIA_SECOND_TREE;
    d.T2 = d.second_tree ? st.threads2 : 1;
    h.dot_partials += d.C;
    h.xs_extent = std::max(h.xs_extent, in.off + in.n);
    b.dots.push_back(d);
    for (int64_t c = 0; c < d.C; ++c) fwd.push_back({8 * d.s, Item{DOT_CHUNK, i, c}});
    for (int64_t e = 0; e < in.n; e += h.bwd_elems_per_item) bwd.push_back({16 * h.bwd_elems_per_item, Item{DOT_BWD, i, e}});
  }
  for (int32_t i = 0; i < ng; ++i) {
    const dpia_gemv_instance &in = gemvs[i];
    const dpia_reduce_strategy &st = in.st;
    if (in.M < 0 || in.N < 1 || in.lda < in.N || in.lda % 4 || in.a_off < 0 || in.a_off % 4 || in.x_off < 0 ||
        in.x_off % 4 || in.y_off < 0 || in.row_split < 1) {
      set_last_error("dpia_batch_plan: gemv %d: bad shape or offsets (offsets and lda must be multiples of 4, "
                     "N >= 1, row_split >= 1)", i);
      return DPIA_ERR_SHAPE;
    }
    if (st.map_level != DPIA_LVL_WARP || st.inner_level != DPIA_LVL_THREAD || st.vec != V || st.compensated ||
        st.stage != DPIA_STAGE_PRIVATE ||
        st.split <= 0 || st.split % (32 * V) || st.second != DPIA_SECOND_SEQ ||
        (st.thread_map != DPIA_MAP_INTERLEAVED && st.thread_map != DPIA_MAP_CONTIG)) {
      set_last_error("dpia_batch_plan: gemv %d: row strategy must be WARP/THREAD, vec 4, split a multiple of 128, "
                     "SEQ second level, plain", i);
      return DPIA_ERR_STRATEGY;
    }
    GemvDesc g{};
    g.a_off = in.a_off;
    g.x_off = in.x_off;
    g.y_off = in.y_off;
    g.M = in.M;
    g.N = in.N;
    g.lda = in.lda;
    g.s = st.split;
    g.Crow = (in.N + g.s - 1) / g.s;
    g.Rc = g.s / (32 * V);
    if (st.thread_map == DPIA_MAP_INTERLEAVED) {
      g.step = 32 * V;
      g.tstride = V;
    } else {
      g.step = V;
      g.tstride = g.Rc * V;
    }
    g.Rs = in.row_split;
    g.Cr = in.M > 0 ? (in.M + g.Rs - 1) / g.Rs : 1;  // no rows: one empty chunk, so dx = +0 is written
    g.Npad = round_up(in.N, 4);
    g.part_base = h.dx_partials;
    g.tiles = (int32_t)((in.N + kDxTile - 1) / kDxTile);
    g.da_rows = (int32_t)da_rows_for(in.N);
    g.tile_cnt = (int32_t)h.dx_tiles;
    h.dx_partials += g.Cr * g.Npad;
    h.dx_tiles += g.tiles;
    h.as_extent = std::max(h.as_extent, in.M > 0 ? in.a_off + (in.M - 1) * in.lda + in.N : in.a_off);
    h.gx_extent = std::max(h.gx_extent, in.x_off + in.N);
    h.gy_extent = std::max(h.gy_extent, in.y_off + in.M);
    b.gemvs.push_back(g);
    for (int64_t r = 0; r < in.M; r += h.rows_per_item)
      fwd.push_back({4 * std::min<int64_t>(h.rows_per_item, in.M - r) * in.N, Item{GEMV_ROWS, i, r}});
    for (int64_t r = 0; r < in.M; r += g.da_rows)
      bwd.push_back({4 * std::min<int64_t>(g.da_rows, in.M - r) * in.N, Item{GEMV_DA, i, r}});
    for (int64_t t = 0; t < g.tiles; ++t)
      for (int64_t k = 0; k < g.Cr; ++k) {
        const int64_t rows = std::min<int64_t>(g.Rs, std::max<int64_t>(in.M - k * g.Rs, 1));
        bwd.push_back({4 * rows * std::min<int64_t>(kDxTile, in.N - t * kDxTile), Item{GEMV_DX, i, t * g.Cr + k}});
      }
  }
  // schedule 0: longest first, dealt round robin at launch; schedule 1: instance
  // order, with the running sums of the costs each block finds its share by
  if (h.schedule != 1) {  // 0 and 2: longest first
    auto by_cost = [](const std::pair<int64_t, Item> &x, const std::pair<int64_t, Item> &y) {
      return x.first > y.first;
    };
    std::stable_sort(fwd.begin(), fwd.end(), by_cost);
    std::stable_sort(bwd.begin(), bwd.end(), by_cost);
  }
  int64_t acc = 0;
  for (auto &p : fwd) {
    b.fwd.push_back(p.second);
    acc += std::max<int64_t>(p.first, 1);
    b.fwd_cost.push_back(acc);
  }
  h.fwd_total = acc;
  acc = 0;
  for (auto &p : bwd) {
    b.bwd.push_back(p.second);
    acc += std::max<int64_t>(p.first, 1);
    b.bwd_cost.push_back(acc);
  }
  h.bwd_total = acc;
  h.n_fwd = (int64_t)b.fwd.size();
  h.n_bwd = (int64_t)b.bwd.size();
  if (h.schedule == 2 && h.n_bwd > (int64_t)1 << 30) {  // the 32-bit counter also counts every warp's last grab
    set_last_error("dpia_batch_plan: schedule 2 takes at most 2^30 backward items (%lld)", (long long)h.n_bwd);
    return DPIA_ERR_SHAPE;
  }
  int64_t off = round_up(sizeof(PlanHeader), 128);
  h.dots_off = off;
  off += round_up((int64_t)b.dots.size() * sizeof(DotDesc), 128);
  h.gemvs_off = off;
  off += round_up((int64_t)b.gemvs.size() * sizeof(GemvDesc), 128);
  h.fwd_off = off;
  off += round_up(h.n_fwd * (int64_t)sizeof(Item), 128);
  h.bwd_off = off;
  off += round_up(h.n_bwd * (int64_t)sizeof(Item), 128);
  h.fwd_cost_off = off;
  off += round_up(h.n_fwd * 8, 128);
  h.bwd_cost_off = off;
  off += round_up(h.n_bwd * 8, 128);
  h.total_bytes = off;
  return DPIA_OK;
}

struct FwdArgs {
  const char *plan;
  const float *xs, *ys;
  float *dot_out;
  const float *As, *gx;
  float *gy;
  WsLayout ws;
};

struct BwdArgs {
  const char *plan;
  const float *xs, *ys, *dot_g;
  float *dxs, *dys;
  const float *As, *gx, *gdy;
  float *dAs, *dgx;
  WsLayout ws;
};

// The contiguous run of items whose start cost lies in this block's share
// [total*b/G, total*(b+1)/G) of the running sums `end` (item i starts at
// end[i-1], item 0 at 0). Computed by thread 0, broadcast through shared memory.
__device__ __forceinline__ void block_item_range(const int64_t *end, int64_t n, int64_t total, int64_t *lo_hi) {
  if (threadIdx.x == 0) {
    auto first_at = [&](int64_t c) -> int64_t {  // first i with start(i) >= c
      if (c <= 0) return 0;
      int64_t lo = 0, hi = n;  // first j with end[j] >= c, then i = j + 1
      while (lo < hi) {
        const int64_t mid = (lo + hi) / 2;
        if (end[mid] >= c) hi = mid; else lo = mid + 1;
      }
      return lo + 1 < n ? lo + 1 : n;
    };
    const int64_t G = gridDim.x, b = blockIdx.x;
    lo_hi[0] = first_at(total / G * b + total % G * b / G);
    lo_hi[1] = b + 1 == G ? n : first_at(total / G * (b + 1) + total % G * (b + 1) / G);
  }
  __syncthreads();
}

constexpr int kSeqStage = 1024;

// The forward kernel runs at 3 blocks of 256 per SM (85 registers): its GEMV
// rows keep 32 items per lane in flight, which measured faster than 4 blocks
// with 16 (64 registers). The backward kernel keeps 4 blocks (64 registers).

// Rows of an interleaved GEMV whose one chunk gives each lane at most RC
// vectors (N <= 128 RC): the warp takes 8 / RC of its rows at once, so that up
// to eight 128-bit loads per lane are in flight as for wider rows, then folds
// each row exactly as thread_fold does (lane vectors in r order, items at or
// past N as the identity (0, 0), the lane's four sums from zero in lane
// order), the warp tree, and the row's one chunk added to zero.
template <int RC>
__device__ __forceinline__ void gemv_rows_narrow(const float *A, int64_t lda, const float *x, float *y, int64_t N,
                                                 int64_t r0, int64_t r_end, int64_t stride, int lane) {
  constexpr int G = 8 / RC;
  constexpr bool HOLD_X = RC <= 4;  // wider rows re-read x (cached) inside the fold: fewer registers
  auto x_at = [&](int q) {
    const int64_t e0 = 4 * lane + 128 * q;
    float4 v;
    if (e0 + 4 <= N) {
      v = ld_cached_v4(x + e0);
    } else {
      v.x = e0 < N ? x[e0] : 0.0f;
      v.y = e0 + 1 < N ? x[e0 + 1] : 0.0f;
      v.z = e0 + 2 < N ? x[e0 + 2] : 0.0f;
      v.w = e0 + 3 < N ? x[e0 + 3] : 0.0f;
    }
    return v;
  };
  float4 xv[HOLD_X ? RC : 1];
  if constexpr (HOLD_X) {
#pragma unroll
    for (int q = 0; q < RC; ++q) xv[q] = x_at(q);
  }
  for (int64_t r = r0; r < r_end; r += stride * G) {
    float4 av[G][RC];
#pragma unroll
    for (int k = 0; k < G; ++k) {
      const int64_t row = r + k * stride;
      const float *p = A + (row < r_end ? row : r0) * lda;
#pragma unroll
      for (int q = 0; q < RC; ++q) {
        const int64_t e0 = 4 * lane + 128 * q;
        if (e0 + 4 <= N) {
          av[k][q] = ld_stream_v4(p + e0);
        } else {
          av[k][q].x = e0 < N ? p[e0] : 0.0f;
          av[k][q].y = e0 + 1 < N ? p[e0 + 1] : 0.0f;
          av[k][q].z = e0 + 2 < N ? p[e0 + 2] : 0.0f;
          av[k][q].w = e0 + 3 < N ? p[e0 + 3] : 0.0f;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < G; ++k) {
      float acc[4] = {SumF32::zero(), SumF32::zero(), SumF32::zero(), SumF32::zero()};
#pragma unroll
      for (int q = 0; q < RC; ++q) {
        const float4 xq = HOLD_X ? xv[HOLD_X ? q : 0] : x_at(q);
        acc[0] = SumF32::step(acc[0], DotF32::elem(av[k][q].x, xq.x));
        acc[1] = SumF32::step(acc[1], DotF32::elem(av[k][q].y, xq.y));
        acc[2] = SumF32::step(acc[2], DotF32::elem(av[k][q].z, xq.z));
        acc[3] = SumF32::step(acc[3], DotF32::elem(av[k][q].w, xq.w));
      }
      float t = SumF32::zero();
#pragma unroll
      for (int v = 0; v < 4; ++v) t = SumF32::combine(t, acc[v]);
      t = warp_tree<SumF32>(t, 32);
      const int64_t row = r + k * stride;
      if (lane == 0 && row < r_end) y[row] = __fadd_rn(0.0f, t);
    }
  }
}

__global__ void __launch_bounds__(256, 3) batch_fwd_kernel(const FwdArgs a) {
  __shared__ float sm[32];
  __shared__ float stage[kSeqStage];
  __shared__ int last;
  __shared__ int64_t range[2];
  const PlanHeader *h = reinterpret_cast<const PlanHeader *>(a.plan);
  const DotDesc *__restrict__ dots = reinterpret_cast<const DotDesc *>(a.plan + h->dots_off);
  const GemvDesc *__restrict__ gemvs = reinterpret_cast<const GemvDesc *>(a.plan + h->gemvs_off);
  const Item *__restrict__ items = reinterpret_cast<const Item *>(a.plan + h->fwd_off);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  int64_t i0 = blockIdx.x, i1 = h->n_fwd, istep = gridDim.x;
  if (h->schedule == 1) {
    block_item_range(reinterpret_cast<const int64_t *>(a.plan + h->fwd_cost_off), h->n_fwd, h->fwd_total, range);
    i0 = range[0];
    i1 = range[1];
    istep = 1;
  }
  // schedule 2 deals the forward's items round robin too: taking each from a
  // counter costs a block two barriers and an atomic per item (6.65 against
  // 6.33 ms on the bench batch)
  for (int64_t it = i0; it < i1; it += istep) {
    const Item w = items[it];
    // descriptors are read field by field through the read-only cache (held
    // whole in registers they would cap the kernel's occupancy)
    const DotDesc &d = dots[w.inst];
    const GemvDesc &g = gemvs[w.inst];
    if (w.type == DOT_CHUNK) {
      const float *x = a.xs + d.off, *y = a.ys + d.off;
      const int64_t c = w.a;
      const bool full = (c + 1) * d.s <= d.n;
      float v = thread_fold<DotF32, SumF32, V, false, 2, true>(x, y, d.n, c * d.s + t * d.tstride, d.Rc, d.step,
                                                              full);
      v = block_tree<SumF32>(v, blockDim.x, sm);
      if (t == 0) a.ws.dot_part[d.part_base + c] = v;
      __threadfence();
      __syncthreads();
      if (t == 0) {
        const unsigned ticket = atomicAdd(a.ws.dot_cnt + w.inst, 1u);
        __threadfence();
        last = ticket == d.C - 1;
      }
      __syncthreads();
      if (last) {  // this block finished the instance's last chunk: second level
        const float *part = a.ws.dot_part + d.part_base;
        float res = 0.0f;
        if (!d.second_tree) {  // stage the partials with one parallel load, fold them in order
          for (int64_t k0 = 0; k0 < d.C; k0 += kSeqStage) {
            const int cnt = d.C - k0 < kSeqStage ? (int)(d.C - k0) : kSeqStage;
            for (int i = t; i < cnt; i += blockDim.x) stage[i] = __ldcg(part + k0 + i);
            __syncthreads();
            if (t == 0)
              for (int i = 0; i < cnt; ++i) res = __fadd_rn(res, stage[i]);
            __syncthreads();
          }
        } else {
          float acc = 0.0f;
          if (t < d.T2) {
            const int64_t R2 = ceil_div(d.C, d.T2);
            for (int64_t r = 0; r < R2; ++r) {
              const int64_t i = r * d.T2 + t;
              acc = __fadd_rn(acc, i < d.C ? __ldcg(part + i) : 0.0f);
            }
          }
          res = block_tree<SumF32>(acc, d.T2, sm);
        }
        if (t == 0) {
          a.dot_out[w.inst] = res;
          a.ws.dot_cnt[w.inst] = 0u;
        }
      }
      __syncthreads();
    } else {  // GEMV_ROWS: a warp per row, the row's chunks folded in order
      const int64_t warps = blockDim.x >> 5;
      const int64_t r_end = w.a + h->rows_per_item < g.M ? w.a + h->rows_per_item : g.M;
      const float *x = a.gx + g.x_off;
      if (g.Crow == 1 && g.Rc >= 2 && g.Rc <= 8 && g.step == 32 * V) {
        const float *A0 = a.As + g.a_off;
        float *y = a.gy + g.y_off;
        // fewer vectors fold as four (or eight): the others lie past N, identity items
        // (+0 added to a sum that starts at +0 and so is never -0: the same bits)
        if (g.Rc <= 4) gemv_rows_narrow<4>(A0, g.lda, x, y, g.N, w.a + warp, r_end, warps, lane);
        else gemv_rows_narrow<8>(A0, g.lda, x, y, g.N, w.a + warp, r_end, warps, lane);
      } else
      for (int64_t r = w.a + warp; r < r_end; r += warps) {
        const float *row = a.As + g.a_off + r * g.lda;
        float acc = 0.0f;
        for (int64_t c = 0; c < g.Crow; ++c) {
          const bool full = (c + 1) * g.s <= g.N;
          float v = thread_fold<DotF32, SumF32, V, true, 1, true>(row, x, g.N, c * g.s + lane * g.tstride, g.Rc,
                                                                  g.step, full);
          v = warp_tree<SumF32>(v, 32);
          if (lane == 0) acc = __fadd_rn(acc, v);
        }
        if (lane == 0) a.gy[g.y_off + r] = acc;
      }
    }
  }
}

// The contiguous run of items whose start cost lies in this warp's share of the
// running sums `end` (the warp version of block_item_range; lane 0 searches,
// the warp shares the result).
__device__ __forceinline__ void warp_item_range(const int64_t *end, int64_t n, int64_t total, int64_t w, int64_t W,
                                                int64_t *lo, int64_t *hi) {
  int64_t a = 0, b = 0;
  if ((threadIdx.x & 31) == 0) {
    auto first_at = [&](int64_t c) -> int64_t {
      if (c <= 0) return 0;
      int64_t l = 0, h = n;
      while (l < h) {
        const int64_t mid = (l + h) / 2;
        if (end[mid] >= c) h = mid; else l = mid + 1;
      }
      return l + 1 < n ? l + 1 : n;
    };
    a = first_at(total / W * w + total % W * w / W);
    b = w + 1 == W ? n : first_at(total / W * (w + 1) + total % W * (w + 1) / W);
  }
  *lo = __shfl_sync(0xffffffffu, a, 0);
  *hi = __shfl_sync(0xffffffffu, b, 0);
}

// Every warp works alone: no block barrier, so no warp idles while others of
// its block finish an item. 64 registers: four blocks of 256 per SM.
__global__ void __launch_bounds__(256, 4) batch_bwd_kernel(const BwdArgs a) {
  const PlanHeader *h = reinterpret_cast<const PlanHeader *>(a.plan);
  const DotDesc *__restrict__ dots = reinterpret_cast<const DotDesc *>(a.plan + h->dots_off);
  const GemvDesc *__restrict__ gemvs = reinterpret_cast<const GemvDesc *>(a.plan + h->gemvs_off);
  const Item *__restrict__ items = reinterpret_cast<const Item *>(a.plan + h->bwd_off);
  const int lane = threadIdx.x & 31;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int64_t i0 = wid, i1 = h->n_bwd, istep = nw;
  if (h->schedule == 1) {
    warp_item_range(reinterpret_cast<const int64_t *>(a.plan + h->bwd_cost_off), h->n_bwd, h->bwd_total, wid, nw,
                    &i0, &i1);
    istep = 1;
  }
  const bool dyn = h->schedule == 2;
  auto next_item = [&]() -> int64_t {  // schedule 2: the warp's next item from the shared counter
    unsigned v = 0;
    if (lane == 0) v = atomicAdd(a.ws.sched + 2, 1u);
    return (int64_t)__shfl_sync(0xffffffffu, v, 0);
  };
  if (dyn) i0 = next_item();
  for (int64_t it = i0; it < i1; it = dyn ? next_item() : it + istep) {
    const Item w = items[it];
    const DotDesc &d = dots[w.inst];
    const GemvDesc &g = gemvs[w.inst];
    if (w.type == DOT_BWD) {  // dx = g*y, dy = g*x over [e0, e1)
      const float gv = __ldg(a.dot_g + w.inst);
      const int64_t e0 = w.a;
      const int64_t e1 = e0 + kDotBwdElems < d.n ? e0 + kDotBwdElems : d.n;
      const float *x = a.xs + d.off, *y = a.ys + d.off;
      float *dx = a.dxs + d.off, *dy = a.dys + d.off;
      const int64_t v1 = e0 + (e1 - e0) / 4 * 4;
#pragma unroll 4
      for (int64_t e = e0 + 4 * lane; e < v1; e += 128) {
        const float4 yv = ld_stream_v4(y + e), xv = ld_stream_v4(x + e);
        st_stream_v4(dx + e, make_float4(__fmul_rn(gv, yv.x), __fmul_rn(gv, yv.y), __fmul_rn(gv, yv.z),
                                         __fmul_rn(gv, yv.w)));
        st_stream_v4(dy + e, make_float4(__fmul_rn(gv, xv.x), __fmul_rn(gv, xv.y), __fmul_rn(gv, xv.z),
                                         __fmul_rn(gv, xv.w)));
      }
      for (int64_t e = v1 + lane; e < e1; e += 32) {
        dx[e] = __fmul_rn(gv, y[e]);
        dy[e] = __fmul_rn(gv, x[e]);
      }
    } else if (w.type == GEMV_DA) {  // dA rows [r0, r1) = dy_r * x; a lane per column group of 4
      const float *x = a.gx + g.x_off;
      const float *dyv = a.gdy + g.y_off;
      const int64_t r0 = w.a, r1 = w.a + g.da_rows < g.M ? w.a + g.da_rows : g.M;
      const int nr = (int)(r1 - r0);  // at most kDaMaxRows = 64
      // the item's dy values, two per lane, handed to the store loop by shuffles:
      // no load waits between the stores
      const float dlo = lane < nr ? __ldg(dyv + r0 + lane) : 0.0f;
      const float dhi = lane + 32 < nr ? __ldg(dyv + r0 + 32 + lane) : 0.0f;
      const int64_t cgv = g.N / 4;  // full column groups
      float *base = a.dAs + g.a_off;
      float *rows = base + r0 * g.lda;
      for (int64_t jb = 0; jb < cgv; jb += 32) {  // every lane runs every trip (the shuffles)
        const int64_t j = jb + lane;
        const bool on = j < cgv;
        const float4 xv = on ? ld_cached_v4(x + 4 * j) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll 4
        for (int r = 0; r < nr; ++r) {
          const float dv = __shfl_sync(0xffffffffu, r < 32 ? dlo : dhi, r & 31);
          if (on)
            st_stream_v4(rows + r * g.lda + 4 * j, make_float4(__fmul_rn(dv, xv.x), __fmul_rn(dv, xv.y),
                                                              __fmul_rn(dv, xv.z), __fmul_rn(dv, xv.w)));
        }
      }
      if (4 * cgv < g.N)  // the ragged last columns, element by element
        for (int64_t q = lane; q < (r1 - r0) * (g.N - 4 * cgv); q += 32) {
          const int64_t r = r0 + q / (g.N - 4 * cgv), e = 4 * cgv + q % (g.N - 4 * cgv);
          base[r * g.lda + e] = __fmul_rn(__ldg(dyv + r), __ldg(x + e));
        }
    } else {  // GEMV_DX: (column tile, row chunk); a lane per column group of 4
      const int64_t tile = w.a / g.Cr, chunk = w.a % g.Cr;
      const int64_t j0 = tile * kDxTile + 4 * lane;
      const float *A = a.As + g.a_off;
      const float *dyv = a.gdy + g.y_off;
      if (j0 < g.N) {
        const int64_t r0 = chunk * g.Rs;
        const int64_t r1 = r0 + g.Rs < g.M ? r0 + g.Rs : g.M;
        float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (j0 + 4 <= g.N) {
          int64_t i = r0;
          for (; i + 8 <= r1; i += 8) {  // eight rows of loads in flight per lane
            float4 av[8];
            float dv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              av[u] = ld_stream_v4(A + (i + u) * g.lda + j0);
              dv[u] = __ldg(dyv + i + u);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              acc[0] = __fadd_rn(acc[0], __fmul_rn(av[u].x, dv[u]));
              acc[1] = __fadd_rn(acc[1], __fmul_rn(av[u].y, dv[u]));
              acc[2] = __fadd_rn(acc[2], __fmul_rn(av[u].z, dv[u]));
              acc[3] = __fadd_rn(acc[3], __fmul_rn(av[u].w, dv[u]));
            }
          }
          for (; i < r1; ++i) {
            const float4 av = ld_stream_v4(A + i * g.lda + j0);
            const float dv = __ldg(dyv + i);
            acc[0] = __fadd_rn(acc[0], __fmul_rn(av.x, dv));
            acc[1] = __fadd_rn(acc[1], __fmul_rn(av.y, dv));
            acc[2] = __fadd_rn(acc[2], __fmul_rn(av.z, dv));
            acc[3] = __fadd_rn(acc[3], __fmul_rn(av.w, dv));
          }
        } else {
          for (int64_t i = r0; i < r1; ++i) {
            const float dv = __ldg(dyv + i);
#pragma unroll
            for (int v = 0; v < 4; ++v)
              if (j0 + v < g.N) acc[v] = __fadd_rn(acc[v], __fmul_rn(A[i * g.lda + j0 + v], dv));
          }
        }
        float *part = a.ws.dx_part + g.part_base + chunk * g.Npad;
#pragma unroll
        for (int v = 0; v < 4; ++v)
          if (j0 + v < g.N) part[j0 + v] = acc[v];
      }
      // every lane's partials are visible before the warp takes its ticket
      __threadfence();
      __syncwarp();
      unsigned ticket = 0;
      if (lane == 0) ticket = atomicAdd(a.ws.dx_cnt + g.tile_cnt + tile, 1u);
      ticket = __shfl_sync(0xffffffffu, ticket, 0);
      if (ticket == (unsigned)(g.Cr - 1)) {
        // the last warp of this tile folds its chunk partials in chunk order, a lane
        // per column group (rows of partials are Npad floats: 128-bit loads, eight
        // chunks of loads ahead of the dependent adds)
        __threadfence();
        const float *pb = a.ws.dx_part + g.part_base;
        if (j0 < g.N) {
          float res[4] = {0.0f, 0.0f, 0.0f, 0.0f};
          int64_t c = 0;
          for (; c + 8 <= g.Cr; c += 8) {
            float4 b[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) b[u] = __ldcg(reinterpret_cast<const float4 *>(pb + (c + u) * g.Npad + j0));
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              res[0] = __fadd_rn(res[0], b[u].x);
              res[1] = __fadd_rn(res[1], b[u].y);
              res[2] = __fadd_rn(res[2], b[u].z);
              res[3] = __fadd_rn(res[3], b[u].w);
            }
          }
          for (; c < g.Cr; ++c) {
            const float4 b = __ldcg(reinterpret_cast<const float4 *>(pb + c * g.Npad + j0));
            res[0] = __fadd_rn(res[0], b.x);
            res[1] = __fadd_rn(res[1], b.y);
            res[2] = __fadd_rn(res[2], b.z);
            res[3] = __fadd_rn(res[3], b.w);
          }
#pragma unroll
          for (int v = 0; v < 4; ++v)
            if (j0 + v < g.N) a.dgx[g.x_off + j0 + v] = res[v];
        }
        if (lane == 0) a.ws.dx_cnt[g.tile_cnt + tile] = 0u;
      }
    }
  }
  // schedule 2: the last warp to finish puts the counters back to zero
  if (dyn && lane == 0 && atomicAdd(a.ws.sched + 3, 1u) == (unsigned)nw - 1) {
    a.ws.sched[2] = 0u;
    a.ws.sched[3] = 0u;
  }
}

const PlanHeader *check_plan(const char *fn, const void *plan_dev, const void *plan_host) {
  if (!plan_dev || !plan_host) {
    set_last_error("%s: plan is NULL", fn);
    return nullptr;
  }
  const PlanHeader *h = static_cast<const PlanHeader *>(plan_host);
  if (h->magic != kPlanMagic) {
    set_last_error("%s: not a batch plan (bad magic)", fn);
    return nullptr;
  }
  if (reinterpret_cast<uintptr_t>(plan_dev) % 128) {
    set_last_error("%s: device plan must be 128-byte aligned", fn);
    return nullptr;
  }
  return h;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

int persistent(const void *k, int threads, int64_t items) {
  int64_t cap = (int64_t)sm_count() * resident_blocks(k, threads);
  int64_t g = items < cap ? items : cap;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

}  // namespace dpia

using namespace dpia;

extern "C" {

size_t dpia_batch_plan_size(int32_t n_dots, const dpia_dot_instance *dots, int32_t n_gemvs,
                            const dpia_gemv_instance *gemvs, const dpia_batch_options *opt) {
  Built b;
  if (build_plan(n_dots, dots, n_gemvs, gemvs, opt, b) != DPIA_OK) return 0;
  return (size_t)b.h.total_bytes;
}

dpia_status dpia_batch_plan(int32_t n_dots, const dpia_dot_instance *dots, int32_t n_gemvs,
                            const dpia_gemv_instance *gemvs, const dpia_batch_options *opt, void *plan_host,
                            size_t plan_bytes) {
  set_last_error("");
  Built b;
  dpia_status rc = build_plan(n_dots, dots, n_gemvs, gemvs, opt, b);
  if (rc) return rc;
  if (!plan_host) {
    set_last_error("dpia_batch_plan: plan_host is NULL");
    return DPIA_ERR_NULL;
  }
  if ((int64_t)plan_bytes < b.h.total_bytes) {
    set_last_error("dpia_batch_plan: plan buffer of %zu bytes, %lld needed", plan_bytes, (long long)b.h.total_bytes);
    return DPIA_ERR_WORKSPACE;
  }
  char *p = static_cast<char *>(plan_host);
  std::memset(p, 0, (size_t)b.h.total_bytes);
  std::memcpy(p, &b.h, sizeof b.h);
  if (!b.dots.empty()) std::memcpy(p + b.h.dots_off, b.dots.data(), b.dots.size() * sizeof(DotDesc));
  if (!b.gemvs.empty()) std::memcpy(p + b.h.gemvs_off, b.gemvs.data(), b.gemvs.size() * sizeof(GemvDesc));
  if (!b.fwd.empty()) std::memcpy(p + b.h.fwd_off, b.fwd.data(), b.fwd.size() * sizeof(Item));
  if (!b.bwd.empty()) std::memcpy(p + b.h.bwd_off, b.bwd.data(), b.bwd.size() * sizeof(Item));
  if (!b.fwd_cost.empty()) std::memcpy(p + b.h.fwd_cost_off, b.fwd_cost.data(), b.fwd_cost.size() * 8);
  if (!b.bwd_cost.empty()) std::memcpy(p + b.h.bwd_cost_off, b.bwd_cost.data(), b.bwd_cost.size() * 8);
  return DPIA_OK;
}

size_t dpia_batch_workspace_size(const void *plan_host) {
  if (!plan_host) return 0;
  const PlanHeader *h = static_cast<const PlanHeader *>(plan_host);
  if (h->magic != kPlanMagic) return 0;
  return (size_t)ws_bytes_of(*h);
}

dpia_status dpia_batch_forward_f32(const void *plan_dev, const void *plan_host, const float *xs, const float *ys,
                                   float *dot_out, const float *As, const float *gx, float *gy, void *ws,
                                   size_t ws_bytes, int32_t grid, dpia_stream_t stream) {
  const char *fn = "dpia_batch_forward_f32";
  set_last_error("");
  const PlanHeader *h = check_plan(fn, plan_dev, plan_host);
  if (!h) return DPIA_ERR_NULL;
  if (h->n_fwd == 0) return DPIA_OK;
  if (h->n_dots > 0 && (!xs || !ys || !dot_out)) {
    set_last_error("%s: dot arrays are NULL", fn);
    return DPIA_ERR_NULL;
  }
  if (h->n_gemvs > 0 && (!As || !gx || !gy)) {
    set_last_error("%s: GEMV arrays are NULL", fn);
    return DPIA_ERR_NULL;
  }
  if ((xs && !aligned16(xs)) || (ys && !aligned16(ys)) || (As && !aligned16(As)) || (gx && !aligned16(gx))) {
    set_last_error("%s: packed inputs must be 16-byte aligned", fn);
    return DPIA_ERR_ALIGN;
  }
  if (!ws || (int64_t)ws_bytes < ws_bytes_of(*h) || reinterpret_cast<uintptr_t>(ws) % 128) {
    set_last_error("%s: workspace NULL, unaligned or smaller than %lld bytes", fn, (long long)ws_bytes_of(*h));
    return DPIA_ERR_WORKSPACE;
  }
  if (grid < 0) {
    set_last_error("%s: grid=%d", fn, grid);
    return DPIA_ERR_STRATEGY;
  }
  FwdArgs a{static_cast<const char *>(plan_dev), xs, ys, dot_out, As, gx, gy, ws_layout(*h, ws)};
  const void *k = (const void *)batch_fwd_kernel;
  const int g = grid > 0 ? grid : persistent(k, h->threads, h->n_fwd);
  void *args[] = {&a};
  cudaError_t e = cudaLaunchKernel(k, dim3(g), dim3(h->threads), args, 0, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    set_last_error("%s: CUDA error %d (%s)", fn, (int)e, cudaGetErrorString(e));
    return DPIA_ERR_CUDA;
  }
  return DPIA_OK;
}

dpia_status dpia_batch_backward_f32(const void *plan_dev, const void *plan_host, const float *xs, const float *ys,
                                    const float *dot_g, float *dxs, float *dys, const float *As, const float *gx,
                                    const float *gdy, float *dAs, float *dgx, void *ws, size_t ws_bytes, int32_t grid,
                                    dpia_stream_t stream) {
  const char *fn = "dpia_batch_backward_f32";
  set_last_error("");
  const PlanHeader *h = check_plan(fn, plan_dev, plan_host);
  if (!h) return DPIA_ERR_NULL;
  if (h->n_bwd == 0) return DPIA_OK;
  if (h->n_dots > 0 && (!xs || !ys || !dot_g || !dxs || !dys)) {
    set_last_error("%s: dot arrays are NULL", fn);
    return DPIA_ERR_NULL;
  }
  if (h->n_gemvs > 0 && (!As || !gx || !gdy || !dAs || !dgx)) {
    set_last_error("%s: GEMV arrays are NULL", fn);
    return DPIA_ERR_NULL;
  }
  const void *vp[] = {xs, ys, dxs, dys, As, gx, dAs};
  for (const void *p : vp)
    if (p && !aligned16(p)) {
      set_last_error("%s: packed arrays must be 16-byte aligned", fn);
      return DPIA_ERR_ALIGN;
    }
  if (!ws || (int64_t)ws_bytes < ws_bytes_of(*h) || reinterpret_cast<uintptr_t>(ws) % 128) {
    set_last_error("%s: workspace NULL, unaligned or smaller than %lld bytes", fn, (long long)ws_bytes_of(*h));
    return DPIA_ERR_WORKSPACE;
  }
  if (grid < 0) {
    set_last_error("%s: grid=%d", fn, grid);
    return DPIA_ERR_STRATEGY;
  }
  BwdArgs a{static_cast<const char *>(plan_dev), xs, ys, dot_g, dxs, dys, As, gx, gdy, dAs, dgx, ws_layout(*h, ws)};
  const void *k = (const void *)batch_bwd_kernel;
  const int g = grid > 0 ? grid : persistent(k, h->threads, h->n_bwd);
  void *args[] = {&a};
  cudaError_t e = cudaLaunchKernel(k, dim3(g), dim3(h->threads), args, 0, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    set_last_error("%s: CUDA error %d (%s)", fn, (int)e, cudaGetErrorString(e));
    return DPIA_ERR_CUDA;
  }
  return DPIA_OK;
}

}  // extern "C"
