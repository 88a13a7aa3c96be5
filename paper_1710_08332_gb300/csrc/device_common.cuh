// Device building blocks of the strategy reduction: vector loads (asVector),
// accumulator policies (binary32 sums, Kahan pairs, int64 sums), the
// per-thread sequential fold (reduceSeq over a thread's column, Section 4.2's
// reduceI as new + for) and the halving trees over lanes and warps.
//
// Every floating-point + and * goes through __fadd_rn / __fmul_rn / __fsub_rn,
// which the compiler never contracts into an FMA, so a reduction is bit-equal
// to any other evaluation of the same strategy tree.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dpia {

// ---------------------------------------------------------------------------
// loads
// ---------------------------------------------------------------------------

// Streaming loads: read once, do not allocate in L1.
__device__ __forceinline__ float4 ld_stream_v4(const float *p) {
  float4 v;
  asm("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
      : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
      : "l"(p));
  return v;
}
__device__ __forceinline__ float2 ld_stream_v2(const float *p) {
  float2 v;
  asm("ld.global.nc.L1::no_allocate.v2.f32 {%0,%1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ float ld_stream_1(const float *p) {
  float v;
  asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ int4 ld_stream_v4(const int32_t *p) {
  int4 v;
  asm("ld.global.nc.L1::no_allocate.v4.s32 {%0,%1,%2,%3}, [%4];"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
      : "l"(p));
  return v;
}
__device__ __forceinline__ int2 ld_stream_v2(const int32_t *p) {
  int2 v;
  asm("ld.global.nc.L1::no_allocate.v2.s32 {%0,%1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ int32_t ld_stream_1(const int32_t *p) {
  int32_t v;
  asm("ld.global.nc.L1::no_allocate.s32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

// Streaming store: written once, evict first.
__device__ __forceinline__ void st_stream_v4(float *p, float4 v) {
  asm volatile("st.global.cs.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z),
               "f"(v.w)
               : "memory");
}

// Cached read-only loads (an operand many blocks re-read, e.g. GEMV's x).
__device__ __forceinline__ float4 ld_cached_v4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ float2 ld_cached_v2(const float *p) { return __ldg(reinterpret_cast<const float2 *>(p)); }
__device__ __forceinline__ float ld_cached_1(const float *p) { return __ldg(p); }

// V consecutive elements starting at p (p aligned to min(4V,16) bytes).
template <int V, bool CACHED, class T>
__device__ __forceinline__ void load_vec(const T *p, T (&r)[V]) {
  if constexpr (V == 1) {
    if constexpr (CACHED) r[0] = ld_cached_1(p); else r[0] = ld_stream_1(p);
  } else if constexpr (V == 2) {
    if constexpr (CACHED) {
      float2 a = ld_cached_v2(p); r[0] = a.x; r[1] = a.y;
    } else {
      auto a = ld_stream_v2(p); r[0] = a.x; r[1] = a.y;
    }
  } else {
#pragma unroll
    for (int q = 0; q < V / 4; ++q) {
      if constexpr (CACHED) {
        float4 a = ld_cached_v4(p + 4 * q);
        r[4 * q] = a.x; r[4 * q + 1] = a.y; r[4 * q + 2] = a.z; r[4 * q + 3] = a.w;
      } else {
        auto a = ld_stream_v4(p + 4 * q);
        r[4 * q] = a.x; r[4 * q + 1] = a.y; r[4 * q + 2] = a.z; r[4 * q + 3] = a.w;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// element maps: what one zipped item contributes to the sum
// ---------------------------------------------------------------------------

struct DotF32 {  // map (lambda p. fst p * snd p)
  using in_t = float;
  using e_t = float;
  static constexpr bool kTwo = true;
  __device__ static __forceinline__ float elem(float a, float b) { return __fmul_rn(a, b); }
};
struct AsumF32 {  // map abs
  using in_t = float;
  using e_t = float;
  static constexpr bool kTwo = false;
  __device__ static __forceinline__ float elem(float a, float) { return fabsf(a); }
};
struct DotI32 {  // int32 inputs, int64 products
  using in_t = int32_t;
  using e_t = long long;
  static constexpr bool kTwo = true;
  __device__ static __forceinline__ long long elem(int32_t a, int32_t b) {
    return (long long)a * (long long)b;
  }
};

// ---------------------------------------------------------------------------
// accumulator policies: zero, step (fold one element in), combine (merge two
// partial results), warp shuffle
// ---------------------------------------------------------------------------

struct SumF32 {
  using acc_t = float;
  using out_t = float;
  __device__ static __forceinline__ float zero() { return 0.0f; }
  __device__ static __forceinline__ float step(float a, float e) { return __fadd_rn(a, e); }
  __device__ static __forceinline__ float combine(float a, float b) { return __fadd_rn(a, b); }
  __device__ static __forceinline__ float shfl_down(float v, int off) {
    return __shfl_down_sync(0xffffffffu, v, off);
  }
  __device__ static __forceinline__ float result(float a) { return a; }
};

// Kahan pairs (sum, compensation): y = e - c; t = s + y; c' = (t - s) - y; s' = t.
struct KahanF32 {
  using acc_t = float2;
  using out_t = float;
  __device__ static __forceinline__ float2 zero() { return make_float2(0.0f, 0.0f); }
  __device__ static __forceinline__ float2 step(float2 a, float e) {
    float y = __fsub_rn(e, a.y);
    float t = __fadd_rn(a.x, y);
    float c = __fsub_rn(__fsub_rn(t, a.x), y);
    return make_float2(t, c);
  }
  __device__ static __forceinline__ float2 combine(float2 a, float2 b) {
    return step(a, __fsub_rn(b.x, b.y));
  }
  __device__ static __forceinline__ float2 shfl_down(float2 v, int off) {
    return make_float2(__shfl_down_sync(0xffffffffu, v.x, off),
                       __shfl_down_sync(0xffffffffu, v.y, off));
  }
  __device__ static __forceinline__ float result(float2 a) { return a.x; }
};

struct SumI64 {
  using acc_t = long long;
  using out_t = long long;
  __device__ static __forceinline__ long long zero() { return 0; }
  __device__ static __forceinline__ long long step(long long a, long long e) { return a + e; }
  __device__ static __forceinline__ long long combine(long long a, long long b) { return a + b; }
  __device__ static __forceinline__ long long shfl_down(long long v, int off) {
    return __shfl_down_sync(0xffffffffu, v, off);
  }
  __device__ static __forceinline__ long long result(long long a) { return a; }
};

// ---------------------------------------------------------------------------
// per-thread fold of one chunk column
// ---------------------------------------------------------------------------

// Fold-step loads in flight per thread: 128 bytes of streamed operands, i.e.
// 16 elements per operand when both operands stream from HBM, 32 when one does
// (asum, or GEMV whose x is re-read from cache); at most 8 vectors per operand,
// and 16 elements for V >= 8 (wider vectors would spill).
template <int V, int STREAMS>
struct Unroll {
  static constexpr int elems = V >= 8 ? 16 : 32 / STREAMS;
  static constexpr int value = V >= elems ? 1 : elems / V > 8 ? 8 : elems / V;
};

// Thread's column of a chunk: Rc vectors of V items at base, base+step, ...
// Lanes fold their items in order from zero, then the lanes are folded in lane
// order (asScalar then reduce). Items at index >= n are the identity items
// (0, 0): they are still folded in (the padded split of a ragged length).
// STREAMS sets the loads in flight (Unroll); callers short of registers pass 2.
// RAGGED_BATCHED: a chunk reaching past n folds its whole vectors with the
// batched loads too (for callers whose chunks are often padded: GEMV rows,
// batched instances); otherwise such a chunk is folded one vector at a time,
// which keeps the kernel's register count down.
template <class E, class A, int V, bool CACHE_Y, int STREAMS = (E::kTwo && !CACHE_Y) ? 2 : 1,
          bool RAGGED_BATCHED = false>
__device__ __forceinline__ typename A::acc_t thread_fold(const typename E::in_t *__restrict__ x,
                                                         const typename E::in_t *__restrict__ y,
                                                         int64_t n, int64_t base, int64_t Rc,
                                                         int64_t step, bool full) {
  using in_t = typename E::in_t;
  using acc_t = typename A::acc_t;
  constexpr int U = Unroll<V, STREAMS>::value;
  acc_t acc[V];
#pragma unroll
  for (int v = 0; v < V; ++v) acc[v] = A::zero();
  if (full) {
    int64_t r = 0;
    for (; r + U <= Rc; r += U) {
      in_t xv[U][V], yv[U][V];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        load_vec<V, false>(x + base + (r + u) * step, xv[u]);
        if constexpr (E::kTwo) load_vec<V, CACHE_Y>(y + base + (r + u) * step, yv[u]);
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int v = 0; v < V; ++v)
          acc[v] = A::step(acc[v], E::elem(xv[u][v], E::kTwo ? yv[u][v] : xv[u][v]));
    }
    // what is left of the column in a half and a quarter batch (a short column,
    // e.g. a narrow GEMV row's, keeps its loads in flight together), then singly;
    // the vectors are still folded in r order
    if constexpr (U >= 4) {
      constexpr int H = U / 2;
      if (r + H <= Rc) {
        in_t xv[H][V], yv[H][V];
#pragma unroll
        for (int u = 0; u < H; ++u) {
          load_vec<V, false>(x + base + (r + u) * step, xv[u]);
          if constexpr (E::kTwo) load_vec<V, CACHE_Y>(y + base + (r + u) * step, yv[u]);
        }
#pragma unroll
        for (int u = 0; u < H; ++u)
#pragma unroll
          for (int v = 0; v < V; ++v)
            acc[v] = A::step(acc[v], E::elem(xv[u][v], E::kTwo ? yv[u][v] : xv[u][v]));
        r += H;
      }
    }
    if constexpr (U >= 8) {
      constexpr int Q = U / 4;
      if (r + Q <= Rc) {
        in_t xv[Q][V], yv[Q][V];
#pragma unroll
        for (int u = 0; u < Q; ++u) {
          load_vec<V, false>(x + base + (r + u) * step, xv[u]);
          if constexpr (E::kTwo) load_vec<V, CACHE_Y>(y + base + (r + u) * step, yv[u]);
        }
#pragma unroll
        for (int u = 0; u < Q; ++u)
#pragma unroll
          for (int v = 0; v < V; ++v)
            acc[v] = A::step(acc[v], E::elem(xv[u][v], E::kTwo ? yv[u][v] : xv[u][v]));
        r += Q;
      }
    }
    for (; r < Rc; ++r) {
      in_t xv[V], yv[V];
      load_vec<V, false>(x + base + r * step, xv);
      if constexpr (E::kTwo) load_vec<V, CACHE_Y>(y + base + r * step, yv);
#pragma unroll
      for (int v = 0; v < V; ++v) acc[v] = A::step(acc[v], E::elem(xv[v], E::kTwo ? yv[v] : xv[v]));
    }
  } else if constexpr (!RAGGED_BATCHED) {
    // a chunk reaching past n, one vector at a time: items at index >= n are
    // the identity items (0, 0), folded in all the same
    for (int64_t r = 0; r < Rc; ++r) {
      const int64_t e0 = base + r * step;
      in_t xv[V], yv[V];
      if (e0 + V <= n) {
        load_vec<V, false>(x + e0, xv);
        if constexpr (E::kTwo) load_vec<V, CACHE_Y>(y + e0, yv);
      } else {
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const bool in = e0 + v < n;
          xv[v] = in ? x[e0 + v] : in_t(0);
          yv[v] = (E::kTwo && in) ? y[e0 + v] : in_t(0);
        }
      }
#pragma unroll
      for (int v = 0; v < V; ++v) acc[v] = A::step(acc[v], E::elem(xv[v], E::kTwo ? yv[v] : xv[v]));
    }
  } else {
    // a chunk reaching past n: vectors r < Rin lie wholly below n and take the
    // same batched loads; at most one vector straddles n, the rest are the
    // identity items (0, 0), folded in all the same
    const int64_t room = n - V - base;  // e0(r) + V <= n  <=>  r * step <= room
    int64_t Rin = room < 0 ? 0 : room / step + 1;
    if (Rin > Rc) Rin = Rc;
    int64_t r = 0;
    for (; r + U <= Rin; r += U) {
      in_t xv[U][V], yv[U][V];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        load_vec<V, false>(x + base + (r + u) * step, xv[u]);
        if constexpr (E::kTwo) load_vec<V, CACHE_Y>(y + base + (r + u) * step, yv[u]);
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int v = 0; v < V; ++v)
          acc[v] = A::step(acc[v], E::elem(xv[u][v], E::kTwo ? yv[u][v] : xv[u][v]));
    }
    if constexpr (U >= 4) {
      constexpr int H = U / 2;
      if (r + H <= Rin) {  // half a batch left
        in_t xv[H][V], yv[H][V];
#pragma unroll
        for (int u = 0; u < H; ++u) {
          load_vec<V, false>(x + base + (r + u) * step, xv[u]);
          if constexpr (E::kTwo) load_vec<V, CACHE_Y>(y + base + (r + u) * step, yv[u]);
        }
#pragma unroll
        for (int u = 0; u < H; ++u)
#pragma unroll
          for (int v = 0; v < V; ++v)
            acc[v] = A::step(acc[v], E::elem(xv[u][v], E::kTwo ? yv[u][v] : xv[u][v]));
        r += H;
      }
    }
    if constexpr (U >= 8) {
      constexpr int Q = U / 4;
      if (r + Q <= Rin) {  // a quarter batch left
        in_t xv[Q][V], yv[Q][V];
#pragma unroll
        for (int u = 0; u < Q; ++u) {
          load_vec<V, false>(x + base + (r + u) * step, xv[u]);
          if constexpr (E::kTwo) load_vec<V, CACHE_Y>(y + base + (r + u) * step, yv[u]);
        }
#pragma unroll
        for (int u = 0; u < Q; ++u)
#pragma unroll
          for (int v = 0; v < V; ++v)
            acc[v] = A::step(acc[v], E::elem(xv[u][v], E::kTwo ? yv[u][v] : xv[u][v]));
        r += Q;
      }
    }
    for (; r < Rc; ++r) {
      const int64_t e0 = base + r * step;
      in_t xv[V], yv[V];
      if (r < Rin) {
        load_vec<V, false>(x + e0, xv);
        if constexpr (E::kTwo) load_vec<V, CACHE_Y>(y + e0, yv);
      } else {
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const bool in = e0 + v < n;
          xv[v] = in ? x[e0 + v] : in_t(0);
          yv[v] = (E::kTwo && in) ? y[e0 + v] : in_t(0);
        }
      }
#pragma unroll
      for (int v = 0; v < V; ++v) acc[v] = A::step(acc[v], E::elem(xv[v], E::kTwo ? yv[v] : xv[v]));
    }
  }
  acc_t t = A::zero();
#pragma unroll
  for (int v = 0; v < V; ++v) t = A::combine(t, acc[v]);
  return t;
}

// ---------------------------------------------------------------------------
// halving trees
// ---------------------------------------------------------------------------

// Lane l combines lane l + L/2, then l + L/4, .., l + 1; lane 0 ends with the
// tree over lanes 0..L-1 (L a power of two <= 32). Other lanes hold junk.
template <class A>
__device__ __forceinline__ typename A::acc_t warp_tree(typename A::acc_t v, int L) {
  for (int off = L >> 1; off >= 1; off >>= 1) v = A::combine(v, A::shfl_down(v, off));
  return v;
}

// Tree over the first `count` threads of the block (count a power of two,
// <= blockDim.x): 32-lane trees inside warps, then the tree over the warp
// sums. Threads >= count must pass any value. Result valid in thread 0.
// `sm` holds >= 32 entries; the call ends with a __syncthreads().
template <class A>
__device__ __forceinline__ typename A::acc_t block_tree(typename A::acc_t v, int count,
                                                        typename A::acc_t *sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int L = count < 32 ? count : 32;
  const int W = count / L;
  v = warp_tree<A>(v, L);
  if (W == 1) {
    __syncthreads();
    return v;
  }
  if (lane == 0 && warp < W) sm[warp] = v;
  __syncthreads();
  if (warp == 0) {
    typename A::acc_t w = lane < W ? sm[lane] : A::zero();
    v = warp_tree<A>(w, W);
  }
  __syncthreads();
  return v;
}

__host__ __device__ constexpr int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Largest block for a vector width: wide vectors keep 2V..4V values per
// thread in registers, so V >= 8 is limited to 512 threads (128 registers).
__host__ __device__ constexpr int max_threads_for_vec(int V) { return V >= 8 ? 512 : 1024; }

}  // namespace dpia
