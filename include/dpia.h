/*
 * dpia.h -- C ABI of the strategy-preserving map/reduce hot path for GB300 (sm_103a).
 *
 * Each entry point computes one pattern instance "out := E" (Section 4.1 states
 * the translation problem as producing a command equal to the assignment of a
 * functional expression E to an output acceptor) with the parallelisation
 * strategy passed explicitly, as the strategy-annotated dot product of Section
 * 2.1 carries it in its split sizes and map levels. Temporaries that the
 * strategy allocates in global memory are not allocated here: as in Section
 * 6.4 (allocation hoisting of newGlobal out of parallel loops) they become a
 * caller-provided workspace of (#chunks x partial) entries.
 *
 * Conventions for every call:
 *   - Pointers are DEVICE pointers owned by the caller, unless stated.
 *   - Calls are asynchronous on `stream` (NULL = the legacy default stream);
 *     the library never synchronises and never allocates device memory.
 *   - All arguments are validated on the host before anything is launched; a
 *     non-OK status means nothing was enqueued (except DPIA_ERR_CUDA, which
 *     reports a launch failure). dpia_last_error_message() then describes it.
 *   - Outputs and workspaces must not overlap inputs (the paper's interference
 *     control: a parallel loop writes only through its own acceptor). The only
 *     exception is scal's exact in-place form y == x.
 *   - A workspace serves one call at a time. It holds completion counters
 *     and must be zero-filled before its first use (e.g. one memset); every
 *     call leaves the counters zero again, so it can be reused without a new
 *     memset by calls with the same counter layout: dot / asum / int32-dot
 *     calls of any shape keep theirs in the first 128 bytes; a GEMV backward's
 *     counters depend on (M, N, row_split), so reuse its workspace only for
 *     that shape (or zero it again). It must be 128-byte aligned.
 *   - Floating point is IEEE binary32 with round-to-nearest-even, subnormals
 *     kept; every + and * of a reduction is rounded separately (no contraction),
 *     so a result is bit-identical to any evaluation of the same strategy tree.
 */
#ifndef DPIA_H
#define DPIA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t / CUstream. */
typedef struct CUstream_st *dpia_stream_t;

typedef enum {
  DPIA_OK = 0,
  DPIA_ERR_NULL = 1,        /* a required pointer is NULL */
  DPIA_ERR_SHAPE = 2,       /* negative size, split not dividing the length (without pad), ... */
  DPIA_ERR_ALIGN = 3,       /* pointer or leading dimension not aligned for the requested vector width */
  DPIA_ERR_STRATEGY = 4,    /* illegal strategy: bad sizes or an illegal nesting of levels */
  DPIA_ERR_WORKSPACE = 5,   /* workspace NULL or smaller than the *_workspace_size() answer */
  DPIA_ERR_ALIAS = 6,       /* an output or the workspace overlaps an input */
  DPIA_ERR_CUDA = 7,        /* the CUDA runtime reported an error at launch */
  DPIA_ERR_TIMEOUT = 8,     /* a bounded device-side wait gave up (reported via a status word) */
  DPIA_ERR_UNSUPPORTED = 9  /* a legal strategy this build does not implement */
} dpia_status;

/*
 * Levels of the GPU hierarchy a map can run at (Section 6.2: mapGlobal,
 * mapWorkgroup, mapLocal, mapSeq; WARP is the sm_103a level between a
 * work-group and a work-item, where reductions use register shuffles).
 *   GRID   -- mapGlobal: iterations spread over all threads of the grid;
 *   BLOCK  -- mapWorkgroup: one thread block per iteration;
 *   WARP   -- one warp (32 threads) per iteration;
 *   THREAD -- mapLocal: one thread of the enclosing block/warp per iteration;
 *   SEQ    -- mapSeq: a sequential loop in one thread.
 * A map nested in another must run at a strictly finer level; a map at GRID
 * level runs on single threads, so only SEQ may be nested in it (the legality
 * rule the paper's conclusion asks for: no work-group map inside a local map).
 */
typedef enum {
  DPIA_LVL_GRID = 0,
  DPIA_LVL_BLOCK = 1,
  DPIA_LVL_WARP = 2,
  DPIA_LVL_THREAD = 3,
  DPIA_LVL_SEQ = 4
} dpia_level;

enum { DPIA_MAP_INTERLEAVED = 0, DPIA_MAP_CONTIG = 1 };
enum { DPIA_SECOND_SEQ = 0, DPIA_SECOND_TREE = 1 };
enum { DPIA_STAGE_PRIVATE = 0, DPIA_STAGE_LOCAL = 1 };

/*
 * Reduction strategy R (dot, asum, the rows of GEMV):
 *
 *   reduce2nd (join (map@map_level (lambda chunk.
 *       tree (map@inner_level (lambda col. foldV (reduce (+) 0 (map f col)))
 *                              (columns of (asVector vec chunk)))))
 *     (split split (input)))
 *
 * split       -- s, elements per chunk (Section 2.1's split 2048*128).
 * threads     -- T, threads per block (power of two, 32..1024; <= 512 when vec >= 8).
 * vec         -- V in {1,2,4,8,16}: lanes per thread (asVector V, Section 6.2);
 *                V >= 4 uses 128-bit loads. Inputs must be aligned to
 *                min(4V, 16) bytes.
 * map_level   -- level of the map over chunks: BLOCK (a block per chunk,
 *                inner THREAD: T threads), WARP (a warp per chunk, inner
 *                THREAD: 32 threads), or GRID (one thread per chunk, inner
 *                SEQ). These three pairs are implemented.
 * inner_level -- level of the map over the chunk's columns (see above).
 * thread_map  -- INTERLEAVED: thread t folds vectors r*Tc + t, r = 0,1,..
 *                (coalesced); CONTIG: thread t folds vectors t*Rc .. t*Rc+Rc-1
 *                (the paper's per-thread contiguous sub-chunk). Tc = threads
 *                per chunk, Rc = s / (Tc*V).
 * The Tc per-thread results are reduced by a halving tree (lane l adds lane
 * l+16, l+8, .., l+1 inside each warp, then the same over the warp sums).
 * second      -- SEQ: the chunk results are folded in chunk order from +0 (the
 *                final sequential loop of Section 2.2); TREE: they are reduced
 *                by threads2 threads of one block, thread t folding result
 *                r*threads2 + t, then the halving tree. threads2 is a power of
 *                two <= threads. The second level runs in the last block to
 *                finish (no second launch, no device-side wait).
 * compensated -- 1: every fold step is a Kahan step on (sum, compensation)
 *                pairs; tree nodes merge pairs (f32 only).
 * pad         -- 1: n need not be a multiple of split; the last chunk is
 *                padded with (+0,+0) items (the reduce's identity). 0: a
 *                non-dividing split is DPIA_ERR_SHAPE.
 * grid        -- blocks to launch; 0 = a persistent grid of (SMs x resident
 *                blocks per SM), capped by the work. The grid never changes
 *                the result (chunks map to blocks by a grid-stride loop).
 * stage       -- address space the chunk passes through on its way to the
 *                fold (Section 6.2's toPrivate / toLocal, both the identity on
 *                values): PRIVATE loads it straight into registers; LOCAL
 *                copies it tile by tile into shared memory with bulk
 *                asynchronous copies (a four-stage ring per block), and the
 *                threads fold from there. LOCAL is implemented for
 *                dot/asum (f32, int32) with map_level BLOCK, vec 4 and the
 *                interleaved map (otherwise DPIA_ERR_UNSUPPORTED); a ragged
 *                last chunk is loaded directly. Every wait on a copy is
 *                bounded (2 s); one that runs out sets the device status word
 *                (dpia_poll_device_status), and the call's result is then
 *                undefined while its workspace stays usable.
 */
typedef struct {
  int64_t split;
  int32_t threads;
  int32_t vec;
  int32_t map_level;
  int32_t inner_level;
  int32_t thread_map;
  int32_t second;
  int32_t threads2;
  int32_t compensated;
  int32_t pad;
  int32_t grid;
  int32_t stage;
} dpia_reduce_strategy;

/* Version of this ABI (major*10000 + minor*100 + patch). */
int32_t dpia_version(void);

/* Description of the last error of the calling host thread ("" if none). */
const char *dpia_last_error_message(void);

/*
 * Workspace bytes a dot/asum call with this n and strategy needs: 128 bytes of
 * counter plus one partial per chunk (4 bytes f32, 8 bytes for a compensated
 * pair or an int64 partial; the larger is returned). Returns 0 if the
 * strategy is invalid for n (the call would fail with the same error).
 */
size_t dpia_dot_workspace_size(int64_t n, const dpia_reduce_strategy *st);

/*
 * out[0] := reduce (+) 0 (map (lambda p. fst p * snd p) (zip x y)) under
 * strategy st (Section 2.1, the dot product and its two-level strategy).
 * x, y: n floats each; out: one float. n == 0 gives +0.
 */
dpia_status dpia_dot_f32(const float *x, const float *y, int64_t n,
                         const dpia_reduce_strategy *st, float *out, void *ws,
                         size_t ws_bytes, dpia_stream_t stream);

/*
 * out[0] := the same reduction on int32 inputs with int64 products and int64
 * sums (exact, wrapping modulo 2^64 only beyond the int64 range). st as for
 * dpia_dot_f32 (compensated must be 0).
 */
dpia_status dpia_dot_i32(const int32_t *x, const int32_t *y, int64_t n,
                         const dpia_reduce_strategy *st, int64_t *out, void *ws,
                         size_t ws_bytes, dpia_stream_t stream);

/* out[0] := reduce (+) 0 (map abs x) under strategy st (asum of Section 7). */
dpia_status dpia_asum_f32(const float *x, int64_t n, const dpia_reduce_strategy *st,
                          float *out, void *ws, size_t ws_bytes, dpia_stream_t stream);

/*
 * y := map (lambda v. a * v) x (scal of Section 7). n floats; vec in
 * {1,2,4,8,16} is the asVector width of the map (alignment as above). y == x
 * (in place) is allowed; any other overlap is DPIA_ERR_ALIAS.
 */
dpia_status dpia_scal_f32(float a, const float *x, float *y, int64_t n, int32_t vec,
                          dpia_stream_t stream);

/*
 * Backward of out = dot(x, y): with g the incoming gradient (ONE float in
 * device memory), dx := map (lambda v. g * v) y and dy := map (lambda v. g * v) x
 * (the adjoint of reduce(+) is a broadcast of g, the adjoint of the pointwise
 * product map multiplies by the other operand). dx or dy may be NULL to skip it.
 */
dpia_status dpia_dot_bwd_f32(const float *x, const float *y, const float *g, int64_t n,
                             float *dx, float *dy, dpia_stream_t stream);

/*
 * y := map (lambda row. R (zip row x)) A for A of M rows x N columns, row-major
 * with leading dimension lda >= N (elements). R is the reduction strategy st
 * applied to each row: map_level BLOCK (a block per row) or WARP (a warp per
 * row), inner THREAD; split divides N (or pad = 1) and the row's chunk
 * results are folded in chunk order (second must be SEQ). With V >= 4, A,
 * lda*4 bytes and x must be 16-byte aligned.
 */
dpia_status dpia_gemv_f32(const float *A, int64_t M, int64_t N, int64_t lda, const float *x,
                          float *y, const dpia_reduce_strategy *st, dpia_stream_t stream);

/* Workspace bytes of dpia_gemv_bwd_f32 for dx: 128 + ceil(M/row_split)*N*4 (+ counters). */
size_t dpia_gemv_bwd_workspace_size(int64_t M, int64_t N, int64_t row_split);

/*
 * Backward of y = A x:
 *   dx := map (lambda col. reduce2nd (map fold (split row_split (zip col dy)))) (transpose A)
 *         -- each column's rows are split into chunks of row_split rows, each
 *         chunk folded in row order from +0, the chunk results folded in chunk
 *         order from +0 (rows past M are the identity);
 *   dA := map (lambda d. map (lambda v. d * v) x) dy   (dA = dy x^T, ldda >= N).
 * dx or dA may be NULL to skip it. ws (for dx) as dpia_gemv_bwd_workspace_size.
 * Pointers 4-byte aligned; 16-byte alignment of A, dA, x with lda and ldda
 * multiples of 4 enables 128-bit loads and stores (the values do not change).
 */
dpia_status dpia_gemv_bwd_f32(const float *A, int64_t M, int64_t N, int64_t lda,
                              const float *x, const float *dy, float *dx, float *dA,
                              int64_t ldda, int64_t row_split, void *ws, size_t ws_bytes,
                              dpia_stream_t stream);

enum { DPIA_CONTRACT_OFF = 0, DPIA_CONTRACT_FMA = 1 };

/*
 * GEMM strategy. contract: how the FP32 fold rounds each step (OFF: a
 * separately rounded multiply and add; FMA: one fused multiply-add, the
 * contraction declared explicitly -- the paper's num is abstract, so the
 * rounding of a step is part of the strategy). tile_m/n/k: 0 for the
 * implemented tiles or exactly those values -- FP32: 128 x 128 x 16; BF16:
 * tile_m x tile_n x 64 with tile_m 256 (512 on CTA pairs) and tile_n in
 * {128, 160, 192, 224, 256} (0 = the width whose tiles fill the fewest
 * waves). grid: CTAs of the persistent BF16 kernel (0 = one per SM, or as
 * many CTA pairs as fit at once).
 * cluster (BF16 only): 1: one CTA (one SM) per 256-row tile, two M=128 MMAs
 * per k step (tcgen05 cta_group::1). 2: a cluster of two CTAs on two SMs per
 * tile, each staging 128 rows of every 256-row block of A and half of B's
 * columns, one M=256 MMA per block across the pair (cta_group::2); tile_m 512
 * gives each SM two blocks that share its half of B. 0: a pair with 512-row
 * tiles when M >= 512 and pairs fit on the device, else one CTA. cluster = 2
 * where no CTA pair fits returns DPIA_ERR_CUDA. The value of C does not
 * depend on it. The FP32 fold ignores grid and cluster.
 * schedule (FP32 fold only; BF16 ignores it): how the tiles of a last wave
 * that 128 x 128 tiles leave partly empty are spread over the SMs. 1: every
 * tile a CTA, one launch. 2: the tile rows of a last wave at most half full
 * as 64 x 128 tiles in a second launch (else as 1). 3: k-range pieces over
 * two launches: the (tile, k-slice) units cut into one equal range per
 * resident CTA; the first launch folds the low-k part of every cut tile and
 * leaves its accumulators in C, the second continues those folds from C
 * (needs at least two tiles' k-slices per CTA of the device, else
 * DPIA_ERR_STRATEGY). 0: 3 where it fits and the last wave gives some SM
 * two tiles while more than 8% of the launch's tile slots stay empty, else
 * 1. Every schedule runs each C_ij's one sequential fold: C is the same bits
 * under all of them. Outside 0..3: DPIA_ERR_STRATEGY.
 */
typedef struct {
  int32_t contract;
  int32_t tile_m;
  int32_t tile_n;
  int32_t tile_k;
  int32_t grid;
  int32_t cluster;
  int32_t schedule;
} dpia_gemm_strategy;

/*
 * C := map (lambda a. map (lambda b. fold_k (a_k * b_k)) (transpose op(B))) op(A)
 * in FP32 on the CUDA cores: op(A) is M x K (A stored M x K row-major with
 * lda, or K x M when transA = 1), op(B) is K x N (B stored K x N with ldb, or
 * N x K when transB = 1), C is M x N with ldc (f32). Each C_ij is one
 * sequential fold over k = 0..K-1 from +0 (Section 4.2's reduceI), so the
 * result is bit-identical to a plain loop with the same contraction. No
 * alignment is required; 16-byte alignment with leading dimensions a multiple
 * of 4 enables 128-bit loads. K == 0 gives C = +0.
 */
dpia_status dpia_gemm_f32(const float *A, const float *B, float *C, int64_t M, int64_t N, int64_t K,
                          int64_t lda, int64_t ldb, int64_t ldc, int32_t transA, int32_t transB,
                          const dpia_gemm_strategy *st, dpia_stream_t stream);

/*
 * The same map of maps of reduce with bf16 operands (raw bit patterns,
 * uint16) and f32 accumulation on the tensor cores (tcgen05.mma, TMA, tensor
 * memory). Layout arguments as dpia_gemm_f32 (transA = 1 / transB = 0 are the
 * MN-major operand layouts, read directly). A and B must be 16-byte aligned
 * and lda, ldb multiples of 8 (TMA). The order of the accumulation inside the
 * tensor core is fixed by the hardware, so results are defined up to the
 * f32 rounding of a k-reduction (checked against FP64 by tolerance).
 */
dpia_status dpia_gemm_bf16(const uint16_t *A, const uint16_t *B, float *C, int64_t M, int64_t N,
                           int64_t K, int64_t lda, int64_t ldb, int64_t ldc, int32_t transA,
                           int32_t transB, const dpia_gemm_strategy *st, dpia_stream_t stream);

/* y := map bf16_round_nearest_even x (n floats to n bf16 bit patterns); x 16-byte, y 8-byte aligned. */
dpia_status dpia_cast_f32_bf16(const float *x, uint16_t *y, int64_t n, dpia_stream_t stream);

/*
 * Synchronous: writes to *status DPIA_ERR_TIMEOUT if a bounded device-side wait
 * of any kernel of this library gave up since the previous poll on the
 * current device (the kernel then returned early, leaving its output
 * undefined), else DPIA_OK; clears the flag.
 */
dpia_status dpia_poll_device_status(int32_t *status);

/*
 * Self-test of the bounded device-side waits (no counterpart in the paper):
 * launches one block whose wait on an mbarrier that nothing completes gives up
 * after timeout_us microseconds (1 .. 2,000,000) and records DPIA_ERR_TIMEOUT
 * in the device status word, which dpia_poll_device_status then reports. No
 * memory is touched and the context stays usable. Asynchronous on stream;
 * timeout_us out of range is DPIA_ERR_SHAPE.
 */
dpia_status dpia_selftest_bounded_wait(uint32_t timeout_us, dpia_stream_t stream);

/*
 * Batches of uneven instances in one persistent launch.
 *
 * Thousands of dot products and GEMVs of different lengths are packed into
 * shared arrays (each instance at its own offset) and computed by a single
 * persistent kernel: the plan lists every instance with its own reduction
 * strategy (Section 2.1's split sizes chosen per instance) and a work table
 * of (instance, chunk) and (instance, row group) items, longest first, that
 * the blocks walk in a grid-stride loop. Each instance's second-level reduce
 * runs in the block that finishes its last chunk (a per-instance ticket; no
 * block waits). The backward launch covers dx = g*y, dy = g*x of every dot and
 * dA = dy x^T, dx = A^T dy of every GEMV the same way.
 *
 * Instance strategies: dots at BLOCK level (threads = the batch's threads,
 * vec 4), any split (a multiple of threads*4), interleaved or contiguous,
 * SEQ or TREE second level, pad implied; GEMV rows at WARP level (a warp per
 * row, vec 4), split a multiple of 128, the row's chunks folded in order, and
 * a backward row_split. Offsets are in elements; every instance must start on
 * a 16-byte boundary (offsets multiples of 4) and GEMV rows too (lda a
 * multiple of 4).
 */
typedef struct {
  int64_t off;                /* offset of x_i (and y_i) in the packed arrays */
  int64_t n;                  /* length */
  dpia_reduce_strategy st;    /* BLOCK / THREAD, vec 4, threads = the batch's */
} dpia_dot_instance;

typedef struct {
  int64_t a_off;              /* offset of A_i (M x N, row-major, lda) in the packed A array */
  int64_t x_off;              /* offset of x_i (N) in the packed x array (and of dx_i in dx) */
  int64_t y_off;              /* offset of y_i (M) in the packed y array (and of dy_i in dy) */
  int64_t M, N, lda;
  dpia_reduce_strategy st;    /* WARP / THREAD rows, vec 4 */
  int64_t row_split;          /* backward: rows per chunk of dx = A^T dy */
} dpia_gemv_instance;

/*
 * How the blocks of a batched launch share the work (the values never depend
 * on it):
 *   threads       -- block size (a power of two, 32..256);
 *   schedule      -- 0: items sorted longest first and dealt to the blocks
 *                    round robin; 1: items in instance order, each block takes
 *                    the contiguous run whose byte costs make up its equal share;
 *                    2: items sorted longest first, dealt round robin in the
 *                    forward, and in the backward each warp takes the next one
 *                    from a counter in the workspace when it is free (launches
 *                    sharing a workspace must not overlap: run them on one stream;
 *                    at most 2^30 backward items, else DPIA_ERR_SHAPE).
 */
typedef struct {
  int32_t threads;
  int32_t schedule;
  int32_t reserved[2];
} dpia_batch_options;

/* Bytes of the plan of a batch (0 if an instance or an option is invalid). */
size_t dpia_batch_plan_size(int32_t n_dots, const dpia_dot_instance *dots, int32_t n_gemvs,
                            const dpia_gemv_instance *gemvs, const dpia_batch_options *opt);

/*
 * Build the plan in host memory (plan_bytes from dpia_batch_plan_size),
 * validating every instance. The plan is plain data: copy it to device
 * memory once (cudaMemcpy) and pass both copies to the launches below; it is
 * reused for every launch with the same shapes.
 */
dpia_status dpia_batch_plan(int32_t n_dots, const dpia_dot_instance *dots, int32_t n_gemvs,
                            const dpia_gemv_instance *gemvs, const dpia_batch_options *opt,
                            void *plan_host, size_t plan_bytes);

/* Workspace bytes the batched launches of this plan need (zero-filled once). */
size_t dpia_batch_workspace_size(const void *plan_host);

/*
 * Forward of every instance in one launch: dot_out[i] := dot_i(xs, ys) and
 * gy_i := A_i gx_i. Pointers of a kind (dots or GEMVs) may be NULL when the
 * plan has no instance of that kind. grid = 0: one persistent grid.
 */
dpia_status dpia_batch_forward_f32(const void *plan_dev, const void *plan_host, const float *xs,
                                   const float *ys, float *dot_out, const float *As,
                                   const float *gx, float *gy, void *ws, size_t ws_bytes,
                                   int32_t grid, dpia_stream_t stream);

/*
 * Backward of every instance in one launch: for each dot, with g = dot_g[i],
 * dxs_i := g * y_i and dys_i := g * x_i; for each GEMV, with dy_i in gdy,
 * dA_i := dy_i x_i^T (stored with the instance's lda in dAs) and
 * dgx_i := A_i^T dy_i (row chunks of row_split folded in order).
 */
dpia_status dpia_batch_backward_f32(const void *plan_dev, const void *plan_host, const float *xs,
                                    const float *ys, const float *dot_g, float *dxs, float *dys,
                                    const float *As, const float *gx, const float *gdy, float *dAs,
                                    float *dgx, void *ws, size_t ws_bytes, int32_t grid,
                                    dpia_stream_t stream);

/*
 * Allocation-free dot product. The paper has no counterpart: this entry exists
 * for callers that cannot allocate device memory -- e.g. a plugin inside a
 * host framework that owns all device memory and offers it no allocator, or a
 * latency-critical path that cannot afford cudaMalloc's possible device
 * synchronisation. It computes exactly what dpia_dot_f32 computes (same
 * strategy, same bits) but takes no workspace: its scratch (the per-chunk
 * partials and the completion counter) is a static device array of
 * DPIA_NOALLOC_SCRATCH_BYTES (1 MiB) that every GPU loading the library keeps
 * until the process exits. Its layout is that of dpia_dot_f32's workspace: a
 * 128-byte counter, then 8 bytes per chunk whatever the strategy (room for a
 * Kahan pair), so at most (1 MiB - 128) / 8 = 131056 chunks (n / split,
 * rounded up) are allowed; larger requests return DPIA_ERR_WORKSPACE with an
 * explanation and enqueue nothing.
 *   - The first call on a device (with that device current) looks up the
 *     array's device address; make that first call before any stream capture.
 *   - The address is kept for the life of the process. cudaDeviceReset (or
 *     any reset of the device's primary context) unloads the library's device
 *     code together with the array, so this entry point must not be called
 *     on a device after it has been reset; the entries that take a caller
 *     workspace are not affected.
 *   - Every call clears the array's counter (an asynchronous memset on
 *     `stream`) and then reuses the array: calls whose executions overlap on
 *     the GPU race on it and must be ordered by the caller.
 *   - No cudaMalloc, cudaFree or allocating library routine is called.
 * Arguments and errors otherwise as dpia_dot_f32.
 */
#define DPIA_NOALLOC_SCRATCH_BYTES (1u << 20)
dpia_status dpia_dot_f32_noalloc(const float *x, const float *y, int64_t n,
                                 const dpia_reduce_strategy *st, float *out,
                                 dpia_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* DPIA_H */
