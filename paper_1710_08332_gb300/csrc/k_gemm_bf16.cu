// BF16 GEMM on the 5th-generation tensor cores: C (f32) = op(A) op(B) with
// bf16 operands and f32 accumulation in tensor memory.
//
// The same map-of-maps-of-reduce as the FP32 fold (each C_ij is a reduce over
// k of a_ik * b_kj), but the reduce is carried by tcgen05.mma, whose internal
// accumulation order is fixed by the hardware: results are checked against
// FP64 by tolerance, not bit for bit.
//
// Structure (one CTA per SM, persistent over 256 x BN output tiles):
//   warp 0     -- TMA producer: cp.async.bulk.tensor loads of the A (256 x 64)
//                 and B (BN x 64) k-slices into a 3-stage shared-memory ring,
//                 128-byte swizzled, completion counted on mbarriers;
//   warp 1     -- allocates 512 TMEM columns (two 128 x BN f32 accumulators,
//                 rows 0..127 and 128..255 of the tile); one thread issues two
//                 tcgen05.mma (M=128, N=BN, K=16) per k step, both reading the
//                 same B slice, and commits each stage back to the producer
//                 and each finished tile to the epilogue;
//   warps 2..9 -- epilogue: warp w reads TMEM lanes 32*(w%4) .. +31 of
//                 accumulator (w-2)/4 with tcgen05.ld and stores them as f32
//                 (below).
// Two M=128 products per B slice halve the operand bytes per flop against a
// 128-row tile. BN (<= 256, a multiple of 32) is chosen per shape so that the
// tiles fill whole waves of SMs. The producer keeps prefetching the next tile
// while the epilogue drains TMEM. (Six 32 KiB stages of 32-wide k-slices were
// measured slower than three 64 KiB stages: the per-request cost of the
// smaller TMA loads outweighs the deeper pipeline.)
// Operands may be K-major or MN-major (transposed) independently: the
// shared-memory descriptors select the canonical 128-byte-swizzle layout of
// either major-ness, so the transposes of the backward pass need no copies.
//
// A second kernel runs each tile on a CTA pair (cta_group::2, below); with
// 512-row tiles it stages 23% fewer operand bytes per flop and is the
// default when M >= 512. The epilogue of both kernels stages each warp's
// 32 x 32 block in shared memory and hands it to the TMA engine, which writes
// whole 128-byte rows of C; writing C is the part of a tile the MMAs cannot
// overlap (both accumulators fill tensor memory). Measured at 4096^3, each
// launch alone: 512-row pairs 1.60 PFLOP/s, one SM per tile 1.53-1.60,
// 256-row pairs 1.20-1.29; B shared by TMA multicast within clusters of
// one-SM CTAs measured slower and was not kept.
//
// Every mbarrier wait is bounded by the global timer. A wait that runs out
// sets the CTA's abort flag and the library's device status word
// (dpia_poll_device_status reports it), the CTA drains what it has in flight,
// frees its tensor memory and returns; nothing spins forever.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "../../include/dpia.h"
#include "async_copy.cuh"
#include "device_common.cuh"
#include "kernels.h"

namespace dpia {

__device__ unsigned g_device_status;  // sticky DPIA_ERR_TIMEOUT flag, read by dpia_poll_device_status

namespace {

constexpr int BM = 256, BN_MAX = 256, BK = 64, STAGES = 3;
constexpr int A_BYTES = BM * BK * 2;             // 32 KiB
constexpr int B_BYTES = BN_MAX * BK * 2;         // 32 KiB (room for the widest B slice)
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;   // 64 KiB
// Shared-memory layouts of one k-slice (BK = 64 bf16), 128-byte swizzle:
//   K-major operand : rows of 128 bytes (the 64 k values), 8-row atoms of
//                     1024 bytes (SBO 1024), k step of 16 = +32 bytes;
//   MN-major operand: TMA boxes of 64 (m or n) x 64 (k), rows of 128 bytes,
//                     8-row atoms of 1024 bytes (SBO 1024), boxes 8192 bytes
//                     apart (LBO 8192), k step of 16 = +2048 bytes.
constexpr uint32_t KMAJ_SBO = 1024, MN_LBO = 8192, MN_SBO = 1024;
constexpr uint32_t LAYOUT_SW128 = 2;
constexpr int NUM_EPI_WARPS = 8;
constexpr int NUM_THREADS = 64 + 32 * NUM_EPI_WARPS;
constexpr uint32_t TMEM_COLS = 512;
constexpr int EPI_BUF_BYTES = 32 * 32 * 4;  // a warp's 32 x 32 f32 staging block
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + NUM_EPI_WARPS * EPI_BUF_BYTES + 1024 + 256;

struct Params {
  float *C;
  int64_t M, N, K, ldc;
  int BN, tiles_n, num_tiles, k_blocks;
  int a_mn, b_mn;
  int vec_ok;         // C has a tensor map: the epilogue stores through the TMA engine
  int a_3d;           // MN-major A loaded as one 3-D box {64 m, 64 k, 4 m-blocks}
  uint32_t stage_tx;  // bytes the TMA loads of one stage deliver
};

// Bounded wait on a phase parity; false if it timed out or the CTA aborted.
__device__ __noinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255) == 0) {
      if (*abort_flag) return false;
      if (globaltimer() - t0 > kTimeoutNs) {
        *abort_flag = 1;
        atomicExch(&g_device_status, (unsigned)DPIA_ERR_TIMEOUT);
        return false;
      }
    }
  }
}

__device__ __forceinline__ void tma_load_2d(const CUtensorMap *map, uint64_t *bar, void *dst, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(const CUtensorMap *map, uint64_t *bar, void *dst, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: start address, leading/stride byte
// offsets, descriptor version 1, swizzle layout.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo, uint32_t layout) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)layout << 61;
  return d;
}

// Descriptor of rows [128h, 128h+128) (A) or of the whole slice (B, h = 0)
// for the k-th 16-wide step of a stage.
__device__ __forceinline__ uint64_t operand_desc(uint32_t base, int mn_major, int h, int k) {
  return mn_major ? sdesc(base + h * (2 * MN_LBO) + k * 2048, MN_LBO, MN_SBO, LAYOUT_SW128)
                  : sdesc(base + h * (128 * BK * 2) + k * 32, 16, KMAJ_SBO, LAYOUT_SW128);
}

// Instruction descriptor of kind::f16: f32 accumulator, bf16 A and B,
// operand major-ness, N >> 3 and M >> 4.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, int a_mn, int b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 lanes x 32 columns of 32-bit values from tensor memory (lane = row);
// the registers are valid after tmem_wait_ld().
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Bulk tensor store of a shared-memory box to global memory (the TMA engine
// writes it while the warp goes on; elements outside the tensor are skipped).
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, const void *src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(smem_u32(src)), "r"(x), "r"(y)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the committed stores have read their shared-memory source
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// the committed stores have completed
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Stores one 32 x 32 block of an accumulator into C: lane i holds the 32
// values of row row0 + i, columns col0 .. col0 + 31. With a tensor map of C
// (C 16-byte aligned, rows a multiple of 16 bytes apart) the block goes into
// the warp's 4 KiB of shared memory in the 128-byte swizzle (16-byte chunk j
// of row i at chunk j ^ (i % 8): conflict-free for the writing lanes) and one
// lane hands it to the TMA engine, which writes whole rows and skips what
// lies outside C; the warp does not wait for the writes. Otherwise the block
// is stored element by element.
__device__ __forceinline__ void store_block(float *buf, const uint32_t (&r)[32], const CUtensorMap *tma_c, float *C,
                                            int64_t ldc, int64_t M, int64_t N, int64_t row0, int64_t col0,
                                            int tma_ok, int lane) {
  if (tma_ok) {
    if (row0 < M && col0 < N) {  // the same for the whole warp
      if (lane == 0) bulk_wait_read();  // the warp's previous block has left the buffer
      __syncwarp();
#pragma unroll
      for (int j = 0; j < 8; ++j)
        *reinterpret_cast<float4 *>(buf + lane * 32 + ((j ^ (lane & 7)) << 2)) =
            make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]), __uint_as_float(r[4 * j + 2]),
                        __uint_as_float(r[4 * j + 3]));
      fence_proxy_async_smem();  // the generic-proxy writes, before the TMA engine reads them
      __syncwarp();
      if (lane == 0) {
        tma_store_2d(tma_c, buf, (int)col0, (int)row0);
        bulk_commit();
      }
    }
  } else if (row0 + lane < M) {
    float *crow = C + (row0 + lane) * ldc;
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (col0 + j < N) crow[col0 + j] = __uint_as_float(r[j]);
  }
}

__global__ void __launch_bounds__(NUM_THREADS, 1)
    gemm_bf16_tcgen05_kernel(const __grid_constant__ CUtensorMap tma_a, const __grid_constant__ CUtensorMap tma_b,
                             const __grid_constant__ CUtensorMap tma_c, const Params p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float *epi_buf = reinterpret_cast<float *>(smem + STAGES * STAGE_BYTES);  // [NUM_EPI_WARPS][32 * 32]
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES + NUM_EPI_WARPS * EPI_BUF_BYTES);
  uint64_t *empty = full + STAGES;
  uint64_t *tfull = empty + STAGES;
  uint64_t *tempty = tfull + 1;
  uint64_t *drain = tempty + 1;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int BN = p.BN;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(tfull, 1);
    mbar_init(tempty, 32 * NUM_EPI_WARPS);
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tma_a)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tma_b)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ producer
    uint32_t stage = 0, phase = 0;
    int pending[STAGES] = {0, 0, 0};
    uint32_t pend_phase[STAGES] = {0, 0, 0};
    bool ok = true;
    for (int tile = blockIdx.x; ok && tile < p.num_tiles; tile += gridDim.x) {
      const int tm = tile / p.tiles_n, tn = tile % p.tiles_n;
      for (int kb = 0; kb < p.k_blocks; ++kb) {
        if (!mbar_wait(&empty[stage], phase ^ 1, abort_flag)) {
          ok = false;
          break;
        }
        pending[stage] = 0;  // the previous load of this stage was consumed
        mbar_expect_tx(&full[stage], p.stage_tx);
        uint8_t *sa = smem + stage * STAGE_BYTES;
        uint8_t *sb = sa + A_BYTES;
        if (!p.a_mn) {
          tma_load_2d(&tma_a, &full[stage], sa, kb * BK, tm * BM);
        } else if (p.a_3d) {
          tma_load_3d(&tma_a, &full[stage], sa, 0, kb * BK, tm * (BM / 64));
        } else {
#pragma unroll
          for (int j = 0; j < BM / 64; ++j) tma_load_2d(&tma_a, &full[stage], sa + j * MN_LBO, tm * BM + 64 * j, kb * BK);
        }
        if (!p.b_mn) {
          tma_load_2d(&tma_b, &full[stage], sb, kb * BK, tn * BN);
        } else {
          for (int j = 0; j * 64 < BN; ++j) tma_load_2d(&tma_b, &full[stage], sb + j * MN_LBO, tn * BN + 64 * j, kb * BK);
        }
        pending[stage] = 1;
        pend_phase[stage] = phase;
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1;
        }
      }
    }
    if (!ok) {
      // drain copies still in flight before the CTA's shared memory goes away
      for (int s = 0; s < STAGES; ++s) {
        if (!pending[s]) continue;
        const uint64_t t0 = globaltimer();
        while (!mbar_try_wait(&full[s], pend_phase[s]) && globaltimer() - t0 < kTimeoutNs) {
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------------ MMA issuer
    const uint32_t idesc = idesc_bf16(128, BN, p.a_mn, p.b_mn);
    uint32_t stage = 0, phase = 0;
    bool ok = true;
    int iter = 0;
    for (int tile = blockIdx.x; ok && tile < p.num_tiles; tile += gridDim.x, ++iter) {
      if (!mbar_wait(tempty, (iter & 1) ^ 1, abort_flag)) {
        ok = false;
        break;
      }
      fence_after();
      for (int kb = 0; kb < p.k_blocks; ++kb) {
        if (!mbar_wait(&full[stage], phase, abort_flag)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t a0 = smem_u32(smem + stage * STAGE_BYTES);
        const uint32_t b0 = a0 + A_BYTES;
#pragma unroll
        for (int k = 0; k < BK / 16; ++k) {
          const uint64_t db = operand_desc(b0, p.b_mn, 0, k);
#pragma unroll
          for (int h = 0; h < 2; ++h)  // rows 128*h .. 128*h+127 of the tile
            umma(tmem_base + h * 256, operand_desc(a0, p.a_mn, h, k), db, idesc, (kb | k) != 0);
        }
        umma_commit(&empty[stage]);
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1;
        }
      }
      if (ok) umma_commit(tfull);
    }
    // every MMA of this CTA has completed once this commit arrives
    umma_commit(drain);
    const uint64_t t0 = globaltimer();
    while (!mbar_try_wait(drain, 0) && globaltimer() - t0 < kTimeoutNs) {
    }
  } else if (warp >= 2) {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;         // TMEM lane quarter this warp may access
    const int h = (warp - 2) >> 2;  // accumulator (row half of the tile)
    int iter = 0;
    for (int tile = blockIdx.x; tile < p.num_tiles; tile += gridDim.x, ++iter) {
      const int tm = tile / p.tiles_n, tn = tile % p.tiles_n;
      if (!mbar_wait(tfull, iter & 1, abort_flag)) break;
      fence_after();
      const int64_t row0 = (int64_t)tm * BM + 128 * h + 32 * q;  // this warp's 32 rows
      const uint32_t tbase = tmem_base + h * 256 + ((uint32_t)(32 * q) << 16);
      float *buf = epi_buf + (warp - 2) * (32 * 32);
#pragma unroll 1
      for (int c = 0; c < BN; c += 64) {  // two 32-column blocks per round trip to tensor memory
        uint32_t r0[32], r1[32];
        const bool two = c + 32 < BN;  // the same for the whole warp
        tmem_ld32_async(tbase + c, r0);
        if (two) tmem_ld32_async(tbase + c + 32, r1);
        tmem_wait_ld();
        if (c + 64 >= BN) {
          fence_before();
          mbar_arrive(tempty);
        }
        store_block(buf, r0, &tma_c, p.C, p.ldc, p.M, p.N, row0, (int64_t)tn * BN + c, p.vec_ok, lane);
        if (two) store_block(buf, r1, &tma_c, p.C, p.ldc, p.M, p.N, row0, (int64_t)tn * BN + c + 32, p.vec_ok, lane);
      }
    }
    if (lane == 0) bulk_wait_all();  // the stores of C have completed (and left shared memory)
  }

  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                 : "memory");
  }
}

// ---------------------------------------------------------------- CTA pairs
// The same product with each 256-row block of the tile on two SMs (a cluster
// of two CTAs, tcgen05 cta_group::2): each CTA stages 128 rows of the block's
// A slice and half of the B slice's columns; one M=256 MMA issued by the even
// CTA reads both CTAs' shared memory and writes rows 0..127 of the block's
// accumulator to its own tensor memory and rows 128..255 to its peer's. A
// tile has MH such blocks (256 * MH rows) that share the B slice:
//   MH = 1: each SM's accumulator is 128 x BN, so two fit in tensor memory
//           and the epilogue of one tile overlaps the MMAs of the next; six
//           32 KiB stages;
//   MH = 2: each SM holds two 128 x BN accumulators (one tile, as in the
//           one-SM kernel) but stages only half of each B slice: 23% fewer
//           operand bytes per flop than the one-SM tile; four 48 KiB stages.
//   warp 0 -- TMA producer (both CTAs): its A rows and B columns of a
//             k-slice; the copies of both CTAs complete on the even CTA's
//             full barrier;
//   warp 1 -- allocates 512 TMEM columns in both CTAs (collectively); in the
//             even CTA one thread issues the MMAs (M=256, N=BN, K=16) and
//             commits stage releases and finished accumulators to the
//             barriers of both CTAs;
//   warps 2.. -- epilogue (both CTAs, 4 * MH warps): its rows of the
//             accumulators, then a release arrival on the even CTA's tempty.
template <int MH>
struct Pair {
  static constexpr int A_BYTES = MH * 128 * BK * 2;  // this CTA's 128 rows of each 256-row block
  static constexpr int B_BYTES = 128 * BK * 2;       // this CTA's half of the widest B slice
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int STAGES = MH == 1 ? 6 : 4;
  static constexpr int SLOTS = MH == 1 ? 2 : 1;  // accumulator sets in tensor memory
  static constexpr int EPI_WARPS = 4 * MH;
  static constexpr int THREADS = 64 + 32 * EPI_WARPS;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + EPI_WARPS * EPI_BUF_BYTES + 1024 + 256;
};

struct PairParams {
  float *C;
  int64_t M, N, K, ldc;
  int BN, tiles_n, k_blocks, units;  // units: (256 * MH) x BN tiles
  int a_mn, b_mn;
  int vec_ok;         // C has a tensor map: the epilogue stores through the TMA engine
  int a_3d;           // MN-major A loaded as one 3-D box {64 m, 64 k, 2 m-blocks}
  uint32_t stage_tx;  // bytes both CTAs' copies of one stage deliver to the even CTA's barrier
};

__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_id() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_count() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return r;
}
// All threads of both CTAs; release/acquire orders shared-memory writes (the
// mbarrier initialisation) before the peer's accesses.
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Address in the cluster window of the variable at this CTA-relative shared
// address in the CTA of the given rank.
__device__ __forceinline__ uint32_t map_to_rank(uint32_t smem_addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Copies into this CTA's shared memory whose bytes complete on an mbarrier of
// either CTA of the pair (bar: its address in the cluster window).
__device__ __forceinline__ void tma2_load_2d(const CUtensorMap *map, uint32_t bar, void *dst, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void tma2_load_3d(const CUtensorMap *map, uint32_t bar, void *dst, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y), "r"(z)
      : "memory");
}
__device__ __forceinline__ void umma2(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
// One arrival on the mbarrier at this offset in both CTAs once the MMAs
// issued so far have completed.
__device__ __forceinline__ void umma2_commit_both(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"((uint16_t)3)
      : "memory");
}
__device__ __forceinline__ void umma2_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

template <int MH>
__global__ void __launch_bounds__(Pair<MH>::THREADS, 1)
    gemm_bf16_pair_kernel(const __grid_constant__ CUtensorMap tma_a, const __grid_constant__ CUtensorMap tma_b,
                          const __grid_constant__ CUtensorMap tma_c, const PairParams p) {
  using PC = Pair<MH>;
  constexpr int STAGES_ = PC::STAGES, SLOTS = PC::SLOTS;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float *epi_buf = reinterpret_cast<float *>(smem + STAGES_ * PC::STAGE_BYTES);  // [EPI_WARPS][32 * 32]
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES_ * PC::STAGE_BYTES +
                                                PC::EPI_WARPS * EPI_BUF_BYTES);  // used in the even CTA
  uint64_t *empty = full + STAGES_;
  uint64_t *tfull = empty + STAGES_;  // [SLOTS]: accumulators ready
  uint64_t *tempty = tfull + 2;       // [SLOTS]: accumulators drained by both CTAs (used in the even CTA)
  uint64_t *drain = tempty + 2;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_ctarank();  // 0: issues the MMAs; 1: its peer
  const int BN = p.BN, HN = BN / 2;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES_; ++s) {
      mbar_init(&full[s], 1);   // the even CTA's expect_tx arrival, plus both CTAs' bytes
      mbar_init(&empty[s], 1);  // the MMA commit
    }
    for (int b = 0; b < SLOTS; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 2 * PC::EPI_WARPS);  // one arrival per epilogue warp of both CTAs
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tma_a)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tma_b)) : "memory");
  }
  if (warp == 1) {  // one warp of each CTA of the pair allocates, collectively
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  cluster_sync();  // both CTAs' barriers are initialised before any copy or commit reaches them
  const uint32_t tmem_base = *tmem_slot;
  const int cid = (int)cluster_id(), ncl = (int)cluster_count();
  constexpr int TILE_M = 256 * MH;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ producer (both CTAs)
    const uint32_t full0 = map_to_rank(smem_u32(full), 0);
    uint32_t stage = 0, phase = 0;
    int pending[STAGES_] = {};
    uint32_t pend_phase[STAGES_] = {};
    bool ok = true;
    for (int u = cid; ok && u < p.units; u += ncl) {
      const int tm = u / p.tiles_n, tn = u % p.tiles_n;
      const int col0 = tn * BN + (int)rank * HN;  // this CTA's columns of op(B)
      for (int kb = 0; kb < p.k_blocks; ++kb) {
        if (!mbar_wait(&empty[stage], phase ^ 1, abort_flag)) {
          ok = false;
          break;
        }
        pending[stage] = 0;
        if (rank == 0) mbar_expect_tx(&full[stage], p.stage_tx);
        const uint32_t fb = full0 + stage * 8u;
        uint8_t *sa = smem + stage * PC::STAGE_BYTES;
        uint8_t *sb = sa + PC::A_BYTES;
#pragma unroll
        for (int h = 0; h < MH; ++h) {
          const int row0 = tm * TILE_M + h * 256 + (int)rank * 128;  // this CTA's rows of op(A) in block h
          uint8_t *sah = sa + h * (128 * BK * 2);
          if (!p.a_mn) {
            tma2_load_2d(&tma_a, fb, sah, kb * BK, row0);
          } else if (p.a_3d) {
            tma2_load_3d(&tma_a, fb, sah, 0, kb * BK, row0 / 64);
          } else {
            for (int j = 0; j < 2; ++j) tma2_load_2d(&tma_a, fb, sah + j * MN_LBO, row0 + 64 * j, kb * BK);
          }
        }
        if (!p.b_mn) {
          tma2_load_2d(&tma_b, fb, sb, kb * BK, col0);
        } else {
          for (int j = 0; j * 64 < HN; ++j) tma2_load_2d(&tma_b, fb, sb + j * MN_LBO, col0 + 64 * j, kb * BK);
        }
        pending[stage] = 1;
        pend_phase[stage] = phase;
        if (++stage == STAGES_) {
          stage = 0;
          phase ^= 1;
        }
      }
    }
    // each stage's last use released: no commit reaches this CTA's barriers after it exits
    for (int i = 0; ok && i < STAGES_; ++i) {
      ok = mbar_wait(&empty[stage], phase ^ 1, abort_flag);
      if (++stage == STAGES_) {
        stage = 0;
        phase ^= 1;
      }
    }
    if (!ok && rank == 0) {
      // drain copies still in flight (both CTAs' bytes complete on these barriers)
      for (int s = 0; s < STAGES_; ++s) {
        if (!pending[s]) continue;
        const uint64_t t0 = globaltimer();
        while (!mbar_try_wait(&full[s], pend_phase[s]) && globaltimer() - t0 < kTimeoutNs) {
        }
      }
    }
  } else if (warp == 1 && lane == 0 && rank == 0) {
    // ------------------------------------------------------------ MMA issuer (even CTA)
    const uint32_t idesc = idesc_bf16(256, BN, p.a_mn, p.b_mn);
    uint32_t stage = 0, phase = 0;
    bool ok = true;
    int iter = 0;
    for (int u = cid; ok && u < p.units; u += ncl, ++iter) {
      const int sl = iter % SLOTS;
      const uint32_t use = (uint32_t)(iter / SLOTS);
      if (!mbar_wait(&tempty[sl], (use & 1) ^ 1, abort_flag)) {
        ok = false;
        break;
      }
      fence_after();
      for (int kb = 0; kb < p.k_blocks; ++kb) {
        if (!mbar_wait(&full[stage], phase, abort_flag)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t a0 = smem_u32(smem + stage * PC::STAGE_BYTES);
        const uint32_t b0 = a0 + PC::A_BYTES;
#pragma unroll
        for (int k = 0; k < BK / 16; ++k) {
          const uint64_t db = operand_desc(b0, p.b_mn, 0, k);
#pragma unroll
          for (int h = 0; h < MH; ++h)  // accumulator of block h: columns (sl + h) * 256 ..
            umma2(tmem_base + (uint32_t)(sl + h) * 256, operand_desc(a0 + h * (128 * BK * 2), p.a_mn, 0, k), db,
                  idesc, (kb | k) != 0);
        }
        umma2_commit_both(&empty[stage]);
        if (++stage == STAGES_) {
          stage = 0;
          phase ^= 1;
        }
      }
      if (ok) umma2_commit_both(&tfull[sl]);
    }
    umma2_commit(drain);
    const uint64_t t0 = globaltimer();
    while (!mbar_try_wait(drain, 0) && globaltimer() - t0 < kTimeoutNs) {
    }
  } else if (warp >= 2) {
    // ------------------------------------------------------------ epilogue (both CTAs)
    const int q = warp & 3;         // TMEM lane quarter this warp may access
    const int h = (warp - 2) >> 2;  // 256-row block of the tile
    const uint32_t tempty0 = map_to_rank(smem_u32(tempty), 0);
    int iter = 0;
    for (int u = cid; u < p.units; u += ncl, ++iter) {
      const int sl = iter % SLOTS;
      const uint32_t use = (uint32_t)(iter / SLOTS);
      const int tm = u / p.tiles_n, tn = u % p.tiles_n;
      if (!mbar_wait(&tfull[sl], use & 1, abort_flag)) break;
      fence_after();
      const int64_t row0 = (int64_t)tm * TILE_M + 256 * h + 128 * rank + 32 * q;  // this warp's 32 rows
      const uint32_t tbase = tmem_base + (uint32_t)(sl + h) * 256 + ((uint32_t)(32 * q) << 16);
      float *buf = epi_buf + (warp - 2) * (32 * 32);
#pragma unroll 1
      for (int c = 0; c < BN; c += 64) {  // two 32-column blocks per round trip to tensor memory
        uint32_t r0[32], r1[32];
        const bool two = c + 32 < BN;  // the same for the whole warp
        tmem_ld32_async(tbase + c, r0);
        if (two) tmem_ld32_async(tbase + c + 32, r1);
        tmem_wait_ld();
        if (c + 64 >= BN) {  // accumulator read out: the MMAs may refill it
          fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive_cluster(tempty0 + (uint32_t)sl * 8u);
        }
        store_block(buf, r0, &tma_c, p.C, p.ldc, p.M, p.N, row0, (int64_t)tn * BN + c, p.vec_ok, lane);
        if (two) store_block(buf, r1, &tma_c, p.C, p.ldc, p.M, p.N, row0, (int64_t)tn * BN + c + 32, p.vec_ok, lane);
      }
    }
    if (lane == 0) bulk_wait_all();  // the stores of C have completed (and left shared memory)
  }

  fence_before();
  __syncthreads();
  cluster_sync();  // no CTA frees its tensor memory or leaves while its peer's MMAs or copies may reach it
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                 : "memory");
  }
}

// 3-D view of a row-major K x M bf16 matrix (M contiguous) as {64 m, K, M/64
// blocks}: a box {64, 64, blocks} lands in shared memory as that many
// [64 k][64 m] blocks, the MN-major layout the descriptors read, in one copy.
// Needs M a multiple of 64 (the view never reads past a row).
bool make_map_mn3d(CUtensorMap *map, const void *base, int64_t K, int64_t M, int64_t ld, int blocks);

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  }
  return fn;
}

// 2-D bf16 tensor map of a row-major matrix rows x cols (leading dimension ld
// elements), box {box_inner (along cols), box_outer (along rows)}; the swizzle
// span equals the box's inner extent in bytes (64 or 128).
bool make_map(CUtensorMap *map, const void *base, int64_t rows, int64_t cols, int64_t ld, int box_inner,
              int box_outer) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE,
                  box_inner * 2 == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// f32 tensor map of C (rows x cols, leading dimension ld elements) for the
// epilogue's stores: 32 x 32 boxes of 128-byte rows, 128-byte swizzle.
bool make_map_c(CUtensorMap *map, float *base, int64_t rows, int64_t cols, int64_t ld) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  cuuint32_t box[2] = {32, 32};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool make_map_mn3d(CUtensorMap *map, const void *base, int64_t K, int64_t M, int64_t ld, int blocks) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {64, (cuuint64_t)K, (cuuint64_t)(M / 64)};
  cuuint64_t strides[2] = {(cuuint64_t)ld * 2, 128};
  cuuint32_t box[3] = {64, (cuuint32_t)BK, (cuuint32_t)blocks};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

// Tile width: the BN in {256, 224, ..., 128} whose tiles (tile_m rows) fill
// the fewest waves of the slots that run at once (CTAs, or CTA pairs),
// weighted by the tile's cost (proportional to BN).
int pick_bn(int64_t M, int64_t N, int slots, int tile_m) {
  int best = 256;
  int64_t best_cost = -1;
  for (int bn = 256; bn >= 128; bn -= 32) {
    const int64_t tiles = ceil_div(M, tile_m) * ceil_div(N, bn);
    const int64_t waves = ceil_div(tiles, slots);
    const int64_t cost = waves * bn;
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = bn;
    }
  }
  return best;
}

template <int MH>
cudaLaunchConfig_t pair_config(cudaLaunchAttribute *attr, int grid, cudaStream_t stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(Pair<MH>::THREADS);
  cfg.dynamicSmemBytes = Pair<MH>::SMEM_BYTES;
  cfg.stream = stream;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// CTA pairs of the pair kernel that fit on the GPU at once (0 if none), per device.
template <int MH>
int pair_slots() {
  static int cached[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  if (cached[dev] == 0) {
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = pair_config<MH>(attr, 2 * 64, nullptr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, reinterpret_cast<const void *>(gemm_bf16_pair_kernel<MH>), &cfg) !=
        cudaSuccess) {
      cudaGetLastError();
      n = 0;
    }
    cached[dev] = n > 0 ? n : -1;
  }
  return cached[dev] > 0 ? cached[dev] : 0;
}

cudaError_t set_smem_attrs() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void *>(gemm_bf16_tcgen05_kernel),
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(reinterpret_cast<const void *>(gemm_bf16_pair_kernel<1>),
                             cudaFuncAttributeMaxDynamicSharedMemorySize, Pair<1>::SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(reinterpret_cast<const void *>(gemm_bf16_pair_kernel<2>),
                             cudaFuncAttributeMaxDynamicSharedMemorySize, Pair<2>::SMEM_BYTES);
  if (e == cudaSuccess) done = true;
  return e;
}

// The pair kernel: (256 * MH) x BN tiles, each on a cluster of two CTAs.
template <int MH>
cudaError_t launch_pair(const uint16_t *A, const uint16_t *B, float *C, int64_t M, int64_t N, int64_t K,
                        int64_t lda, int64_t ldb, int64_t ldc, int transA, int transB, int grid, int tile_n,
                        int vec_ok, int fit, cudaStream_t stream) {
  const int clusters = grid > 0 ? (grid / 2 > 0 ? grid / 2 : 1) : fit;
  const int BN = tile_n > 0 ? tile_n : pick_bn(M, N, clusters, 256 * MH);
  const int HN = BN / 2;
  alignas(64) CUtensorMap ma, mb;
  const int a_3d = transA && M % 64 == 0;
  bool ok = transA ? (a_3d ? make_map_mn3d(&ma, A, K, M, lda, 2) : make_map(&ma, A, K, M, lda, 64, BK))
                   : make_map(&ma, A, M, K, lda, BK, 128);
  ok = ok && (transB ? make_map(&mb, B, N, K, ldb, BK, HN) : make_map(&mb, B, K, N, ldb, 64, BK));
  if (!ok) return cudaErrorInvalidValue;
  PairParams p;
  p.C = C;
  p.M = M;
  p.N = N;
  p.K = K;
  p.ldc = ldc;
  p.BN = BN;
  p.tiles_n = (int)ceil_div(N, BN);
  p.k_blocks = (int)ceil_div(K, BK);
  p.units = (int)(ceil_div(M, 256 * MH) * p.tiles_n);
  p.a_mn = transA ? 1 : 0;
  p.b_mn = transB ? 0 : 1;
  alignas(64) CUtensorMap mc;
  p.vec_ok = vec_ok && make_map_c(&mc, C, M, N, ldc);  // else C is stored element by element
  p.a_3d = a_3d;
  const uint32_t b_half = p.b_mn ? (uint32_t)ceil_div(HN, 64) * (64u * BK * 2u) : (uint32_t)HN * BK * 2u;
  p.stage_tx = 2u * ((uint32_t)Pair<MH>::A_BYTES + b_half);
  const int g = 2 * (clusters < p.units ? clusters : p.units);
  void *args[] = {&ma, &mb, &mc, &p};
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg = pair_config<MH>(attr, g, stream);
  return cudaLaunchKernelExC(&cfg, reinterpret_cast<const void *>(gemm_bf16_pair_kernel<MH>), args);
}

// op(A) is M x K: A stored M x K (transA = 0, K-major) or K x M (transA = 1,
// MN-major). op(B) is K x N: B stored K x N (transB = 0, MN-major) or N x K
// (transB = 1, K-major). tile_n = 0 picks BN per shape. cluster: 1 = one CTA
// per 256-row tile (cta_group::1), 2 = a CTA pair per tile of tile_m = 256
// or 512 rows (cta_group::2), 0 = a CTA pair per 512-row tile when M >= 512,
// else one CTA per tile. grid > 0: CTAs of the persistent grid (a pair
// kernel takes whole pairs).
cudaError_t launch_gemm_bf16(const uint16_t *A, const uint16_t *B, float *C, int64_t M, int64_t N, int64_t K,
                             int64_t lda, int64_t ldb, int64_t ldc, int transA, int transB, int grid, int tile_m,
                             int tile_n, int cluster, int vec_ok, cudaStream_t stream) {
  cudaError_t e = set_smem_attrs();
  if (e != cudaSuccess) return e;
  if (cluster == 0 && M >= 512 && pair_slots<2>() > 0) {  // the default for tiles that fill 512 rows
    cluster = 2;
    tile_m = 512;
  }
  if (cluster == 2) {
    const int fit = tile_m == 512 ? pair_slots<2>() : pair_slots<1>();
    if (fit == 0) return cudaErrorInvalidConfiguration;
    return tile_m == 512
               ? launch_pair<2>(A, B, C, M, N, K, lda, ldb, ldc, transA, transB, grid, tile_n, vec_ok, fit, stream)
               : launch_pair<1>(A, B, C, M, N, K, lda, ldb, ldc, transA, transB, grid, tile_n, vec_ok, fit, stream);
  }
  const void *kfn = reinterpret_cast<const void *>(gemm_bf16_tcgen05_kernel);
  const int ctas = grid > 0 ? grid : sm_count();
  const int BN = tile_n > 0 ? tile_n : pick_bn(M, N, ctas, BM);
  alignas(64) CUtensorMap ma, mb;
  const int a_3d = transA && M % 64 == 0;
  bool ok = transA ? (a_3d ? make_map_mn3d(&ma, A, K, M, lda, BM / 64) : make_map(&ma, A, K, M, lda, 64, BK))
                   : make_map(&ma, A, M, K, lda, BK, BM);
  ok = ok && (transB ? make_map(&mb, B, N, K, ldb, BK, BN) : make_map(&mb, B, K, N, ldb, 64, BK));
  if (!ok) return cudaErrorInvalidValue;
  Params p;
  p.C = C;
  p.M = M;
  p.N = N;
  p.K = K;
  p.ldc = ldc;
  p.BN = BN;
  p.tiles_n = (int)ceil_div(N, BN);
  p.num_tiles = (int)(ceil_div(M, BM) * p.tiles_n);
  p.k_blocks = (int)ceil_div(K, BK);
  p.a_mn = transA ? 1 : 0;
  p.b_mn = transB ? 0 : 1;
  alignas(64) CUtensorMap mc;
  p.vec_ok = vec_ok && make_map_c(&mc, C, M, N, ldc);  // else C is stored element by element
  p.a_3d = a_3d;
  const uint32_t b_tx = p.b_mn ? (uint32_t)ceil_div(BN, 64) * (64u * BK * 2u) : (uint32_t)BN * BK * 2u;
  p.stage_tx = (uint32_t)A_BYTES + b_tx;
  int g = ctas < p.num_tiles ? ctas : p.num_tiles;
  void *args[] = {&ma, &mb, &mc, &p};
  return cudaLaunchKernel(kfn, dim3(g), dim3(NUM_THREADS), args, SMEM_BYTES, stream);
}

unsigned *device_status_word() {
  static unsigned *addr[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  if (!addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_device_status) != cudaSuccess) return nullptr;
    addr[dev] = static_cast<unsigned *>(p);
  }
  return addr[dev];
}

cudaError_t poll_device_status(unsigned *out) {
  unsigned zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(out, g_device_status, sizeof(unsigned));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(g_device_status, &zero, sizeof(unsigned));
}

}  // namespace dpia
