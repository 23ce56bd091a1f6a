// tc_gemm.cuh -- tcgen05 tensor-core tiles for the update GEMMs of the mixed
// modes (SYRK U_J = L_RJ L_RJ^T and the blocked trailing update of a panel).
//
// One CTA computes one 128 x 128 tile D = A B^T, where A and B are 128-row slices
// of a row-major panel (K contiguous, i.e. both operands K-major):
// - TMA loads 128-byte-wide K chunks (32 binary32 / 64 bf16 elements per row) with
//   the 128-byte swizzle into a shared-memory ring of 2 or 6 stages (chosen per
//   launch: 2 stages leave room for three CTAs per SM when the launch has tiles
//   for all of them, 6 give one CTA a deeper pipeline when it does not). Rows or
//   columns past the panel read as zeros (out-of-bounds fill).
// - One thread issues tcgen05.mma (kind::tf32 or kind::f16 with bf16 operands)
//   into a 128 x 128 binary32 accumulator in tensor memory and releases each
//   stage with tcgen05.commit.
// - Four warps read the accumulator back with tcgen05.ld (32 columns per load)
//   and apply the masked epilogue (overwrite for U, subtract for the panel),
//   with 16-byte loads and stores where a 32-column run is entirely in the
//   mask; the subtracting epilogue reads the first run of C while the MMAs
//   run and each later run while the previous one is processed.
// Every wait is bounded: on a timeout the CTA records an error code, stops
// issuing, waits (bounded) for its own copies in flight, frees its tensor memory
// and returns.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cstdint>

namespace tc {

constexpr int kMaxStages = 6;
constexpr int kFewStages = 2;
constexpr int kTileM = 128;
constexpr int kTileN = 128;
constexpr int kChunkBytes = 128;                   // K extent of one stage, per row
constexpr int kOperandBytes = kTileM * kChunkBytes;   // 16 KiB per operand per stage
constexpr int kStageBytes = 2 * kOperandBytes;
constexpr int kSmemMax = kMaxStages * kStageBytes + 1024;   // + alignment slack
__host__ __device__ constexpr int smem_bytes(int stages) { return stages * kStageBytes + 1024; }
// Stages for a launch of `tiles` CTAs on `sms` SMs: 2 (three CTAs per SM) when
// every SM gets at least two tiles, else the deep ring.
inline int stages_for(int tiles, int sms) { return tiles >= 2 * sms ? kFewStages : kMaxStages; }
constexpr int kThreads = 128;
constexpr int kTmemCols = 128;

enum : int { kErrNone = 0, kErrTimeoutEmpty = 1, kErrTimeoutFull = 2, kErrTimeoutAccum = 3 };

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

// Bounded wait: gives up after ~2^31 cycles (about a second at 2 GHz).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (it > 16) __nanosleep(32);
    if ((it & 255) == 255 && clock64() - t0 > (1ll << 31)) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);   // start address
  d |= (uint64_t)1 << 16;                      // leading byte offset (unused with this swizzle)
  d |= (uint64_t)(1024 >> 4) << 32;            // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                      // descriptor version
  d |= (uint64_t)2 << 61;                      // 128-byte swizzle
  return d;
}

// Instruction descriptor: D binary32, A/B format (1 = bf16, 2 = tf32), both
// K-major, N = 128, M = 128.
__host__ __device__ constexpr uint32_t instr_desc(uint32_t fmt) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kTileN >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);
}

template <int KIND>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  if (KIND == 0) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
  }
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Geometry of one tile: operand rows a_row / b_row in the panel's tensor map,
// K range [k_begin, k_end), output C (row-major, ldc) with m x n valid entries,
// entry (i, j) written only when i + rdiag >= j; SUB: C -= D, else C = D.
struct TileJob {
  const CUtensorMap* map;
  int a_row, b_row, k_begin, k_end;
  float* C;
  int64_t ldc;
  int m, n, rdiag;
  bool sub;
};

// The CTA body. KIND 0: tf32 operands (32 elements per 128-byte chunk, K = 8 per
// MMA); KIND 1: bf16 operands (64 per chunk, K = 16 per MMA).
template <int KIND>
__device__ __forceinline__ void tile_body(const TileJob& job, uint8_t* smem_raw, int kStages, int* err) {
  __shared__ __align__(8) uint64_t full_bar[kMaxStages];
  __shared__ __align__(8) uint64_t empty_bar[kMaxStages];
  __shared__ __align__(8) uint64_t accum_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ int issued;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  constexpr int kElem = KIND == 0 ? 32 : 64;           // elements per 128-byte chunk row
  constexpr int kInstK = KIND == 0 ? 8 : 16;           // K of one MMA
  constexpr int kMmaPerChunk = kElem / kInstK;         // = 4
  constexpr uint32_t kIdesc = instr_desc(KIND == 0 ? 2u : 1u);
  const int nk = (job.k_end - job.k_begin + kElem - 1) / kElem;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    mbar_init(smem_u32(&accum_bar), 1);
    abort_flag = 0;
    issued = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0 && lane == 0) {
    // producer: TMA loads of the A and B chunks
    int it = 0;
    for (; it < nk; ++it) {
      const int s = it % kStages, round = it / kStages;
      if (round > 0 && !mbar_wait_bounded(smem_u32(&empty_bar[s]), (uint32_t)((round - 1) & 1))) {
        atomicExch(err, kErrTimeoutEmpty);
        abort_flag = 1;
        break;
      }
      if (*(volatile int*)&abort_flag) break;
      const uint32_t fb = smem_u32(&full_bar[s]);
      mbar_expect_tx(fb, (uint32_t)kStageBytes);
      const int kx = job.k_begin + it * kElem;
      tma_load_2d(base + s * kStageBytes, job.map, kx, job.a_row, fb);
      tma_load_2d(base + s * kStageBytes + kOperandBytes, job.map, kx, job.b_row, fb);
    }
    issued = it;
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    int it = 0;
    for (; it < nk; ++it) {
      const int s = it % kStages, round = it / kStages;
      if (!mbar_wait_bounded(smem_u32(&full_bar[s]), (uint32_t)(round & 1))) {
        atomicExch(err, kErrTimeoutFull);
        *(volatile int*)&abort_flag = 1;
        break;
      }
      fence_after();
      const uint32_t a0 = base + s * kStageBytes, b0 = a0 + kOperandBytes;
      const uint64_t ad = sw128_desc(a0), bd = sw128_desc(b0);
#pragma unroll
      for (int kk = 0; kk < kMmaPerChunk; ++kk)
        mma<KIND>(tmem, ad + (uint64_t)(2 * kk), bd + (uint64_t)(2 * kk), kIdesc, (it > 0 || kk > 0) ? 1u : 0u);
      mma_commit(smem_u32(&empty_bar[s]));
    }
    mma_commit(smem_u32(&accum_bar));
  }
  __syncwarp();
  const int row = warp * 32 + lane;
  float* crow = job.C + (int64_t)row * job.ldc;
  // a 32-column run of this thread's row lies inside the tile and the mask and
  // is 16-byte aligned
  auto full_run = [&](int c0) {
    return row < job.m && c0 + 32 <= job.n && row + job.rdiag >= c0 + 31 &&
           (reinterpret_cast<uintptr_t>(crow + c0) & 15u) == 0;
  };
  // subtracting epilogue: the first run of C is read while the MMAs still run,
  // each later run while the one before it is processed
  float4 cbuf[2][8];
  if (job.sub && full_run(0)) {
#pragma unroll
    for (int q = 0; q < 8; ++q) cbuf[0][q] = reinterpret_cast<const float4*>(crow)[q];
  }
  // one thread waits for the accumulator, then the whole CTA reads it
  __shared__ int acc_ready;
  if (threadIdx.x == 0) {
    const bool ok = mbar_wait_bounded(smem_u32(&accum_bar), 0u);
    if (!ok) atomicExch(err, kErrTimeoutAccum);
    acc_ready = ok && !*(volatile int*)&abort_flag;
  }
  __syncthreads();
  fence_after();
  if (acc_ready) {
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
    for (int cb = 0; cb < kTileN / 32; ++cb) {
      const int c0 = cb * 32;
      if (c0 >= job.n) break;                            // uniform across the CTA
      const bool full = full_run(c0);
      if (cb + 1 < kTileN / 32 && job.sub && full_run(c0 + 32)) {
#pragma unroll
        for (int q = 0; q < 8; ++q) cbuf[(cb + 1) & 1][q] = reinterpret_cast<const float4*>(crow + c0 + 32)[q];
      }
      float v[32];
      tmem_ld32(trow + (uint32_t)c0, v);
      if (full) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          float4 o = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
          if (job.sub) {
            const float4 c = cbuf[cb & 1][q];
            o = make_float4(c.x - o.x, c.y - o.y, c.z - o.z, c.w - o.w);
          }
          reinterpret_cast<float4*>(crow + c0)[q] = o;
        }
      } else if (row < job.m) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = c0 + j;
          if (col < job.n && row + job.rdiag >= col) {
            if (job.sub) crow[col] -= v[j];
            else crow[col] = v[j];
          }
        }
      }
    }
  }
  // teardown: after an abort, wait (bounded) for the last copy issued into each
  // stage to land
  if (warp == 0 && lane == 0 && *(volatile int*)&abort_flag) {
    for (int s = 0; s < kStages && s < issued; ++s) {
      const int last_round = (issued - 1 - s) / kStages;
      mbar_wait_bounded(smem_u32(&full_bar[s]), (uint32_t)(last_round & 1));
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

}  // namespace tc
