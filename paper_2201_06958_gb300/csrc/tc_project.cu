// tc_project.cu - the projection of Eqs. 2.15/2.16 with the snapshot difference
// fused in, on the 5th-generation tensor cores (sm_103a).
//
// The snapshot is viewed as N1 x N2 x S (S = product of the modes after the second)
// and cut into 128 x 128 (i1 x i2) tile positions.  Every CTA of the persistent grid
// keeps one tile position and walks a strided set of the slices s:
//   * TMA (cp.async.bulk.tensor) streams each 128 x 16 FP32 strip of V_{k+1} and V_k as
//     two 64 x 16 halves (4 KB boxes) into two 8 KB shared-memory stages, eight strips per
//     tile, sixteen stages, each refilled by its own lane of the TMA warp as soon as it
//     frees;
//   * eight converter warps, one per strip (two stages each), form dV = V_{k+1} - V_k in
//     FP32 (before any rounding), accumulate ||dV||_W^2, round to BF16 and write the tile
//     128-byte-swizzled, releasing each half's stage once it is converted;
//   * one thread issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32 in TMEM) on that tile
//     twice: as the K-major A operand of Z1 = dV x_1 A_1^T (M = i2, K = i1) and as the
//     MN-major A operand of Z2 = dV x_2 A_2^T (M = i1, K = i2); the tile position's rows of
//     the weighted bases A_n = W_n U_n are packed into shared memory as BF16 by the
//     epilogue warps at the start;
//   * four epilogue warps drain the TMEM accumulators (tcgen05.ld) into partial sums
//     over the i1 tiles (Z1) and i2 tiles (Z2).
// A finishing launch sums the partials and contracts the remaining modes, giving every
// Y_n (dS = Y_2 x_2 A_2^T follows in the update kernel or in a mode product).
// Every wait is bounded: on timeout the kernel records a flag, stops issuing, drains
// its own copies and frees TMEM before returning.
#include <cstdio>
#include <cstdlib>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "tc_project.h"

namespace tdb {
namespace {

constexpr int TILE = 128;
constexpr int SUB_I1 = 64, SUB_I2 = 16;                  // one TMA box: half the tile's i1 width x 16 rows of i2
constexpr int NSTRIP = TILE / SUB_I2;                    // 8 strips per tile
constexpr int NHALF = TILE / SUB_I1;                     // 2 halves (along i1) per strip
constexpr int BOX_BYTES = SUB_I1 * SUB_I2 * 4;           // 4 KB
constexpr int STAGE_BYTES = 2 * BOX_BYTES;               // V_{k+1} and V_k boxes of one half strip: 8 KB
constexpr int NSTAGE = NSTRIP * NHALF;                   // stage 2c + h: half h of strip c (converter warp c)
constexpr int BF_TILE_BYTES = TILE * TILE * 2;           // 32 KB
constexpr int HALF_BYTES = BF_TILE_BYTES / 2;            // one 64-wide i1 half: 128 rows x 128 B
constexpr int NUM_EPI_WARPS = 4;                         // warps 0..3 (TMEM lane quadrants 0..3)
constexpr int TMA_WARP = 4;
constexpr int MMA_WARP = 5;
constexpr int CONV_WARP0 = 6;
constexpr int NUM_CONV_WARPS = NSTRIP;                   // converter warp c owns strip c
constexpr int NUM_WARPS = CONV_WARP0 + NUM_CONV_WARPS;   // 14
constexpr int NUM_THREADS = NUM_WARPS * 32;              // 448
constexpr uint32_t TMEM_COLS = 128;                      // 2 buffers x (D1 32 cols + D2 32 cols)
constexpr long long TIMEOUT_CYCLES = 4000000000ll;       // ~2 s at 2 GHz
constexpr int kSmemLimit = 227 * 1024 - 512;             // dynamic shared memory (static use 256 B)

// Every CTA keeps one tile position (q1, q2) and walks the slices s0, s0 + cstep, ...,
// so only that position's two K blocks of each operand image are resident.
struct Params {
  int N1, N2, nslice;
  int nq1, nq2, nq12;            // tile positions: nq1 x nq2
  int cstep;                     // CTAs per tile position
  int r1, r2, r1pad, r2pad;
  int b1_bytes, b2_bytes;        // the position's two K blocks of A_1 and A_2 (BF16 images)
  float* Z1p;                    // [nq1][nslice][r1][N2]  (i2 fastest)
  float* Z2p;                    // [nq2][nslice][r2][N1]  (i1 fastest)
  const float* A1;               // weighted bases A_1 = W_1 U_1 (N1 x r1) and A_2 (N2 x r2), FP32
  const float* A2;
  const float* w1f;             // float copies of w_1, w_2, zero-padded to whole tiles
  const float* w2f;
  const double* wsl;             // slice weights (product over modes >= 3)
  double* npart;                 // ||dV||_W^2 per converter warp: [CTA][NUM_CONV_WARPS]
  unsigned* flags;
  unsigned long long* span;      // profiling: {first CTA start, last CTA end, ...} (global timer), or null
  float dscale;                  // dV = dscale (V_{k+1} - V_k) (1; 1/4 or 1/2 for a central difference): a
                                 // power of two, applied to the accumulators and the norm (exact)
};

// Shared memory of the fused kernel: 1 KB alignment slack, two BF16 tiles, the two image
// blocks, the stages, the barriers.
__host__ __device__ constexpr int smem_fixed_bytes(int b1, int b2) {
  return 1024 + 2 * BF_TILE_BYTES + ((b1 + 1023) & ~1023) + ((b2 + 1023) & ~1023) + 512;
}

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(bar),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* tm) {
  asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)tm) : "memory");
}

// Programmatic launch: wait until the stream's previous kernel has completed and its
// writes are visible (a no-op when the kernel was launched the ordinary way).
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Bounded wait on a phase parity.  Returns false (and raises the abort flag) on
// timeout or when another role already aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, unsigned* flags,
                                          long long limit = TIMEOUT_CYCLES) {
  long long t0 = clock64();
  for (int it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255) == 255) {
      if (*abort_flag) return false;
      if (clock64() - t0 > limit) {
        *abort_flag = 1;
        grid_dep_wait();                 // the previous kernel clears the step's flags
        atomicOr(flags, kFlagTimeout);
        return false;
      }
    }
  }
}

// The same wait for a whole warp: lane 0 polls, the outcome is broadcast (so the lanes
// leave together even when the wait runs out), then every lane takes the completed phase
// itself (it cannot move on before this warp's own next arrival).
__device__ __forceinline__ bool mbar_wait_warp(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                               unsigned* flags) {
  int ok = 0;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, abort_flag, flags) ? 1 : 0;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (ok) mbar_try_wait(bar, parity);
  return ok != 0;
}

// L2 policy for the Z partials: kept in L2 against the streamed snapshots (the finishing
// launch reads them right after this kernel)
__device__ __forceinline__ uint64_t l2_evict_last_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void st_l2_keep(float* p, float v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol) : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* tm, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"((uint64_t)tm), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// Untiled bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"((uint64_t)src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: start, leading / stride byte offsets, version 1,
// 128-byte swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, B K-major, A K- or MN-major.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N, int a_mn_major) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn_major << 15) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Packed FP32 pairs (the .f32x2 forms of sm_100+): two lanes of arithmetic per instruction,
// each element rounded as the scalar instruction would round it.
__device__ __forceinline__ uint64_t f2(float x, float y) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
  return r;
}
__device__ __forceinline__ void f2_split(uint64_t v, float& x, float& y) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(v));
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// ---------------------------------------------------------------------------
// The fused kernel
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NUM_THREADS, 1)
    k_tc_project(const __grid_constant__ CUtensorMap tmVn, const __grid_constant__ CUtensorMap tmVp, Params P) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* bf_tiles = smem;                                          // 2 x 32 KB
  unsigned char* b1_smem = bf_tiles + 2 * BF_TILE_BYTES;                   // A_1 blocks of this position
  unsigned char* b2_smem = b1_smem + ((P.b1_bytes + 1023) & ~1023);        // A_2 blocks
  unsigned char* stages = b2_smem + ((P.b2_bytes + 1023) & ~1023);        // 16 x 8 KB
  uint64_t* bars = (uint64_t*)(stages + NSTAGE * STAGE_BYTES);
  uint64_t* full = bars;                    // [NSTAGE]
  uint64_t* empty = bars + NSTAGE;          // [NSTAGE]
  uint64_t* bf_full = bars + 2 * NSTAGE;
  uint64_t* mma_done = bf_full + 2;
  uint64_t* epi_done = mma_done + 2;
  uint64_t* bimg_full = epi_done + 2;       // the operand images are in place
  uint32_t* tmem_slot = (uint32_t*)(bimg_full + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (P.span && tid == 0) atomicMin(&P.span[0], global_ns());
  // the finishing launch may be scheduled now: it waits for this grid before it reads
  // anything this grid writes
  if (tid == 0) grid_dep_launch();
  // this CTA's tile position and its first slice
  const int pos = blockIdx.x % P.nq12;
  const int q1 = pos % P.nq1, q2 = pos / P.nq1;
  const int s_first = blockIdx.x / P.nq12;

  // lane 0 of the TMA warp initialises the barriers; then lane j (< 16) of that warp, the
  // owner of stage j (half j % 2 of strip j / 2), issues the first slice's half strip at once
  // (every stage is free).  A stage whose rows lie past N2 or whose columns lie past N1 is
  // neither loaded nor waited for, on both sides.  No other warp touches a barrier before
  // the block-wide sync below.
  const int x_tile = q1 * TILE;
  if (warp == TMA_WARP) {
    if (lane == 0) {
      prefetch_tmap(&tmVn);
      prefetch_tmap(&tmVp);
      for (int s = 0; s < NSTAGE; ++s) {
        mbar_init(smem_u32(&full[s]), 1);
        mbar_init(smem_u32(&empty[s]), 1);
      }
      for (int b = 0; b < 2; ++b) {
        mbar_init(smem_u32(&bf_full[b]), NUM_CONV_WARPS);
        mbar_init(smem_u32(&mma_done[b]), 1);
        mbar_init(smem_u32(&epi_done[b]), NUM_EPI_WARPS);
      }
      mbar_init(smem_u32(bimg_full), NUM_EPI_WARPS);
      *abort_flag = 0;
      fence_mbar_init();
      fence_proxy_async();
    }
    __syncwarp();
    const int y = q2 * TILE + (lane >> 1) * SUB_I2, x = x_tile + (lane & 1) * SUB_I1;
    if (lane < NSTAGE && s_first < P.nslice && y < P.N2 && x < P.N1) {
      const uint32_t fb = smem_u32(&full[lane]);
      mbar_arrive_expect_tx(fb, STAGE_BYTES);
      const uint32_t dst = smem_u32(stages + lane * STAGE_BYTES);
      tma_load_3d(dst, &tmVn, x, y, s_first, fb);
      tma_load_3d(dst + BOX_BYTES, &tmVp, x, y, s_first, fb);
    }
  }
  if (warp == MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const uint32_t bf_base = smem_u32(bf_tiles);
  double acc_norm = 0.0;

  if (warp == TMA_WARP) {
    if (lane < NSTAGE) {
      // lane j refills stage j with its half strip of each of this CTA's slices, as soon as
      // its converter releases it; the sixteen lanes poll and issue side by side, so a burst
      // of releases is refilled at once.
      const int j = lane;
      const int nt = s_first < P.nslice ? (P.nslice - 1 - s_first) / P.cstep + 1 : 0;
      const int y = q2 * TILE + (j >> 1) * SUB_I2, x = x_tile + (j & 1) * SUB_I1;
      const bool in = y < P.N2 && x < P.N1;
      int tj = in ? (nt > 0 ? 1 : 0) : nt;      // slices loaded so far (the first at the start)
      const uint32_t fb = smem_u32(&full[j]), eb = smem_u32(&empty[j]);
      const uint32_t dst = smem_u32(stages + j * STAGE_BYTES);
      long long t0 = clock64();
      int it = 0;
      while (tj < nt) {
        if (mbar_test_wait(eb, (tj & 1) ^ 1)) {
          mbar_arrive_expect_tx(fb, STAGE_BYTES);
          const int sl = s_first + tj * P.cstep;
          tma_load_3d(dst, &tmVn, x, y, sl, fb);
          tma_load_3d(dst + BOX_BYTES, &tmVp, x, y, sl, fb);
          ++tj;
          t0 = clock64();
          continue;
        }
        if ((++it & 63) == 63) {
          if (*abort_flag) break;
          if (clock64() - t0 > TIMEOUT_CYCLES) {
            *abort_flag = 1;
            grid_dep_wait();
            atomicOr(P.flags, kFlagTimeout);
            break;
          }
        }
      }
      // drain: every armed copy of this stage has landed before the CTA may leave
      if (in && tj > 0) {
        long long t1 = clock64();
        while (!mbar_try_wait(fb, (tj - 1) & 1) && clock64() - t1 < TIMEOUT_CYCLES) {
        }
      }
    }
  } else if (warp == MMA_WARP) {
    if (lane == 0) {
      const uint32_t idesc1 = instr_desc(128, P.r1pad, 0);
      const uint32_t idesc2 = instr_desc(128, P.r2pad, 1);
      const uint32_t b1 = smem_u32(b1_smem), b2 = smem_u32(b2_smem);
      const uint32_t blk1 = (uint32_t)P.r1pad * 128u, blk2 = (uint32_t)P.r2pad * 128u;
      int t = 0;
      for (int sl = s_first; sl < P.nslice; sl += P.cstep, ++t) {
        const int buf = t & 1;
        if (t == 0 && !mbar_wait(smem_u32(bimg_full), 0, abort_flag, P.flags)) break;
        if (!mbar_wait(smem_u32(&bf_full[buf]), (t >> 1) & 1, abort_flag, P.flags)) break;
        if (t >= 2 && !mbar_wait(smem_u32(&epi_done[buf]), ((t >> 1) - 1) & 1, abort_flag, P.flags)) break;
        tc_fence_after();
        const uint32_t tile = bf_base + buf * BF_TILE_BYTES;
        const uint32_t d1 = tmem_base + buf * 64;
        const uint32_t d2 = tmem_base + buf * 64 + 32;
        // Z1 tile: D1[i2, a] = sum_{i1} dV[i1, i2] A1[i1, a]  (A: K-major view, K = i1)
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          uint64_t ad = smem_desc(tile + (kk >> 2) * HALF_BYTES + (kk & 3) * 32, 16, 1024);
          uint64_t bd = smem_desc(b1 + (kk >> 2) * blk1 + (kk & 3) * 32, 16, 1024);
          mma_bf16(d1, ad, bd, idesc1, kk > 0 ? 1u : 0u);
        }
        // Z2 tile: D2[i1, b] = sum_{i2} dV[i1, i2] A2[i2, b]  (A: MN-major view, M = i1, K = i2)
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          uint64_t ad = smem_desc(tile + kk * 2048, HALF_BYTES, 1024);
          uint64_t bd = smem_desc(b2 + (kk >> 2) * blk2 + (kk & 3) * 32, 16, 1024);
          mma_bf16(d2, ad, bd, idesc2, kk > 0 ? 1u : 0u);
        }
        mma_commit(smem_u32(&mma_done[buf]));
      }
      // make sure the last committed MMAs have finished before TMEM is released
      if (t > 0) {
        const int tl = t - 1;
        long long t0 = clock64();
        while (!mbar_try_wait(smem_u32(&mma_done[tl & 1]), (tl >> 1) & 1) && clock64() - t0 < TIMEOUT_CYCLES) {
        }
      }
    }
  } else if (warp < NUM_EPI_WARPS) {
    // First the BF16 operand images of this tile position: rows q1*128 .. q1*128+127 of
    // A_1 and q2*128 .. of A_2 as two 64-row K blocks each, in the 128-byte-swizzled
    // K-major layout the MMA reads (element (k, a) of block g at g rpad 128 + a 128 +
    // ((k / 8) ^ (a % 8)) 16 + (k % 8) 2 bytes; zero past N_n and r_n).  A thread packs
    // eight consecutive k of one column a per item: one 16-byte shared store.
    {
      const int et = tid;                              // 0 .. 127
      for (int img = 0; img < 2; ++img) {
        const float* A = img == 0 ? P.A1 : P.A2;
        const int N = img == 0 ? P.N1 : P.N2, r = img == 0 ? P.r1 : P.r2, rpad = img == 0 ? P.r1pad : P.r2pad;
        const int i0 = (img == 0 ? q1 : q2) * TILE;
        unsigned char* dst = img == 0 ? b1_smem : b2_smem;
        // float4 reads only where every column of A starts on a 16-byte boundary (N a
        // multiple of 4; a whole float4 is then in or out); otherwise element by element
        const bool vec = (N & 3) == 0;
        for (int item = et; item < 2 * rpad * 8; item += NUM_EPI_WARPS * 32) {
          const int kc = item & 7, a = (item >> 3) % rpad, g = (item >> 3) / rpad;
          const int i = i0 + g * 64 + kc * 8;
          float v[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) v[u] = 0.f;
          if (a < r) {
            const float* col = A + (int64_t)N * a;
            if (vec) {
#pragma unroll
              for (int h = 0; h < 2; ++h)
                if (i + 4 * h < N) {
                  const float4 x = __ldg((const float4*)(col + i + 4 * h));
                  v[4 * h] = x.x; v[4 * h + 1] = x.y; v[4 * h + 2] = x.z; v[4 * h + 3] = x.w;
                }
            } else {
#pragma unroll
              for (int u = 0; u < 8; ++u)
                if (i + u < N) v[u] = __ldg(col + i + u);
            }
          }
          const uint4 pk = make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]),
                                      pack_bf16x2(v[6], v[7]));
          *(uint4*)(dst + g * rpad * 128 + a * 128 + ((kc ^ (a & 7)) << 4)) = pk;
        }
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(bimg_full));
    }
    // epilogue: TMEM lanes 32*warp .. 32*warp+31
    const uint64_t keep = l2_evict_last_policy();
    int t = 0;
    for (int sl = s_first; sl < P.nslice; sl += P.cstep, ++t) {
      const int buf = t & 1;
      if (!mbar_wait_warp(smem_u32(&mma_done[buf]), (t >> 1) & 1, abort_flag, P.flags)) break;
      tc_fence_after();
      const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
      float v[32];
      // Z1 partial, row i2 = q2*128 + 32*warp + lane: column a of the slice's block is
      // contiguous in i2, so each store of the warp covers 32 consecutive floats
      tmem_ld16(tmem_base + lane_base + buf * 64, v);
      if (P.r1pad > 16) tmem_ld16(tmem_base + lane_base + buf * 64 + 16, v + 16);
      {
        const int i2 = q2 * TILE + 32 * warp + lane;
        if (i2 < P.N2) {
          float* dst = P.Z1p + ((size_t)q1 * P.nslice + sl) * (size_t)P.r1 * P.N2 + i2;
#pragma unroll
          for (int a = 0; a < 32; ++a)
            if (a < P.r1) st_l2_keep(dst + (size_t)a * P.N2, v[a] * P.dscale, keep);
        }
      }
      // Z2 partial, row i1 = q1*128 + 32*warp + lane
      tmem_ld16(tmem_base + lane_base + buf * 64 + 32, v);
      if (P.r2pad > 16) tmem_ld16(tmem_base + lane_base + buf * 64 + 48, v + 16);
      {
        const int i1 = q1 * TILE + 32 * warp + lane;
        if (i1 < P.N1) {
          float* dst = P.Z2p + ((size_t)q2 * P.nslice + sl) * (size_t)P.r2 * P.N1 + i1;
#pragma unroll
          for (int b = 0; b < 32; ++b)
            if (b < P.r2) st_l2_keep(dst + (size_t)b * P.N1, v[b] * P.dscale, keep);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&epi_done[buf]));
    }
  } else if (warp >= CONV_WARP0) {
    // converter warp c owns strip c (rows c*16 .. c*16+15 of the tile's i2) and its two
    // half-strip stages 2c, 2c + 1 (i1 halves): it forms dV in FP32, adds its weighted
    // square to ||dV||_W^2, rounds to BF16 and writes the half into the 128-byte-swizzled
    // tile, releasing each stage as soon as that half is converted (its refill then
    // overlaps the other half's conversion)
    const int c = warp - CONV_WARP0;
    const int cx = lane & 15, ry = lane >> 4;
    const int chunk = cx >> 1, hoff = (cx & 1) * 8;
    const bool strip_in = q2 * TILE + c * SUB_I2 < P.N2;
    bool half_in[2];
    uint64_t w1p[2][2];                 // w_1 of this lane's four columns in each half, as pairs
    float w2v[8];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      half_in[h] = q1 * TILE + h * 64 < P.N1;
      const float4 w = __ldg((const float4*)(P.w1f + q1 * TILE + h * 64 + 4 * cx));
      w1p[h][0] = f2(w.x, w.y);
      w1p[h][1] = f2(w.z, w.w);
    }
    // weights of the rows this lane converts (zero past N_2)
#pragma unroll
    for (int k = 0; k < 8; ++k) w2v[k] = __ldg(&P.w2f[q2 * TILE + c * SUB_I2 + ry + 2 * k]);
    int t = 0;
    bool ok = true;
    for (int sl = s_first; sl < P.nslice && ok; sl += P.cstep, ++t) {
      const int buf = t & 1;
      if (t >= 2 && !mbar_wait_warp(smem_u32(&mma_done[buf]), ((t >> 1) - 1) & 1, abort_flag, P.flags)) break;
      const double wsl = __ldg(&P.wsl[sl]);
      float acc = 0.f;
#pragma unroll
      for (int h = 0; h < NHALF; ++h) {
        const int j = 2 * c + h;                      // this half's stage
        const bool loaded = strip_in && half_in[h];
        const bool have = loaded && mbar_wait_warp(smem_u32(&full[j]), t & 1, abort_flag, P.flags);
        if (loaded && !have) { ok = false; break; }
        const float4* vn = (const float4*)(stages + j * STAGE_BYTES);
        const float4* vp = (const float4*)(stages + j * STAGE_BYTES + BOX_BYTES);
        unsigned char* half = bf_tiles + buf * BF_TILE_BYTES + h * HALF_BYTES;
        if (!have) {
          // outside the tensor: zeros in the BF16 tile
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const int r = c * SUB_I2 + ry + 2 * k;
            *(uint2*)(half + r * 128 + ((chunk ^ (r & 7)) << 4) + hoff) = make_uint2(0u, 0u);
          }
          continue;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int row = ry + 2 * k;                 // 0..15 within the strip
          const float4 a = vn[row * 16 + cx];
          const float4 b = vp[row * 16 + cx];
          // dV in FP32 pairs; sum_j w_1(j) dV_j^2 of the row's four columns, then times w_2
          const uint64_t d01 = f2_sub(f2(a.x, a.y), f2(b.x, b.y));
          const uint64_t d23 = f2_sub(f2(a.z, a.w), f2(b.z, b.w));
          const uint64_t q = f2_fma(f2_mul(w1p[h][1], d23), d23, f2_mul(f2_mul(w1p[h][0], d01), d01));
          float q0, q1v, d0, d1, d2, d3;
          f2_split(q, q0, q1v);
          acc = fmaf(w2v[k], q0 + q1v, acc);
          f2_split(d01, d0, d1);
          f2_split(d23, d2, d3);
          const int r = c * SUB_I2 + row;             // tile row (i2 within the tile)
          uint2 pk = make_uint2(pack_bf16x2(d0, d1), pack_bf16x2(d2, d3));
          *(uint2*)(half + r * 128 + ((chunk ^ (r & 7)) << 4) + hoff) = pk;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&empty[j]));
      }
      if (!ok) break;
      acc_norm += (double)acc * wsl;
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bf_full[buf]));
    }
    // this warp's share of ||dV||_W^2, written as soon as its strips are done (the finishing
    // launch adds the partials); dV carries the factor dscale, a power of two (exact)
    const double s = warp_sum(acc_norm);
    if (lane == 0) P.npart[(size_t)blockIdx.x * NUM_CONV_WARPS + c] = s * ((double)P.dscale * (double)P.dscale);
  }

  // TMEM is released once every role is done with it; the kernel completes only after the
  // stream's previous kernel (programmatic launch)
  tc_fence_before();
  __syncthreads();
  if (tid == 0) {
    grid_dep_wait();
    if (P.span) atomicMax(&P.span[1], global_ns());
  }
  if (warp == MMA_WARP) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS) : "memory");
  }
}

// Diagnostic: the projection kernel's bounded mbarrier wait on a barrier that no thread
// and no copy ever arrives at, so that the wait runs out and raises the timeout flag.
__global__ void k_selftest_mbar(unsigned* flags, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait(smem_u32(&bar), 0, &abort_flag, flags, limit);
  __syncthreads();
}

// Finish, first launch.  The fused kernel leaves partial first contractions over the
// tiles q of the contracted mode: Z1p at e + n1 (s + S q), e = i2 + N2 a, n1 = r1 N2
// (mode 1 contracted), and Z2p at f + n2 (s + S q), f = i1 + N1 b, n2 = N1 r2 (mode 2
// contracted), s the slice (i3 + N3 i4).  This launch sums them over q and contracts the
// slices with B (S x J):
//   Y_2[a + r1 (i2 + N2 j)] = sum_s Z1[e, s] B[s, j],    Y_1[f + n2 j] = sum_s Z2[f, s] B[s, j],
// with B = A_3 (three modes), B[i3 + N3 i4, c + r3 d] = A_3[i3, c] A_4[i4, d] (four modes,
// the Kronecker product that contracts modes 3 and 4 at once) or the 1 x 1 identity (two
// modes).  It also writes Z1 = sum_q Z1p when there is more than one tile along mode 1
// (the next launch forms Y_3 from it) and, in its first CTA, ||dV||_W^2 from the fused
// kernel's per-CTA partials.  A CTA owns 256 elements of one side (a thread per element,
// its slice values in registers) and one of `nsplit` slice ranges; the slices' rows of B
// are staged in shared memory and read as float4 broadcasts, 32 outputs j at a time.
// With nsplit > 1 each CTA writes its partial and k_tc_finish_red adds the partials of
// every output in split order (so results do not vary from run to run).
constexpr int FS_TE = 256, FS_SC = 16, FS_JB = 32, FS_JMAX = 128, FS_SPLIT_MAX = 32;
constexpr int FS_CTAS = 2 * 152;   // split target: about two CTAs per SM
constexpr int FS_NQ_MAX = 8;   // tiles along mode 1 or 2 loaded at once; more are added in order after them
struct FinArgs {
  const float* Z1p;
  const float* Z2p;
  int N1, N2, S, nq1, nq2, r1, r2;
  const float* A3;       // N3 x r3 (null: two modes, B = [1])
  const float* A4;       // N4 x r4 (null: three modes)
  int N3, r3, N4, r4, J;
  float* Z1;             // N2 x r1 x S, i2 fastest (written when nq1 > 1 and W is not fused)
  // W = Z1 x_2 A_2^T (r1 x r2 x S: Y_3 for three modes) formed here when a first-side CTA
  // holds whole i2 columns (te1 = N2 floor(256 / N2) elements, N2 <= 256)
  float* W;
  const float* A2;
  int fuse_w, te1;
  float* Y2;
  float* Y1;
  float* part;           // [tile][split][J][256]
  int nsplit, nt1, nt2;
  const double* npart;
  int nnp;
  unsigned long long* span;     // profiling words of the main kernel (see Params), or null
  double* dv2;
};

// Row stride of A_2 in the fused finish's shared memory: = 4 (mod 32), so that the lanes
// of a warp (eight columns b x four i2 phases) read 32 different banks.
__host__ __device__ constexpr int a2_stride(int N2) { return N2 + ((36 - N2 % 32) % 32); }

template <int NQ>   // tiles along the contracted mode, rounded up to a power of two (<= FS_NQ_MAX)
__global__ void __launch_bounds__(FS_TE, 2) k_tc_finish_sk(FinArgs f) {
  constexpr int SC = NQ <= 2 ? FS_SC : (NQ == 4 ? FS_SC / 2 : FS_SC / 4);   // slices per chunk
  constexpr int BPT = FS_SC * FS_JMAX / FS_TE;      // B values a thread stages per chunk
  extern __shared__ __align__(16) float fs_sm[];    // B rows of a slice chunk: [FS_SC][Jp]
  __shared__ double dsh[32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) grid_dep_launch();
  const int tile = blockIdx.x / f.nsplit, sp = blockIdx.x % f.nsplit;
  const bool first = tile < f.nt1;
  const bool fw = first && f.fuse_w;
  const int Jp0 = (f.J + 3) & ~3;
  float* zs = fs_sm + FS_SC * Jp0;                     // fw: the chunk's z values [FS_SC][FS_TE]
  float* a2s = zs + FS_SC * FS_TE;                     // fw: A_2 (N2 x r2, ld a2_stride(N2))
  const int a2st = a2_stride(f.N2);
  if (fw) {
    // A_2 is an input of the step (not written by the main kernel): staged before the wait
    for (int i0 = tid; i0 < f.N2 * f.r2; i0 += 4 * FS_TE) {
      float v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = i0 + k * FS_TE < f.N2 * f.r2 ? __ldg(&f.A2[i0 + k * FS_TE]) : 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int idx = i0 + k * FS_TE;
        if (idx < f.N2 * f.r2) a2s[idx % f.N2 + a2st * (idx / f.N2)] = v[k];
      }
    }
  }
  // programmatic launch: the main kernel's results (partials, norms, span words) are
  // complete and visible after this
  grid_dep_wait();
  if (blockIdx.x == gridDim.x - 1) {
    // ||dV||_W^2: the main kernel's partials, eight loads in flight per thread (in the last
    // CTA, a second-side one whenever there is one: those form no W)
    double t = 0.0;
    for (int i0 = tid; i0 < f.nnp; i0 += 8 * FS_TE) {
      double v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = i0 + k * FS_TE < f.nnp ? __ldcg(&f.npart[i0 + k * FS_TE]) : 0.0;
#pragma unroll
      for (int k = 0; k < 8; ++k) t += v[k];
    }
    t = block_sum(t, dsh);
    if (tid == 0) *f.dv2 = t;
    if (tid == 0 && f.span) {
      // the main kernel has completed: its span into the sums, the words reset for the next
      const unsigned long long a = f.span[0], b = f.span[1];
      if (b > a) {
        f.span[2] += b - a;
        f.span[3] += 1;
      }
      f.span[0] = ~0ull;
      f.span[1] = 0ull;
    }
  }
  const int64_t ne = first ? (int64_t)f.r1 * f.N2 : (int64_t)f.N1 * f.r2;
  const int te = first ? f.te1 : FS_TE;                // elements per CTA on this side
  const int64_t e = (int64_t)(first ? tile : tile - f.nt1) * te + tid;
  const bool in = tid < te && e < ne;
  const int na = fw ? te / f.N2 : 0;                   // a1 values this CTA holds whole
  const int a1_lo = fw ? tile * na : 0;
  const int nq = first ? f.nq1 : f.nq2;
  const float* Pp = (first ? f.Z1p : f.Z2p) + (in ? e : 0);
  const bool write_z = first && f.nq1 > 1 && !f.fuse_w;
  const int J = f.J, Jp = (J + 3) & ~3;
  const int s_lo = (int)((int64_t)f.S * sp / f.nsplit), s_hi = (int)((int64_t)f.S * (sp + 1) / f.nsplit);
  const int64_t qstride = ne * (int64_t)f.S;
  float* mine = f.part + ((int64_t)tile * f.nsplit + sp) * (int64_t)J * FS_TE;
  auto store = [&](int64_t ee, int j, float v) {
    if (first) {
      const int64_t a = ee / f.N2, i2 = ee - a * f.N2;
      f.Y2[a + (int64_t)f.r1 * i2 + ne * (int64_t)j] = v;
    } else {
      f.Y1[ee + ne * (int64_t)j] = v;
    }
  };
  for (int j0 = 0; j0 < J; j0 += FS_JB) {
    const int jn = min(FS_JB, J - j0);
    float acc[FS_JB];
#pragma unroll
    for (int t = 0; t < FS_JB; ++t) acc[t] = 0.f;
    for (int s0 = s_lo; s0 < s_hi; s0 += SC) {
      const int sc = min(SC, s_hi - s0);
      // this element's slice values summed over q: every load of the chunk is issued
      // into registers before the first addition
      float raw[SC * NQ];
#pragma unroll
      for (int u = 0; u < SC; ++u) {
        const float* pe = Pp + ne * (int64_t)(s0 + u);
#pragma unroll
        for (int q = 0; q < NQ; ++q) raw[u * NQ + q] = (in && u < sc && q < nq) ? __ldcg(pe + qstride * q) : 0.f;
      }
      // this chunk's B rows, loaded beside the partials (staged in shared memory below)
      float bpre[BPT];
#pragma unroll
      for (int k = 0; k < BPT; ++k) {
        const int idx = tid + k * FS_TE;
        float bv = 0.f;
        if (idx < SC * Jp) {
          const int sl = idx % SC, j = idx / SC;       // consecutive threads: consecutive slices
          if (sl < sc && j < J) {
            const int s = s0 + sl;
            if (!f.A3) {
              bv = 1.f;
            } else if (!f.A4) {
              bv = __ldg(&f.A3[s + (int64_t)f.N3 * j]);
            } else {
              const int i3 = s % f.N3, i4 = s / f.N3, c = j % f.r3, dd = j / f.r3;
              bv = __ldg(&f.A3[i3 + (int64_t)f.N3 * c]) * __ldg(&f.A4[i4 + (int64_t)f.N4 * dd]);
            }
          }
        }
        bpre[k] = bv;
      }
      float z[SC];
#pragma unroll
      for (int u = 0; u < SC; ++u) {
        float v = raw[u * NQ];
#pragma unroll
        for (int q = 1; q < NQ; ++q) v += raw[u * NQ + q];
        if (NQ == FS_NQ_MAX && nq > NQ && in && u < sc) {
          // a long mode (more than FS_NQ_MAX tiles): the rest in tile order
          const float* pe = Pp + ne * (int64_t)(s0 + u);
          for (int q = NQ; q < nq; ++q) v += __ldcg(pe + qstride * q);
        }
        z[u] = v;
      }
      if (write_z && j0 == 0 && in) {
#pragma unroll
        for (int u = 0; u < SC; ++u)
          if (u < sc) f.Z1[e + ne * (int64_t)(s0 + u)] = z[u];
      }
      __syncthreads();                                   // the previous chunk is done with zs, fs_sm
      if (fw && j0 == 0) {
#pragma unroll
        for (int u = 0; u < SC; ++u) zs[u * FS_TE + tid] = (in && u < sc) ? z[u] : 0.f;
      }
#pragma unroll
      for (int k = 0; k < BPT; ++k) {
        const int idx = tid + k * FS_TE;
        if (idx < SC * Jp) fs_sm[(idx % SC) * Jp + idx / SC] = bpre[k];
      }
      __syncthreads();
      if (fw && j0 == 0) {
        // W[a1, a2, s] = sum_i2 Z1[i2, a1, s] A2[i2, a2] for this CTA's whole columns a1: a
        // warp per (a1, eight a2, four slices); lane (b, phase) sums i2 = phase (mod 4) for
        // the four slices side by side, then the four phases are added by shuffles
        if ((f.N2 & 3) == 0) {
          // whole float4 runs of i2: a thread per output (a1, slice, a2), a2 fastest, two
          // chains (even and odd runs) added at the end
          const int nout = na * sc * f.r2;
          for (int o = tid; o < nout; o += FS_TE) {
            const int b = o % f.r2, rest = o / f.r2, u = rest % sc, al = rest / sc;
            const float4* zc = reinterpret_cast<const float4*>(zs + u * FS_TE + al * f.N2);
            const float4* ac = reinterpret_cast<const float4*>(a2s + a2st * b);
            float w0 = 0.f, w1 = 0.f;
            const int nq4 = f.N2 >> 2;
            int q = 0;
#pragma unroll 2
            for (; q + 1 < nq4; q += 2) {
              const float4 z0 = zc[q], a0 = ac[q], z1 = zc[q + 1], a1v = ac[q + 1];
              w0 = fmaf(z0.x, a0.x, w0); w0 = fmaf(z0.y, a0.y, w0); w0 = fmaf(z0.z, a0.z, w0); w0 = fmaf(z0.w, a0.w, w0);
              w1 = fmaf(z1.x, a1v.x, w1); w1 = fmaf(z1.y, a1v.y, w1); w1 = fmaf(z1.z, a1v.z, w1); w1 = fmaf(z1.w, a1v.w, w1);
            }
            if (q < nq4) {
              const float4 z0 = zc[q], a0 = ac[q];
              w0 = fmaf(z0.x, a0.x, w0); w0 = fmaf(z0.y, a0.y, w0); w0 = fmaf(z0.z, a0.z, w0); w0 = fmaf(z0.w, a0.w, w0);
            }
            const int a1 = a1_lo + al;
            if (a1 < f.r1) f.W[a1 + (int64_t)f.r1 * (b + (int64_t)f.r2 * (s0 + u))] = w0 + w1;
          }
        } else {
          const int nbg = (f.r2 + 7) >> 3, nug = (sc + 3) >> 2;
          const int nitem = na * nbg * nug;
          const int bl = lane & 7, ph = lane >> 3;
          for (int item = warp; item < nitem; item += FS_TE / 32) {
            const int bg = item % nbg, rest = item / nbg, al = rest % na, u0 = 4 * (rest / na);
            const int b = bg * 8 + bl;
            const float* zc = zs + u0 * FS_TE + al * f.N2;
            const float* ac = a2s + a2st * (b < f.r2 ? b : f.r2 - 1);
            float w[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
            for (int i2 = ph; i2 < f.N2; i2 += 4) {
              const float av = ac[i2];
#pragma unroll
              for (int u = 0; u < 4; ++u) w[u] = fmaf(zc[u * FS_TE + i2], av, w[u]);
            }
            const int a1 = a1_lo + al;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              float x = w[u];
              x += __shfl_xor_sync(0xffffffffu, x, 8);
              x += __shfl_xor_sync(0xffffffffu, x, 16);
              if (ph == 0 && b < f.r2 && a1 < f.r1 && u0 + u < sc)
                f.W[a1 + (int64_t)f.r1 * (b + (int64_t)f.r2 * (s0 + u0 + u))] = x;
            }
          }
        }
      }
#pragma unroll
      for (int u = 0; u < SC; ++u) {
        const float* brow = fs_sm + u * Jp + j0;
#pragma unroll
        for (int t4 = 0; t4 < FS_JB / 4; ++t4) {
          if (4 * t4 < jn) {
            const float4 bb = *reinterpret_cast<const float4*>(brow + 4 * t4);
            acc[4 * t4] = fmaf(bb.x, z[u], acc[4 * t4]);
            acc[4 * t4 + 1] = fmaf(bb.y, z[u], acc[4 * t4 + 1]);
            acc[4 * t4 + 2] = fmaf(bb.z, z[u], acc[4 * t4 + 2]);
            acc[4 * t4 + 3] = fmaf(bb.w, z[u], acc[4 * t4 + 3]);
          }
        }
      }
    }
    if (f.nsplit == 1) {
      if (in) {
#pragma unroll
        for (int t = 0; t < FS_JB; ++t)
          if (t < jn) store(e, j0 + t, acc[t]);
      }
    } else {
#pragma unroll
      for (int t = 0; t < FS_JB; ++t)
        if (t < jn) mine[(int64_t)(j0 + t) * FS_TE + tid] = acc[t];
    }
  }
}

// Finish, split partials: output (e, j) of a tile is the sum of its nsplit partials in
// split order (one thread per output, every load issued before the additions).
__global__ void __launch_bounds__(256) k_tc_finish_red(FinArgs f) {
  grid_dep_wait();                  // programmatic launch: the split partials are complete
  const int J = f.J;
  const int64_t per_tile = (int64_t)J * FS_TE;
  const int64_t total = (int64_t)(f.nt1 + f.nt2) * per_tile;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < total; o += (int64_t)gridDim.x * blockDim.x) {
    const int tile = (int)(o / per_tile);
    const int rem = (int)(o % per_tile);
    const int j = rem / FS_TE, x = rem % FS_TE;
    const bool first = tile < f.nt1;
    const int64_t ne = first ? (int64_t)f.r1 * f.N2 : (int64_t)f.N1 * f.r2;
    const int te = first ? f.te1 : FS_TE;
    const int64_t e = (int64_t)(first ? tile : tile - f.nt1) * te + x;
    if (x >= te || e >= ne) continue;
    const float* base = f.part + (int64_t)tile * f.nsplit * per_tile + (int64_t)j * FS_TE + x;
    float vals[FS_SPLIT_MAX];
#pragma unroll
    for (int q = 0; q < FS_SPLIT_MAX; ++q) vals[q] = q < f.nsplit ? __ldcg(&base[(int64_t)q * per_tile]) : 0.f;
    float v = 0.f;
#pragma unroll
    for (int q = 0; q < FS_SPLIT_MAX; ++q) v += vals[q];
    if (first) {
      const int64_t a = e / f.N2, i2 = e - a * f.N2;
      f.Y2[a + (int64_t)f.r1 * i2 + ne * (int64_t)j] = v;
    } else {
      f.Y1[e + ne * (int64_t)j] = v;
    }
  }
}


// Three-mode finish, second launch: Y_3 = Z1 x_2 A_2^T (r1 x r2 x S), a CTA per
// slice, i2 in chunks of FB_CH staged in shared memory (thread per output (a1, a2)).
// dS = Y_3 x_3 A_3^T follows in the update kernel.
constexpr int FB_CH = 128;
constexpr size_t kFinishBSmem = (size_t)(32 * FB_CH + 32 * (FB_CH + 1)) * sizeof(float);
__global__ void __launch_bounds__(256) k_tc_finish_b(const float* __restrict__ Z1, int N2, int S, int r1, int r2,
                                                     const float* __restrict__ A2, float* __restrict__ Y3) {
  extern __shared__ float fb_sm[];
  float* zs = fb_sm;                   // r1 x FB_CH (element a + r1 il), from Z1 at i2 + N2 a + r1 N2 s
  float* as = zs + 32 * FB_CH;         // FB_CH x r2 (ld FB_CH + 1)
  const int tid = threadIdx.x;
  const int64_t n1 = (int64_t)r1 * N2;
  for (int sl = blockIdx.x; sl < S; sl += gridDim.x) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int i0 = 0; i0 < N2; i0 += FB_CH) {
      const int ch = min(FB_CH, N2 - i0);
      const float* src = Z1 + i0 + n1 * sl;
#pragma unroll 4
      for (int e = tid; e < r1 * ch; e += 256) {
        const int il = e % ch, a = e / ch;
        zs[a + r1 * il] = __ldcg(&src[il + (int64_t)N2 * a]);
      }
#pragma unroll 4
      for (int e = tid; e < ch * r2; e += 256) {
        const int il = e % ch, b = e / ch;
        as[il + (FB_CH + 1) * b] = __ldg(&A2[i0 + il + (int64_t)N2 * b]);
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int o = tid + 256 * j;
        const int a1 = o % r1, a2 = o / r1;
        if (a2 < r2)
          for (int il = 0; il < ch; ++il) acc[j] = fmaf(as[il + (FB_CH + 1) * a2], zs[a1 + r1 * il], acc[j]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int o = tid + 256 * j;
      const int a1 = o % r1, a2 = o / r1;
      if (a2 < r2) Y3[a1 + (int64_t)r1 * (a2 + (int64_t)r2 * sl)] = acc[j];
    }
  }
}

// Copies of V_{k+1} and V_k with the rows of mode 1 padded to N1p (a multiple of 4, the
// 16-byte row stride TMA needs) by zeros: a[i + N1p c] = (i < N1 ? V[i + N1 c] : 0).
__global__ void k_pad_rows(const float* __restrict__ Vn, const float* __restrict__ Vp, int N1, int N1p, int64_t ncol,
                           float* __restrict__ an, float* __restrict__ ap) {
  const int64_t tot = (int64_t)N1p * ncol;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / N1p;
    const int i = (int)(e - c * N1p);
    const bool in = i < N1;
    an[e] = in ? __ldcs(&Vn[i + (int64_t)N1 * c]) : 0.f;
    ap[e] = in ? __ldcs(&Vp[i + (int64_t)N1 * c]) : 0.f;
  }
}

// Float copies of w_1 and w_2, zero-padded to whole 128-wide tiles (read by the converters).
__global__ void k_weights_f(const double* w1, int N1, int L1, const double* w2, int N2, int L2, float* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L1 + L2; i += gridDim.x * blockDim.x)
    out[i] = (i < L1) ? (i < N1 ? (float)w1[i] : 0.f) : (i - L1 < N2 ? (float)w2[i - L1] : 0.f);
}

__global__ void k_slice_weights(int p, const double* w3, int N3, const double* w4, int N4, double* out) {
  int n = (p >= 3 ? N3 : 1) * (p >= 4 ? N4 : 1);
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    double v = 1.0;
    if (p >= 3) v *= w3[s % N3];
    if (p >= 4) v *= w4[s / N3];
    out[s] = v;
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

bool get_encoder(std::string& err) {
  if (g_encode) return true;
  cudaDriverEntryPointQueryResult q;
  void* fn = nullptr;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
    err = "cuTensorMapEncodeTiled unavailable";
    return false;
  }
  g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  return true;
}

// ld1: row pitch of mode 1 in elements (N1, or N1 rounded up to 4 for a padded copy)
bool encode_map(CUtensorMap* tm, const float* base, int N1, int ld1, int N2, int nslice, std::string& err) {
  cuuint64_t dims[3] = {(cuuint64_t)ld1, (cuuint64_t)N2, (cuuint64_t)nslice};
  cuuint64_t strides[2] = {(cuuint64_t)ld1 * 4, (cuuint64_t)ld1 * N2 * 4};
  cuuint32_t box[3] = {SUB_I1, SUB_I2, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
    return false;
  }
  return true;
}

int rpad_of(int r) { return r <= 16 ? 16 : 32; }

}  // namespace

// ---------------------------------------------------------------------------
// Launch-shape tuner.  The tile (128 x 128, eight 16-row strips) is fixed by the MMA
// shape and the TMEM layout; what varies with the tensor's shape is the work split: how
// many CTAs share a tile position in the persistent grid (all SMs for a large tensor;
// fewer can win for a small one, whose per-CTA start-up then dominates), and how many
// slice ranges the finishing contraction splits into.  On a plan's first call outside
// stream capture every candidate is timed with CUDA events on the call's own inputs (one
// warm-up and three timed launches) and the fastest kept; choices are cached per shape
// and device for the process.
// ---------------------------------------------------------------------------
struct TuneKey {
  int dev, N1, ld1, N2, nslice, r1pad, r2pad, J, p;
  bool operator<(const TuneKey& o) const {
    return std::tie(dev, N1, ld1, N2, nslice, r1pad, r2pad, J, p) <
           std::tie(o.dev, o.N1, o.ld1, o.N2, o.nslice, o.r1pad, o.r2pad, o.J, o.p);
  }
};
struct TuneChoice {
  int cstep, fin_target;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneChoice> g_tune_cache;

bool tune_lookup(const TuneKey& k, TcPlan& plan) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune_cache.find(k);
  if (it == g_tune_cache.end()) return false;
  plan.cstep = it->second.cstep;
  plan.fin_target = it->second.fin_target;
  plan.ncand = 0;
  plan.from_cache = true;
  return true;
}

void tune_store(const TuneKey& k, const TcPlan& plan) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[k] = TuneChoice{plan.cstep, plan.fin_target};
}

template <typename FP, typename FF>
void tune_shape(TcPlan& plan, int cmax, FP&& project, FF&& finish, cudaStream_t s) {
  cudaEvent_t ea = nullptr, eb = nullptr;
  cudaEventCreate(&ea);
  cudaEventCreate(&eb);
  auto time_us = [&](auto&& fn) {
    fn();
    cudaEventRecord(ea, s);
    for (int i = 0; i < 3; ++i) fn();
    cudaEventRecord(eb, s);
    cudaEventSynchronize(eb);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ea, eb);
    return ms * 1000.f / 3.f;
  };
  int cands[TcPlan::kMaxCand];
  int nc = 0;
  for (int c : {cmax, (3 * cmax + 3) / 4, (cmax + 1) / 2, (cmax + 3) / 4}) {
    c = std::max(1, c);
    bool dup = false;
    for (int i = 0; i < nc; ++i) dup |= cands[i] == c;
    if (!dup && nc < TcPlan::kMaxCand) cands[nc++] = c;
  }
  plan.ncand = nc;
  int best = cmax;
  float best_us = 1e30f;
  for (int i = 0; i < nc; ++i) {
    const float us = time_us([&] { project(cands[i]); });
    plan.cand[i] = cands[i];
    plan.cand_us[i] = us;
    if (us < best_us) { best_us = us; best = cands[i]; }
  }
  plan.cstep = best;
  project(best);                      // partials of the chosen shape for the finish candidates
  int fbest = FS_CTAS;
  float fbest_us = 1e30f;
  const int targets[3] = {152, 2 * 152, 4 * 152};
  for (int i = 0; i < 3; ++i) {
    const float us = time_us([&] { finish(targets[i]); });
    plan.fin_cand[i] = targets[i];
    plan.fin_us[i] = us;
    if (us < fbest_us) { fbest_us = us; fbest = targets[i]; }
  }
  plan.fin_target = fbest;
  plan.from_cache = false;
  cudaEventDestroy(ea);
  cudaEventDestroy(eb);
}

tdb_status tc_selftest_mbar_wait(unsigned* flags, long long limit, cudaStream_t s) {
  k_selftest_mbar<<<1, 32, 0, s>>>(flags, limit);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? TDB_OK : TDB_ERR_CUDA;
}

bool tc_supported(int p, const int64_t* N, const int* cap, std::string& err) {
  if (p < 2 || p > 4) { err = "needs 2..4 modes"; return false; }
  if (cap[0] > 32 || cap[1] > 32) { err = "ranks of modes 1, 2 must be <= 32"; return false; }
  int dev = 0, major = 0, minor = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (major != 10) { err = "needs a compute capability 10.x GPU (tcgen05)"; return false; }
  // each CTA holds its tile position's two K blocks of each image
  const int b1 = 2 * rpad_of(cap[0]) * 128, b2 = 2 * rpad_of(cap[1]) * 128;
  if (smem_fixed_bytes(b1, b2) + NSTAGE * STAGE_BYTES > kSmemLimit) {
    err = "shared memory budget exceeded";
    return false;
  }
  return get_encoder(err);
}

void tc_carve(TcPlan& plan, Carver& cv, int p, const int64_t* N, const int* cap) {
  plan.p = p;
  int64_t nslice = 1;
  for (int n = 2; n < p; ++n) nslice *= N[n];
  int nq1 = (int)((N[0] + TILE - 1) / TILE), nq2 = (int)((N[1] + TILE - 1) / TILE);
  plan.z1p = cv.take<float>((size_t)nq1 * nslice * N[1] * cap[0]);
  plan.z2p = cv.take<float>((size_t)nq2 * nslice * N[0] * cap[1]);
  plan.wsl = cv.take<double>((size_t)nslice);
  if (N[0] % 4 != 0) {
    const size_t padn = (size_t)((N[0] + 3) & ~3) * N[1] * nslice;
    plan.pad[0] = cv.take<float>(padn);
    plan.pad[1] = cv.take<float>(padn);
  }
  plan.w12f = cv.take<float>((size_t)(nq1 + nq2) * TILE);
  plan.npart = cv.take<double>((size_t)1024 * NUM_CONV_WARPS);
  // finish: split partials ((FS_CTAS + tiles) x 256 x J floats bound nsplit x tiles x 256 x J
  // for the split count the launch picks)
  const int jmax = p == 2 ? 1 : (p == 3 ? cap[2] : cap[2] * cap[3]);
  const int64_t ntmax = ((int64_t)cap[0] * N[1] + FS_TE - 1) / FS_TE + ((int64_t)N[0] * cap[1] + FS_TE - 1) / FS_TE;
  plan.fpart_cap = (size_t)(FS_CTAS + ntmax) * FS_TE * jmax;
  plan.fpart = cv.take<float>(plan.fpart_cap);
}

tdb_status tc_project(TcPlan& plan, const float* Vn, const float* Vp, int p, const int64_t* N, const int* r,
                      const void* const* A, const double* const* w, float* Z1, float* Z2, float* scratch,
                      float* dS, float* const* Y, double* dv2, unsigned* flags, cudaStream_t s, cudaEvent_t* evm,
                      std::string& err, bool defer_ds, float dscale, bool pdl) {
  if (!get_encoder(err)) return TDB_ERR_UNSUPPORTED;
  const int N1 = (int)N[0], N2 = (int)N[1];
  int nslice = 1;
  for (int n = 2; n < p; ++n) nslice *= (int)N[n];
  const int nq1 = (N1 + TILE - 1) / TILE, nq2 = (N2 + TILE - 1) / TILE;
  const int r1pad = rpad_of(r[0]), r2pad = rpad_of(r[1]);
  if (!plan.wsl_ready) {
    k_slice_weights<<<(nslice + 255) / 256, 256, 0, s>>>(p, p >= 3 ? w[2] : nullptr, p >= 3 ? (int)N[2] : 1,
                                                         p >= 4 ? w[3] : nullptr, p >= 4 ? (int)N[3] : 1, plan.wsl);
    count_launch();
    k_weights_f<<<((nq1 + nq2) * TILE + 255) / 256, 256, 0, s>>>(w[0], N1, nq1 * TILE, w[1], N2, nq2 * TILE,
                                                                plan.w12f);
    count_launch();
    plan.wsl_ready = true;
  }
  // rows of mode 1 whose byte length is not a multiple of 16: the kernel streams zero-padded
  // copies of both snapshots instead (TMA's row stride rule)
  const int ld1 = (N1 + 3) & ~3;
  if (ld1 != N1) {
    if (!plan.pad[0] || !plan.pad[1]) {
      err = "no padded snapshot buffers (N_1 not a multiple of 4)";
      return TDB_ERR_UNSUPPORTED;
    }
    const int64_t tot = (int64_t)ld1 * N2 * nslice;
    k_pad_rows<<<(int)std::min<int64_t>((tot + 255) / 256, 152 * 16), 256, 0, s>>>(Vn, Vp, N1, ld1,
                                                                                   (int64_t)N2 * nslice, plan.pad[0],
                                                                                   plan.pad[1]);
    count_launch();
    Vn = plan.pad[0];
    Vp = plan.pad[1];
  }
  CUtensorMap tmn, tmp;
  if (!encode_map(&tmn, Vn, N1, ld1, N2, nslice, err) || !encode_map(&tmp, Vp, N1, ld1, N2, nslice, err))
    return TDB_ERR_UNSUPPORTED;
  Params P;
  memset(&P, 0, sizeof(P));
  P.N1 = N1;
  P.N2 = N2;
  P.nslice = nslice;
  P.nq1 = nq1;
  P.nq2 = nq2;
  P.r1 = r[0];
  P.r2 = r[1];
  P.r1pad = r1pad;
  P.r2pad = r2pad;
  P.nq12 = nq1 * nq2;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  // persistent grid: for every tile position the same number of CTAs (at most one per SM
  // in all), each walking a strided set of the slices; how many is the tuner's choice
  const int cmax = std::max(1, std::min(nslice, std::min(nsm, 1024) / P.nq12));
  P.b1_bytes = 2 * r1pad * 128;
  P.b2_bytes = 2 * r2pad * 128;
  const int fixed = smem_fixed_bytes(P.b1_bytes, P.b2_bytes);
  if (fixed + NSTAGE * STAGE_BYTES > kSmemLimit) {
    err = "shared memory budget exceeded";
    return TDB_ERR_UNSUPPORTED;
  }
  const size_t smem = (size_t)fixed + (size_t)NSTAGE * STAGE_BYTES;
  P.Z1p = plan.z1p;
  P.Z2p = plan.z2p;
  P.A1 = (const float*)A[0];
  P.A2 = (const float*)A[1];
  P.w1f = plan.w12f;
  P.w2f = plan.w12f + nq1 * TILE;
  P.wsl = plan.wsl;
  P.npart = plan.npart;
  P.flags = flags;
  P.dscale = dscale;
  P.span = plan.tuned ? plan.span : nullptr;
  if (!plan.attr_set) {
    cudaFuncSetAttribute(k_tc_project, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    plan.attr_set = true;
  }
  // (the tuner launches it plainly: a programmatic launch would overlap the launch before)
  auto launch_project = [&](int cstep, bool prog) {
    P.cstep = cstep;
    if (prog) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(P.nq12 * cstep);
      cfg.blockDim = dim3(NUM_THREADS);
      cfg.dynamicSmemBytes = smem;
      cfg.stream = s;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      at[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      cudaLaunchKernelEx(&cfg, k_tc_project, tmn, tmp, P);
    } else {
      k_tc_project<<<P.nq12 * cstep, NUM_THREADS, smem, s>>>(tmn, tmp, P);
    }
    count_launch();
  };
  // finish: Y_1, Y_2 (and Z1) from the tile partials, the slices contracted with
  // B = A_3 (x A_4); then Y_3 (three modes) or W = Z1 x_2 A_2^T (four modes) per slice
  const int J = p == 2 ? 1 : (p == 3 ? r[2] : r[2] * r[3]);
  // W = Z1 x_2 A_2^T inside the finish when its first-side CTAs can hold whole i2 columns
  const bool fuse_w = p >= 3 && N2 <= FS_TE;
  const int te1 = fuse_w ? N2 * (FS_TE / N2) : FS_TE;
  const int nt1 = (int)(((int64_t)r[0] * N2 + te1 - 1) / te1);
  const int nt2 = (int)(((int64_t)N1 * r[1] + FS_TE - 1) / FS_TE);
  if (J > FS_JMAX) {
    err = "finish: r_3 r_4 above 128";
    return TDB_ERR_UNSUPPORTED;
  }
  // splits per tile: the grid stays within the target (whole waves of resident CTAs: two
  // per SM), at least one split
  auto nsplit_for = [&](int target) {
    int ns = (int)std::max<int64_t>(1, target / (nt1 + nt2));
    ns = std::min({ns, std::max(1, nslice / FS_SC), FS_SPLIT_MAX});
    while (ns > 1 && (size_t)ns * (nt1 + nt2) * FS_TE * J > plan.fpart_cap) --ns;
    return ns;
  };
  FinArgs f;
  f.Z1p = plan.z1p;
  f.Z2p = plan.z2p;
  f.N1 = N1;
  f.N2 = N2;
  f.S = nslice;
  f.nq1 = nq1;
  f.nq2 = nq2;
  f.r1 = r[0];
  f.r2 = r[1];
  f.A3 = p >= 3 ? (const float*)A[2] : nullptr;
  f.A4 = p >= 4 ? (const float*)A[3] : nullptr;
  f.N3 = p >= 3 ? (int)N[2] : 1;
  f.r3 = p >= 3 ? r[2] : 1;
  f.N4 = p >= 4 ? (int)N[3] : 1;
  f.r4 = p >= 4 ? r[3] : 1;
  f.J = J;
  f.Z1 = Z1;
  f.W = p == 3 ? Y[2] : scratch;
  f.A2 = (const float*)A[1];
  f.fuse_w = fuse_w ? 1 : 0;
  f.te1 = te1;
  f.Y2 = Y[1];
  f.Y1 = Y[0];
  f.part = plan.fpart;
  f.nt1 = nt1;
  f.nt2 = nt2;
  f.npart = plan.npart;
  f.span = nullptr;
  f.dv2 = dv2;
  const size_t fsm = sizeof(float) * (FS_SC * ((J + 3) & ~3) +
                                      (fuse_w ? FS_SC * FS_TE + (size_t)a2_stride(N2) * r[1] : 0));
  if (fsm > 48 * 1024) {
    static bool fs_attr = false;
    if (!fs_attr) {
      const int lim = 100 * 1024;
      cudaFuncSetAttribute(k_tc_finish_sk<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
      cudaFuncSetAttribute(k_tc_finish_sk<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
      cudaFuncSetAttribute(k_tc_finish_sk<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
      cudaFuncSetAttribute(k_tc_finish_sk<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
      fs_attr = true;
    }
  }
  const int nqm = std::max(nq1, nq2);
  // both finishing kernels start by programmatic launch behind the kernel before them (their
  // set-up overlaps its tail; they wait for it before reading its results)
  auto launch_pdl = [&](auto kern, int grid, int block, size_t sm) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, f);
    count_launch();
  };
  auto launch_finish = [&](int nsplit) {
    f.nsplit = nsplit;
    const int fgrid = (nt1 + nt2) * nsplit;
    if (nqm <= 1) launch_pdl(k_tc_finish_sk<1>, fgrid, FS_TE, fsm);
    else if (nqm <= 2) launch_pdl(k_tc_finish_sk<2>, fgrid, FS_TE, fsm);
    else if (nqm <= 4) launch_pdl(k_tc_finish_sk<4>, fgrid, FS_TE, fsm);
    else launch_pdl(k_tc_finish_sk<8>, fgrid, FS_TE, fsm);
    if (nsplit > 1) {
      const int64_t outs = (int64_t)(nt1 + nt2) * J * FS_TE;
      launch_pdl(k_tc_finish_red, (int)std::min<int64_t>((outs + 255) / 256, 152 * 16), 256, 0);
    }
  };
  // launch shape: tuned once per plan on its first call outside stream capture (cached
  // process-wide per shape); under capture before that, the full grid
  if (!plan.tuned) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
      const TuneKey key{dev, N1, ld1, N2, nslice, r1pad, r2pad, J, p};
      // a fixed shape from the environment (reproducible profiles): TDB_TC_SHAPE="ctas,target"
      const char* fixed = getenv("TDB_TC_SHAPE");
      int fc = 0, ft = 0;
      if (fixed && sscanf(fixed, "%d,%d", &fc, &ft) == 2 && fc > 0 && ft > 0) {
        plan.cstep = std::min(fc, cmax);
        plan.fin_target = ft;
        plan.ncand = 0;
        plan.from_cache = false;
      } else if (!tune_lookup(key, plan)) {
        tune_shape(plan, cmax, [&](int c) { launch_project(c, false); }, [&](int target) {
          f.nnp = P.nq12 * plan.cstep * NUM_CONV_WARPS;
          launch_finish(nsplit_for(target));
        }, s);
        tune_store(key, plan);
      }
      plan.tuned = true;
    } else {
      cudaGetLastError();
    }
  }
  const int cstep = plan.tuned ? std::min(plan.cstep, cmax) : cmax;
  const int grid = P.nq12 * cstep;
  if (evm && !pdl) record_timing_event(evm[0], s);
  launch_project(cstep, pdl);
  if (evm) record_timing_event(evm[1], s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    err = std::string("k_tc_project launch: ") + cudaGetErrorString(e);
    return TDB_ERR_CUDA;
  }
  f.nnp = grid * NUM_CONV_WARPS;
  f.span = P.span;
  launch_finish(nsplit_for(plan.tuned ? plan.fin_target : FS_CTAS));
  if (p >= 3) {
    if (!fuse_w) {
      // Z1 summed over the mode-1 tiles: the partials themselves when there is one tile
      const float* z1 = nq1 > 1 ? Z1 : plan.z1p;
      float* out = p == 3 ? Y[2] : scratch;
      k_tc_finish_b<<<std::min(nslice, 152 * 8), 256, kFinishBSmem, s>>>(z1, N2, nslice, r[0], r[1],
                                                                         (const float*)A[1], out);
      count_launch();
    }
    if (p == 4) {
      // Y_3 = W x_4 A_4^T and Y_4 = W x_3 A_3^T from W = Z1 x_2 A_2^T (r1 x r2 x N3 x N4)
      const int64_t L12 = (int64_t)r[0] * r[1];
      launch_modeprod<float, float, float>(scratch, Y[2], (const float*)A[3], L12 * N[2], (int)N[3], r[3], 1, N[3], 1,
                                           s);
      launch_modeprod<float, float, float>(scratch, Y[3], (const float*)A[2], L12, (int)N[2], r[2], N[3], N[2], 1, s);
    }
  }
  if (!defer_ds) {
    // dS = Y_2 x_2 A_2^T (otherwise the update kernel forms it)
    int64_t Q = 1;
    for (int n = 2; n < p; ++n) Q *= r[n];
    launch_modeprod<float, float, float>(Y[1], dS, (const float*)A[1], r[0], N2, r[1], Q, N2, 1, s);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    err = std::string("projection finish: ") + cudaGetErrorString(e);
    return TDB_ERR_CUDA;
  }
  return TDB_OK;
}


// ---------------------------------------------------------------------------
// Allocation-free variant of the fused projection (see tdb_project_noalloc in
// include/tdb.h).  Its scratch lives in this file-scope device array; host code
// may not use the array's name as a device address, so the address is fetched
// once per device with cudaGetSymbolAddress.
// ---------------------------------------------------------------------------
constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_addr[64] = {nullptr};

// Bytes of scratch the projection needs for these sizes, laid out by `lay`.
size_t noalloc_layout(Carver& cv, TcPlan& plan, int p, const int64_t* N, const int* r, float** Z1, float** Z2,
                      float** scratch, unsigned** status) {
  *status = cv.take<unsigned>(64);
  int cap[kMaxModes] = {r[0], r[1], p > 2 ? r[2] : 1, p > 3 ? r[3] : 1};
  tc_carve(plan, cv, p, N, cap);
  int64_t S = 1;
  for (int n = 0; n < p; ++n) S *= N[n];
  *Z1 = cv.take<float>((size_t)(S / N[0]) * r[0]);
  *Z2 = nullptr;                                       // (the finish does not form Z2)
  // W = Z1 x_2 A_2^T of four modes (r1 r2 N3 N4); at least one element
  int64_t sc = (int64_t)r[0] * r[1];
  for (int n = 2; n < p; ++n) sc *= N[n];
  *scratch = cv.take<float>((size_t)std::max<int64_t>(sc, 1));
  return cv.off;
}
}  // namespace

}  // namespace tdb

extern "C" tdb_status tdb_project_noalloc(int ndim, const int64_t* dims, const int* ranks, const float* V_next,
                                          const float* V_prev, const float* const* A, const double* const* w,
                                          float* dS, float* const* Y, double* dv2, void* stream) {
  using namespace tdb;
  std::string err;
  if (ndim < 2 || ndim > kMaxModes || !dims || !ranks || !V_next || !V_prev || !A || !w || !dS || !Y || !dv2)
    return TDB_ERR_INVALID_ARG;
  int64_t N[kMaxModes] = {1, 1, 1, 1};
  int r[kMaxModes] = {1, 1, 1, 1};
  for (int n = 0; n < ndim; ++n) {
    N[n] = dims[n];
    r[n] = ranks[n];
    if (N[n] < 1 || N[n] > 1024) return TDB_ERR_SHAPE;
    if (r[n] < 1 || r[n] > kMaxRank || r[n] > N[n] || !A[n] || !w[n] || !Y[n]) return TDB_ERR_RANK;
  }
  if (N[0] % 4 != 0) return TDB_ERR_UNSUPPORTED;       // (no room for padded copies in the static scratch)
  if (!tc_supported(ndim, N, r, err)) return TDB_ERR_UNSUPPORTED;
  // sizes beyond the static scratch are refused before anything is launched
  TcPlan plan;
  float *Z1 = nullptr, *Z2 = nullptr, *scr = nullptr;
  unsigned* status = nullptr;
  {
    Carver measure(nullptr);
    if (noalloc_layout(measure, plan, ndim, N, r, &Z1, &Z2, &scr, &status) > kNoAllocScratchBytes)
      return TDB_ERR_WORKSPACE;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return TDB_ERR_CUDA;
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return TDB_ERR_CUDA;
      g_noalloc_addr[dev] = ptr;
    }
    base = g_noalloc_addr[dev];
  }
  plan = TcPlan();
  Carver cv(base);
  noalloc_layout(cv, plan, ndim, N, r, &Z1, &Z2, &scr, &status);
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(status, 0, sizeof(unsigned), s) != cudaSuccess) return TDB_ERR_CUDA;
  tdb_status st = tc_project(plan, V_next, V_prev, ndim, N, r, (const void* const*)A, w, Z1, Z2, scr, dS, Y, dv2,
                             status, s, nullptr, err);
  if (st != TDB_OK) return st;
  unsigned h_status = 0;
  if (cudaMemcpyAsync(&h_status, status, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return TDB_ERR_CUDA;
  return (h_status & kFlagTimeout) ? TDB_ERR_TIMEOUT : TDB_OK;
}
