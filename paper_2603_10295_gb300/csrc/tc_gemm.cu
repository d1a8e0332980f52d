// Split-precision GEMM on the 5th-generation tensor cores (tcgen05, kind::tf32):
//
//   C[q][m][n] = sum_k (Ahi Bhi + Ahi Blo + Alo Bhi)[m][k] [q][n][k]      (FP32 result)
//
// with A = Ahi + Alo and B = Bhi + Blo the two-term TF32 splits of FP32 operands
// (3-term product: the lo*lo term, 2^-22 relative, is dropped).  The large term
// accumulates in one TMEM accumulator and the two correction terms in a second
// one; they are added once in the epilogue (compensated recombination: the
// small terms are not rounded against the large running sum).
//
// In the mixed form this is the Re->k contraction of Eq. 10 on the real
// embedding of the complex product (A = [Re P_k, Im P_k] interleaved, B the
// 2x2 real blocks of G2), so C holds G3 as interleaved complex64.
//
// CTA tile 128 (m) x 256 (n), K in 32-float (128-byte) slices; 2-stage TMA ->
// shared memory (128B swizzle) pipeline; warp 0 lane 0 issues TMA, warp 1
// lane 0 issues tcgen05.mma (M=128, N=256, K=8 per instruction) and commits to
// mbarriers; all four warps drain TMEM (32 lanes each) in the epilogue.  Every
// mbarrier wait is bounded: on a timeout the CTA sets *err, stops issuing,
// drains what it issued (bounded again), frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "eph_kernels.cuh"

namespace eph {

namespace tc {

constexpr int BM = 128, BN = 256, BK = 32, STAGES = 2;
constexpr int A_BYTES = BM * BK * 4;                         // 16 KiB
constexpr int B_BYTES = BN * BK * 4;                         // 32 KiB
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;       // 96 KiB
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 128;
constexpr uint32_t TMEM_COLS = 512;                          // acc0: columns 0..255, acc1: 256..511
constexpr long long WAIT_LIMIT_CYCLES = 4000000000LL;       // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Bounded wait for the completion of the phase with the given parity.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t addr = smem_u32(bar);
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > WAIT_LIMIT_CYCLES) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major tile, rows of 128 B, 128-byte swizzle,
// 8-row core-matrix groups 1024 B apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;              // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
  d |= (uint64_t)1 << 46;              // version
  d |= (uint64_t)2 << 61;              // SWIZZLE_128B
  return d;
}

// Instruction descriptor, kind::tf32: D f32, A/B tf32, both K-major, M = 128, N = 256.
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

}  // namespace tc

__global__ void __launch_bounds__(128, 1) k_tc_split_gemm(const __grid_constant__ CUtensorMap mAhi,
                                                          const __grid_constant__ CUtensorMap mAlo,
                                                          const __grid_constant__ CUtensorMap mBhi,
                                                          const __grid_constant__ CUtensorMap mBlo, int M,
                                                          int a_row0, int Nr, int Kp, float* __restrict__ C, long ldc,
                                                          long sC, int* __restrict__ err) {
  using namespace tc;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM, q = blockIdx.z;
  const int nkb = Kp / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
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
  const uint32_t tmem = *tmem_slot;

  auto stage_ptr = [&](int s, int which) -> unsigned char* {
    const int off[4] = {0, A_BYTES, 2 * A_BYTES, 2 * A_BYTES + B_BYTES};
    return smem + s * STAGE_BYTES + off[which];
  };

  int issued = 0;  // producer: k blocks whose loads were issued
  int mma_ok = 1;  // MMA thread: all k blocks consumed
  if (warp == 0 && lane == 0) {
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % STAGES;
      if (kb >= STAGES && !mbar_wait(&empty[s], ((kb / STAGES) - 1) & 1)) {
        *abort_flag = 1;
        atomicOr(err, 1);
        break;
      }
      if (*abort_flag) break;
      mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
      tma_load_2d(stage_ptr(s, 0), &mAhi, kb * BK, a_row0 + m0, &full[s]);
      tma_load_2d(stage_ptr(s, 1), &mAlo, kb * BK, a_row0 + m0, &full[s]);
      tma_load_2d(stage_ptr(s, 2), &mBhi, kb * BK, q * Nr + n0, &full[s]);
      tma_load_2d(stage_ptr(s, 3), &mBlo, kb * BK, q * Nr + n0, &full[s]);
      ++issued;
    }
  } else if (warp == 1 && lane == 0) {
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % STAGES;
      if (*abort_flag || !mbar_wait(&full[s], (kb / STAGES) & 1)) {
        *abort_flag = 1;
        atomicOr(err, 2);
        mma_ok = 0;
        break;
      }
      fence_after();
      const uint64_t dAhi = smem_desc(smem_u32(stage_ptr(s, 0)));
      const uint64_t dAlo = smem_desc(smem_u32(stage_ptr(s, 1)));
      const uint64_t dBhi = smem_desc(smem_u32(stage_ptr(s, 2)));
      const uint64_t dBlo = smem_desc(smem_u32(stage_ptr(s, 3)));
#pragma unroll
      for (int kk = 0; kk < BK / 8; ++kk) {
        const uint64_t o = (uint64_t)(kk * 32) >> 4;  // 8 tf32 = 32 bytes along K inside the swizzle atom
        const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
        mma_tf32(tmem, dAhi + o, dBhi + o, acc);
        mma_tf32(tmem + 256, dAhi + o, dBlo + o, acc);
        mma_tf32(tmem + 256, dAlo + o, dBhi + o, 1u);
      }
      mma_commit(&empty[s]);  // stage s is free once these MMAs have read it
    }
    mma_commit(done);  // all MMAs issued by this thread have completed
  }
  __syncwarp();

  const bool ok = mbar_wait(done, 0);
  if (!ok) atomicOr(err, 4);
  fence_after();
  if (ok && mma_ok && !*abort_flag) {
    const int row = m0 + warp * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
    float* crow = C + (long)q * sC + (long)row * ldc;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
      uint32_t r0[16], r1[16];
      tmem_ld16(tl + c0, r0);
      tmem_ld16(tl + 256 + c0, r1);
      tmem_ld_wait();
      if (row < M) {  // four 16-byte stores per lane where the row has them
        const bool vec_ok = (reinterpret_cast<uintptr_t>(crow) & 15) == 0;
#pragma unroll
        for (int i = 0; i < 16; i += 4) {
          const int col = n0 + c0 + i;
          if (col + 3 < Nr && vec_ok) {
            *reinterpret_cast<float4*>(crow + col) =
                make_float4(__uint_as_float(r0[i]) + __uint_as_float(r1[i]),
                            __uint_as_float(r0[i + 1]) + __uint_as_float(r1[i + 1]),
                            __uint_as_float(r0[i + 2]) + __uint_as_float(r1[i + 2]),
                            __uint_as_float(r0[i + 3]) + __uint_as_float(r1[i + 3]));
          } else {
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (col + u < Nr) crow[col + u] = __uint_as_float(r0[i + u]) + __uint_as_float(r1[i + u]);
          }
        }
      }
    }
  }
  // drain: after an abort the producer waits (bounded) for its last loads of each stage
  if (warp == 0 && lane == 0 && *abort_flag) {
    for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; ++kb) {
      const int s = kb % STAGES;
      mbar_wait(&full[s], (kb / STAGES) & 1);
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// ----------------------------------------------------------------------------- fixed-point BF16 digits
// C[q][m][n] = sA * sB[q*Nr+n] * 2^-16 * (L0 + L123),
//   L0   = sum_k a_0[m][k] b_0[n][k],                       a_i = d_i 2^-8i, b_j = e_j 2^-8j
//   L123 = sum_{1 <= i+j <= 3} sum_k a_i[m][k] b_j[n][k]
// where x/s = sum_i d_i 2^-8(i+1) with integer digits |d| <= 128 (A: 3 digits, B: 4; s a
// power of two >= 2 max|x| of the row), each digit stored pre-scaled by 2^-8i, exactly,
// in bf16.  Level-0 products are integers below 2^14, so L0 over K <= 1024 stays below 2^24
// and its FP32 tensor-core accumulation is exact; L123 is at most 2^-7 of L0, so its FP32
// rounding is ~2^-31 of the result.  B carries a 4th digit because the mode-rotated
// g(Re,q) columns decay over Re and the fixed-point error is relative to the row maximum.
//
// Persistent kernel, one CTA (6 warps) per SM: warp 0 issues TMA into a 2-stage ring of
// 112 KiB stages, warp 1 issues the 9 tcgen05.mma (M=128, N=128, K=16) per K step into one
// of two TMEM accumulator pairs (L0, L123 at columns b*256 + {0, 128}), warps 2-5 drain the
// other pair (epilogue of tile i overlaps the MMAs of tile i+1).  Tiles (m, q, n) are taken
// in steps of gridDim.x with n fastest, then q: the CTAs that need one A row tile (every
// q and n) run at the same time and read it from DRAM once.
namespace tcf {
constexpr int BM = 128, BN = 128, BK = 64, STAGES = 2, NA = 3, NB = 4;   // BK bf16 = 128 B rows

__device__ __forceinline__ void tile_coords(long t, int ntn, int nq, int* q, int* m0, int* n0) {
  const long per_m = (long)ntn * nq;
  const long mt = t / per_m;
  const int rem = (int)(t - mt * per_m);
  *q = rem / ntn;
  *m0 = (int)mt * BM;
  *n0 = (rem - *q * ntn) * BN;
}
constexpr int A_BYTES = BM * BK * 2;                              // 16 KiB per digit slice
constexpr int B_BYTES = BN * BK * 2;                              // 16 KiB
constexpr int STAGE_BYTES = NA * A_BYTES + NB * B_BYTES;          // 112 KiB
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;     // 225 KiB
constexpr uint32_t TMEM_COLS = 512;                               // 2 buffers x (L0, L123) x 128 columns
constexpr int THREADS = 192;
// kind::f16 instruction descriptor: D f32, A/B bf16, K-major, M = 128, N = 128 (K = 16 per MMA)
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}
}  // namespace tcf

struct TcMaps7 {
  CUtensorMap a[3];
  CUtensorMap b[4];
};

__global__ void __launch_bounds__(tcf::THREADS, 1) k_tc_fixed_gemm(const __grid_constant__ TcMaps7 maps, int M, int a_row0,
                                                                  int Nr, int Kp, int nq, float sA,
                                                                  const float* __restrict__ sB,
                                                                  float* __restrict__ C, long ldc, long sC,
                                                                  int* __restrict__ err) {
  using namespace tc;
  using tcf::BM;
  using tcf::BN;
  using tcf::BK;
  using tcf::STAGES;
  using tcf::NA;
  using tcf::NB;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * tcf::STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* accf = empty + STAGES;   // [2] accumulator pair b holds a finished tile
  uint64_t* acce = accf + 2;         // [2] accumulator pair b has been drained
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acce + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkb = Kp / BK;
  const int ntn = (Nr + BN - 1) / BN, ntm = (M + BM - 1) / BM;
  const long ntiles = (long)ntn * ntm * nq;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], 4);  // one arrival per epilogue warp
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(tcf::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  auto tile = [&](int s, int which) -> unsigned char* { return smem + s * tcf::STAGE_BYTES + which * tcf::A_BYTES; };

  if (warp == 0) {
    if (lane == 0) {  // ---- TMA producer
      long it = 0;
      for (long t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
        int q, m0, n0;
        tcf::tile_coords(t, ntn, nq, &q, &m0, &n0);
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = (int)(it % STAGES);
          if (it >= STAGES && !mbar_wait(&empty[s], (uint32_t)(((it / STAGES) - 1) & 1))) {
            *abort_flag = 1;
            atomicOr(err, 1);
            break;
          }
          if (*abort_flag) break;
          mbar_arrive_expect_tx(&full[s], tcf::STAGE_BYTES);
#pragma unroll
          for (int d = 0; d < NA; ++d) tma_load_2d(tile(s, d), &maps.a[d], kb * BK, a_row0 + m0, &full[s]);
#pragma unroll
          for (int d = 0; d < NB; ++d) tma_load_2d(tile(s, NA + d), &maps.b[d], kb * BK, q * Nr + n0, &full[s]);
        }
      }
      // after an abort: wait (bounded) for the loads still in flight
      if (*abort_flag)
        for (long j = (it > STAGES ? it - STAGES : 0); j < it; ++j) mbar_wait(&full[j % STAGES], (uint32_t)((j / STAGES) & 1));
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {  // ---- MMA issuer
      long it = 0, lt = 0;
      for (long t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x, ++lt) {
        const int b = (int)(lt & 1);
        if (lt >= 2 && !mbar_wait(&acce[b], (uint32_t)(((lt / 2) - 1) & 1))) {
          *abort_flag = 1;
          atomicOr(err, 8);
          break;
        }
        fence_after();
        const uint32_t d0 = tmem + (uint32_t)(b * 256), d1 = d0 + 128;
        bool ok = true;
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = (int)(it % STAGES);
          if (*abort_flag || !mbar_wait(&full[s], (uint32_t)((it / STAGES) & 1))) {
            *abort_flag = 1;
            atomicOr(err, 2);
            ok = false;
            break;
          }
          fence_after();
          uint64_t da[NA], db[NB];
#pragma unroll
          for (int d = 0; d < NA; ++d) da[d] = smem_desc(smem_u32(tile(s, d)));
#pragma unroll
          for (int d = 0; d < NB; ++d) db[d] = smem_desc(smem_u32(tile(s, NA + d)));
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint64_t o = (uint64_t)(kk * 32) >> 4;  // 16 bf16 = 32 bytes along K inside the swizzle atom
            const uint32_t first = (kb > 0 || kk > 0) ? 1u : 0u;
            tcf::mma_bf16(d0, da[0] + o, db[0] + o, first);  // level 0 (exact)
            tcf::mma_bf16(d1, da[0] + o, db[1] + o, first);  // levels 1-3 (pre-scaled digits)
            tcf::mma_bf16(d1, da[1] + o, db[0] + o, 1u);
            tcf::mma_bf16(d1, da[0] + o, db[2] + o, 1u);
            tcf::mma_bf16(d1, da[1] + o, db[1] + o, 1u);
            tcf::mma_bf16(d1, da[2] + o, db[0] + o, 1u);
            tcf::mma_bf16(d1, da[0] + o, db[3] + o, 1u);
            tcf::mma_bf16(d1, da[1] + o, db[2] + o, 1u);
            tcf::mma_bf16(d1, da[2] + o, db[1] + o, 1u);
          }
          mma_commit(&empty[s]);  // stage s is free once these MMAs have read it
        }
        mma_commit(&accf[b]);  // the tile's accumulators are complete (or the loop was aborted)
        if (!ok) break;
      }
    }
    __syncwarp();
  } else {  // ---- epilogue, warps 2..5: TMEM lane quarter = warp % 4
    const int quarter = warp & 3;
    long lt = 0;
    for (long t = blockIdx.x; t < ntiles; t += gridDim.x, ++lt) {
      const int b = (int)(lt & 1);
      const bool ok = mbar_wait(&accf[b], (uint32_t)((lt / 2) & 1));
      if (!ok || *abort_flag) {
        if (!ok) atomicOr(err, 4);
        break;
      }
      fence_after();
      int q, m0, n0;
      tcf::tile_coords(t, ntn, nq, &q, &m0, &n0);
      const int row = m0 + quarter * 32 + lane;
      const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * 256);
      float* crow = C + (long)q * sC + (long)row * ldc;
      const float* srow = sB + (long)q * Nr;
      const bool vec_ok = ((reinterpret_cast<uintptr_t>(crow) | reinterpret_cast<uintptr_t>(srow)) & 15) == 0;
      const float sc = sA * 0x1p-16f;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 16) {
        uint32_t r0[16], r1[16];
        tmem_ld16(tl + c0, r0);
        tmem_ld16(tl + 128 + c0, r1);
        tmem_ld_wait();
        if (row < M) {
          // 16 consecutive columns of one row per lane: four 16-byte stores where the row has
          // them (scalar 4-byte stores, one row per lane, had left most of every 32-byte
          // sector unused and made the epilogue the limiter)
#pragma unroll
          for (int i = 0; i < 16; i += 4) {
            const int col = n0 + c0 + i;
            if (col + 3 < Nr && vec_ok) {
              const float4 sv = *reinterpret_cast<const float4*>(srow + col);
              float4 o;
              o.x = (__uint_as_float(r0[i]) + __uint_as_float(r1[i])) * (sc * sv.x);
              o.y = (__uint_as_float(r0[i + 1]) + __uint_as_float(r1[i + 1])) * (sc * sv.y);
              o.z = (__uint_as_float(r0[i + 2]) + __uint_as_float(r1[i + 2])) * (sc * sv.z);
              o.w = (__uint_as_float(r0[i + 3]) + __uint_as_float(r1[i + 3])) * (sc * sv.w);
              *reinterpret_cast<float4*>(crow + col) = o;
            } else {
#pragma unroll
              for (int u = 0; u < 4; ++u)
                if (col + u < Nr)
                  crow[col + u] = (__uint_as_float(r0[i + u]) + __uint_as_float(r1[i + u])) * (sc * srow[col + u]);
            }
          }
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) tcf::mbar_arrive(&acce[b]);
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcf::TMEM_COLS) : "memory");
  }
}

// ----------------------------------------------------------------------------- H(k+q) to FP64 class
// H(k+q) = P_k (e^{iq.Re} H(Re)) needs ~1e-12 for the eigensolve, so this contraction carries
// five fixed-point BF16 digits per operand (40 bits) and keeps every product of digit levels
// i + j <= 4 (15 MMAs per K step).  Levels 0, 1 and 2 accumulate in separate TMEM accumulators,
// where their integer sums are exact in FP32 (K <= 1024); levels 3 and 4 share one (its FP32
// rounding is 2^-48 of the result).  The epilogue adds the four with two-sums into a float pair
// (hi, lo), exact to ~2^-48 relative, scaled by the (power-of-two) operand scales.
// Tiles 128 x 128 with K slices of 32 bf16 (64-byte rows, 64-byte swizzle) so that the ten
// digit tiles of a stage (80 KiB) fit twice in shared memory; one accumulator set (512 TMEM
// columns), so the next tile's MMAs wait for the epilogue.
namespace tch {
constexpr int BM = 128, BN = 128, BK = 32, STAGES = 2, ND = 5;
constexpr int T_BYTES = BM * BK * 2;                           // 8 KiB per digit tile
constexpr int STAGE_BYTES = 2 * ND * T_BYTES;                  // 80 KiB (five digits; four use 64)
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr uint32_t TMEM_COLS = 512;                            // L0, L1, L2, L34 x 128 columns
constexpr int THREADS = 192;

// K-major tile of 64-byte rows with 64-byte swizzle: 8-row groups 512 B apart, descriptor v1.
__device__ __forceinline__ uint64_t smem_desc64(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;  // SWIZZLE_64B
  return d;
}

// Tile order with the m tile fastest: the m tiles that share one B tile run back to back
// (batched products with M <= 2 BM rows per batch read each B tile from DRAM once).
__device__ __forceinline__ void tile_coords_mfast(long t, int ntm, int ntn, int* q, int* m0, int* n0) {
  const int m = (int)(t % ntm);
  const long r = t / ntm;
  const int n = (int)(r % ntn);
  *q = (int)(r / ntn);
  *m0 = m * BM;
  *n0 = n * BN;
}

__device__ __forceinline__ void two_sum(float& h, float& l, float x) {
  const float s = __fadd_rn(h, x);
  const float bb = __fsub_rn(s, h);
  const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(x, bb));
  h = s;
  l = __fadd_rn(l, e);
}
}  // namespace tch

struct TcMaps10 {
  CUtensorMap a[5];
  CUtensorMap b[5];
};

// Batch q reads A rows a_row0 + ((q + a_qoff) mod a_mod) a_stride + m (a_mod = 1: A shared by
// every batch); morder = 1 takes the m tiles fastest.
// NDG = 5: the scheme above; NDG = 4: four digits (32 bits) per operand, levels <= 3 kept
// (10 MMAs per K step into the same four accumulators L0, L1, L2, L3), ~2^-32 relative.
template <int NDG>
__global__ void __launch_bounds__(tch::THREADS, 1) k_tc_hkq_gemm(const __grid_constant__ TcMaps10 maps, int M,
                                                                int a_row0, int Nr, int Kp, int nq, float sA,
                                                                const float* __restrict__ sB, float2* __restrict__ C,
                                                                long ldc, long sC, int* __restrict__ err, int a_mod,
                                                                int a_qoff, int a_stride, int morder) {
  using namespace tc;
  using tch::BM;
  using tch::BN;
  using tch::BK;
  using tch::STAGES;
  using tch::ND;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  constexpr int SBYTES = 2 * NDG * tch::T_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * tch::STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* accf = empty + STAGES;  // the accumulators hold a finished tile
  uint64_t* acce = accf + 1;        // the accumulators have been drained
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acce + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkb = Kp / BK;
  const int ntn = (Nr + BN - 1) / BN, ntm = (M + BM - 1) / BM;
  const long ntiles = (long)ntn * ntm * nq;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    mbar_init(acce, 4);  // one arrival per epilogue warp
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(tch::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  auto tile = [&](int s, int which) -> unsigned char* { return smem + s * SBYTES + which * tch::T_BYTES; };

  if (warp == 0) {
    if (lane == 0) {  // ---- TMA producer
      long it = 0;
      for (long t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
        int q, m0, n0;
        if (morder)
          tch::tile_coords_mfast(t, ntm, ntn, &q, &m0, &n0);
        else
          tcf::tile_coords(t, ntn, nq, &q, &m0, &n0);
        const int arow = a_row0 + ((q + a_qoff) % a_mod) * a_stride + m0;
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = (int)(it % STAGES);
          if (it >= STAGES && !mbar_wait(&empty[s], (uint32_t)(((it / STAGES) - 1) & 1))) {
            *abort_flag = 1;
            atomicOr(err, 1);
            break;
          }
          if (*abort_flag) break;
          mbar_arrive_expect_tx(&full[s], SBYTES);
#pragma unroll
          for (int d = 0; d < NDG; ++d) tma_load_2d(tile(s, d), &maps.a[d], kb * BK, arow, &full[s]);
#pragma unroll
          for (int d = 0; d < NDG; ++d) tma_load_2d(tile(s, NDG + d), &maps.b[d], kb * BK, q * Nr + n0, &full[s]);
        }
      }
      if (*abort_flag)
        for (long j = (it > STAGES ? it - STAGES : 0); j < it; ++j) mbar_wait(&full[j % STAGES], (uint32_t)((j / STAGES) & 1));
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {  // ---- MMA issuer
      long it = 0, lt = 0;
      for (long t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x, ++lt) {
        if (lt >= 1 && !mbar_wait(acce, (uint32_t)((lt - 1) & 1))) {
          *abort_flag = 1;
          atomicOr(err, 8);
          break;
        }
        fence_after();
        bool ok = true;
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = (int)(it % STAGES);
          if (*abort_flag || !mbar_wait(&full[s], (uint32_t)((it / STAGES) & 1))) {
            *abort_flag = 1;
            atomicOr(err, 2);
            ok = false;
            break;
          }
          fence_after();
          uint64_t da[NDG], db[NDG];
#pragma unroll
          for (int d = 0; d < NDG; ++d) {
            da[d] = tch::smem_desc64(smem_u32(tile(s, d)));
            db[d] = tch::smem_desc64(smem_u32(tile(s, NDG + d)));
          }
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint64_t o = (uint64_t)(kk * 32) >> 4;  // 16 bf16 = 32 bytes along K
            const uint32_t first = (kb > 0 || kk > 0) ? 1u : 0u;
            const uint32_t t0 = tmem, t1 = tmem + 128, t2 = tmem + 256, t3 = tmem + 384;
            tcf::mma_bf16(t0, da[0] + o, db[0] + o, first);  // level 0
            tcf::mma_bf16(t1, da[0] + o, db[1] + o, first);  // level 1
            tcf::mma_bf16(t1, da[1] + o, db[0] + o, 1u);
            tcf::mma_bf16(t2, da[0] + o, db[2] + o, first);  // level 2
            tcf::mma_bf16(t2, da[1] + o, db[1] + o, 1u);
            tcf::mma_bf16(t2, da[2] + o, db[0] + o, 1u);
            tcf::mma_bf16(t3, da[0] + o, db[3] + o, first);  // level 3 (and 4)
            tcf::mma_bf16(t3, da[1] + o, db[2] + o, 1u);
            tcf::mma_bf16(t3, da[2] + o, db[1] + o, 1u);
            tcf::mma_bf16(t3, da[3] + o, db[0] + o, 1u);
            if constexpr (NDG == 5) {
              tcf::mma_bf16(t3, da[0] + o, db[4] + o, 1u);
              tcf::mma_bf16(t3, da[1] + o, db[3] + o, 1u);
              tcf::mma_bf16(t3, da[2] + o, db[2] + o, 1u);
              tcf::mma_bf16(t3, da[3] + o, db[1] + o, 1u);
              tcf::mma_bf16(t3, da[4] + o, db[0] + o, 1u);
            }
          }
          mma_commit(&empty[s]);
        }
        mma_commit(accf);
        if (!ok) break;
      }
    }
    __syncwarp();
  } else {  // ---- epilogue, warps 2..5: TMEM lane quarter = warp % 4
    const int quarter = warp & 3;
    long lt = 0;
    for (long t = blockIdx.x; t < ntiles; t += gridDim.x, ++lt) {
      const bool ok = mbar_wait(accf, (uint32_t)(lt & 1));
      if (!ok || *abort_flag) {
        if (!ok) atomicOr(err, 4);
        break;
      }
      fence_after();
      int q, m0, n0;
      if (morder)
        tch::tile_coords_mfast(t, ntm, ntn, &q, &m0, &n0);
      else
        tcf::tile_coords(t, ntn, nq, &q, &m0, &n0);
      const int row = m0 + quarter * 32 + lane;
      const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
      float2* crow = C + (long)q * sC + (long)row * ldc;
      const float* srow = sB + (long)q * Nr;
      const float sc = sA * 0x1p-16f;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 16) {
        uint32_t r0[16], r1[16], r2[16], r3[16];
        tmem_ld16(tl + c0, r0);
        tmem_ld16(tl + 128 + c0, r1);
        tmem_ld16(tl + 256 + c0, r2);
        tmem_ld16(tl + 384 + c0, r3);
        tmem_ld_wait();
        if (row < M) {
#pragma unroll
          for (int i = 0; i < 16; i += 2) {
            const int col = n0 + c0 + i;
            float2 v[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              float h = __uint_as_float(r0[i + u]), l = 0.f;
              tch::two_sum(h, l, __uint_as_float(r1[i + u]));
              tch::two_sum(h, l, __uint_as_float(r2[i + u]));
              tch::two_sum(h, l, __uint_as_float(r3[i + u]));
              const float f = (col + u < Nr) ? sc * srow[col + u] : 0.f;  // powers of two: exact
              v[u] = make_float2(h * f, l * f);
            }
            if (col + 1 < Nr) {
              *reinterpret_cast<float4*>(crow + col) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
            } else if (col < Nr) {
              crow[col] = v[0];
            }
          }
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) tcf::mbar_arrive(acce);
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tch::TMEM_COLS) : "memory");
  }
}

// ----------------------------------------------------------------------------- batched band products
// The band rotation's products (complex64 result): four digits per operand, levels <= 3, with
// level 0 exact in its own accumulator and levels 1-3 in a second one (their sum is at most 2^-7
// of level 0, so its FP32 rounding is ~2^-31 of the result), which leaves room for two
// accumulator sets: the epilogue of one tile runs under the MMAs of the next.  The result is
// written as one FP32 per element, the two sums added and rounded once (2^-24 of the element):
// the second stage's digits and the complex64 g need no more, and a float pair would double the
// bytes the epilogue writes and the next step reads.
// 32-wide K slices (64-byte swizzle), three 64 KiB stages.  Batch q reads A rows
// a_row0 + ((q + a_qoff) mod a_mod) a_stride + m; tiles (m fastest, then n, then q).
namespace tcb {
constexpr int BM = 128, BN = 128, BK = 32, STAGES = 3, ND = 4;
constexpr int T_BYTES = BM * BK * 2;                       // 8 KiB per digit tile
constexpr int STAGE_BYTES = 2 * ND * T_BYTES;              // 64 KiB
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr uint32_t TMEM_COLS = 512;                        // 2 sets x (L0, L123) x 128 columns
constexpr int THREADS = 192;
}  // namespace tcb

__global__ void __launch_bounds__(tcb::THREADS, 1) k_tc_band_gemm(const __grid_constant__ TcMaps10 maps, int M,
                                                                 int a_row0, int Nr, int Kp, int nq, float sA,
                                                                 const float* __restrict__ sB, float* __restrict__ C,
                                                                 long ldc, long sC, int* __restrict__ err, int a_mod,
                                                                 int a_qoff, int a_stride) {
  using namespace tc;
  using tcb::BM;
  using tcb::BN;
  using tcb::BK;
  using tcb::STAGES;
  using tcb::ND;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * tcb::STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* accf = empty + STAGES;  // [2] accumulator set b holds a finished tile
  uint64_t* acce = accf + 2;        // [2] accumulator set b has been drained
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acce + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkb = Kp / BK;
  const int ntn = (Nr + BN - 1) / BN, ntm = (M + BM - 1) / BM;
  const long ntiles = (long)ntn * ntm * nq;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], 4);  // one arrival per epilogue warp
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(tcb::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  auto tile = [&](int s, int which) -> unsigned char* { return smem + s * tcb::STAGE_BYTES + which * tcb::T_BYTES; };

  if (warp == 0) {
    if (lane == 0) {  // ---- TMA producer
      long it = 0;
      for (long t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
        int q, m0, n0;
        tch::tile_coords_mfast(t, ntm, ntn, &q, &m0, &n0);
        const int arow = a_row0 + ((q + a_qoff) % a_mod) * a_stride + m0;
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = (int)(it % STAGES);
          if (it >= STAGES && !mbar_wait(&empty[s], (uint32_t)(((it / STAGES) - 1) & 1))) {
            *abort_flag = 1;
            atomicOr(err, 1);
            break;
          }
          if (*abort_flag) break;
          mbar_arrive_expect_tx(&full[s], tcb::STAGE_BYTES);
#pragma unroll
          for (int d = 0; d < ND; ++d) tma_load_2d(tile(s, d), &maps.a[d], kb * BK, arow, &full[s]);
#pragma unroll
          for (int d = 0; d < ND; ++d) tma_load_2d(tile(s, ND + d), &maps.b[d], kb * BK, q * Nr + n0, &full[s]);
        }
      }
      // after an abort: wait (bounded) for the loads still in flight
      if (*abort_flag)
        for (long j = (it > STAGES ? it - STAGES : 0); j < it; ++j) mbar_wait(&full[j % STAGES], (uint32_t)((j / STAGES) & 1));
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {  // ---- MMA issuer
      long it = 0, lt = 0;
      for (long t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x, ++lt) {
        const int b = (int)(lt & 1);
        if (lt >= 2 && !mbar_wait(&acce[b], (uint32_t)(((lt / 2) - 1) & 1))) {
          *abort_flag = 1;
          atomicOr(err, 8);
          break;
        }
        fence_after();
        const uint32_t d0 = tmem + (uint32_t)(b * 256), d1 = d0 + 128;
        bool ok = true;
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = (int)(it % STAGES);
          if (*abort_flag || !mbar_wait(&full[s], (uint32_t)((it / STAGES) & 1))) {
            *abort_flag = 1;
            atomicOr(err, 2);
            ok = false;
            break;
          }
          fence_after();
          uint64_t da[ND], db[ND];
#pragma unroll
          for (int d = 0; d < ND; ++d) {
            da[d] = tch::smem_desc64(smem_u32(tile(s, d)));
            db[d] = tch::smem_desc64(smem_u32(tile(s, ND + d)));
          }
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint64_t o = (uint64_t)(kk * 32) >> 4;  // 16 bf16 = 32 bytes along K
            const uint32_t first = (kb > 0 || kk > 0) ? 1u : 0u;
            tcf::mma_bf16(d0, da[0] + o, db[0] + o, first);  // level 0 (exact)
            tcf::mma_bf16(d1, da[0] + o, db[1] + o, first);  // levels 1-3
            tcf::mma_bf16(d1, da[1] + o, db[0] + o, 1u);
            tcf::mma_bf16(d1, da[0] + o, db[2] + o, 1u);
            tcf::mma_bf16(d1, da[1] + o, db[1] + o, 1u);
            tcf::mma_bf16(d1, da[2] + o, db[0] + o, 1u);
            tcf::mma_bf16(d1, da[0] + o, db[3] + o, 1u);
            tcf::mma_bf16(d1, da[1] + o, db[2] + o, 1u);
            tcf::mma_bf16(d1, da[2] + o, db[1] + o, 1u);
            tcf::mma_bf16(d1, da[3] + o, db[0] + o, 1u);
          }
          mma_commit(&empty[s]);  // stage s is free once these MMAs have read it
        }
        mma_commit(&accf[b]);  // the tile's accumulators are complete (or the loop was aborted)
        if (!ok) break;
      }
    }
    __syncwarp();
  } else {  // ---- epilogue, warps 2..5: TMEM lane quarter = warp % 4
    const int quarter = warp & 3;
    long lt = 0;
    for (long t = blockIdx.x; t < ntiles; t += gridDim.x, ++lt) {
      const int b = (int)(lt & 1);
      const bool ok = mbar_wait(&accf[b], (uint32_t)((lt / 2) & 1));
      if (!ok || *abort_flag) {
        if (!ok) atomicOr(err, 4);
        break;
      }
      fence_after();
      int q, m0, n0;
      tch::tile_coords_mfast(t, ntm, ntn, &q, &m0, &n0);
      const int row = m0 + quarter * 32 + lane;
      const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * 256);
      float* crow = C + (long)q * sC + (long)row * ldc;
      const float* srow = sB + (long)q * Nr;
      const float sc = sA * 0x1p-16f;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 16) {
        uint32_t r0[16], r1[16];
        tmem_ld16(tl + c0, r0);
        tmem_ld16(tl + 128 + c0, r1);
        tmem_ld_wait();
        if (row < M) {
#pragma unroll
          for (int i = 0; i < 16; i += 4) {
            const int col = n0 + c0 + i;
            float v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const float f = (col + u < Nr) ? sc * srow[col + u] : 0.f;  // powers of two: exact
              v[u] = __fadd_rn(__uint_as_float(r0[i + u]), __uint_as_float(r1[i + u])) * f;
            }
            if (col + 3 < Nr && ((reinterpret_cast<uintptr_t>(crow + col) & 15) == 0)) {
              *reinterpret_cast<float4*>(crow + col) = make_float4(v[0], v[1], v[2], v[3]);
            } else {
#pragma unroll
              for (int u = 0; u < 4; ++u)
                if (col + u < Nr) crow[col + u] = v[u];
            }
          }
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) tcf::mbar_arrive(&acce[b]);
    }
  }
  // drain: after an abort the producer waits (bounded) for its last loads (above); every warp
  // then meets here before the TMEM is released
  fence_before();
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcb::TMEM_COLS) : "memory");
  }
}

// ----------------------------------------------------------------------------- FP64-accuracy complex GEMM
// C = A B^T on the real embedding of a complex product (the Re->k contraction of Eq. 10 on a k
// list in the FP64 form): A rows m with K = (e, re/im), B rows n = the output's real columns with
// the same K.  Every operand value x is seven balanced base-128 digits of x / s, with s =
// 2^(emax - 1021) a power of two per A row and per B row (emax >= the biased exponent of every
// value of the row, so |x / s| < 1/2):
//   x / s = sum_{i<7} d_i 2^-7(i+1),  |d_i| <= 64,  stored as d_i 2^-7i (exact in bf16).
// The digit products of levels l = i + j <= 7 (34 MMAs per K step) go to six accumulators: levels
// 0-4 each alone, where the sum is n_l 2^-7l with an integer |n_l| <= K 5 2^12 < 2^24 for K <= 512
// (exact in FP32), levels 5-7 together.  That sum is 2^-35 below level 0 and takes 19 MMAs per K
// step, each rounding it in FP32: ~K 2^-24 of it, 2^-50 of the result (with levels 4-7 together,
// 2^-28 below level 0, the same roundings measured ~1e-12).  The dropped levels >= 8 are below
// 2^-53 of the result.  The epilogue forms the integer Z = sum_l n_l 2^7(6-l) (units of
// 2^-56 s_A s_B; |Z| < K 2^54 <= 2^63 for K <= 512) and assembles the double from Z with integer
// operations, rounded to nearest.  One accumulator set of 6 x 80 TMEM columns: the next tile's
// MMAs wait for the epilogue, which twelve warps share (three per TMEM lane quarter) so that its
// dependent integer chains overlap.
namespace tz {
constexpr int BM = 128, BN = 80, BK = 32, STAGES = 2, ND = 7, NACC = 6;
constexpr int A_T = BM * BK * 2;                   // 8 KiB per digit tile
constexpr int B_T = BN * BK * 2;                   // 5 KiB loaded per B digit tile ...
constexpr int B_SLOT = 8192;                       // ... in an 8 KiB slot (every tile 1 KiB aligned)
constexpr int STAGE_BYTES = ND * (A_T + B_SLOT);   // 112 KiB
constexpr int TX_BYTES = ND * (A_T + B_T);         // 91 KiB delivered per stage
constexpr int META_BYTES = BN * 12;               // per tile: column offsets (8 B) and exponents (4 B)
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256 + META_BYTES;  // 226.2 KiB
constexpr uint32_t TMEM_COLS = 512;                // accumulators at columns 0, 80, ..., 400
constexpr int EPI_WARPS = 12;                      // three per TMEM lane quarter, every third 16-column chunk
constexpr int THREADS = 64 + 32 * EPI_WARPS;       // producer, MMA issuer, epilogue
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);
// x + OFF7 makes all seven base-128 fields of a value |X| <= 2^48 non-negative: OFF7 = 64 sum 128^i
constexpr long long OFF7 = 64LL * (((1LL << 49) - 1) / 127);

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(IDESC), "r"(acc)
      : "memory");
}

// the integer nearest to v (finite, |v| < 2^62), from the IEEE bits
__device__ __forceinline__ long long f2ll(float v) {
  const uint32_t b = __float_as_uint(v);
  const int be = (int)((b >> 23) & 0xFF);
  if (be == 0) return 0;
  const long long m = (long long)((b & 0x7FFFFFu) | 0x800000u);
  const int e = be - 150;  // v = m 2^e
  long long r = 0;
  if (e >= 0)
    r = m << e;
  else if (e > -25)
    r = (m + (1LL << (-e - 1))) >> (-e);
  return (b >> 31) ? -r : r;
}

// Z 2^E as a double rounded to nearest (|Z| < 2^63), from integer operations
__device__ __forceinline__ double ll2d(long long Z, int E) {
  if (Z == 0) return 0.0;
  const unsigned long long sgn = Z < 0 ? (1ULL << 63) : 0ULL;
  const unsigned long long M = Z < 0 ? 0ULL - (unsigned long long)Z : (unsigned long long)Z;
  const int lz = __clzll((long long)M);
  const unsigned long long N = M << lz;  // leading one at bit 63
  unsigned long long r = N + 0x400ULL;   // round at bit 11: 53 significant bits remain
  int ex = 63 - lz + E;                  // exponent of the leading bit
  if (r < N) {                           // the rounding carried out of bit 63
    r = 1ULL << 63;
    ++ex;
  }
  const long long be = (long long)ex + 1023;
  if (be <= 0) return 0.0;  // below the normal range
  return __longlong_as_double((long long)(sgn | ((unsigned long long)be << 52) | ((r >> 11) & 0xFFFFFFFFFFFFFULL)));
}

// the integer v (|v| < 2^24, an exact integer in FP32), from the IEEE bits in 32-bit operations
__device__ __forceinline__ int f2i24(float v) {
  const uint32_t b = __float_as_uint(v);
  const uint32_t m = (b & 0x7FFFFFu) | 0x800000u;
  const int sh = 150 - (int)((b >> 23) & 0xFFu);  // 0 .. 150; >= 24 only for v = 0
  const int r = sh < 24 ? (int)(m >> sh) : 0;
  return (int)b < 0 ? -r : r;
}

// Z from the six level sums (levels 0-4 exact integers times 2^-7l, levels 5-7 rounded)
__device__ __forceinline__ long long combine(uint32_t l0, uint32_t l1, uint32_t l2, uint32_t l3, uint32_t l4,
                                             uint32_t l5) {
  unsigned long long z = (unsigned long long)(long long)f2i24(__uint_as_float(l0)) << 42;
  z += (unsigned long long)(long long)f2i24(__uint_as_float(l1) * 0x1p7f) << 35;
  z += (unsigned long long)(long long)f2i24(__uint_as_float(l2) * 0x1p14f) << 28;
  z += (unsigned long long)(long long)f2i24(__uint_as_float(l3) * 0x1p21f) << 21;
  z += (unsigned long long)(long long)f2i24(__uint_as_float(l4) * 0x1p28f) << 14;
  z += (unsigned long long)f2ll(__uint_as_float(l5) * 0x1p42f);
  return (long long)z;
}

__device__ __forceinline__ int dexp(double x) { return (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FF); }

// the seven digits of x relative to 2^(emax - 1021) (emax >= its biased exponent), as bf16 bits
__device__ __forceinline__ void digits7(double x, int emax, uint32_t (&h)[ND]) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  long long X = 0;  // round(x / 2^(emax - 1021) * 2^49), |X| <= 2^48
  if (e != 0) {
    const long long m = (long long)((b & 0xFFFFFFFFFFFFFULL) | (1ULL << 52));
    const int sh = emax + 5 - e;  // >= 5
    X = sh < 54 ? (m + (1LL << (sh - 1))) >> sh : 0LL;
    if (b >> 63) X = -X;
  }
  const unsigned long long Y = (unsigned long long)(X + OFF7);
#pragma unroll
  for (int i = 0; i < ND; ++i) {
    const uint32_t f = i == 0 ? (uint32_t)(Y >> 42) : (uint32_t)((Y >> (7 * (ND - 1 - i))) & 127u);
    // (f - 64) 2^-7i: exact FP32 arithmetic from the bits of 2^23 + f; its bf16 is the top half
    const float v = (__uint_as_float(0x4B000000u | f) - 8388672.0f) * __uint_as_float((uint32_t)(127 - 7 * i) << 23);
    h[i] = __float_as_uint(v) >> 16;
  }
}
}  // namespace tz

struct TzMaps {
  CUtensorMap a[tz::ND];
  CUtensorMap b[tz::ND];
};

// A planes [7][rows][Kp] of P (element (r, e) at P[r sr + e se], ne complex values per row):
// K = (e, re/im).  ea[row] = the largest biased exponent of the row.
__global__ void k_zdig_rows_exp(const double2* __restrict__ P, long sr, long se, int rows, int ne,
                                int* __restrict__ ea) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  int m = 0;
  for (int e = 0; e < ne; ++e) {
    const double2 z = P[(long)r * sr + (long)e * se];
    m = max(m, max(tz::dexp(z.x), tz::dexp(z.y)));
  }
  ea[r] = m;
}

__global__ void k_zdig_rows(const double2* __restrict__ P, long sr, long se, int rows, int ne, int Kp,
                            const int* __restrict__ ea, uint32_t* __restrict__ planes, long plane_words) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int half = Kp / 2;
  if (t >= (long)rows * half) return;
  const int r = (int)(t / half), e = (int)(t - (long)r * half);
  uint32_t hr[tz::ND], hi[tz::ND];
  if (e < ne) {
    const double2 z = P[(long)r * sr + (long)e * se];
    tz::digits7(z.x, ea[r], hr);
    tz::digits7(z.y, ea[r], hi);
  } else {
#pragma unroll
    for (int d = 0; d < tz::ND; ++d) hr[d] = hi[d] = 0u;
  }
#pragma unroll
  for (int d = 0; d < tz::ND; ++d) planes[d * plane_words + t] = hr[d] | (hi[d] << 16);
}

// B planes [7][nq ncq][Kp] of W[q][e][c] (complex, row stride ldw, q stride sW, ncq / 2 columns;
// conj(W) with cj): row 2c holds (Re W, -Im W) and row 2c + 1 (Im W, Re W) along K = (e, re/im),
// so that A B^T gives Re and Im of P W.  eb[row] = the largest biased exponent of the column (both
// rows).
__global__ void k_zdig_cols_exp(const double2* __restrict__ W, long ldw, long sW, int nq, int ne, int ncol,
                                int* __restrict__ eb) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)nq * ncol) return;
  const int q = (int)(t / ncol), c = (int)(t - (long)q * ncol);
  int m = 0;
  for (int e = 0; e < ne; ++e) {
    const double2 z = W[(long)q * sW + (long)e * ldw + c];
    m = max(m, max(tz::dexp(z.x), tz::dexp(z.y)));
  }
  eb[2 * t] = m;
  eb[2 * t + 1] = m;
}

__global__ void k_zdig_cols(const double2* __restrict__ W, long ldw, long sW, int nq, int ne, int ncol, int Kp,
                            int cj, const int* __restrict__ eb, uint32_t* __restrict__ planes, long plane_words) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;  // (q, c, e), e fastest
  const int half = Kp / 2;
  if (t >= (long)nq * ncol * half) return;
  const long qc = t / half;
  const int e = (int)(t - qc * half);
  const int q = (int)(qc / ncol), c = (int)(qc - (long)q * ncol);
  uint32_t hr[tz::ND], hi[tz::ND];
  if (e < ne) {
    const double2 z = W[(long)q * sW + (long)e * ldw + c];
    const int em = eb[2 * qc];
    tz::digits7(z.x, em, hr);
    tz::digits7(cj ? -z.y : z.y, em, hi);
  } else {
#pragma unroll
    for (int d = 0; d < tz::ND; ++d) hr[d] = hi[d] = 0u;
  }
  const long w0 = (2 * qc) * half + e, w1 = (2 * qc + 1) * half + e;  // words of rows 2c and 2c + 1
#pragma unroll
  for (int d = 0; d < tz::ND; ++d) {
    const uint32_t nhi = hi[d] ? hi[d] ^ 0x8000u : 0u;  // the digits of -Im W
    planes[d * plane_words + w0] = hr[d] | (nhi << 16);
    planes[d * plane_words + w1] = hi[d] | (hr[d] << 16);
  }
}

// C[q sCq + row ldc + c scol] (complex128; q = n / ncq, c = (n mod ncq) / 2 for the real column n;
// added to what C holds with acc) from the A rows a_row0 .. a_row0 + M - 1 and the N B rows;
// tiles 128 x 80, n tiles fastest (the CTAs on one A row
// tile run together and share it through L2).  Bounded waits: on a timeout *err is set and the
// CTA stops, drains what it issued and frees its TMEM.
__global__ void __launch_bounds__(tz::THREADS, 1) k_tc_zgemm64(const __grid_constant__ TzMaps maps, int M, int a_row0,
                                                              int N, int Kp, const int* __restrict__ ea,
                                                              const int* __restrict__ eb, double2* __restrict__ C,
                                                              int ncq, long ldc, long sCq, long scol, int acc,
                                                              int* __restrict__ err) {
  using namespace tc;
  using tz::BK;
  using tz::BM;
  using tz::BN;
  using tz::ND;
  using tz::STAGES;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * tz::STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* accf = empty + STAGES;  // the accumulators hold a finished tile
  uint64_t* acce = accf + 1;        // the accumulators have been drained
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acce + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  // barriers and flags take the first 64 bytes after the stages; the column data follow at +128
  long* coff = reinterpret_cast<long*>(smem + STAGES * tz::STAGE_BYTES + 128);  // [BN] C offset of column
  int* cexp = reinterpret_cast<int*>(coff + BN);                                  // [BN] its scale exponent

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkb = Kp / BK;
  const int ntn = (N + BN - 1) / BN, ntm = (M + BM - 1) / BM;
  const long ntiles = (long)ntn * ntm;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    mbar_init(acce, tz::EPI_WARPS);  // one arrival per epilogue warp
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(tz::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  auto atile = [&](int s, int d) -> unsigned char* { return smem + s * tz::STAGE_BYTES + d * tz::A_T; };
  auto btile = [&](int s, int d) -> unsigned char* { return smem + s * tz::STAGE_BYTES + ND * tz::A_T + d * tz::B_SLOT; };

  if (warp == 0) {
    if (lane == 0) {  // ---- TMA producer
      long it = 0;
      for (long t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
        const int m0 = (int)(t / ntn) * BM, n0 = (int)(t % ntn) * BN;
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = (int)(it % STAGES);
          if (it >= STAGES && !mbar_wait(&empty[s], (uint32_t)(((it / STAGES) - 1) & 1))) {
            *abort_flag = 1;
            atomicOr(err, 1);
            break;
          }
          if (*abort_flag) break;
          mbar_arrive_expect_tx(&full[s], tz::TX_BYTES);
#pragma unroll
          for (int d = 0; d < ND; ++d) tma_load_2d(atile(s, d), &maps.a[d], kb * BK, a_row0 + m0, &full[s]);
#pragma unroll
          for (int d = 0; d < ND; ++d) tma_load_2d(btile(s, d), &maps.b[d], kb * BK, n0, &full[s]);
        }
      }
      // after an abort: wait (bounded) for the loads still in flight
      if (*abort_flag)
        for (long j = (it > STAGES ? it - STAGES : 0); j < it; ++j) mbar_wait(&full[j % STAGES], (uint32_t)((j / STAGES) & 1));
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {  // ---- MMA issuer
      long it = 0, lt = 0;
      for (long t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x, ++lt) {
        if (lt >= 1 && !mbar_wait(acce, (uint32_t)((lt - 1) & 1))) {
          *abort_flag = 1;
          atomicOr(err, 8);
          break;
        }
        fence_after();
        bool ok = true;
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = (int)(it % STAGES);
          if (*abort_flag || !mbar_wait(&full[s], (uint32_t)((it / STAGES) & 1))) {
            *abort_flag = 1;
            atomicOr(err, 2);
            ok = false;
            break;
          }
          fence_after();
          uint64_t da[ND], db[ND];
#pragma unroll
          for (int d = 0; d < ND; ++d) {
            da[d] = tch::smem_desc64(smem_u32(atile(s, d)));
            db[d] = tch::smem_desc64(smem_u32(btile(s, d)));
          }
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint64_t o = (uint64_t)(kk * 32) >> 4;  // 16 bf16 = 32 bytes along K
            const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
#pragma unroll
            for (int l = 0; l <= 7; ++l) {
              const uint32_t dst = tmem + (uint32_t)((l < 5 ? l : 5) * BN);
#pragma unroll
              for (int i = (l > ND - 1 ? l - (ND - 1) : 0); i <= (l < ND - 1 ? l : ND - 1); ++i) {
                const bool first = (l < 5) ? (i == 0) : (l == 5 && i == 0);
                tz::mma(dst, da[i] + o, db[l - i] + o, first ? acc : 1u);
              }
            }
          }
          mma_commit(&empty[s]);  // stage s is free once these MMAs have read it
        }
        mma_commit(accf);  // the tile's accumulators are complete (or the loop was aborted)
        if (!ok) break;
      }
    }
    __syncwarp();
  } else {  // ---- epilogue, warps 2..13: TMEM lane quarter = warp % 4, chunk share (warp - 2) / 4
    const int quarter = warp & 3, share = (warp - 2) >> 2;
    long lt = 0;
    for (long t = blockIdx.x; t < ntiles; t += gridDim.x, ++lt) {
      const bool ok = mbar_wait(accf, (uint32_t)(lt & 1));
      if (!ok || *abort_flag) {
        if (!ok) atomicOr(err, 4);
        break;
      }
      fence_after();
      const int m0 = (int)(t / ntn) * BM, n0 = (int)(t % ntn) * BN;
      // the tile's column offsets into C and scale exponents, once per tile (the epilogue threads,
      // named barrier 1: the previous tile's readers are done before the rewrite)
      {
        const int et = threadIdx.x - 64;
        asm volatile("bar.sync 1, %0;" ::"n"(32 * tz::EPI_WARPS) : "memory");
        if (et < BN) {
          const int n = n0 + et;
          if (n < N) {
            const int q = n / ncq;
            coff[et] = (long)q * sCq + (long)((n - q * ncq) >> 1) * scol;
            cexp[et] = eb[n] - 1021;
          }
        }
        asm volatile("bar.sync 1, %0;" ::"n"(32 * tz::EPI_WARPS) : "memory");
      }
      const int row = m0 + quarter * 32 + lane;
      const bool live = row < M;
      const int erow = live ? ea[a_row0 + row] - 1021 - 56 : 0;
      double2* crow = C + (long)row * ldc;
      const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
#pragma unroll 1
      for (int c0 = 16 * share; c0 < BN; c0 += 16 * (tz::EPI_WARPS / 4)) {
        uint32_t r0[16], r1[16], r2[16], r3[16], r4[16], r5[16];
        tmem_ld16(tl + c0, r0);
        tmem_ld16(tl + BN + c0, r1);
        tmem_ld16(tl + 2 * BN + c0, r2);
        tmem_ld16(tl + 3 * BN + c0, r3);
        tmem_ld16(tl + 4 * BN + c0, r4);
        tmem_ld16(tl + 5 * BN + c0, r5);
        tmem_ld_wait();
        if (live) {
#pragma unroll
          for (int i = 0; i < 16; i += 2) {
            const int n = n0 + c0 + i;  // even; N is even, so n + 1 < N with n
            if (n < N) {
              const int E = erow + cexp[c0 + i];
              const double re = tz::ll2d(tz::combine(r0[i], r1[i], r2[i], r3[i], r4[i], r5[i]), E);
              const double im =
                  tz::ll2d(tz::combine(r0[i + 1], r1[i + 1], r2[i + 1], r3[i + 1], r4[i + 1], r5[i + 1]), E);
              double2* o = crow + coff[c0 + i];
              if (acc) {
                const double2 v = *o;
                *o = make_double2(v.x + re, v.y + im);
              } else {
                *o = make_double2(re, im);
              }
            }
          }
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) tcf::mbar_arrive(acce);
    }
  }
  // drain: after an abort the producer waits (bounded) for its last loads (above); every warp
  // then meets here before the TMEM is released
  fence_before();
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tz::TMEM_COLS) : "memory");
  }
}

// ----------------------------------------------------------------------------- host side
namespace {
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

bool encode_fn() {
  if (g_encode) return true;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult qr;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr) != cudaSuccess ||
      qr != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    return false;
  }
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return true;
}
}  // namespace

// 2-D FP32 tensor map over a row-major [rows][kp] array, box 32 x box_rows, 128-byte swizzle.
cudaError_t make_tc_map(void* map_out, const float* base, long rows, int kp, int box_rows) {
  if (!encode_fn()) return cudaErrorNotSupported;
  if (kp % tc::BK != 0 || (reinterpret_cast<uintptr_t>(base) & 15) != 0 || rows < 1) return cudaErrorInvalidValue;
  cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kp * sizeof(float)};
  cuuint32_t box[2] = {(cuuint32_t)tc::BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(static_cast<CUtensorMap*>(map_out), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                        const_cast<float*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// 2-D BF16 tensor map over a row-major [rows][kp] array, box 64 x box_rows, 128-byte swizzle.
cudaError_t make_tc_map_bf16(void* map_out, const void* base, long rows, int kp, int box_rows) {
  if (!encode_fn()) return cudaErrorNotSupported;
  if (kp % tcf::BK != 0 || (reinterpret_cast<uintptr_t>(base) & 15) != 0 || rows < 1) return cudaErrorInvalidValue;
  cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kp * 2};
  cuuint32_t box[2] = {(cuuint32_t)tcf::BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(static_cast<CUtensorMap*>(map_out), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base),
                        dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// 2-D BF16 tensor map over a row-major [rows][kp] array, box 32 x box_rows, 64-byte swizzle.
cudaError_t make_tc_map_bf16_sw64(void* map_out, const void* base, long rows, int kp, int box_rows) {
  if (!encode_fn()) return cudaErrorNotSupported;
  if (kp % tch::BK != 0 || (reinterpret_cast<uintptr_t>(base) & 15) != 0 || rows < 1) return cudaErrorInvalidValue;
  cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kp * 2};
  cuuint32_t box[2] = {(cuuint32_t)tch::BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(static_cast<CUtensorMap*>(map_out), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base),
                        dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_tc_hkq_gemm(const void* maps_a5, const void* maps_b5, int M, int a_row0, int Nr, int Kp, int nq,
                               float sA, const float* sB, float2* C, long ldc, long sC, int* err, cudaStream_t st) {
  return launch_tc_hkq_gemm_b(maps_a5, maps_b5, M, a_row0, Nr, Kp, nq, sA, sB, C, ldc, sC, err, 1, 0, 0, 0, 5, st);
}

cudaError_t launch_tc_hkq_gemm_b(const void* maps_a5, const void* maps_b5, int M, int a_row0, int Nr, int Kp, int nq,
                                 float sA, const float* sB, float2* C, long ldc, long sC, int* err, int a_mod,
                                 int a_qoff, int a_stride, int morder, int ndig, cudaStream_t st) {
  if (M <= 0 || Nr <= 0 || nq <= 0) return cudaSuccess;
  if (a_mod < 1 || a_qoff < 0 || a_stride < 0 || (ndig != 4 && ndig != 5)) return cudaErrorInvalidValue;
  if (Kp % tch::BK != 0 || Kp <= 0 || Kp > 1024) return cudaErrorInvalidValue;  // exact level sums need K <= 1024
  if ((reinterpret_cast<uintptr_t>(C) & 15) != 0 || (ldc & 1) || (sC & 1)) return cudaErrorInvalidValue;
  auto kern = ndig == 5 ? k_tc_hkq_gemm<5> : k_tc_hkq_gemm<4>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, tch::SMEM_BYTES);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return cudaErrorInvalidDevice;
  TcMaps10 maps;
  for (int d = 0; d < ndig; ++d) {
    maps.a[d] = static_cast<const CUtensorMap*>(maps_a5)[d];
    maps.b[d] = static_cast<const CUtensorMap*>(maps_b5)[d];
  }
  const long ntiles = (long)((Nr + tch::BN - 1) / tch::BN) * ((M + tch::BM - 1) / tch::BM) * nq;
  const int grid = (int)(ntiles < sms ? ntiles : sms);
  kern<<<grid, tch::THREADS, tch::SMEM_BYTES, st>>>(maps, M, a_row0, Nr, Kp, nq, sA, sB, C, ldc, sC, err, a_mod, a_qoff,
                                                    a_stride, morder), note_launch();
  return cudaGetLastError();
}

cudaError_t launch_tc_band_gemm(const void* maps_a4, const void* maps_b4, int M, int a_row0, int Nr, int Kp, int nq,
                                float sA, const float* sB, float* C, long ldc, long sC, int* err, int a_mod,
                                int a_qoff, int a_stride, cudaStream_t st) {
  if (M <= 0 || Nr <= 0 || nq <= 0) return cudaSuccess;
  if (Kp % tcb::BK != 0 || Kp <= 0 || Kp > 1024) return cudaErrorInvalidValue;  // exact level-0 sums need K <= 1024
  if (a_mod < 1 || a_qoff < 0 || a_stride < 0) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(C) & 15) != 0) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_tc_band_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, tcb::SMEM_BYTES);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return cudaErrorInvalidDevice;
  TcMaps10 maps;
  for (int d = 0; d < tcb::ND; ++d) {
    maps.a[d] = static_cast<const CUtensorMap*>(maps_a4)[d];
    maps.b[d] = static_cast<const CUtensorMap*>(maps_b4)[d];
  }
  const long ntiles = (long)((Nr + tcb::BN - 1) / tcb::BN) * ((M + tcb::BM - 1) / tcb::BM) * nq;
  const int grid = (int)(ntiles < sms ? ntiles : sms);
  k_tc_band_gemm<<<grid, tcb::THREADS, tcb::SMEM_BYTES, st>>>(maps, M, a_row0, Nr, Kp, nq, sA, sB, C, ldc, sC, err,
                                                               a_mod, a_qoff, a_stride), note_launch();
  return cudaGetLastError();
}

cudaError_t launch_tc_fixed_gemm(const void* maps_a3, const void* maps_b4, int M, int a_row0, int Nr, int Kp, int nq,
                                 float sA, const float* sB, float* C, long ldc, long sC, int* err, cudaStream_t st) {
  if (M <= 0 || Nr <= 0 || nq <= 0) return cudaSuccess;
  if (Kp % tcf::BK != 0 || Kp <= 0 || Kp > 1024) return cudaErrorInvalidValue;  // exact level-0 sums need K <= 1024
  cudaError_t e = cudaFuncSetAttribute(k_tc_fixed_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, tcf::SMEM_BYTES);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return cudaErrorInvalidDevice;
  TcMaps7 maps;
  for (int d = 0; d < 3; ++d) maps.a[d] = static_cast<const CUtensorMap*>(maps_a3)[d];
  for (int d = 0; d < 4; ++d) maps.b[d] = static_cast<const CUtensorMap*>(maps_b4)[d];
  const long ntiles = (long)((Nr + tcf::BN - 1) / tcf::BN) * ((M + tcf::BM - 1) / tcf::BM) * nq;
  const int grid = (int)(ntiles < sms ? ntiles : sms);
  k_tc_fixed_gemm<<<grid, tcf::THREADS, tcf::SMEM_BYTES, st>>>(maps, M, a_row0, Nr, Kp, nq, sA, sB, C, ldc, sC, err), note_launch();
  return cudaGetLastError();
}

cudaError_t launch_tc_split_gemm(const void* mAhi, const void* mAlo, const void* mBhi, const void* mBlo, int M,
                                 int a_row0, int Nr, int Kp, int nq, float* C, long ldc, long sC, int* err,
                                 cudaStream_t st) {
  if (M <= 0 || Nr <= 0 || nq <= 0) return cudaSuccess;
  if (Kp % tc::BK != 0 || Kp <= 0) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_tc_split_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES);
  if (e != cudaSuccess) return e;
  dim3 grid((Nr + tc::BN - 1) / tc::BN, (M + tc::BM - 1) / tc::BM, nq);
  if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidConfiguration;
  k_tc_split_gemm<<<grid, 128, tc::SMEM_BYTES, st>>>(*static_cast<const CUtensorMap*>(mAhi),
                                                     *static_cast<const CUtensorMap*>(mAlo),
                                                     *static_cast<const CUtensorMap*>(mBhi),
                                                     *static_cast<const CUtensorMap*>(mBlo), M, a_row0, Nr, Kp, C,
                                                     ldc, sC, err), note_launch();
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------- FP64-accuracy complex GEMM, host
cudaError_t launch_zdigits_rows(const double2* P, long sr, long se, int rows, int ne, int Kp, int* ea, void* planes,
                                cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  if (Kp % tz::BK != 0 || 2 * ne > Kp) return cudaErrorInvalidValue;
  k_zdig_rows_exp<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(P, sr, se, rows, ne, ea), note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long words = (long)rows * (Kp / 2);
  k_zdig_rows<<<(unsigned)((words + 255) / 256), 256, 0, st>>>(P, sr, se, rows, ne, Kp, ea,
                                                               static_cast<uint32_t*>(planes), words), note_launch();
  return cudaGetLastError();
}

cudaError_t launch_zdigits_cols(const double2* W, long ldw, long sW, int nq, int ne, int ncol, int Kp, int cj, int* eb,
                                void* planes, cudaStream_t st) {
  if (nq <= 0 || ncol <= 0) return cudaSuccess;
  if (Kp % tz::BK != 0 || 2 * ne > Kp) return cudaErrorInvalidValue;
  const long cols = (long)nq * ncol;
  k_zdig_cols_exp<<<(unsigned)((cols + 255) / 256), 256, 0, st>>>(W, ldw, sW, nq, ne, ncol, eb), note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long words = cols * (Kp / 2);
  k_zdig_cols<<<(unsigned)((words + 255) / 256), 256, 0, st>>>(W, ldw, sW, nq, ne, ncol, Kp, cj, eb,
                                                               static_cast<uint32_t*>(planes), 2 * words), note_launch();
  return cudaGetLastError();
}

cudaError_t launch_tc_zgemm64(const void* a_planes, long a_rows, int a_row0, int M, const int* ea, const void* b_planes,
                              int N, const int* eb, int Kp, double2* C, int ncq, long ldc, long sCq, long scol, int acc,
                              int* err, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  // exact sums of levels 0-4 and the int64 combination need K <= 512
  if (Kp % tz::BK != 0 || Kp <= 0 || Kp > 512 || (N & 1) || (ncq & 1) || ncq <= 0) return cudaErrorInvalidValue;
  if (a_row0 < 0 || a_row0 + (long)M > a_rows) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(C) & 15) != 0) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_tc_zgemm64, cudaFuncAttributeMaxDynamicSharedMemorySize, tz::SMEM_BYTES);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return cudaErrorInvalidDevice;
  TzMaps maps;
  const size_t aplane = (size_t)a_rows * Kp * 2, bplane = (size_t)N * Kp * 2;
  for (int d = 0; d < tz::ND; ++d) {
    if ((e = make_tc_map_bf16_sw64(&maps.a[d], static_cast<const char*>(a_planes) + d * aplane, a_rows, Kp, tz::BM)) !=
        cudaSuccess)
      return e;
    if ((e = make_tc_map_bf16_sw64(&maps.b[d], static_cast<const char*>(b_planes) + d * bplane, N, Kp, tz::BN)) !=
        cudaSuccess)
      return e;
  }
  const long ntiles = (long)((N + tz::BN - 1) / tz::BN) * ((M + tz::BM - 1) / tz::BM);
  const int grid = (int)(ntiles < sms ? ntiles : sms);
  k_tc_zgemm64<<<grid, tz::THREADS, tz::SMEM_BYTES, st>>>(maps, M, a_row0, N, Kp, ea, eb, C, ncq, ldc, sCq, scol, acc,
                                                          err), note_launch();
  return cudaGetLastError();
}

}  // namespace eph
