// Band rotation g_nu = V_{k+q}^H G3_nu V_k (the last step of Eq. 7's evaluation, Eqs. 4-5
// gauges) for shapes beyond the shared-memory kernels, on the tcgen05 tensor cores: the mixed
// form's large-Nb path.  Two batched products of the fixed-point digit scheme of the H(k+q)
// contraction with four digits per operand (levels <= 3, ~2^-32 of each row's scale; results
// rounded to one FP32 per element), on the real embedding of the complex matrices (K = 2 Nb,
// re/im interleaved):
//   stage 1, per pair:  C1[2n' + c][nu Nb + a] = (re, im)_c of T[(nu, a)][n'],  T = G3_nu V_k,
//                       A = V_k embedded (rows 2n' + c, K = 2b + t), B = the G3 rows (nu, a);
//   stage 2, per pair:  C2[2m + c][nu Nb + n'] = (re, im)_c of g_nu[m][n'],
//                       A = V_{k+q}^H embedded (rows 2m + c, K = 2a + t),
//                       B rows (nu, n') with K = 2a + t gathered from C1.
// Every B row carries its own power-of-two scale (fixed point relative to the row maximum);
// V is unitary, so its scale is 2.
#include <algorithm>
#include <mutex>
#include <vector>

#include <cuda.h>
#include <cuda_bf16.h>

#include "eph_kernels.cuh"

namespace eph {
namespace {

constexpr int MAXKL = 16;  // K values per lane in the row kernels (Kp <= 512, Nb <= 256)
constexpr int NDIG = 4;    // digits per operand: 32 bits, ~2^-32 of each row's scale (complex64 g)
constexpr int FBITS = 8 * NDIG;

// The digit kernels run on the integer pipe: FP64 arithmetic (and FP64 <-> integer conversion)
// is ~1/64 of the FP32 rate on GB300, so the fixed-point value round(x 2^(F - es)) of
// x / s (s = 2^es, F = 8 NDIG bits) is formed from the IEEE bits.
__device__ __forceinline__ long long fixedF_d(double x, int es) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e == 0) return 0;  // zero or subnormal: below the row's last digit
  const long long m = (long long)((b & 0xFFFFFFFFFFFFFULL) | (1ULL << 52));
  const int sh = (e - 1023) - 52 + FBITS - es;  // x 2^(F - es) = m 2^sh
  long long X;
  if (sh >= 0)
    X = m << sh;  // |x / s| <= 1/2 keeps this below 2^F
  else if (sh > -63)
    X = (m + (1LL << (-sh - 1))) >> (-sh);
  else
    X = 0;
  return (long long)(b >> 63) ? -X : X;
}
__device__ __forceinline__ long long fixedF_f(float x, int es) {
  const unsigned int b = __float_as_uint(x);
  const int e = (int)((b >> 23) & 0xFF);
  if (e == 0) return 0;
  const long long m = (long long)((b & 0x7FFFFFu) | 0x800000u);
  const int sh = (e - 127) - 23 + FBITS - es;
  long long X;
  if (sh >= 0)
    X = m << sh;
  else if (sh > -62)
    X = (m + (1LL << (-sh - 1))) >> (-sh);
  else
    X = 0;
  return (b >> 31) ? -X : X;
}

// NDIG signed base-256 digits of X = round(y 2^F), |y| <= 1/2 (+ 2^-24): y = sum_i d_i
// 2^-8(i+1) + O(2^-(F+1)), |d_i| <= 128; digit i stored pre-scaled by 2^-8i (exact in bf16).
__device__ __forceinline__ void put_digits(long long R, __nv_bfloat16* __restrict__ D, long slice, long idx) {
  float scale = 1.f;
#pragma unroll
  for (int i = 0; i < NDIG - 1; ++i) {
    const int sh = FBITS - 8 - 8 * i;
    const long long d = (R + (1LL << (sh - 1))) >> sh;  // round to nearest (arithmetic shift)
    R -= d * (1LL << sh);
    D[i * slice + idx] = __float2bfloat16_rn((float)(int)d * scale);
    scale *= 0x1p-8f;
  }
  D[(NDIG - 1) * slice + idx] = __float2bfloat16_rn((float)(int)R * scale);
}

// exponent es of the row scale s = 2^es >= 2 max|x| from the largest biased exponent eb of the
// row (max|x| in [2^(eb - bias), 2^(eb - bias + 1))): es = eb - bias + 2; an all-zero row gets 0
__device__ __forceinline__ int warp_max_int(int v) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// A digits of embedded unitary matrices V[b] (nb x nb, stride sV): rows r = 2i + c, K = 2j + t;
// mode 0: [[Vr, -Vi], [Vi, Vr]][c][t] of V[j][i] (V^T applied to G3 rows), mode 1:
// [[Vr, Vi], [-Vi, Vr]][c][t] of V[j][i] (V^H applied to T).  s = 2.
__global__ void k_vdigits(const double2* __restrict__ V, long sV, int nb, long nmat, int kp, int mode,
                          __nv_bfloat16* __restrict__ D, long slice) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long per = 2L * nb * kp;
  if (idx >= per * nmat) return;
  const long b = idx / per;
  const long rem = idx - b * per;
  const int r = (int)(rem / kp), kk = (int)(rem - (long)r * kp);
  double x = 0.0;
  if (kk < 2 * nb) {
    const int i = r >> 1, c = r & 1, j = kk >> 1, t = kk & 1;
    const double2 v = V[b * sV + (long)j * nb + i];
    if (mode == 0)
      x = (c == t) ? v.x : (c == 0 ? -v.y : v.y);
    else
      x = (c == t) ? v.x : (c == 0 ? v.y : -v.y);
  }
  put_digits(fixedF_d(x, 1), D, slice, idx);
}

// Stage-1 B digits, one warp per row w = p nrow + j: K = 2b + t of G3[p][j][b] (complex row of nb
// elements at Y + p ldy + off + j nb: complex128 from the FP64 contraction or complex64 from the
// tensor-core one); sB[w] = the row's scale.
__device__ __forceinline__ int biased_exp(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF); }
__device__ __forceinline__ int biased_exp(float x) { return (int)((__float_as_uint(x) >> 23) & 0xFF); }
__device__ __forceinline__ long long fixedF(double x, int es) { return fixedF_d(x, es); }
__device__ __forceinline__ long long fixedF(float x, int es) { return fixedF_f(x, es); }

template <typename TC>  // double2 or float2
__global__ void k_gdigits(const TC* __restrict__ Y, long ldy, long off, int nrow, int nb, long rows, int kp,
                          float* __restrict__ sB, __nv_bfloat16* __restrict__ D, long slice) {
  using T = decltype(TC::x);
  constexpr int bias = sizeof(T) == 8 ? 1023 : 127;
  const long w = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= rows) return;  // whole warps
  const long p = w / nrow;
  const int j = (int)(w - p * nrow);
  const T* src = reinterpret_cast<const T*>(Y + p * ldy + off + (long)j * nb);
  T x[MAXKL];
  int eb = 0;
#pragma unroll
  for (int i = 0; i < MAXKL; ++i) {
    const int kk = lane + 32 * i;
    x[i] = kk < 2 * nb ? src[kk] : (T)0;
    eb = max(eb, biased_exp(x[i]));
  }
  eb = warp_max_int(eb);
  const int es = eb ? eb - bias + 2 : 0;
  if (lane == 0) sB[w] = ldexpf(1.f, es);
#pragma unroll
  for (int i = 0; i < MAXKL; ++i) {
    const int kk = lane + 32 * i;
    if (kk < kp) put_digits(fixedF(x[i], es), D, slice, w * kp + kk);
  }
}

// Stage-2 B digits, one warp per row w = p nrow + j, j = nu nb + n': K = 2a + t of
// T[(nu, a)][n'] part t = C1[p][2n' + t][nu nb + a].
__global__ void k_tdigits(const float* __restrict__ C1, long sC, int nrow, int nb, long rows, int kp,
                          float* __restrict__ sB, __nv_bfloat16* __restrict__ D, long slice) {
  const long w = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= rows) return;
  const long p = w / nrow;
  const int j = (int)(w - p * nrow);
  const int nu = j / nb, np_ = j - nu * nb;
  const float* src = C1 + p * sC + (long)nu * nb;
  float x[MAXKL];
  int eb = 0;
#pragma unroll
  for (int i = 0; i < MAXKL; ++i) {
    const int kk = lane + 32 * i;
    x[i] = kk < 2 * nb ? src[(long)(2 * np_ + (kk & 1)) * nrow + (kk >> 1)] : 0.f;
    eb = max(eb, (int)((__float_as_uint(x[i]) >> 23) & 0xFF));
  }
  eb = warp_max_int(eb);
  const int es = eb ? eb - 127 + 2 : 0;
  if (lane == 0) sB[w] = ldexpf(1.f, es);
#pragma unroll
  for (int i = 0; i < MAXKL; ++i) {
    const int kk = lane + 32 * i;
    if (kk < kp) put_digits(fixedF_f(x[i], es), D, slice, w * kp + kk);
  }
}

// g[iq][kk][nu][m][n'] = complex64 of C2[p][2m + c][nu nb + n'], pair p0 + p = iq nk + kk.
__global__ void k_gout(const float* __restrict__ C2, long sC, int nrow, int nb, int nm, long npairs, int nk, long p0,
                       float2* __restrict__ g, long sgq) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long per = (long)nm * nb * nb;
  if (idx >= per * npairs) return;
  const long p = idx / per;
  const long rem = idx - p * per;
  const int nu = (int)(rem / (nb * nb));
  const int r2 = (int)(rem - (long)nu * nb * nb);
  const int m = r2 / nb, n = r2 - m * nb;
  const float* src = C2 + p * sC + (long)nu * nb + n;
  const long P = p0 + p;
  const long iq = P / nk, kk = P - iq * nk;
  g[iq * sgq + kk * per + rem] = make_float2(src[(long)(2 * m) * nrow], src[(long)(2 * m + 1) * nrow]);
}

size_t align_up(size_t x) { return (x + 1023) & ~(size_t)1023; }

struct BandTcShape {
  int kp, M;
  long Nr;
  size_t a1, per_pair;
};

BandTcShape band_tc_shape(int nk, int nm, int nb) {
  BandTcShape s;
  s.kp = ((2 * nb + 31) / 32) * 32;
  s.M = 2 * nb;
  s.Nr = (long)nm * nb;
  s.a1 = align_up((size_t)NDIG * nk * s.M * s.kp * 2);
  // B digits (shared by both stages), C in FP32 (C1 then C2), A2 digits, B row scales
  s.per_pair =
      (size_t)NDIG * s.Nr * s.kp * 2 + (size_t)s.M * s.Nr * 4 + (size_t)NDIG * s.M * s.kp * 2 + (size_t)s.Nr * 4;
  return s;
}

}  // namespace

bool band_tc_supported(int nm, int nb) {
  // exact level sums need K = 2 Nb <= 1024; the epilogue's paired stores need an even row length
  return nb >= 1 && nb <= 256 && ((long)nm * nb) % 2 == 0;
}

size_t band_tc_work_bytes(int nk, int nm, int nb, long pairs) {
  const BandTcShape s = band_tc_shape(nk, nm, nb);
  return s.a1 + (size_t)pairs * s.per_pair + 4 * 1024;
}

cudaError_t launch_band_tc(const void* Y, int y_f32, long ldy, long y_off, const double2* Ukq, const double2* Uk, int nq,
                           int nk, int nm, int nb, float2* g, long sgq, void* work, size_t work_bytes, int* err,
                           cudaStream_t st) {
  const long npairs = (long)nq * nk;
  if (npairs <= 0) return cudaSuccess;
  if (!band_tc_supported(nm, nb) || nk < 1) return cudaErrorInvalidValue;
  const BandTcShape sh = band_tc_shape(nk, nm, nb);
  if (work_bytes < band_tc_work_bytes(nk, nm, nb, 1)) return cudaErrorInvalidValue;
  long PB = (long)((work_bytes - sh.a1 - 4 * 1024) / sh.per_pair);
  if (PB > npairs) PB = npairs;
  const int kp = sh.kp, M = sh.M;
  const long Nr = sh.Nr;
  char* base = static_cast<char*>(work);
  __nv_bfloat16* A1 = reinterpret_cast<__nv_bfloat16*>(base);
  char* chunk = base + sh.a1;
  __nv_bfloat16* Bd = reinterpret_cast<__nv_bfloat16*>(chunk);
  float* C = reinterpret_cast<float*>(chunk + align_up((size_t)NDIG * PB * Nr * kp * 2));
  __nv_bfloat16* A2 = reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<char*>(C) + align_up((size_t)PB * M * Nr * 4));
  float* sB = reinterpret_cast<float*>(reinterpret_cast<char*>(A2) + align_up((size_t)NDIG * PB * M * kp * 2));
  cudaError_t e;
  // A digits of V_k for every k of the tile (stage 1)
  {
    const long slice = (long)nk * M * kp;
    k_vdigits<<<(unsigned)((slice + 255) / 256), 256, 0, st>>>(Uk, (long)nb * nb, nb, nk, kp, 0, A1, slice), note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  CUtensorMap mA1[5], mA2[5], mB[5];
  for (int d = 0; d < NDIG; ++d)
    if ((e = make_tc_map_bf16_sw64(&mA1[d], A1 + (long)d * nk * M * kp, (long)nk * M, kp, 128)) != cudaSuccess) return e;
  for (long p0 = 0; p0 < npairs; p0 += PB) {
    const long pb = npairs - p0 < PB ? npairs - p0 : PB;
    const long rows = pb * Nr, bslice = rows * kp, aslice = pb * M * kp;
    for (int d = 0; d < NDIG; ++d) {
      if ((e = make_tc_map_bf16_sw64(&mB[d], Bd + d * bslice, rows, kp, 128)) != cudaSuccess) return e;
      if ((e = make_tc_map_bf16_sw64(&mA2[d], A2 + d * aslice, pb * M, kp, 128)) != cudaSuccess) return e;
    }
    // stage 1: T^T = V_k^T G3^T per pair
    const unsigned gblocks = (unsigned)((rows * 32 + 255) / 256);
    if (y_f32)
      k_gdigits<float2><<<gblocks, 256, 0, st>>>(static_cast<const float2*>(Y) + p0 * ldy, ldy, y_off, (int)Nr, nb,
                                                 rows, kp, sB, Bd, bslice), note_launch();
    else
      k_gdigits<double2><<<gblocks, 256, 0, st>>>(static_cast<const double2*>(Y) + p0 * ldy, ldy, y_off, (int)Nr, nb,
                                                  rows, kp, sB, Bd, bslice), note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_tc_band_gemm(mA1, mB, M, 0, (int)Nr, kp, (int)pb, 2.0f, sB, C, Nr, (long)M * Nr, err, nk,
                                 (int)(p0 % nk), M, st)) != cudaSuccess)
      return e;
    // stage 2: g = V_{k+q}^H T per pair
    k_tdigits<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, st>>>(C, (long)M * Nr, (int)Nr, nb, rows, kp, sB, Bd,
                                                                   bslice), note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_vdigits<<<(unsigned)((aslice + 255) / 256), 256, 0, st>>>(Ukq + p0 * nb * nb, (long)nb * nb, nb, pb, kp, 1, A2,
                                                                aslice), note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_tc_band_gemm(mA2, mB, M, 0, (int)Nr, kp, (int)pb, 2.0f, sB, C, Nr, (long)M * Nr, err, (int)pb, 0, M,
                                 st)) != cudaSuccess)
      return e;
    const long tot = pb * nm * nb * nb;
    k_gout<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(C, (long)M * Nr, (int)Nr, nb, nm, pb, nk, p0, g, sgq), note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}


// ---------------------------------------------------------------------------------------------
// Band rotation for Nb <= 16 and Nm Nb <= 128 (the Si- and MoS2-shaped workloads of the mixed
// form), both products of a tile of pairs fused in one CTA on the tcgen05 tensor cores.  A tile
// holds PPT pairs (q, k) with one k:
//   stage 1, per pair:  U_nu = V_{k+q}^H G3_nu     A rows (nu, n'), K = (a, re/im); B = conj(V_{k+q})
//                       on the real embedding, columns (m, re/im), one column block per pair (the
//                       cross products of one pair's rows with another's block are never read);
//   stage 2, per tile:  g_nu = U_nu V_k            A rows (m, nu), K = (n', re/im); B = V_k on the
//                       real embedding, columns (n, re/im), shared by the tile's pairs.
// Pair j takes the accumulator rows j*RS .. j*RS + Nm Nb - 1 (RS a multiple of 32: each warp's TMEM
// lanes belong to one pair).  Operands are four fixed-point BF16 digits (32 bits; levels i + j <= 3,
// 10 MMAs per K step): level 0 in its own accumulator, where its sum is exact, levels 1-3 in a second
// one (~2^-31 of the result).  G3 (rounded to FP32 when it comes in FP64) carries a
// power-of-two scale per row, U one per pair (errors are measured against each pair's largest
// |g|^2), V scale 2.  Digits of FP32 values come from FP32 arithmetic: adding and subtracting
// 1.5 * 2^23 rounds to an integer and each remainder is exact.  V (FP64) goes through an exact
// 32-bit fixed-point integer.  The threads write the digits straight into shared memory in the
// no-swizzle K-major layout (8-row x 16-byte core matrices); U never leaves the SM.
// Every wait on the MMA completion barrier is bounded: on a timeout the CTA sets *err and stops.
namespace {
namespace bts {
constexpr int THREADS = 128, ND = 4;
constexpr long long WAIT_LIMIT = 2000000000LL;  // ~1 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// byte offset of element (r, k) in a K-major tile with KP columns, no swizzle: core matrices of
// 8 rows x 8 bf16 (128 contiguous bytes), K-adjacent ones 128 B apart (LBO), 8-row groups
// KP/8 x 128 B apart (SBO)
template <int KP>
__device__ __forceinline__ uint32_t off(int r, int k) {
  return (uint32_t)((r >> 3) * (KP * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}
template <int KP>
__device__ __forceinline__ uint64_t desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)(128 >> 4) << 16;       // LBO: next core matrix along K
  d |= (uint64_t)((KP * 16) >> 4) << 32;  // SBO: next 8-row group
  d |= (uint64_t)1 << 46;                 // descriptor version
  return d;                               // swizzle mode 0: none
}
// kind::f16 instruction descriptor: D f32, A/B bf16, both K-major, M = 128, N = n
__device__ __forceinline__ uint32_t idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc)
      : "memory");
}
// the ten digit products of levels <= 3 over KP/16 K steps: level 0 into d0, levels 1-3 into d1
template <int KP>
__device__ __forceinline__ void mma_levels(uint32_t d0, uint32_t d1, uint32_t sA, int a_tile, uint32_t sB, int b_tile,
                                           uint32_t id) {
#pragma unroll
  for (int ks = 0; ks < KP / 16; ++ks) {
    uint64_t da[ND], db[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      da[d] = desc<KP>(sA + d * a_tile + ks * 256);
      db[d] = desc<KP>(sB + d * b_tile + ks * 256);
    }
    const uint32_t f = ks > 0 ? 1u : 0u;
    mma(d0, da[0], db[0], id, f);
    mma(d1, da[0], db[1], id, f);
    mma(d1, da[1], db[0], id, 1u);
    mma(d1, da[0], db[2], id, 1u);
    mma(d1, da[1], db[1], id, 1u);
    mma(d1, da[2], db[0], id, 1u);
    mma(d1, da[0], db[3], id, 1u);
    mma(d1, da[1], db[2], id, 1u);
    mma(d1, da[2], db[1], id, 1u);
    mma(d1, da[3], db[0], id, 1u);
  }
}
__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool wait(uint64_t* bar, uint32_t parity) {
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
    if (clock64() - t0 > WAIT_LIMIT) return false;
  }
}
__device__ __forceinline__ void ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
template <int BYTES>
__device__ __forceinline__ void cp_async(uint32_t dst, const void* src) {
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(dst), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void st32(uint32_t addr, uint32_t v) {
  asm volatile("st.shared.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void st128(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}
// the bf16 pair (lo, hi) of two FP32 values that are exact in bf16 (digits), lo at the lower address
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}
// Digits e_i = D_i 2^-8(i+1), integers |D_i| <= 128, of y + yl with |y + yl| <= 1/2 (y and yl two
// parts of one value): y + yl = e_0 + e_1 + e_2 + e_3 + O(2^-31).  Adding and subtracting
// 1.5 * 2^(23 - 8(i+1)) rounds to a multiple of 2^-8(i+1); the remainders are exact up to the one
// rounding that folds yl in.  Level-0 products e_0 f_0 are multiples of 2^-16 below 2^-2, so their
// sums over K <= 32 stay exact in FP32.
constexpr float MG0 = 0x1.8p15f, MG1 = 0x1.8p7f, MG2 = 0x1.8p-1f, MG3 = 0x1.8p-9f;
__device__ __forceinline__ float rnd_at(float y, float M) { return __fsub_rn(__fadd_rn(y, M), M); }
__device__ __forceinline__ void fdigits(float y, float yl, float (&e)[ND]) {
  float q = rnd_at(__fadd_rn(y, yl), MG0);
  e[0] = q;
  y = __fadd_rn(__fsub_rn(y, q), yl);
  q = rnd_at(y, MG1);
  e[1] = q;
  y = __fsub_rn(y, q);
  q = rnd_at(y, MG2);
  e[2] = q;
  e[3] = rnd_at(__fsub_rn(y, q), MG3);
}
__device__ __forceinline__ float i2f(int q) { return __fsub_rn(__int_as_float(0x4B400000 + q), 12582912.0f); }  // |q| < 2^22
// the same digits of X 2^-32 for an integer X = round(y 2^32), |X| <= 2^31, from integer arithmetic
__device__ __forceinline__ void idigits(long long X, float (&d)[ND]) {
  const int q0 = (int)((X + (1LL << 23)) >> 24);
  int r = (int)(X - ((long long)q0 << 24));
  const int q1 = (r + (1 << 15)) >> 16;
  r -= q1 << 16;
  const int q2 = (r + (1 << 7)) >> 8;
  r -= q2 << 8;
  d[0] = __fmul_rn(i2f(q0), 0x1p-8f);
  d[1] = __fmul_rn(i2f(q1), 0x1p-16f);
  d[2] = __fmul_rn(i2f(q2), 0x1p-24f);
  d[3] = __fmul_rn(i2f(r), 0x1p-32f);
}
// FP64 -> FP32, rounded to nearest (ties away), by integer operations (normal FP32 range; smaller
// magnitudes give 0)
__device__ __forceinline__ float d2f_int(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x) + (1ULL << 28);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned e = (hi >> 20) & 0x7FFu;
  const unsigned mag = __funnelshift_l(lo, hi, 3) - (896u << 23);
  return (e > 896u && e < 1151u) ? __uint_as_float(mag | (hi & 0x80000000u)) : 0.f;
}
__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(double x) { return d2f_int(x); }
__device__ __forceinline__ float pow2f(int e) { return ldexpf(1.f, e); }  // once per row and tile
__device__ __forceinline__ int fexp(float x) { return (int)((__float_as_uint(x) >> 23) & 0xFF); }
}  // namespace bts

template <typename TC, int KP>  // TC: double2 (FP64 contraction) or float2 (tensor-core contraction)
__global__ void __launch_bounds__(bts::THREADS, KP == 16 ? 6 : 4) k_band_tc_small(const TC* __restrict__ Y, long ldy,
                                                                   const double2* __restrict__ Ukq,
                                                                   const double2* __restrict__ Uk, int nq, int nk,
                                                                   int nm, int nb, int RS, int PPT,
                                                                   float2* __restrict__ g, long sgq,
                                                                   const int* __restrict__ keep, int* __restrict__ err,
                                                                   uint32_t tmem_cols, int vec16) {
  using namespace bts;
  constexpr int A_TILE = 128 * KP * 2;
  constexpr int B2_TILE = KP * KP * 2;
  extern __shared__ __align__(1024) unsigned char sm[];
  const int N1 = PPT * KP;  // stage-1 MMA N: PPT column blocks of KP
  const int B1_TILE = N1 * KP * 2;
  unsigned char* A = sm;                    // [ND][128 x KP] (stage 1, then stage 2)
  unsigned char* B1 = A + ND * A_TILE;      // [ND][N1 x KP]
  unsigned char* B2 = B1 + ND * B1_TILE;    // [ND][KP x KP]
  const int per = nm * nb * nb;             // G3 elements of one pair
  // raw inputs of the next tile, copied asynchronously while the current one computes:
  // G3 of each pair [PPT][per], then V_{k+q} of each pair and V_k [PPT + 1][nb2]
  unsigned char* rawG = B2 + ND * B2_TILE;
  unsigned char* rawV = rawG + (((size_t)PPT * per * sizeof(TC) + 15) & ~(size_t)15);
  int* smax = reinterpret_cast<int*>(rawV + (size_t)(PPT + 1) * nb * nb * sizeof(double2));  // [4] exponent of U
  uint64_t* bar = reinterpret_cast<uint64_t*>(smax + 4);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int nb2 = nb * nb, R = nm * nb, K2 = 2 * nb;
  const uint32_t sA = smem_u32(A), sB1 = smem_u32(B1), sB2 = smem_u32(B2);
  const uint32_t sRawG = smem_u32(rawG), sRawV = smem_u32(rawV);
  const TC* gsm = reinterpret_cast<const TC*>(rawG);
  const double2* vsm = reinterpret_cast<const double2*>(rawV);

  // zero the operand tiles once: K padding and unused rows stay zero
  for (int i = tid; i < (ND * (A_TILE + B1_TILE + B2_TILE)) / 16; i += THREADS)
    reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t acc0 = tmem, acc1 = tmem + (uint32_t)N1;  // L0 | L123 (stage 2 uses their first KP columns)
  // this thread's accumulator row: pair j of the tile, row rr of that pair
  const int j = tid / RS, rr = tid - j * RS;
  const bool row_ok = j < PPT && rr < R;
  const int nu1 = rr / nb, x1 = rr - nu1 * nb;  // stage 1 row (nu, n')
  const int m2 = rr / nm, nu2 = rr - m2 * nm;   // stage 2 row (m, nu)
  const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
  const uint32_t tl1 = lane_base + (uint32_t)(j < PPT ? j * KP : 0);
  uint32_t phase = 0;
  const unsigned div_nb = (65536u + nb - 1) / nb, div_nb2 = (65536u + nb2 - 1) / nb2;
  const int nqg = (nq + PPT - 1) / PPT;
  const long ntiles = (long)nqg * nk;
  const bool vec_out = (nb % 2 == 0) && ((reinterpret_cast<uintptr_t>(g) & 15) == 0) && (sgq % 2 == 0);
  // asynchronous copies of tile tt's inputs into rawG / rawV (one commit group)
  auto prefetch = [&](long tt) {
    if (tt >= ntiles) return;
    const int kk = (int)(tt % nk), qg = (int)(tt / nk);
    for (int jj = 0; jj < PPT; ++jj) {
      const int iq = qg * PPT + jj;
      if (iq >= nq) break;
      const long P = (long)iq * nk + kk;
      const TC* src = Y + P * ldy;
      const uint32_t dst = sRawG + (uint32_t)((size_t)jj * per * sizeof(TC));
      if (sizeof(TC) == 16 || !vec16) {
        for (int i = tid; i < per; i += THREADS) cp_async<(int)sizeof(TC)>(dst + (uint32_t)(i * sizeof(TC)), src + i);
      } else {  // complex64 rows 16-byte aligned, even length: two elements per copy
        for (int i = tid; 2 * i < per; i += THREADS) cp_async<16>(dst + (uint32_t)(i * 16), src + 2 * i);
      }
      const double2* vs = Ukq + P * nb2;
      for (int i = tid; i < nb2; i += THREADS) cp_async<16>(sRawV + (uint32_t)((jj * nb2 + i) * 16), vs + i);
    }
    const double2* vk = Uk + (long)kk * nb2;
    for (int i = tid; i < nb2; i += THREADS) cp_async<16>(sRawV + (uint32_t)((PPT * nb2 + i) * 16), vk + i);
    cp_async_commit();
  };
  prefetch(blockIdx.x);

  for (long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int kk = (int)(t % nk), qg = (int)(t / nk);
    // ---- stage-1 A (digits of the G3 rows) and both B operands, from this tile's raw inputs
    if (tid < 4) smax[tid] = 0;
    cp_async_wait_all();
    __syncthreads();
    const int iq = qg * PPT + j;
    const bool live = row_ok && iq < nq;
    const long P = (long)iq * nk + kk;
    int es = 0;  // row scale 2^es of this thread's G3 row
    if (live) {
      const TC* src = gsm + (long)j * per + (long)nu1 * nb2 + x1;
      float v[KP];
      float mx = 0.f;
#pragma unroll
      for (int a = 0; a < KP / 2; ++a) {
        if (a < nb) {
          const TC z = src[(long)a * nb];
          v[2 * a] = to_f(z.x);
          v[2 * a + 1] = to_f(z.y);
          mx = fmaxf(mx, fmaxf(fabsf(v[2 * a]), fabsf(v[2 * a + 1])));
        } else {
          v[2 * a] = 0.f;
          v[2 * a + 1] = 0.f;
        }
      }
      const int eb = fexp(mx);
      es = eb ? eb - 127 + 2 : 0;
      const float sc = pow2f(-es);
#pragma unroll
      for (int c = 0; c < KP / 8; ++c) {  // 16-byte chunk c: K = 8c .. 8c + 7, i.e. a = 4c .. 4c + 3
        uint32_t w[ND][4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          float dr[ND], di[ND];
          fdigits(__fmul_rn(v[8 * c + 2 * i], sc), 0.f, dr);
          fdigits(__fmul_rn(v[8 * c + 2 * i + 1], sc), 0.f, di);
#pragma unroll
          for (int d = 0; d < ND; ++d) w[d][i] = pack2(dr[d], di[d]);
        }
        const uint32_t o = off<KP>(tid, 8 * c);
#pragma unroll
        for (int d = 0; d < ND; ++d) st128(sA + d * A_TILE + o, w[d][0], w[d][1], w[d][2], w[d][3]);
      }
    }
    for (int e = tid; e < (PPT + 1) * nb2; e += THREADS) {
      // e / nb2 and r2 / nb by multiply-shift (exact for e < 2^16 / nb2, r2 < 2^16 / nb)
      const int jj = (int)(((unsigned)e * div_nb2) >> 16), r2 = e - jj * nb2;
      const int a = (int)(((unsigned)r2 * div_nb) >> 16), c = r2 - a * nb;
      float vr[ND], vi[ND];
      if (jj < PPT) {
        // stage 1, block jj: conj(V_{k+q})[a][m = c]; rows (m, re) = (Vr, Vi), (m, im) = (-Vi, Vr) along K = (a, re/im)
        const int iqj = qg * PPT + jj;
        if (iqj >= nq) continue;
        const double2 u = vsm[jj * nb2 + r2];
        idigits(fixedF_d(u.x, 1), vr);
        idigits(fixedF_d(u.y, 1), vi);
        const uint32_t o0 = off<KP>(jj * KP + 2 * c, 2 * a), o1 = off<KP>(jj * KP + 2 * c + 1, 2 * a);
#pragma unroll
        for (int d = 0; d < ND; ++d) {
          st32(sB1 + d * B1_TILE + o0, pack2(vr[d], vi[d]));
          st32(sB1 + d * B1_TILE + o1, pack2(-vi[d], vr[d]));
        }
      } else {
        // stage 2: V_k[n' = a][n = c]; rows (n, re) = (Vr, -Vi), (n, im) = (Vi, Vr) along K = (n', re/im)
        const double2 u = vsm[PPT * nb2 + r2];
        idigits(fixedF_d(u.x, 1), vr);
        idigits(fixedF_d(u.y, 1), vi);
        const uint32_t o0 = off<KP>(2 * c, 2 * a), o1 = off<KP>(2 * c + 1, 2 * a);
#pragma unroll
        for (int d = 0; d < ND; ++d) {
          st32(sB2 + d * B2_TILE + o0, pack2(vr[d], -vi[d]));
          st32(sB2 + d * B2_TILE + o1, pack2(vi[d], vr[d]));
        }
      }
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    prefetch(t + gridDim.x);  // the raw buffers are free again
    if (tid == 0) {  // ---- stage 1 MMAs
      fence_after();
      mma_levels<KP>(acc0, acc1, sA, A_TILE, sB1, B1_TILE, idesc(N1));
      commit(bar);
    }
    bool ok = wait(bar, phase & 1);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(err, 16);
        wait(bar, phase & 1);  // bounded: the MMAs must be done before the TMEM is released
      }
      break;
    }
    ++phase;
    fence_after();
    // ---- epilogue 1: this thread's U row (nu, n'), columns (m, re/im): U = 2^(es + 1) (L0 + L123)
    // (h: L0, l: L123); pair maximum of the exponents of U
    float h[KP], l[KP];
#pragma unroll
    for (int c = 0; c < KP; c += 16) {
      ld16(tl1 + c, h + c);
      ld16(tl1 + (uint32_t)N1 + c, l + c);
    }
    ld_wait();
    {
      float mx = 0.f;
#pragma unroll
      for (int c = 0; c < KP; ++c)
        if (c < K2) mx = fmaxf(mx, fabsf(__fadd_rn(h[c], l[c])));
      const int eb = fexp(mx);
      if (live && eb) atomicMax(&smax[j], eb + es + 1);  // biased exponent of 2^(es + 1) max|L0 + L123|
    }
    fence_before();
    __syncthreads();
    // ---- stage-2 A: digits of U / 2^esu at rows (m, nu), K = (n', re/im) (overwrites stage 1's A)
    const int ebu = j < PPT ? smax[j] : 0;
    const int esu = ebu ? ebu - 127 + 2 : 0;
    if (live) {
      const float sc = pow2f(es + 1 - esu);
#pragma unroll
      for (int m = 0; m < KP / 2; ++m) {
        if (m < nb) {
          float dr[ND], di[ND];
          fdigits(__fmul_rn(h[2 * m], sc), __fmul_rn(l[2 * m], sc), dr);
          fdigits(__fmul_rn(h[2 * m + 1], sc), __fmul_rn(l[2 * m + 1], sc), di);
          const uint32_t o = off<KP>(j * RS + m * nm + nu1, 2 * x1);
#pragma unroll
          for (int d = 0; d < ND; ++d) st32(sA + d * A_TILE + o, pack2(dr[d], di[d]));
        }
      }
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {  // ---- stage 2 MMAs (into the first KP columns of the same accumulators)
      fence_after();
      mma_levels<KP>(acc0, acc1, sA, A_TILE, sB2, B2_TILE, idesc(KP));
      commit(bar);
    }
    ok = wait(bar, phase & 1);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(err, 16);
        wait(bar, phase & 1);
      }
      break;
    }
    ++phase;
    fence_after();
    // ---- epilogue 2: g rows (m, nu), columns (n, re/im)
#pragma unroll
    for (int c = 0; c < KP; c += 16) {
      ld16(lane_base + c, h + c);
      ld16(lane_base + (uint32_t)N1 + c, l + c);
    }
    ld_wait();
    if (live) {
      float2* out = g + (long)iq * sgq + (long)kk * nm * nb2 + (long)nu2 * nb2 + (long)m2 * nb;
      const bool zero = keep && !keep[P];
      const float f = zero ? 0.f : pow2f(esu + 1);  // g = 2^(esu + 1) (L0 + L123), one rounding
#pragma unroll
      for (int c = 0; c < KP; ++c) h[c] = __fmul_rn(__fadd_rn(h[c], l[c]), f);
      if (vec_out) {
#pragma unroll
        for (int n = 0; n < KP / 2; n += 2)
          if (n < nb) reinterpret_cast<float4*>(out)[n / 2] = make_float4(h[2 * n], h[2 * n + 1], h[2 * n + 2], h[2 * n + 3]);
      } else {
#pragma unroll
        for (int n = 0; n < KP / 2; ++n)
          if (n < nb) out[n] = make_float2(h[2 * n], h[2 * n + 1]);
      }
    }
    fence_before();
    __syncthreads();
  }
  cp_async_wait_all();  // no copy may land in shared memory after the CTA has left
  fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
  }
}

struct SmallShape {
  int kp, rs, ppt, n1;
  uint32_t cols;
  size_t smem;
};

// nacc accumulators of PPT * KP columns each must fit the 512 TMEM columns
SmallShape small_shape(int nm, int nb, int nacc = 2) {
  SmallShape s{};
  const int R = nm * nb;
  s.kp = 2 * nb <= 16 ? 16 : 32;
  s.rs = ((R + 31) / 32) * 32;
  s.ppt = s.rs > 0 ? 128 / s.rs : 0;
  if (s.ppt > 4) s.ppt = 4;
  while (s.ppt > 1 && nacc * s.ppt * s.kp > 512) --s.ppt;
  s.n1 = s.ppt * s.kp;
  uint32_t c = 32;
  while (c < (uint32_t)(2 * s.n1)) c <<= 1;
  s.cols = c;
  s.smem = (size_t)bts::ND * (128 * s.kp * 2 + (size_t)s.n1 * s.kp * 2 + (size_t)s.kp * s.kp * 2) + 64;
  return s;
}

// shared memory of one CTA: operand tiles, raw inputs of a tile (G3 in elem_bytes, V), scalars
size_t small_smem(const SmallShape& s, int nm, int nb, size_t elem_bytes) {
  const size_t g3 = (((size_t)s.ppt * nm * nb * nb * elem_bytes) + 15) & ~(size_t)15;
  return s.smem + g3 + (size_t)(s.ppt + 1) * nb * nb * 16;
}

// ---------------------------------------------------------------------------------------------
// The same fused band rotation at FP64 accuracy (the FP64 form, complex128 g), still on the
// tensor cores: every operand is six balanced base-256 digits (48 bits, |D| <= 128, exact in bf16)
// of a fixed-point value relative to a power-of-two scale (G3 and U: one scale per pair; V: 2).
// Digit products of levels i + j <= 6 (26 MMAs per K step) go to five accumulators: levels 0-3
// each alone, where their sums are exact integers in FP32 (|sum| < 2^22 for K <= 32), levels 4-6
// together (2^-32 below level 0: the tensor core's per-instruction FP32 rounding of that sum, ~2^-23
// of it, is ~2^-55 of the result).  The five sums become integers on a 2^-48 grid (adding
// 1.5 * 2^23 after scaling; the combined levels in two exact pieces) combined in 64-bit integers; U
// is re-digitised from that integer and g is assembled from it as an IEEE double with integer
// operations.  No FP64 instruction runs; the error is the digits' rounding (2^-49 of the scale) and
// the dropped levels >= 7: ~5e-14 of each pair's largest |g|^2 (an exact integer model of these
// steps on random inputs).
namespace bt64 {
constexpr int ND = 6;
constexpr int NACC = 5;
// balanced digits of X (|X| < 2^47), value X 2^-48 = sum_i e_i, e_i = D_i 2^-8(i+1), |D_i| <= 128:
// Y = X + 0x808080808080 is in [0, 2^48 + 2^40] and gives D = b - 128 from its bytes b_i (the added
// 128 in every byte position is the carry-free offset of balanced base-256 digits); the top digit
// takes bits 40..48 (b up to 256, D up to +128).  Each digit: one byte permute (or a shift) builds
// the FP32 bits of 2^23 + b, one FMA subtracts 2^23 + 128 and scales, exactly.
__device__ __forceinline__ float dig(uint32_t w, uint32_t sel, float s) {
  return __fmaf_rn(__uint_as_float(__byte_perm(w, 0x4B000000u, sel)), s, -8388736.0f * s);
}
__device__ __forceinline__ void xdigits(long long X, float (&e)[ND]) {
  const unsigned long long Y = (unsigned long long)X + 0x808080808080ULL;
  const uint32_t hi = (uint32_t)(Y >> 32), lo = (uint32_t)Y;
  e[0] = __fmaf_rn(__uint_as_float(0x4B000000u | (hi >> 8)), 0x1p-8f, -8388736.0f * 0x1p-8f);  // bits 40..48
  e[1] = dig(hi, 0x7540, 0x1p-16f);  // byte 4
  e[2] = dig(lo, 0x7543, 0x1p-24f);
  e[3] = dig(lo, 0x7542, 0x1p-32f);
  e[4] = dig(lo, 0x7541, 0x1p-40f);
  e[5] = dig(lo, 0x7540, 0x1p-48f);
}
// x / 2^(emax - 1021) as a signed 48-bit fixed-point integer (rounded), emax >= the biased
// exponent of x, so that |x| / 2^(emax - 1021) < 1/2
__device__ __forceinline__ long long dfixed48(double x, int emax) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e == 0) return 0LL;
  const long long m = (long long)((b & 0xFFFFFFFFFFFFFULL) | (1ULL << 52));
  const int sh = emax + 6 - e;  // X = m 2^(e - 1075) 2^(48 - (emax - 1021)) = m >> (emax + 6 - e), rounded
  const long long M = sh < 53 ? ((m + (1LL << (sh - 1))) >> sh) : 0LL;
  return (b >> 63) ? -M : M;
}
__device__ __forceinline__ int dexp(double x) { return (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FF); }
// the integer n = L 2^k of a level sum (|n| < 2^22; rounded for the combined levels)
// X = n0 2^32 + n1 2^24 + n2 2^16 + n3 2^8 + n4, in units of 2^-48 of the product of the operand
// scales: n0..n3 exact; n4 = the combined levels 4-6 rounded to 2^-48
__device__ __forceinline__ int lvl32(float L, float twok) {
  return __float_as_int(__fmaf_rn(L, twok, 12582912.0f)) - 0x4B400000;
}
__device__ __forceinline__ long long combine(float l0, float l1, float l2, float l3, float l4) {
  long long X = (long long)lvl32(l4, 0x1p48f);
  X += (long long)lvl32(l3, 0x1p40f) * 256;  // widening multiply-adds
  X += (long long)lvl32(l2, 0x1p32f) * 65536;
  X += (long long)lvl32(l1, 0x1p24f) * 16777216;
  return X + ((long long)lvl32(l0, 0x1p16f) << 32);
}
// X 2^E as an IEEE double, exactly (|X| < 2^53), from integer operations
__device__ __forceinline__ double i2d_scaled(long long X, int E) {
  if (X == 0) return 0.0;
  const unsigned long long sgn = X < 0 ? (1ULL << 63) : 0ULL;
  const unsigned long long M = X < 0 ? (unsigned long long)(-X) : (unsigned long long)X;
  const int lz = __clzll((long long)M);
  const int bl = 64 - lz;  // bit length
  const unsigned long long mant = (M << (lz + 1)) >> 12;
  const long long ex = (long long)(bl - 1 + E + 1023);
  if (ex <= 0) return 0.0;  // below the normal range
  return __longlong_as_double((long long)(sgn | ((unsigned long long)ex << 52) | mant));
}
// the 26 digit products of levels <= 6 over KP/16 K steps into accumulator min(level, 4)
template <int KP>
__device__ __forceinline__ void mma_levels64(uint32_t acc, int ncol, uint32_t sA, int a_tile, uint32_t sB, int b_tile,
                                             uint32_t id) {
#pragma unroll
  for (int ks = 0; ks < KP / 16; ++ks) {
    bool first[NACC] = {ks == 0, ks == 0, ks == 0, ks == 0, ks == 0};
#pragma unroll
    for (int lv = 0; lv <= ND; ++lv) {
      const int a_i = lv < NACC ? lv : NACC - 1;
#pragma unroll
      for (int i = (lv > ND - 1 ? lv - (ND - 1) : 0); i <= (lv < ND - 1 ? lv : ND - 1); ++i) {
        const uint64_t da = bts::desc<KP>(sA + i * a_tile + ks * 256);
        const uint64_t db = bts::desc<KP>(sB + (lv - i) * b_tile + ks * 256);
        bts::mma(acc + (uint32_t)(a_i * ncol), da, db, id, first[a_i] ? 0u : 1u);
        first[a_i] = false;
      }
    }
  }
}
}  // namespace bt64

// One CTA per SM holds nslots independent tile slots of four warps (128 threads, TMEM lanes 0-127),
// each with its own shared memory (slot_bytes), TMEM columns (slot_cols), mbarrier and named
// barrier (1 + slot): the five accumulators of a slot take 160 columns at the Si shapes, so
// three slots share one 512-column allocation where separate CTAs would each round up to 256.
//
// Pair (iq, kk) reads its rows [nu][a][b] at X + iq xq + kk xk and writes [nu][m][n] at
// out + iq oq + kk ok; the two may be the same rows (a tile's input is in shared memory before its
// output is written, and no two tiles share a pair).  ADJ = false: V_{k+q}^H X V_k (the band
// rotation); ADJ: V_{k+q} X V_k^H (its adjoint, the same products with both V conjugate-transposed).
// LOSS: the loss terms of the adjoint, c = w_nk / omega_qnu (0 for omega <= omega_min):
// Lpair[iq nk + kk] = sum c |g|^2 (fixed order) and 2 c g written instead of g.  (Template flags:
// the plain rotation compiles without either path; as runtime switches they cost it ~35 % at the
// MoS2 shapes.)
template <int KP, bool ADJ, bool LOSS>
__global__ void __launch_bounds__((KP == 16 ? 3 : 2) * bts::THREADS, 1) k_band_tc_small64(
    const double2* X, long xq, long xk, const double2* __restrict__ Ukq, const double2* __restrict__ Uk, int nq,
    int nk, int nm, int nb, int RS, int PPT, double2* g, long oq, long ok, const int* __restrict__ keep,
    const double* __restrict__ wk, const double* __restrict__ om, double omega_min, double* __restrict__ Lpair,
    int* __restrict__ err, uint32_t tmem_cols, int nslots, unsigned slot_bytes, unsigned slot_cols) {
  using namespace bts;
  using bt64::ND;
  using bt64::NACC;
  constexpr int A_TILE = 128 * KP * 2;
  constexpr int B2_TILE = KP * KP * 2;
  extern __shared__ __align__(1024) unsigned char sm_all[];
  const int slot = threadIdx.x >> 7;
  unsigned char* sm = sm_all + (size_t)slot * slot_bytes;
  const int N1 = PPT * KP;
  const int B1_TILE = N1 * KP * 2;
  unsigned char* A = sm;                  // [ND][128 x KP]
  unsigned char* B1 = A + ND * A_TILE;    // [ND][N1 x KP]
  unsigned char* B2 = B1 + ND * B1_TILE;  // [ND][KP x KP]
  const int per = nm * nb * nb;
  unsigned char* rawG = B2 + ND * B2_TILE;                                   // [PPT][per] complex128
  unsigned char* rawV = rawG + (size_t)PPT * per * sizeof(double2);          // [PPT + 1][nb2]
  int* gmax = reinterpret_cast<int*>(rawV + (size_t)(PPT + 1) * nb * nb * sizeof(double2));  // [4] G3 exponent
  int* umax = gmax + 4;                                                      // [4] bit length of U
  uint64_t* bar = reinterpret_cast<uint64_t*>(umax + 4);
  double* lred = reinterpret_cast<double*>(bar + 1);                         // [4] loss per warp
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm_all + (size_t)nslots * slot_bytes);  // CTA-wide
  const int tid = threadIdx.x & 127, warp = tid >> 5;  // within the slot; warp = TMEM lane quarter
  auto slot_sync = [&]() { asm volatile("bar.sync %0, 128;" ::"r"(1 + slot) : "memory"); };
  auto slot_or = [&](bool v) -> bool {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, 128, p;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(1 + slot)
        : "memory");
    return r != 0;
  };
  const int nb2 = nb * nb, R = nm * nb;
  const uint32_t sA = smem_u32(A), sB1 = smem_u32(B1), sB2 = smem_u32(B2);
  const uint32_t sRawG = smem_u32(rawG), sRawV = smem_u32(rawV);
  const double2* gsm = reinterpret_cast<const double2*>(rawG);
  const double2* vsm = reinterpret_cast<const double2*>(rawV);

  for (int i = tid; i < (ND * (A_TILE + B1_TILE + B2_TILE)) / 16; i += THREADS)
    reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  // this slot's accumulator a (level a, 4: levels 4-6) at columns a * N1 .. a * N1 + N1 - 1 of its range
  const uint32_t tmem = *tslot + (uint32_t)slot * slot_cols;
  const int j = tid / RS, rr = tid - j * RS;
  const bool row_ok = j < PPT && rr < R;
  const int nu1 = rr / nb, x1 = rr - nu1 * nb;  // stage 1 row (nu, n')
  const int m2 = rr / nm, nu2 = rr - m2 * nm;   // stage 2 row (m, nu)
  const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
  const uint32_t tl1 = lane_base + (uint32_t)(j < PPT ? j * KP : 0);
  const unsigned div_nb = (65536u + nb - 1) / nb, div_nb2 = (65536u + nb2 - 1) / nb2;
  uint32_t phase = 0;
  const int nqg = (nq + PPT - 1) / PPT;
  const long ntiles = (long)nqg * nk;
  const long t0 = (long)blockIdx.x * nslots + slot, tstep = (long)gridDim.x * nslots;
  auto prefetch = [&](long tt) {
    if (tt >= ntiles) return;
    const int kk = (int)(tt % nk), qg = (int)(tt / nk);
    for (int jj = 0; jj < PPT; ++jj) {
      const int iq = qg * PPT + jj;
      if (iq >= nq) break;
      const long P = (long)iq * nk + kk;
      const double2* src = X + (long)iq * xq + (long)kk * xk;
      const uint32_t dst = sRawG + (uint32_t)((size_t)jj * per * sizeof(double2));
      for (int i = tid; i < per; i += THREADS) cp_async<16>(dst + (uint32_t)(i * 16), src + i);
      const double2* vs = Ukq + P * nb2;
      for (int i = tid; i < nb2; i += THREADS) cp_async<16>(sRawV + (uint32_t)((jj * nb2 + i) * 16), vs + i);
    }
    const double2* vk = Uk + (long)kk * nb2;
    for (int i = tid; i < nb2; i += THREADS) cp_async<16>(sRawV + (uint32_t)((PPT * nb2 + i) * 16), vk + i);
    cp_async_commit();
  };
  auto wait_mma = [&]() -> bool {
    const bool ok = wait(bar, phase & 1);
    if (slot_or(!ok)) {
      if (tid == 0) {
        atomicOr(err, 16);
        wait(bar, phase & 1);  // bounded: the MMAs must be done before the TMEM is released
      }
      return false;
    }
    ++phase;
    fence_after();
    return true;
  };
  prefetch(t0);

  for (long t = t0; t < ntiles; t += tstep) {
    const int kk = (int)(t % nk), qg = (int)(t / nk);
    if (tid < 4) {
      gmax[tid] = 0;
      umax[tid] = 0;
    }
    cp_async_wait_all();
    slot_sync();
    const int iq = qg * PPT + j;
    const bool live = row_ok && iq < nq;
    const long P = (long)iq * nk + kk;
    const double2* src = gsm + (long)j * per + (long)nu1 * nb2 + x1;
    // ---- pair maximum of the G3 exponents
    if (live) {
      int eb = 0;
#pragma unroll
      for (int a = 0; a < KP / 2; ++a)
        if (a < nb) {
          const double2 z = src[(long)a * nb];
          eb = max(eb, max(bt64::dexp(z.x), bt64::dexp(z.y)));
        }
      atomicMax(&gmax[j], eb);
    }
    // ---- B operands: digits of conj(V_{k+q}) (stage 1, block per pair) and V_k (stage 2), scale 2
    // (|v| <= 1 for unitary V); the adjoint takes conj(V[c][a]) in place of V[a][c]
    for (int e = tid; e < (PPT + 1) * nb2; e += THREADS) {
      const int jj = (int)(((unsigned)e * div_nb2) >> 16), r2 = e - jj * nb2;
      const int a = (int)(((unsigned)r2 * div_nb) >> 16), c = r2 - a * nb;
      const int rv = ADJ ? c * nb + a : r2;
      float vr[ND], vi[ND];
      if (jj < PPT) {
        if (qg * PPT + jj >= nq) continue;
        double2 u = vsm[jj * nb2 + rv];
        if constexpr (ADJ) u.y = -u.y;
        bt64::xdigits(bt64::dfixed48(u.x, 1022), vr);
        bt64::xdigits(bt64::dfixed48(u.y, 1022), vi);
        const uint32_t o0 = off<KP>(jj * KP + 2 * c, 2 * a), o1 = off<KP>(jj * KP + 2 * c + 1, 2 * a);
#pragma unroll
        for (int d = 0; d < ND; ++d) {
          st32(sB1 + d * B1_TILE + o0, pack2(vr[d], vi[d]));
          st32(sB1 + d * B1_TILE + o1, pack2(-vi[d], vr[d]));
        }
      } else {
        double2 u = vsm[PPT * nb2 + rv];
        if constexpr (ADJ) u.y = -u.y;
        bt64::xdigits(bt64::dfixed48(u.x, 1022), vr);
        bt64::xdigits(bt64::dfixed48(u.y, 1022), vi);
        const uint32_t o0 = off<KP>(2 * c, 2 * a), o1 = off<KP>(2 * c + 1, 2 * a);
#pragma unroll
        for (int d = 0; d < ND; ++d) {
          st32(sB2 + d * B2_TILE + o0, pack2(vr[d], -vi[d]));
          st32(sB2 + d * B2_TILE + o1, pack2(vi[d], vr[d]));
        }
      }
    }
    slot_sync();
    // ---- stage-1 A: digits of the G3 rows relative to 2^(emax - 1021) of the pair
    const int gex = j < PPT ? gmax[j] : 0;
    if (live) {
#pragma unroll
      for (int c = 0; c < KP / 8; ++c) {
        uint32_t w[ND][4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int a = 4 * c + i;
          float dr[ND], di[ND];
          if (a < nb) {
            const double2 z = src[(long)a * nb];
            bt64::xdigits(bt64::dfixed48(z.x, gex), dr);
            bt64::xdigits(bt64::dfixed48(z.y, gex), di);
          } else {
#pragma unroll
            for (int d = 0; d < ND; ++d) dr[d] = di[d] = 0.f;
          }
#pragma unroll
          for (int d = 0; d < ND; ++d) w[d][i] = pack2(dr[d], di[d]);
        }
        const uint32_t o = off<KP>(tid, 8 * c);
#pragma unroll
        for (int d = 0; d < ND; ++d) st128(sA + d * A_TILE + o, w[d][0], w[d][1], w[d][2], w[d][3]);
      }
    }
    fence_async_smem();
    fence_before();
    slot_sync();
    prefetch(t + tstep);
    if (tid == 0) {
      fence_after();
      bt64::mma_levels64<KP>(tmem, N1, sA, A_TILE, sB1, B1_TILE, idesc(N1));
      commit(bar);
    }
    if (!wait_mma()) break;
    // ---- epilogue 1: U (row (nu, n'), columns (m, re/im)) as integers X in units of
    // 2^-48 * 2^(gex - 1021) * 2 (the G3 and V scales); pair maximum of the bit lengths
    long long X[KP];
    {
      float l0[KP], l1[KP], l2[KP], l3[KP], l4[KP];
#pragma unroll
      for (int c = 0; c < KP; c += 16) {
        ld16(tl1 + c, l0 + c);
        ld16(tl1 + (uint32_t)N1 + c, l1 + c);
        ld16(tl1 + (uint32_t)(2 * N1) + c, l2 + c);
        ld16(tl1 + (uint32_t)(3 * N1) + c, l3 + c);
        ld16(tl1 + (uint32_t)(4 * N1) + c, l4 + c);
      }
      ld_wait();
      unsigned long long mx = 0;
#pragma unroll
      for (int c = 0; c < KP; ++c) {
        X[c] = bt64::combine(l0[c], l1[c], l2[c], l3[c], l4[c]);
        const unsigned long long M = X[c] < 0 ? (unsigned long long)(-X[c]) : (unsigned long long)X[c];
        if (c < 2 * nb) mx = M > mx ? M : mx;
      }
      if (live) atomicMax(&umax[j], 64 - __clzll((long long)mx));
    }
    fence_before();
    slot_sync();
    // ---- stage-2 A: digits of U relative to 2^B (B = the pair's largest bit length + 1), rows (m, nu)
    const int B = (j < PPT ? umax[j] : 0) + 1;
    if (live) {
#pragma unroll
      for (int m = 0; m < KP / 2; ++m) {
        if (m < nb) {
          float dr[ND], di[ND];
#pragma unroll
          for (int t2 = 0; t2 < 2; ++t2) {
            const long long x = X[2 * m + t2];
            // x / 2^B as a 48-bit fraction (|x| < 2^(B - 1)); shifts of the magnitude keep the sign exact
            const unsigned long long M = x < 0 ? (unsigned long long)(-x) : (unsigned long long)x;
            const long long F = (long long)(B <= 48 ? (M << (48 - B)) : (M >> (B - 48)));
            bt64::xdigits(x < 0 ? -F : F, t2 == 0 ? dr : di);
          }
          const uint32_t o = off<KP>(j * RS + m * nm + nu1, 2 * x1);
#pragma unroll
          for (int d = 0; d < ND; ++d) st32(sA + d * A_TILE + o, pack2(dr[d], di[d]));
        }
      }
    }
    fence_async_smem();
    slot_sync();
    if (tid == 0) {
      fence_after();
      bt64::mma_levels64<KP>(tmem, N1, sA, A_TILE, sB2, B2_TILE, idesc(KP));
      commit(bar);
    }
    if (!wait_mma()) break;
    // ---- epilogue 2: g rows (m, nu), columns (n, re/im) = X_g 2^-48 * 2 * (2^B 2^-48 2^(gex - 1021) 2)
    {
      float l0[KP], l1[KP], l2[KP], l3[KP], l4[KP];
#pragma unroll
      for (int c = 0; c < KP; c += 16) {
        ld16(lane_base + c, l0 + c);
        ld16(lane_base + (uint32_t)N1 + c, l1 + c);
        ld16(lane_base + (uint32_t)(2 * N1) + c, l2 + c);
        ld16(lane_base + (uint32_t)(3 * N1) + c, l3 + c);
        ld16(lane_base + (uint32_t)(4 * N1) + c, l4 + c);
      }
      ld_wait();
      double lsum = 0.0;
      if (live) {
        double2* out = g + (long)iq * oq + (long)kk * ok + (long)nu2 * nb2 + (long)m2 * nb;
        const bool zero = keep && !keep[P];
        // U = X_U 2^-48 2^(gex - 1021) 2; stage-2 A holds U / (2^B 2^-48 2^(gex - 1021) 2)
        const int E = B - 48 + (gex - 1021) + 1 + 1 - 48;
        double inv = 0.0;  // loss: 1 / omega of the row's mode, 0 at or below omega_min
        if constexpr (LOSS) {
          const double w = om[(long)iq * nm + nu2];
          inv = w > omega_min ? 1.0 / w : 0.0;
        }
#pragma unroll
        for (int n = 0; n < KP / 2; ++n) {
          if (n < nb) {
            const long long xr = bt64::combine(l0[2 * n], l1[2 * n], l2[2 * n], l3[2 * n], l4[2 * n]);
            const long long xi = bt64::combine(l0[2 * n + 1], l1[2 * n + 1], l2[2 * n + 1], l3[2 * n + 1], l4[2 * n + 1]);
            double2 v = zero ? make_double2(0.0, 0.0) : make_double2(bt64::i2d_scaled(xr, E), bt64::i2d_scaled(xi, E));
            if constexpr (LOSS) {
              const double c = wk[(long)kk * nb + n] * inv;
              lsum = fma(c, fma(v.x, v.x, v.y * v.y), lsum);
              v = make_double2(2.0 * c * v.x, 2.0 * c * v.y);
            }
            out[n] = v;
          }
        }
      }
      if constexpr (LOSS) {
        // a pair's rows are whole warps (RS is a multiple of 32): warp sums, then the pair's warps in order
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
        if ((tid & 31) == 0) lred[warp] = lsum;
        slot_sync();
        if (live && rr == 0) {
          double sum = 0.0;
          for (int w = j * (RS / 32); w < (j + 1) * (RS / 32); ++w) sum += lred[w];
          Lpair[P] = sum;
        }
      }
    }
    fence_before();
    slot_sync();
  }
  cp_async_wait_all();
  fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tslot), "r"(tmem_cols) : "memory");
  }
}

// Shared-memory request and CTAs per SM of a launch: what the registers, threads and shared memory
// allow, at most tmem_cap; a larger request enforces the cap, so that no CTA's TMEM allocation waits
// on another.  Shared memory is counted in 256-byte units plus the per-CTA reserve.  Cached per
// (kernel, need, cap, device).
cudaError_t small_occupancy(const void* kern, size_t need, int tmem_cap, size_t* smem_out, int* occ_out,
                            int threads = bts::THREADS) {
  struct Entry {
    const void* kern;
    size_t need;
    int cap, dev, threads;
    size_t smem;
    int occ;
  };
  static std::mutex mu;
  static std::vector<Entry> cache;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  // set on every launch: the attribute belongs to the current context
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024)) != cudaSuccess) return e;
  {
    std::lock_guard<std::mutex> lock(mu);
    for (const Entry& c : cache)
      if (c.kern == kern && c.need == need && c.cap == tmem_cap && c.dev == dev && c.threads == threads) {
        *smem_out = c.smem;
        *occ_out = c.occ;
        return cudaSuccess;
      }
  }
  cudaFuncAttributes fa;
  if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
  int sm_smem = 0, reserve = 0, sm_regs = 0;
  if ((e = cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&reserve, cudaDevAttrReservedSharedMemoryPerBlock, dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&sm_regs, cudaDevAttrMaxRegistersPerMultiprocessor, dev)) != cudaSuccess)
    return e;
  auto unit = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t static_smem = fa.sharedSizeBytes;
  const int warp_regs = ((std::max(fa.numRegs, 1) * 32 + 255) / 256) * 256;
  const int by_regs = sm_regs / (warp_regs * (threads / 32));
  const int by_threads = 2048 / threads;
  auto by_smem = [&](size_t dyn) { return (int)((size_t)sm_smem / (unit(dyn + static_smem) + (size_t)reserve)); };
  int occ = std::min(std::min(by_regs, by_threads), by_smem(need));
  size_t smem = need;
  if (occ > tmem_cap) {  // request more shared memory so that at most tmem_cap CTAs fit
    occ = tmem_cap;
    smem = ((size_t)sm_smem / (size_t)tmem_cap - (size_t)reserve - static_smem) & ~(size_t)255;
    if (smem < need) smem = need;
    while (by_smem(smem) > tmem_cap) smem += 256;
  }
  if (occ < 1 || smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  std::lock_guard<std::mutex> lock(mu);
  cache.push_back(Entry{kern, need, tmem_cap, dev, threads, smem, occ});
  *smem_out = smem;
  *occ_out = occ;
  return cudaSuccess;
}

}  // namespace

bool band_tc_small_supported(int nm, int nb) {
  return nb >= 1 && nb <= 16 && nm >= 1 && nm * nb <= 128;
}

cudaError_t launch_band_tc_small(const void* Y, int y_f32, long ldy, const double2* Ukq, const double2* Uk, int nq,
                                 int nk, int nm, int nb, float2* g, long sgq, const int* keep, int* err,
                                 cudaStream_t st) {
  if ((long)nq * nk <= 0) return cudaSuccess;
  if (!band_tc_small_supported(nm, nb) || nk < 1) return cudaErrorInvalidValue;
  const SmallShape s = small_shape(nm, nb);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return cudaErrorInvalidDevice;
  const long ntiles = (long)((nq + s.ppt - 1) / s.ppt) * nk;
  // complex64 G3 in 16-byte copies when every pair's rows start 16-byte aligned and have even length
  const int vec16 = !y_f32 || ((reinterpret_cast<uintptr_t>(Y) & 15) == 0 && ldy % 2 == 0 && (nm * nb * nb) % 2 == 0);
  cudaError_t e;
  // CTAs per SM: what the registers and shared memory allow (occupancy calculator), at most what the
  // TMEM columns allow; a larger shared-memory request enforces the latter, so that no CTA's TMEM
  // allocation waits on another.  The grid is that many CTAs per SM (one wave).
#define EPH_SMALL_LAUNCH(TCT, KPV)                                                                                    \
  do {                                                                                                                \
    auto kern = k_band_tc_small<TCT, KPV>;                                                                            \
    size_t smem = 0;                                                                                                  \
    int occ = 0;                                                                                                      \
    if ((e = small_occupancy(reinterpret_cast<const void*>(kern), small_smem(s, nm, nb, sizeof(TCT)),                 \
                             (int)(512 / s.cols), &smem, &occ)) != cudaSuccess)                                       \
      return e;                                                                                                       \
    const long grid = std::min(ntiles, (long)sms * occ);                                                              \
    kern<<<(unsigned)grid, bts::THREADS, smem, st>>>(static_cast<const TCT*>(Y), ldy, Ukq, Uk, nq, nk, nm, nb, s.rs,  \
                                                     s.ppt, g, sgq, keep, err, s.cols, vec16), note_launch();                        \
  } while (0)
  if (y_f32) {
    if (s.kp == 16) EPH_SMALL_LAUNCH(float2, 16); else EPH_SMALL_LAUNCH(float2, 32);
  } else {
    if (s.kp == 16) EPH_SMALL_LAUNCH(double2, 16); else EPH_SMALL_LAUNCH(double2, 32);
  }
#undef EPH_SMALL_LAUNCH
  return cudaGetLastError();
}

// FP64-accurate variant (complex128 G3 in, complex128 g out): one CTA per SM with up to three tile
// slots (as many as the 512 TMEM columns and the shared memory hold)
cudaError_t launch_band_tc_small64(const double2* Y, long ldy, const double2* Ukq, const double2* Uk, int nq, int nk,
                                   int nm, int nb, double2* g, long sgq, const int* keep, int* err, cudaStream_t st) {
  return launch_band_tc_small64_ex(Y, (long)nk * ldy, ldy, Ukq, Uk, nq, nk, nm, nb, g, sgq, (long)nm * nb * nb, keep,
                                   false, nullptr, nullptr, 0.0, nullptr, err, st);
}

cudaError_t launch_band_tc_small64_ex(const double2* X, long xq, long xk, const double2* Ukq, const double2* Uk, int nq,
                                      int nk, int nm, int nb, double2* out, long oq, long ok, const int* keep, bool adj,
                                      const double* wk, const double* om, double omega_min, double* Lpair, int* err,
                                      cudaStream_t st) {
  if ((long)nq * nk <= 0) return cudaSuccess;
  if (wk && (!om || !Lpair)) return cudaErrorInvalidValue;
  if (!band_tc_small_supported(nm, nb) || nk < 1) return cudaErrorInvalidValue;
  const SmallShape s = small_shape(nm, nb, bt64::NACC);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return cudaErrorInvalidDevice;
  const long ntiles = (long)((nq + s.ppt - 1) / s.ppt) * nk;
  const unsigned slot_cols = (unsigned)(((bt64::NACC * s.n1) + 31) / 32 * 32);
  const size_t slot_need = (size_t)bt64::ND * (128 * s.kp * 2 + (size_t)s.n1 * s.kp * 2 + (size_t)s.kp * s.kp * 2) +
                           (size_t)s.ppt * nm * nb * nb * 16 + (size_t)(s.ppt + 1) * nb * nb * 16 + 128;
  const unsigned slot_bytes = (unsigned)((slot_need + 1023) & ~(size_t)1023);
  int nslots = (int)(512 / slot_cols);
  nslots = std::min(nslots, (int)((220 * 1024 - 64) / slot_bytes));
  nslots = std::min(nslots, s.kp == 16 ? 3 : 2);  // the kernels' launch bounds
  if (nslots < 1) return cudaErrorInvalidConfiguration;
  uint32_t cols = 32;
  while (cols < (uint32_t)(nslots * slot_cols)) cols <<= 1;
  const bool loss = wk != nullptr;
  if (adj && loss) return cudaErrorInvalidValue;
  using Kern = void (*)(const double2*, long, long, const double2*, const double2*, int, int, int, int, int, int, double2*,
                        long, long, const int*, const double*, const double*, double, double*, int*, uint32_t, int,
                        unsigned, unsigned);
  Kern kern = s.kp == 16 ? (adj ? k_band_tc_small64<16, true, false>
                                : (loss ? k_band_tc_small64<16, false, true> : k_band_tc_small64<16, false, false>))
                         : (adj ? k_band_tc_small64<32, true, false>
                                : (loss ? k_band_tc_small64<32, false, true> : k_band_tc_small64<32, false, false>));
  cudaError_t e;
  size_t smem = 0;
  int occ = 0;
  if ((e = small_occupancy(reinterpret_cast<const void*>(kern), (size_t)nslots * slot_bytes + 64, (int)(512 / cols),
                           &smem, &occ, nslots * bts::THREADS)) != cudaSuccess)
    return e;
  const long grid = std::min((ntiles + nslots - 1) / nslots, (long)sms * occ);
  kern<<<(unsigned)grid, nslots * bts::THREADS, smem, st>>>(X, xq, xk, Ukq, Uk, nq, nk, nm, nb, s.rs, s.ppt, out, oq,
                                                              ok, keep, wk, om, omega_min, Lpair, err, cols, nslots,
                                                              slot_bytes, slot_cols), note_launch();
  return cudaGetLastError();
}

}  // namespace eph
