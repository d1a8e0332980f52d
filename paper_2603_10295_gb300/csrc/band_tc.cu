// Band rotation g_nu = V_{k+q}^H G3_nu V_k (the last step of Eq. 7's evaluation, Eqs. 4-5
// gauges) for shapes beyond the shared-memory kernels, on the tcgen05 tensor cores: the mixed
// form's large-Nb path.  Two batched products of the fixed-point digit scheme of the H(k+q)
// contraction with four digits per operand (levels <= 3, ~2^-32 of each row's scale; float-pair
// results), on the real embedding of the complex matrices (K = 2 Nb, re/im interleaved):
//   stage 1, per pair:  C1[2n' + c][nu Nb + a] = (re, im)_c of T[(nu, a)][n'],  T = G3_nu V_k,
//                       A = V_k embedded (rows 2n' + c, K = 2b + t), B = the G3 rows (nu, a);
//   stage 2, per pair:  C2[2m + c][nu Nb + n'] = (re, im)_c of g_nu[m][n'],
//                       A = V_{k+q}^H embedded (rows 2m + c, K = 2a + t),
//                       B rows (nu, n') with K = 2a + t gathered from C1.
// Every B row carries its own power-of-two scale (fixed point relative to the row maximum);
// V is unitary, so its scale is 2.
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
// T[(nu, a)][n'] part t = C1[p][2n' + t][nu nb + a] (float pair hi + lo).
__global__ void k_tdigits(const float2* __restrict__ C1, long sC, int nrow, int nb, long rows, int kp,
                          float* __restrict__ sB, __nv_bfloat16* __restrict__ D, long slice) {
  const long w = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= rows) return;
  const long p = w / nrow;
  const int j = (int)(w - p * nrow);
  const int nu = j / nb, np_ = j - nu * nb;
  const float2* src = C1 + p * sC + (long)nu * nb;
  float2 x[MAXKL];
  int eb = 0;
#pragma unroll
  for (int i = 0; i < MAXKL; ++i) {
    const int kk = lane + 32 * i;
    x[i] = kk < 2 * nb ? src[(long)(2 * np_ + (kk & 1)) * nrow + (kk >> 1)] : make_float2(0.f, 0.f);
    eb = max(eb, (int)((__float_as_uint(x[i].x) >> 23) & 0xFF));
  }
  eb = warp_max_int(eb);
  const int es = eb ? eb - 127 + 2 : 0;  // |hi + lo| <= |hi| (1 + 2^-24): still within s / 2 + 2^-25 s
  if (lane == 0) sB[w] = ldexpf(1.f, es);
#pragma unroll
  for (int i = 0; i < MAXKL; ++i) {
    const int kk = lane + 32 * i;
    if (kk < kp) put_digits(fixedF_f(x[i].x, es) + fixedF_f(x[i].y, es), D, slice, w * kp + kk);
  }
}

// g[iq][kk][nu][m][n'] = complex64 of C2[p][2m + c][nu nb + n'] (hi + lo), pair p0 + p = iq nk + kk.
__global__ void k_gout(const float2* __restrict__ C2, long sC, int nrow, int nb, int nm, long npairs, int nk, long p0,
                       float2* __restrict__ g, long sgq) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long per = (long)nm * nb * nb;
  if (idx >= per * npairs) return;
  const long p = idx / per;
  const long rem = idx - p * per;
  const int nu = (int)(rem / (nb * nb));
  const int r2 = (int)(rem - (long)nu * nb * nb);
  const int m = r2 / nb, n = r2 - m * nb;
  const float2* src = C2 + p * sC + (long)nu * nb + n;
  const float2 re = src[(long)(2 * m) * nrow], im = src[(long)(2 * m + 1) * nrow];
  const long P = p0 + p;
  const long iq = P / nk, kk = P - iq * nk;
  g[iq * sgq + kk * per + rem] = make_float2(__fadd_rn(re.x, re.y), __fadd_rn(im.x, im.y));
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
  // B digits (shared by both stages), C float pairs (C1 then C2), A2 digits, B row scales
  s.per_pair =
      (size_t)NDIG * s.Nr * s.kp * 2 + (size_t)s.M * s.Nr * 8 + (size_t)NDIG * s.M * s.kp * 2 + (size_t)s.Nr * 4;
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
  float2* C = reinterpret_cast<float2*>(chunk + align_up((size_t)NDIG * PB * Nr * kp * 2));
  __nv_bfloat16* A2 = reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<char*>(C) + align_up((size_t)PB * M * Nr * 8));
  float* sB = reinterpret_cast<float*>(reinterpret_cast<char*>(A2) + align_up((size_t)NDIG * PB * M * kp * 2));
  cudaError_t e;
  // A digits of V_k for every k of the tile (stage 1)
  {
    const long slice = (long)nk * M * kp;
    k_vdigits<<<(unsigned)((slice + 255) / 256), 256, 0, st>>>(Uk, (long)nb * nb, nb, nk, kp, 0, A1, slice);
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
                                                 rows, kp, sB, Bd, bslice);
    else
      k_gdigits<double2><<<gblocks, 256, 0, st>>>(static_cast<const double2*>(Y) + p0 * ldy, ldy, y_off, (int)Nr, nb,
                                                  rows, kp, sB, Bd, bslice);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_tc_band_gemm(mA1, mB, M, 0, (int)Nr, kp, (int)pb, 2.0f, sB, C, Nr, (long)M * Nr, err, nk,
                                 (int)(p0 % nk), M, st)) != cudaSuccess)
      return e;
    // stage 2: g = V_{k+q}^H T per pair
    k_tdigits<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, st>>>(C, (long)M * Nr, (int)Nr, nb, rows, kp, sB, Bd,
                                                                   bslice);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_vdigits<<<(unsigned)((aslice + 255) / 256), 256, 0, st>>>(Ukq + p0 * nb * nb, (long)nb * nb, nb, pb, kp, 1, A2,
                                                                aslice);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_tc_band_gemm(mA2, mB, M, 0, (int)Nr, kp, (int)pb, 2.0f, sB, C, Nr, (long)M * Nr, err, (int)pb, 0, M,
                                 st)) != cudaSuccess)
      return e;
    const long tot = pb * nm * nb * nb;
    k_gout<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(C, (long)M * Nr, (int)Nr, nb, nm, pb, nk, p0, g, sgq);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace eph
